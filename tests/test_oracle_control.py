"""Pins of the oracle's starting step, step-size controller and order choice.

The paper names the integrator family (VODE, Sec. 2) and prints none of its
rules, so these pins hold the oracle to the rules as this project states
them, on problems where everything the rules act on has a closed form:
  * the starting step of Hairer, Norsett and Wanner (Solving ODEs I, Sec.
    II.4, order p = 1) for a one-body decay X -> Y, where the weighted norms
    d0 = ||x0||, d1 = ||f(x0)|| and d2 = ||x''(0)|| = ||J f(x0)|| = lambda d1
    are exact;
  * the step-size sequence of fixed-order backward Euler on the same decay,
    where every step's solution (I - hA)^-1 x_n, predictor and error estimate
    are exact, evaluated in 50-digit arithmetic from the stated rules
    (factor 0.9 err^(-1/2), clamped to [0.2, 5], kept at 1 inside [1, 1.2),
    rejections h <- h max(0.2, 0.9 err^(-1/2)), last step landing on t_end);
  * every decision the controller takes after an accepted step of real
    burns (a stiff Bateman chain, the self-heating chain, the 48-species
    network): the error estimates E_q of orders k-1, k, k+1 recomputed in
    50-digit arithmetic from the taped accepted states (newest point against
    the degree-q extrapolation through the q+1 older ones, scaled by
    h / (t_new - t_{n-q})), the order with the largest factor 0.9
    E_q^(-1/(q+1)) taken only after k+1 steps at order k (order k+1 only
    with k+3 points held, ties keep k then k-1), and the proposed step size.
The expected values come from mpmath, never from the oracle's arithmetic.
"""
import mpmath
import numpy as np
import pytest

import oracle
from tests.test_oracle import make_net



@pytest.fixture(autouse=True)
def fifty_digits():
    with mpmath.workdps(50):
        yield


def decay_net(lam):
    return make_net([(0,)], [(1,)], N=2, lam=[lam])


def wnorm(v, w):
    return mpmath.sqrt(sum((vi / wi) ** 2 for vi, wi in zip(v, w)) / len(v))


def expected_h0(lam, rtol, atol, t_end):
    lam, rtol, atol = mpmath.mpf(lam), mpmath.mpf(rtol), mpmath.mpf(atol)
    w = [atol + rtol, atol]                 # weights at x0 = (1, 0)
    d0 = wnorm([1, 0], w)
    d1 = wnorm([-lam, lam], w)             # f(x0)
    d2 = lam * d1                           # x''(0) = J f(x0) = lam^2 (1, -1)
    hp = mpmath.mpf("1e-6") if (d0 < 1e-5 or d1 < 1e-5) else mpmath.mpf("0.01") * d0 / d1
    hp = min(hp, t_end)
    dm = max(d1, d2)
    h1 = max(mpmath.mpf("1e-6"), hp * mpmath.mpf("1e-3")) if dm <= 1e-15 else mpmath.sqrt(
        mpmath.mpf("0.01") / dm)
    return min(100 * hp, h1, mpmath.mpf(t_end))


@pytest.mark.parametrize("lam,rtol,atol,t_end,branch", [
    (1.0, 1e-6, 1e-10, 1.0, "h1"),          # sqrt(0.01 / d2) governs
    (1.0, 1e-3, 100.0, 1e6, "100hp"),       # 100 * 0.01 d0 / d1 governs
    (1e-9, 1e-3, 1e-3, 1e3, "tiny d1"),     # d1 < 1e-5: hp = 1e-6, then 100 hp
])
def test_starting_step_one_body_decay(lam, rtol, atol, t_end, branch):
    net = decay_net(lam)
    # one attempt only: the first step is taken with h0 and accepted (its
    # error estimate is about 0.005 by construction of h0)
    tp = oracle.burn_tape(net, np.array([1.0, 0.0]), 1.0, 1.0, t_end, rtol, atol,
                          max_attempts=1)
    assert tp["counters"][0] == 1 and len(tp["t"]) == 2
    h0 = expected_h0(lam, rtol, atol, t_end)
    # the oracle estimates d2 by the difference (f(x0 + hp f0) - f(x0)) / hp,
    # which cancels to about eps / (lam hp) ~ 1e-10 relative here
    assert abs(tp["t"][1] - float(h0)) <= 1e-9 * float(h0), (tp["t"][1], h0)
    # the branch of the rule the case exercises
    lamm, r, a = mpmath.mpf(lam), mpmath.mpf(rtol), mpmath.mpf(atol)
    d1 = wnorm([-lamm, lamm], [a + r, a])
    h1 = mpmath.sqrt(mpmath.mpf("0.01") / max(d1, lamm * d1))
    if branch == "h1":
        assert abs(h0 - h1) <= 1e-30 * h1
    elif branch == "100hp":
        assert h0 < h1 and d1 >= 1e-5
    else:
        assert d1 < 1e-5 and abs(h0 - mpmath.mpf("1e-4")) <= 1e-30 * h0


def controller_model(lam, rtol, atol, t_end, nsteps):
    """Accepted times of fixed-order backward Euler with the stated
    controller, exact (50 digits), and the regimes the factor went through."""
    lam, rtol, atol = mpmath.mpf(lam), mpmath.mpf(rtol), mpmath.mpf(atol)
    t_end = mpmath.mpf(t_end)
    x = [mpmath.mpf(1), mpmath.mpf(0)]
    f = lambda v: [-lam * v[0], lam * v[0]]
    h = expected_h0(lam, rtol, atol, t_end)
    t, hist = mpmath.mpf(0), [(mpmath.mpf(0), x)]
    times, regimes, rejects = [], set(), 0
    while len(times) < nsteps and t < t_end:
        if t + h >= t_end:
            h = t_end - t
            t_new = t_end
        else:
            t_new = t + h
        xn = hist[-1][1]
        x_be = [xn[0] / (1 + lam * h), xn[1] + xn[0] * lam * h / (1 + lam * h)]
        if len(hist) == 1:
            xp = [xn[i] + h * f(xn)[i] for i in range(2)]
            c = mpmath.mpf("0.5")
        else:
            tm, xm = hist[-2]
            xp = [xn[i] + (xn[i] - xm[i]) * (t_new - hist[-1][0]) / (hist[-1][0] - tm)
                  for i in range(2)]
            c = h / (t_new - tm)
        w = [atol + rtol * abs(v) for v in xn]
        err = wnorm([c * (x_be[i] - xp[i]) for i in range(2)], w)
        if err > 1:
            rejects += 1
            h = h * max(mpmath.mpf("0.2"), mpmath.mpf("0.9") / mpmath.sqrt(err))
            continue
        hist.append((t_new, x_be))
        t = t_new
        times.append(t)
        fac = mpmath.mpf(5) if err == 0 else mpmath.mpf("0.9") / mpmath.sqrt(err)
        if fac >= 5:
            regimes.add("clamp5")
            fac = mpmath.mpf(5)
        elif fac < mpmath.mpf("0.2"):
            regimes.add("clamp0.2")
            fac = mpmath.mpf("0.2")
        elif 1 <= fac < mpmath.mpf("1.2"):
            regimes.add("hold")
            fac = mpmath.mpf(1)
        elif fac >= mpmath.mpf("1.2"):
            regimes.add("grow")
        else:
            regimes.add("shrink")
        h = h * fac
    return times, regimes, rejects


@pytest.mark.parametrize("lam,rtol,atol,t_end,n", [
    (1.0, 1e-6, 1e-10, 3.0, 60),
    (50.0, 1e-4, 1e-8, 0.5, 60),
])
def test_step_controller_backward_euler_decay(lam, rtol, atol, t_end, n):
    net = decay_net(lam)
    tp = oracle.burn_tape(net, np.array([1.0, 0.0]), 1.0, 1.0, t_end, rtol, atol,
                          fixed_order=1)
    times, regimes, rejects = controller_model(lam, rtol, atol, t_end, n)
    got = tp["t"][1:1 + len(times)]
    assert len(got) == len(times)
    exp = np.array([float(v) for v in times])
    # h0 carries the ~1e-10 of its difference estimate of d2 (see above)
    np.testing.assert_allclose(got, exp, rtol=1e-9)
    # the sequence exercised the clamp at 5, free growth and the hold band
    assert {"clamp5", "grow", "hold"} <= regimes, regimes


def lagrange_at(ts, xs, t):
    """Value at t of the polynomial through (ts[j], xs[j]), exact."""
    out = [mpmath.mpf(0)] * len(xs[0])
    for j in range(len(ts)):
        lj = mpmath.mpf(1)
        for m in range(len(ts)):
            if m != j:
                lj *= (t - ts[m]) / (ts[j] - ts[m])
        out = [o + lj * v for o, v in zip(out, xs[j])]
    return out


def replay_controller(tp, rtol, atol, t_end, kmax=5):
    """Recompute, exactly from the taped accepted states, the decision the
    stated controller takes after each accepted step s >= 2: the order of the
    next step and the step size it proposes.  Returns a list of (s,
    predicted order, predicted h, margin), margin = how far the decision is
    from a tie or a band edge (relative)."""
    T = [mpmath.mpf(float(v)) for v in tp["t"]]
    X = [[mpmath.mpf(float(v)) for v in row] for row in tp["x"]]
    atol, rtol = mpmath.mpf(atol), mpmath.mpf(rtol)
    k, nconsec, out = 1, 0, []
    for s in range(1, len(T)):
        nh = min(s + 1, 7)                  # points held after this step
        h = T[s] - T[s - 1]
        w = [atol + rtol * abs(v) for v in X[s - 1]]

        def E(q):                           # newest point vs degree-q extrapolation
            older = list(range(s - 1, s - q - 2, -1))
            P = lagrange_at([T[j] for j in older], [X[j] for j in older], T[s])
            c = h / (T[s] - T[s - q - 1])
            return wnorm([c * (a - b) for a, b in zip(X[s], P)], w)

        def fac(e, q):
            return mpmath.mpf(5) if e == 0 else mpmath.mpf("0.9") * e ** (-mpmath.mpf(1) / (q + 1))

        if T[s] >= t_end:
            break
        nconsec += 1
        kk = int(tp["k"][s])
        if s == 1:                          # first step: Euler predictor, needs f(x0)
            k_next = k
            out.append((s, min(k, nh), None, 0.0))
            continue
        cands = []
        if nconsec >= k + 1:
            cands.append((fac(E(k), k), k))
            if k > 1:
                cands.append((fac(E(k - 1), k - 1), k - 1))
            if k < kmax and nh >= k + 3:
                cands.append((fac(E(k + 1), k + 1), k + 1))
            best, best_q = cands[0]
            for f, q in cands[1:]:
                if f > best:
                    best, best_q = f, q
            if best_q != k:
                k, nconsec = best_q, 0
            factor = best
        else:
            factor = fac(E(kk), kk)
        vals = sorted(float(f) for f, _ in cands)
        margin = min([abs(vals[-1] - vals[-2]) / vals[-1]] if len(vals) > 1 else [1.0])
        for edge in (0.2, 1.0, 1.2, 5.0):
            margin = min(margin, abs(float(factor) - edge) / edge)
        factor = min(max(factor, mpmath.mpf("0.2")), mpmath.mpf(5))
        if 1 <= factor < mpmath.mpf("1.2"):
            factor = mpmath.mpf(1)
        out.append((s, k, h * factor, margin))
    return out


CONTROL_CASES = [("bateman", 0), ("chain13_heat", 0), ("chain13_heat", 3),
                 ("chain13_heat", 11), ("net48", 0), ("net48", 1)]


@pytest.mark.parametrize("name,zone", CONTROL_CASES)
def test_controller_decisions_replayed_exactly(name, zone):
    if name == "bateman":
        lams = [1e-2, 0.3, 7.0, 150.0, 4000.0, 9e4, 0.0]
        m = len(lams)
        net = make_net([(i,) for i in range(m - 1)], [(i + 1,) for i in range(m - 1)],
                       N=m, lam=lams[:-1])
        Y0 = np.zeros(m)
        Y0[0] = 1.0
        T9, rho, t_end, rtol, atol = 1.0, 1.0, 2.0, 1e-10, 1e-20
    else:
        import gen
        net, z, st = gen.problem(name, zone + 1)
        Y0, T9, rho = z["Y"][zone], z["T9"][zone], z["rho"][zone]
        t_end, rtol, atol = st["t_end"], st["rtol"], st["atol"]
    tp = oracle.burn_tape(net, Y0, T9, rho, t_end, rtol, atol)
    assert tp["status"] == 0
    checked, changes = 0, set()
    prev_k = 1
    for s, k_pred, h_pred, margin in replay_controller(tp, rtol, atol, t_end):
        if s + 1 < len(tp["k"]):
            # the next accepted step runs at the chosen order (capped by the
            # points held, which only binds in the first steps)
            assert int(tp["k"][s + 1]) == min(k_pred, min(s + 1, 7)), (s, tp["k"][s + 1], k_pred)
            if k_pred != prev_k:
                changes.add("up" if k_pred > prev_k else "down")
            prev_k = k_pred
        if h_pred is None or margin < 1e-3:
            continue
        # the taped states carry rounding that the extrapolation differences
        # amplify (x_new - P is ~1e-12 of x for large species): 1e-4
        assert abs(tp["hnext"][s] - float(h_pred)) <= 1e-4 * float(h_pred), (
            s, tp["hnext"][s], float(h_pred))
        checked += 1
    assert checked >= 0.8 * (len(tp["t"]) - 3)
    if name in ("bateman", "net48"):
        assert "up" in changes


@pytest.mark.parametrize("name,zone", [("chain13_heat", 0), ("net48", 1)])
def test_order_sum_counter_is_the_sum_of_the_taped_orders(name, zone):
    # the ninth counter fingerprints the path: the orders of the accepted
    # steps, summed, as the tape records them (record 0 is the start)
    import gen
    net, z, st = gen.problem(name, zone + 1)
    tp = oracle.burn_tape(net, z["Y"][zone], z["T9"][zone], z["rho"][zone], st["t_end"],
                          st["rtol"], st["atol"])
    assert tp["status"] == 0
    cnt = np.asarray(tp["counters"]).reshape(-1)
    assert cnt[0] == len(tp["k"]) - 1
    assert cnt[8] == int(np.sum(tp["k"][1:]))
    assert 1 <= tp["k"][1:].min() and tp["k"][1:].max() <= 5
