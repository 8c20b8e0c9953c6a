"""Pins of the CPU oracle against mathematics it does not contain.

The paper (arXiv:2312.02836) prints no worked example of the burn, so every
pin here is a closed form, an invariant, a textbook constant, brute force,
or a finite difference.  Each is chosen so a plausible slip in the oracle
(a dropped term, a wrong sign or power, a transposed index) fails one.
"""
import math

import mpmath
import numpy as np
import pytest

import gen
import oracle
from gen import NetworkSpec


def make_net(reac, prod, N, lam=None, coeffs=None, Q=None, heat=False,
             scale=None, A=None):
    R = len(reac)
    rt = np.full((R, 3), -1, dtype=np.int16)
    pt = np.full((R, 3), -1, dtype=np.int16)
    for r in range(R):
        for s, v in enumerate(sorted(reac[r])):
            rt[r, s] = v
        for s, v in enumerate(sorted(prod[r])):
            pt[r, s] = v
    if coeffs is None:
        coeffs = np.zeros((R, 7))
        coeffs[:, 0] = np.log(np.asarray(lam, dtype=np.float64))
    return NetworkSpec(name="test", N=N, R=R, reactants=rt, products=pt,
                       A=np.arange(1, N + 1, dtype=np.float64) if A is None else A,
                       coeffs=np.asarray(coeffs, dtype=np.float64),
                       Q=None if Q is None else np.asarray(Q, dtype=np.float64),
                       scale=None if scale is None else np.asarray(scale, dtype=np.float64),
                       self_heating=heat)


# ---------------------------------------------------------------- rates

@pytest.mark.parametrize("T9,phi", [
    (8.0, [1.0, 1 / 8, 1 / 2, 2.0, 8.0, 32.0, 3 * math.log(2.0)]),
    (0.125, [1.0, 8.0, 2.0, 0.5, 0.125, 1 / 32, -3 * math.log(2.0)]),
    (1.0, [1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 0.0]),
])
def test_rate_terms_one_by_one(T9, phi):
    # coefficient vector e_j isolates term j: lambda = exp(phi_j(T9));
    # T9 = 8 and 1/8 have exact cube roots, so every power is hand-known.
    coeffs = np.eye(7)
    net = make_net([(0,)] * 7, [(1,)] * 7, N=2, coeffs=coeffs)
    k, _ = oracle.rate_factors(net, T9, 1.0)
    np.testing.assert_allclose(k, np.exp(phi), rtol=2e-15)


def test_rate_density_power_scale_and_multiplier():
    lam = [2.0, 3.0, 5.0]
    net = make_net([(0,), (0, 1), (0, 1, 2)], [(1,), (2,), (3,)], N=4, lam=lam,
                   scale=[1.0, 0.5, 0.25])
    rho = 7.0
    p = np.array([0.1, -0.2, 0.3])
    k, _ = oracle.rate_factors(net, 2.5, rho, p)
    expect = np.array([2.0, 3.0 * 0.5 * rho, 5.0 * 0.25 * rho ** 2]) * np.exp(p)
    np.testing.assert_allclose(k, expect, rtol=1e-15)


def test_rate_temperature_derivative_fd():
    net = gen.network("net48")
    for T9 in (0.3, 1.0, 3.7, 8.0):
        _, g = oracle.rate_factors(net, T9, 1e6)
        h = 1e-6 * T9
        kp, _ = oracle.rate_factors(net, T9 + h, 1e6)
        km, _ = oracle.rate_factors(net, T9 - h, 1e6)
        fd = (np.log(kp) - np.log(km)) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8 * np.abs(g).max())


# ---------------------------------------------------------------- tabulated rates

def _tab_net(fn, reac=((0,),), prod=((1,),), N=2, charge=(1.0, 1.0)):
    """One tabulated reaction whose table holds fn(log10 rho Ye, T9) at the
    nodes of the generator's grid."""
    net = make_net(list(reac), list(prod), N=N, lam=[1.0])
    D, T = gen.workloads.TAB_DENS, gen.workloads.TAB_T9
    net.tab_of = np.zeros(1, dtype=np.int32)
    net.tab_dens, net.tab_t9 = D.copy(), T.copy()
    net.tab_lnl = fn(D[:, None], T[None, :])[None, :, :].copy()
    net.charge = np.asarray(charge, dtype=np.float64)
    return net


def test_table_bilinear_exact_nodes_derivative_and_clamp():
    # ln lambda = a + b x + c T + d x T is bilinear, so interpolation is exact
    # anywhere in the grid, and d ln lambda / dT9 = c + d x
    a, b, c, d = 1.5, 0.7, -0.4, 0.05
    net = _tab_net(lambda x, T: a + b * x + c * T + d * x * T)
    for T9, rho, ye in ((0.85, 3e5, 0.5), (3.3, 7e6, 0.45), (1.0, 1e6, 1.0), (9.1, 2e7, 0.3)):
        x = math.log10(rho * ye)
        k, g = oracle.rate_factors(net, T9, rho, ye=ye)
        np.testing.assert_allclose(k, [math.exp(a + b * x + c * T9 + d * x * T9)], rtol=1e-13)
        np.testing.assert_allclose(g, [c + d * x], rtol=1e-12)
    # beyond the grid: the edge value, no temperature slope
    k, g = oracle.rate_factors(net, 12.0, 1e6, ye=1.0)
    np.testing.assert_allclose(k, [math.exp(a + b * 6.0 + c * 10.0 + d * 60.0)], rtol=1e-13)
    assert g[0] == 0.0
    k, _ = oracle.rate_factors(net, 2.0, 1e9, ye=1.0)          # log10(rho Ye) = 9 > 8
    np.testing.assert_allclose(k, [math.exp(a + b * 8.0 + c * 2.0 + d * 16.0)], rtol=1e-13)


def test_table_read_equals_scipy_grid_interpolator():
    # the generated tables of the tabulated workload, read by the oracle and
    # by SciPy's linear RegularGridInterpolator (an independent routine)
    from scipy.interpolate import RegularGridInterpolator
    net = gen.network("chain13_heat_tab")
    rng = np.random.default_rng(11)
    for _ in range(20):
        T9 = rng.uniform(0.3, 10.0)
        rho, ye = 10 ** rng.uniform(4.3, 8.3), 0.5
        k, _ = oracle.rate_factors(net, T9, rho, ye=ye)
        x = math.log10(rho * ye)
        for r in np.nonzero(net.tab_of >= 0)[0]:
            f = RegularGridInterpolator((net.tab_dens, net.tab_t9), net.tab_lnl[net.tab_of[r]])
            n_r = int((net.reactants[r] >= 0).sum())
            lnk = math.log(k[r] / rho ** (n_r - 1))
            assert abs(lnk - f([[x, T9]])[0]) < 1e-12


def test_table_reads_rho_ye_of_the_initial_composition():
    # one-body decay 0 -> 1 whose table depends on density only: lambda =
    # exp(-1 + 0.5 log10(rho Ye)) with Ye = sum Z_i Y_i = 3 * 0.1 + 1 * 0.2
    net = _tab_net(lambda x, T: -1.0 + 0.5 * x + 0.0 * T, charge=(3.0, 1.0))
    Y0 = np.array([[0.1, 0.2]])
    rho, t_end = 4e6, 0.7
    ye = 3.0 * 0.1 + 1.0 * 0.2
    lam = math.exp(-1.0 + 0.5 * math.log10(rho * ye))
    o = oracle.burn(net, Y0, np.array([2.0]), np.array([rho]), t_end, 1e-10, 1e-20)
    assert o["status"][0] == 0
    np.testing.assert_allclose(o["Y"][0, 0], 0.1 * math.exp(-lam * t_end), rtol=1e-7)


# ---------------------------------------------------------------- screening

def test_screening_factor_closed_form_and_zero_zeta():
    # alpha + alpha (s = 0.188 * 2 * 2) at T9 = 1 (T6 = 1000):
    # k_screened / k = exp(s sqrt(rho zeta) 1000^(-3/2))
    net = make_net([(0, 0)], [(1,)], N=2, lam=[3.0])
    net.screen = np.array([0.188 * 4.0])
    rho, zeta = 1e6, 1.5
    k0, _ = oracle.rate_factors(net, 1.0, rho)
    k, _ = oracle.rate_factors(net, 1.0, rho, zeta=zeta)
    H = 0.188 * 4.0 * math.sqrt(rho * zeta) * 1000.0 ** -1.5
    np.testing.assert_allclose(k / k0, [math.exp(H)], rtol=1e-14)
    k00, _ = oracle.rate_factors(net, 1.0, rho, zeta=0.0)
    np.testing.assert_array_equal(k00, k0)


def test_screening_coefficient_is_debye_hueckel():
    # Weak screening: H = Z1 Z2 e^2 / (k T lambda_D) with the Debye length
    # lambda_D = sqrt(k T / (4 pi e^2 rho N_A zeta)), in cgs units with
    # CODATA constants.  The oracle's H for s = 0.188 Z1 Z2 (T6 = 1e3 T9)
    # must match it to the 3 digits of 0.188.
    e, kB, NA = 4.80320471e-10, 1.380649e-16, 6.02214076e23
    net = make_net([(0, 1)], [(2,)], N=3, lam=[1.0])
    Z1, Z2 = 6.0, 2.0
    net.screen = np.array([0.188 * Z1 * Z2])
    for T9, rho, zeta in ((0.3, 1e7, 0.8), (2.0, 1e5, 3.0)):
        k0, _ = oracle.rate_factors(net, T9, rho)
        k, _ = oracle.rate_factors(net, T9, rho, zeta=zeta)
        T = T9 * 1e9
        lam_D = math.sqrt(kB * T / (4 * math.pi * e ** 2 * rho * NA * zeta))
        H = Z1 * Z2 * e ** 2 / (kB * T * lam_D)
        assert abs(math.log(k[0] / k0[0]) / H - 1) < 2e-3


def test_screened_rate_temperature_derivative_fd():
    net, z, s = gen.problem("chain13_heat_scr", 8)
    for i in range(4):
        T9, rho, zeta = z["T9"][i], z["rho"][i], z["zeta"][i]
        _, g = oracle.rate_factors(net, T9, rho, zeta=zeta)
        h = 1e-6 * T9
        kp, _ = oracle.rate_factors(net, T9 + h, rho, zeta=zeta)
        km, _ = oracle.rate_factors(net, T9 - h, rho, zeta=zeta)
        fd = (np.log(kp) - np.log(km)) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8 * np.abs(g).max())


# ------------------------------------------ effective (alpha,p)(p,gamma) rate

def _ap_net(lams, reac=((0, 1),), prod=((2,),), N=3, scale=None):
    """One A + alpha -> B reaction as the effective rate, with constant fits
    lams = (ag, ap, pg, pa)."""
    net = make_net(list(reac), list(prod), N=N, lam=[lams[0]], scale=scale)
    net.ap_pg = np.ones(1, dtype=np.int8)
    net.ap_coeffs = np.zeros((1, 3, 7))
    net.ap_coeffs[0, :, 0] = np.log(np.asarray(lams[1:], dtype=np.float64))
    return net


def test_effective_rate_closed_form():
    # lambda = ag + ap pg / (pg + pa) = 2 + 3 * 5 / 12, times s e^p rho^(n-1);
    # constant fits have a zero temperature derivative
    net = _ap_net((2.0, 3.0, 5.0, 7.0), scale=[0.5])
    k, g = oracle.rate_factors(net, 1.7, 4.0, np.array([0.3]))
    np.testing.assert_allclose(k, [0.5 * math.exp(0.3) * 4.0 * (2.0 + 3.0 * 5.0 / 12.0)],
                               rtol=1e-15)
    assert abs(g[0]) < 1e-15


def test_effective_rate_limits():
    # fast (p,g) against a vanishing (p,a): every (a,p) flow reaches B;
    # vanishing (p,g): only the direct channel is left
    k, _ = oracle.rate_factors(_ap_net((2.0, 3.0, 5.0, 1e-300)), 1.0, 1.0)
    np.testing.assert_allclose(k, [5.0], rtol=1e-15)
    k, _ = oracle.rate_factors(_ap_net((2.0, 3.0, 1e-300, 5.0)), 1.0, 1.0)
    np.testing.assert_allclose(k, [2.0], rtol=1e-15)


def test_effective_rate_from_the_fits_in_mpmath():
    # each of the four channels evaluated from its fit in 50-digit arithmetic,
    # then combined: the oracle's lambda and d ln lambda / dT9 (the latter by
    # a central difference of the high-precision lambda)
    net = gen.network("chain13_heat_ap")
    mpmath.mp.dps = 50

    def fit(a, T):
        T = mpmath.mpf(T)
        return mpmath.exp(a[0] + a[1] / T + a[2] * T ** (-mpmath.mpf(1) / 3)
                          + a[3] * T ** (mpmath.mpf(1) / 3) + a[4] * T
                          + a[5] * T ** (mpmath.mpf(5) / 3) + a[6] * mpmath.log(T))

    def lam(r, T):
        ag = fit([mpmath.mpf(float(v)) for v in net.coeffs[r]], T)
        ap, pg, pa = (fit([mpmath.mpf(float(v)) for v in net.ap_coeffs[r, c]], T)
                      for c in range(3))
        return ag + ap * pg / (pg + pa)

    for T9 in (0.6, 1.0, 2.9, 4.7):
        k, g = oracle.rate_factors(net, T9, 1.0)
        for r in np.nonzero(net.ap_pg)[0]:
            assert abs(k[r] / float(lam(r, T9)) - 1) < 1e-13
            h = mpmath.mpf("1e-20")
            d = (mpmath.log(lam(r, T9 + h)) - mpmath.log(lam(r, T9 - h))) / (2 * h)
            assert abs(g[r] - float(d)) <= 1e-12 * max(1.0, abs(float(d)))


def test_effective_rate_equals_the_network_it_replaces():
    # The approximation it stands for: A + a -> X + p, X + p -> A + a,
    # X + p -> B and A + a -> B with proton capture on X fast, against the
    # single effective A + a -> B.  With X and p made and destroyed in pairs,
    # Y_X = Y_p = y relaxes to y^2 = ap Y_A Y_a / (pa + pg) within
    # 1/(2 (pa + pg) y) ~ 2e-6 s, and holds y ~ 2e-7 of the flow; the burns
    # agree to that order, while a wrong split of the flow (or a missing
    # direct channel) changes Y_B by tens of percent.
    ag, ap, pg, pa = 1.0, 10.0, 1e12, 3e11
    full = make_net([(0, 1), (2, 3), (2, 3), (0, 1)], [(2, 3), (0, 1), (4,), (4,)],
                    N=5, lam=[ap, pa, pg, ag], A=np.array([4.0, 12.0, 15.0, 1.0, 16.0]))
    eff = _ap_net((ag, ap, pg, pa))
    Y0f = np.array([0.2, 0.03, 0.0, 0.0, 0.0])
    Y0e = np.array([0.2, 0.03, 0.0])
    t_end = 0.1
    of = oracle.burn(full, Y0f[None], np.array([1.0]), np.array([1.0]), t_end, 1e-10, 1e-20)
    oe = oracle.burn(eff, Y0e[None], np.array([1.0]), np.array([1.0]), t_end, 1e-10, 1e-20)
    assert of["status"][0] == 0 and oe["status"][0] == 0
    yf, ye = of["Y"][0], oe["Y"][0]
    assert 1e-8 < yf[2] < 1e-6 and abs(yf[2] - yf[3]) < 1e-12   # Y_X = Y_p, small
    np.testing.assert_allclose([yf[0], yf[1], yf[4]], ye, rtol=1e-3)
    # the closed form of the effective burn: A + a -> B at the constant rate
    # L = ag + ap pg/(pg+pa), Y_a - Y_A = const: dY_A/dt = -L Y_A (Y_A + d)
    L = ag + ap * pg / (pg + pa)
    d = 0.2 - 0.03
    YA = d * 0.03 / ((0.03 + d) * math.exp(L * d * t_end) - 0.03)
    np.testing.assert_allclose(ye[1], YA, rtol=1e-8)


# ---------------------------------------------------------------- RHS

def test_rhs_single_reactions_by_hand():
    lam = [3.0, 5.0, 7.0, 11.0]
    # 0+0 -> 1 ; 0+0+0 -> 2 ; 1+2 -> 3 ; 3 -> 0+2
    net = make_net([(0, 0), (0, 0, 0), (1, 2), (3,)],
                   [(1,), (2,), (3,), (0, 2)], N=4, lam=lam)
    rho = 2.0
    x = np.array([0.3, 0.2, 0.1, 0.05])
    R0 = 3.0 * rho * x[0] ** 2
    R1 = 5.0 * rho ** 2 * x[0] ** 3
    R2 = 7.0 * rho * x[1] * x[2]
    R3 = 11.0 * x[3]
    expect = np.array([-2 * R0 - 3 * R1 + R3,
                       R0 - R2,
                       R1 - R2 + R3,
                       R2 - R3])
    f, _ = oracle.rhs(net, x, 1.0, rho)
    np.testing.assert_allclose(f, expect, rtol=1e-15)


@pytest.mark.parametrize("name", ["chain13", "net48", "net128_heat"])
def test_rhs_mass_invariant(name):
    # every rate conserves sum_i A_i Y_i, so sum_i A_i f_i = 0
    net = gen.network(name)
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = rng.uniform(0.0, 0.05, net.N)
        T9 = rng.uniform(0.5, 5.0)
        xs = np.concatenate([x, [T9]]) if net.self_heating else x
        f, _ = oracle.rhs(net, xs, T9, 1e6)
        terms = net.A * f[:net.N]
        assert abs(terms.sum()) <= 1e-13 * np.abs(terms).sum()


def test_self_heating_rhs_by_hand():
    net = make_net([(0, 0)], [(1,)], N=2, lam=[4.0], Q=[6.0], heat=True)
    x = np.array([0.4, 0.1, 1.0])   # Y0, Y1, T9 (lambda independent of T9)
    rho = 3.0
    R = 4.0 * rho * 0.4 ** 2
    cv = 1.5 * 0.5 + 1e-3
    f, ed = oracle.rhs(net, x, 0.0, rho)
    np.testing.assert_allclose(f, [-2 * R, R, 6.0 * R / cv], rtol=1e-15)
    assert abs(ed - 6.0 * R) <= 1e-15 * 6.0 * R


# ---------------------------------------------------------------- Jacobian

@pytest.mark.parametrize("name", ["chain13", "chain13_heat", "net48", "net128_heat"])
def test_jacobian_central_fd(name):
    net = gen.network(name)
    onet = oracle.Network(net)
    rng = np.random.default_rng(5)
    x = rng.uniform(0.01, 0.2, net.N)
    T9 = 2.3
    if net.self_heating:
        x = np.concatenate([x, [T9]])
    rho = 3e5
    J = oracle.jacobian(onet, x, T9, rho)
    n = x.shape[0]
    for j in range(n):
        h = 1e-7 * max(abs(x[j]), 1e-10)
        xp = x.copy()
        xm = x.copy()
        xp[j] += h
        xm[j] -= h
        fp, _ = oracle.rhs(onet, xp, T9, rho)
        fm, _ = oracle.rhs(onet, xm, T9, rho)
        fd = (fp - fm) / (2 * h)
        scale = np.abs(J[:, j]).max() + 1e-300
        # central-difference truncation plus the rounding of f at step h
        tol = 1e-6 * np.abs(fd) + 1e-7 * scale + 100 * 2.2e-16 * np.abs(fp) / h
        assert np.all(np.abs(J[:, j] - fd) <= tol), (j, J[:, j], fd)


# ---------------------------------------------------------------- BDF pieces

TEXTBOOK_BDF = {
    1: [1.0, -1.0],
    2: [3 / 2, -2.0, 1 / 2],
    3: [11 / 6, -3.0, 3 / 2, -1 / 3],
    4: [25 / 12, -4.0, 3.0, -4 / 3, 1 / 4],
    5: [137 / 60, -5.0, 5.0, -10 / 3, 5 / 4, -1 / 5],
}


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_bdf_alpha_equal_steps_textbook(k):
    # classical constant-step BDF coefficients (Hairer & Wanner II, Sec. III.1)
    h = 0.37
    t_new = 5.0
    t_old = t_new - h * np.arange(1, k + 1)
    a = oracle.bdf_alpha(k, t_new, t_old, h)
    np.testing.assert_allclose(a, TEXTBOOK_BDF[k], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_bdf_alpha_exact_on_polynomials_variable_steps(k):
    # sum_j alpha_j p(t_{n+1-j}) = h p'(t_{n+1}) for deg p <= k
    rng = np.random.default_rng(k)
    steps = rng.uniform(0.2, 1.0, k)
    t_new = 3.0
    t_old = t_new - np.cumsum(steps)
    h = steps[0]
    a = oracle.bdf_alpha(k, t_new, t_old, h)
    nodes = np.concatenate([[t_new], t_old])
    for deg in range(k + 1):
        c = rng.normal(size=deg + 1)
        p = np.polynomial.Polynomial(c)
        lhs = np.dot(a, p(nodes))
        rhs = h * p.deriv()(t_new)
        assert abs(lhs - rhs) <= 1e-11 * (1 + abs(rhs))
    # and not for degree k+1 (the formula has order exactly k)
    p = np.polynomial.Polynomial(np.eye(k + 2)[k + 1])
    assert abs(np.dot(a, p(nodes)) - h * p.deriv()(t_new)) > 1e-6


def test_extrapolation_exact_and_remainder():
    rng = np.random.default_rng(11)
    for q in range(1, 6):
        t_pts = np.sort(rng.uniform(0, 1, q + 1))[::-1]
        t = 1.3
        coef = rng.normal(size=q + 1)
        p = np.polynomial.Polynomial(coef)
        x_pts = np.stack([p(t_pts), 2 * p(t_pts)], axis=1)
        out = oracle.extrapolate(t_pts, x_pts, t)
        np.testing.assert_allclose(out, [p(t), 2 * p(t)], rtol=1e-11)
        # degree q+1 monomial: remainder = prod (t - t_j)
        mono = t_pts ** (q + 1)
        out = oracle.extrapolate(t_pts, mono[:, None], t)
        assert abs((t ** (q + 1) - out[0]) - np.prod(t - t_pts)) < 1e-11


# ---------------------------------------------------------------- integrator

def bateman(lams, t):
    # N_n(t) for N_0(0) = 1, chain with decay constants lams (last = 0)
    mpmath.mp.dps = 40
    lams = [mpmath.mpf(v) for v in lams]
    out = []
    for n in range(len(lams)):
        pre = mpmath.mpf(1)
        for i in range(n):
            pre *= lams[i]
        s = mpmath.mpf(0)
        for i in range(n + 1):
            den = mpmath.mpf(1)
            for j in range(n + 1):
                if j != i:
                    den *= lams[j] - lams[i]
            s += mpmath.e ** (-lams[i] * t) / den
        out.append(float(pre * s))
    return np.array(out)


@pytest.mark.parametrize("lams,t_end", [
    ([0.5, 1.3, 2.9, 0.7, 0.0], 3.0),                       # non-stiff
    ([1e-2, 0.3, 7.0, 150.0, 4000.0, 9e4, 0.0], 2.0),       # stiff
])
def test_bateman_chain(lams, t_end):
    m = len(lams)
    net = make_net([(i,) for i in range(m - 1)], [(i + 1,) for i in range(m - 1)],
                   N=m, lam=lams[:-1])
    Y0 = np.zeros(m)
    Y0[0] = 1.0
    out = oracle.burn(net, Y0[None], 1.0, 1.0, t_end, 1e-10, 1e-20)
    assert out["status"][0] == 0
    exact = bateman(lams, t_end)
    big = exact > 1e-12
    np.testing.assert_allclose(out["Y"][0][big], exact[big], rtol=1e-7)
    # the order control really raises the order on a smooth problem
    tape = oracle.burn_tape(net, Y0, 1.0, 1.0, t_end, 1e-10, 1e-20)
    assert tape["k"].max() >= 3


@pytest.mark.parametrize("rtol", [1e-6, 1e-8])
def test_bateman_error_follows_tolerance(rtol):
    lams = [0.5, 1.3, 2.9, 0.7, 0.0]
    net = make_net([(i,) for i in range(4)], [(i + 1,) for i in range(4)], N=5,
                   lam=lams[:-1])
    Y0 = np.array([1.0, 0, 0, 0, 0])
    out = oracle.burn(net, Y0[None], 1.0, 1.0, 3.0, rtol, rtol * 1e-4)
    exact = bateman(lams, 3.0)
    err = np.abs(out["Y"][0] - exact).max() / np.abs(exact).max()
    assert err < 100 * rtol


def test_two_body_identical_closed_form():
    k = 1e3
    net = make_net([(0, 0)], [(1,)], N=2, lam=[k])
    out = oracle.burn(net, np.array([[1.0, 0.0]]), 1.0, 1.0, 1.0, 1e-10, 1e-20)
    X = 1.0 / (1.0 + 2 * k * 1.0)
    np.testing.assert_allclose(out["Y"][0], [X, (1 - X) / 2], rtol=1e-7)


def test_three_body_identical_closed_form():
    k, rho, X0, t = 2.0, 10.0, 0.5, 0.8
    net = make_net([(0, 0, 0)], [(1,)], N=2, lam=[k])
    out = oracle.burn(net, np.array([[X0, 0.0]]), 1.0, rho, t, 1e-10, 1e-20)
    kk = k * rho ** 2
    X = X0 / math.sqrt(1 + 6 * kk * X0 ** 2 * t)
    np.testing.assert_allclose(out["Y"][0, 0], X, rtol=1e-7)
    np.testing.assert_allclose(out["Y"][0, 1], (X0 - X) / 3, rtol=1e-7)


def test_two_body_distinct_closed_form():
    k, A0, B0, t = 30.0, 0.3, 0.5, 0.4
    net = make_net([(0, 1)], [(2,)], N=3, lam=[k])
    out = oracle.burn(net, np.array([[A0, B0, 0.0]]), 1.0, 1.0, t, 1e-10, 1e-20)
    d = B0 - A0
    A = d * A0 / (B0 * math.exp(d * k * t) - A0)
    np.testing.assert_allclose(out["Y"][0], [A, A + d, A0 - A], rtol=1e-7)


def test_mass_invariant_every_step():
    net, z, s = gen.problem("net48", 4)
    for i in range(4):
        tp = oracle.burn_tape(net, z["Y"][i], z["T9"][i], z["rho"][i],
                              s["t_end"], s["rtol"], s["atol"])
        assert tp["status"] == 0
        m = tp["x"] @ net.A
        assert np.abs(m - 1.0).max() <= 1e-12
        assert tp["x"].min() >= -10 * s["atol"]


def test_self_heating_against_rk4():
    coeffs = np.zeros((2, 7))
    coeffs[:, 0] = np.log([1.0, 0.5])
    coeffs[:, 4] = [0.3, 0.2]          # lambda grows with T9
    net = make_net([(0, 0), (0, 1)], [(1,), (2,)], N=3, coeffs=coeffs,
                   Q=[2.0, 3.0], heat=True)
    onet = oracle.Network(net)
    x = np.array([0.5, 0.0, 0.0, 1.0])
    t_end = 1.0
    out = oracle.burn(net, x[None, :3], x[3], 2.0, t_end, 1e-11, 1e-16)
    steps = 20000
    h = t_end / steps
    E = 0.0

    def f(v):
        d, ed = oracle.rhs(onet, v, 0.0, 2.0)
        return np.concatenate([d, [ed]])

    v = np.concatenate([x, [E]])
    for _ in range(steps):
        k1 = f(v[:4])
        k2 = f((v + 0.5 * h * k1)[:4])
        k3 = f((v + 0.5 * h * k2)[:4])
        k4 = f((v + h * k3)[:4])
        v = v + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    np.testing.assert_allclose(out["Y"][0], v[:3], rtol=1e-8, atol=1e-14)
    np.testing.assert_allclose(out["T9"][0], v[3], rtol=1e-8)
    np.testing.assert_allclose(out["E"][0], v[4], rtol=1e-8)


def _newton_steps(onet, x0, h, nsteps, coeffs_fn, T9, rho):
    # independent dense full-Newton solve of sum_j c_j x_{n+1-j} = h f(x_{n+1})
    hist = [x0.copy()]
    for s in range(nsteps):
        c = coeffs_fn(s)
        psi = sum(c[j] * hist[-j] for j in range(1, len(c)))
        x = hist[-1].copy()
        for _ in range(60):
            f, _ = oracle.rhs(onet, x, T9, rho)
            J = oracle.jacobian(onet, x, T9, rho)
            G = c[0] * x + psi - h * f
            d = np.linalg.solve(c[0] * np.eye(len(x)) - h * J, -G)
            x = x + d
            if np.all(np.abs(d) <= 1e-16 * (np.abs(x) + 1e-30)):
                break
        hist.append(x)
    return hist[-1]


def _fixed_step_case(order, nsteps):
    # a stiff nonlinear zone of the alpha chain at a step its modified Newton
    # iteration (Jacobian at the predictor) handles without failures
    net, z, s = gen.problem("chain13", 7)
    onet = oracle.Network(net)
    i, h = 6, 1e-8
    out = oracle.burn(onet, z["Y"][i:i + 1], z["T9"][i], z["rho"][i], h * nsteps,
                      s["rtol"], s["atol"], fixed_h=h, fixed_order=order,
                      newton_tol=1e-7, newton_maxit=60)
    assert out["counters"][0, 2] == 0 and out["counters"][0, 0] == nsteps
    return onet, z, i, h, out


def test_fixed_step_backward_euler():
    onet, z, i, h, out = _fixed_step_case(1, 100)
    ref = _newton_steps(onet, z["Y"][i], h, 100, lambda s_: [1.0, -1.0],
                        z["T9"][i], z["rho"][i])
    np.testing.assert_allclose(out["Y"][0], ref, rtol=1e-12, atol=1e-18)


def test_fixed_step_bdf2():
    onet, z, i, h, out = _fixed_step_case(2, 60)
    ref = _newton_steps(onet, z["Y"][i], h, 60,
                        lambda s_: [1.0, -1.0] if s_ == 0 else TEXTBOOK_BDF[2],
                        z["T9"][i], z["rho"][i])
    np.testing.assert_allclose(out["Y"][0], ref, rtol=1e-12, atol=1e-18)


def test_threads_do_not_change_results():
    net, z, s = gen.problem("chain13_heat", 48)
    a = oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"], s["atol"], threads=1)
    b = oracle.burn(net, z["Y"], z["T9"], z["rho"], s["t_end"], s["rtol"], s["atol"], threads=5)
    for key in ("Y", "T9", "E", "counters", "status"):
        assert np.array_equal(a[key], b[key])


def test_nonfinite_input_status():
    net, z, s = gen.problem("chain13", 2)
    T9 = z["T9"].copy()
    T9[1] = np.nan
    out = oracle.burn(net, z["Y"], T9, z["rho"], s["t_end"], s["rtol"], s["atol"])
    assert out["status"][0] == 0 and out["status"][1] == 5


# ---------------------------------------------------------------- sensitivities

def test_sensitivity_one_body_closed_form():
    k, t_end = 3.0, 0.7
    net = make_net([(0,)], [(1,)], N=2, lam=[k])
    Y0 = np.array([1.0, 0.0])
    tp = oracle.burn_tape(net, Y0, 1.0, 1.0, t_end, 1e-10, 1e-20)
    dx, _ = oracle.forward_sensitivity(net, 1.0, 1.0, tp["t"], tp["k"], tp["x"])
    X = math.exp(-k * t_end)
    # d X / d ln(mult) = -k t X ; d X / d X0 = exp(-k t) ; mass: dY1 = -dX
    np.testing.assert_allclose(dx[0, 0], -k * t_end * X, rtol=1e-7)
    np.testing.assert_allclose(dx[1, 0], k * t_end * X, rtol=1e-7)
    np.testing.assert_allclose(dx[0, 1], X, rtol=1e-7)   # column R + 0 = dX0
    np.testing.assert_allclose(dx[1, 1], 1 - X, rtol=1e-7)


@pytest.mark.parametrize("name,zone", [("net48_adjoint", 1), ("chain13_heat", 3)])
def test_sensitivity_against_frozen_schedule_fd(name, zone):
    net, z, s = gen.problem(name, zone + 1)
    onet = oracle.Network(net)
    Y0, T9, rho = z["Y"][zone], z["T9"][zone], z["rho"][zone]
    tp = oracle.burn_tape(onet, Y0, T9, rho, s["t_end"], s["rtol"], s["atol"])
    assert tp["status"] == 0
    dx, dE = oracle.forward_sensitivity(onet, T9, rho, tp["t"], tp["k"], tp["x"])
    eps = 1e-5   # at 1e-6 the ~25-ulp round-off of a 600-step replay dominates small gradients
    R, n = net.R, onet.n
    rng = np.random.default_rng(0)
    params = list(rng.choice(R, 4, replace=False)) + [R + 0, R + 3]
    if not net.self_heating:
        params.append(R + n)       # T9 as a parameter
    else:
        params.append(R + net.N)   # initial T9
    for p in params:
        def run(sign):
            lm = np.zeros(R)
            y0 = Y0.copy()
            t9 = T9
            if p < R:
                lm[p] += sign * eps
            elif p < R + net.N:
                y0[p - R] += sign * eps
            else:
                t9 = T9 * math.exp(sign * eps)
            return oracle.replay(onet, y0, t9, rho, tp["t"], tp["k"], s["rtol"],
                                 s["atol"], ln_mult=lm)
        xp, Ep = run(+1)
        xm, Em = run(-1)
        fd = (xp - xm) / (2 * eps)
        fdE = (Ep - Em) / (2 * eps)
        col = dx[:, p].copy()
        colE = dE[p]
        if p >= R + net.N:        # FD taken in ln T9
            col *= T9
            colE *= T9
        # FD round-off: x is known to ~10 ulps at each end, divided by 2 eps
        floor = 1e-9 * np.abs(col).max() + 1e-8 * np.abs(xp)
        assert np.all(np.abs(col - fd) <= 1e-6 * np.abs(col) + floor), (p, col, fd)
        if net.Q is not None:
            assert abs(colE - fdE) <= 1e-6 * abs(colE) + 1e-8 * abs(Ep), (p, colE, fdE)


def test_per_zone_end_times_equal_separate_burns():
    # the operator-split mode: each zone burns for its own step
    net, z, s = gen.problem("chain13_heat", 6)
    tz = np.array([1e-4, 3e-4, 1e-3, 0.0, 2e-5, 7e-4])
    a = oracle.burn(net, z["Y"], z["T9"], z["rho"], tz, s["rtol"], s["atol"])
    for i in range(6):
        b = oracle.burn(net, z["Y"][i:i + 1], z["T9"][i], z["rho"][i], tz[i], s["rtol"],
                        s["atol"])
        for key in ("Y", "T9", "E", "counters", "status"):
            assert np.array_equal(a[key][i], b[key][0])
    bad = tz.copy()
    bad[1] = np.nan
    bad[2] = -1.0
    c = oracle.burn(net, z["Y"], z["T9"], z["rho"], bad, s["rtol"], s["atol"])
    assert list(c["status"][1:3]) == [5, 5]
    assert np.array_equal(c["Y"][1:3], z["Y"][1:3])


def test_exp_table_of_the_device_code_is_two_to_the_j_over_32():
    # the double-double table of the device exp (Tang's method) against
    # 2^(j/32) from mpmath, regenerated by the script beside the header
    import re
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_2312_02836_gb300", "csrc")
    spec = importlib.util.spec_from_file_location("exp2_table", os.path.join(csrc, "exp2_table.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    text = open(os.path.join(csrc, "expf64.cuh")).read()
    body = text.split("#define NB_EXP2_TABLE", 1)[1].split("\n\n", 1)[0]
    vals = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-f.]+p[+-]\d+", body)]
    assert len(vals) == 64
    assert vals == [v for lt in mod.table() for v in lt]
    mpmath.mp.prec = 200
    for j in range(32):
        err = abs(mpmath.mpf(vals[2 * j]) + mpmath.mpf(vals[2 * j + 1]) - mpmath.mpf(2) ** (mpmath.mpf(j) / 32))
        assert err < mpmath.mpf(2) ** -104
