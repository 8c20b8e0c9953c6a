"""Algorithmic operation counts of a burn, from the per-zone event counters
and the network's per-event counts (``Network.info()``).

Flops count FP64 adds and multiplies (an FMA is 2).  exp, log, cbrt, pow,
sqrt and divisions are special functions: they are counted apart, not as
flops, so the flop rate is a floor on the FP64 pipe's real load.
"""
from __future__ import annotations

import numpy as np

# FP64 peak of a GB300: 152 SMs x 2 FP64 FMA lanes per SM per clock
# (1/64 of the FP32 rate) x 2 flops x 2.070 GHz maximum SM clock
SM_COUNT = 152
FP64_FMA_PER_SM_CLK = 2
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12


def burn_ops(info: dict, counters: np.ndarray, self_heating: bool) -> dict:
    """Totals over the zones of one burn: flops and special functions."""
    counters = np.asarray(counters, dtype=np.int64)
    c = counters.reshape(-1, counters.shape[-1]).sum(0)
    acc, rej_e, rej_n, newton, jac, rhs, teval, edot = (int(v) for v in c[:8])
    attempts = acc + rej_e + rej_n
    n = info["n_state"]
    R = info["n_reactions"]
    flops = (teval * info["flops_rate_eval"]
             + (jac if self_heating else 0) * info["flops_rate_deriv"]
             + (rhs + edot) * info["flops_terms"]
             + rhs * info["flops_rhs"]
             + jac * (info["flops_jacobian"] + info["flops_lu"])
             + newton * (info["flops_solve"] + 8 * n)    # residual, update, norm
             + attempts * 13 * n                          # history sum, predictor, error norm
             + edot * (info["flops_edot"] + 4))
    special = {
        "exp": teval * R,
        "log_cbrt": 2 * teval,
        "div": 2 * teval + jac * n + attempts * n,
        "sqrt": newton + attempts,
        "pow": acc,
    }
    return {"flops": int(flops), "special": special, "events": {
        "accepted": acc, "rejected_error": rej_e, "rejected_newton": rej_n,
        "newton_iters": newton, "jacobians": jac, "rhs": rhs,
        "rate_evals": teval, "edot": edot}}


def adjoint_ops(info: dict, steps: int, K: int, self_heating: bool) -> int:
    """Flops of the reverse sweep over `steps` recorded steps, K cotangents."""
    n, R = info["n_state"], info["n_reactions"]
    per_step = ((info["flops_rate_eval"] + info["flops_rate_deriv"]) if self_heating else 0) \
        + info["flops_terms"] + info["flops_jacobian"] + info["flops_lu"] \
        + K * (info["flops_tsolve"] + 12 * n + 6 * R)
    return int(steps * per_step)
