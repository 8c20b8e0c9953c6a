"""ctypes declarations of the C ABI in ``include/netburn.h`` (argument
marshalling only: every step of the burn runs in the CUDA library)."""
from __future__ import annotations

import ctypes as C
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

NB_OK = 0
ERRORS = {-1: "NB_E_ARG", -2: "NB_E_TOPOLOGY", -3: "NB_E_TOO_LARGE",
          -4: "NB_E_CUDA", -5: "NB_E_NOMEM", -6: "NB_E_TAPE", -7: "NB_E_COMPILE"}
ZONE_STATUS = {0: "OK", 1: "MAX_STEPS", 2: "DT_UNDERFLOW", 3: "NEWTON_FAIL",
               4: "TAPE_FULL", 5: "NONFINITE", 6: "TIMEOUT", 7: "SINGULAR"}
NCOUNT = 9
COUNTER_NAMES = ("accepted", "rejected_error", "rejected_newton", "newton_iters",
                 "jacobians", "rhs_evals", "rate_evals", "edot_evals", "order_sum")
KERNEL_AUTO = -1
KERNEL_PERSISTENT = 0
KERNEL_PLAIN = 1
KERNEL_COOP = 2

# every symbol declared in include/netburn.h
EXPORTS = ("nb_net_load", "nb_net_free", "nb_net_get_info", "nb_default_options",
           "nb_burn_batch", "nb_burn_batch_host", "nb_tape_alloc", "nb_tape_free",
           "nb_tape_steps", "nb_tape_read", "nb_burn_adjoint", "nb_burn_adjoint_ex", "nb_burn_batch_noalloc",
           "nb_burn_multi", "nb_net_specialize", "nb_specialize_source",
           "nb_specialize_compile",
           "nb_exp_eval", "nb_zone_costs", "nb_strerror")


class Topology(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_reactions", C.c_int32),
                ("reactants", C.c_void_p), ("products", C.c_void_p),
                ("Q", C.c_void_p), ("scale", C.c_void_p),
                ("self_heating", C.c_int32), ("ap_pg", C.c_void_p),
                ("ap_coeffs", C.c_void_p), ("screen", C.c_void_p),
                ("tab_of", C.c_void_p), ("tab_nd", C.c_int32), ("tab_nt", C.c_int32),
                ("tab_dens", C.c_void_p), ("tab_t9", C.c_void_p),
                ("tab_lnl", C.c_void_p), ("charge", C.c_void_p)]


class NetInfo(C.Structure):
    _fields_ = [("n_state", C.c_int32), ("n_reactions", C.c_int32),
                ("nnz_jacobian", C.c_int32), ("nnz_lu", C.c_int32),
                ("n_dterms", C.c_int32), ("lane_doubles", C.c_int32),
                ("blob_bytes", C.c_int32), ("has_energy", C.c_int32),
                ("flops_rate_eval", C.c_int64), ("flops_rate_deriv", C.c_int64),
                ("flops_terms", C.c_int64), ("flops_rhs", C.c_int64),
                ("flops_jacobian", C.c_int64), ("flops_lu", C.c_int64),
                ("flops_solve", C.c_int64), ("flops_edot", C.c_int64),
                ("flops_tsolve", C.c_int64),
                ("exp_per_rate_eval", C.c_int32), ("specialize_auto", C.c_int32),
                ("last_specialized", C.c_int32), ("reserved", C.c_int32)]


MULTI_MAX_SETS = 12


class BurnSet(C.Structure):
    _fields_ = [("net", C.c_void_p), ("Z", C.c_int64), ("Y0", C.c_void_p),
                ("T9_0", C.c_void_p), ("rho", C.c_void_p), ("ln_mult", C.c_void_p),
                ("ln_mult_per_zone", C.c_int32), ("t_end_zone", C.c_void_p),
                ("zeta_zone", C.c_void_p),
                ("Y", C.c_void_p), ("T9", C.c_void_p), ("E", C.c_void_p),
                ("counters", C.c_void_p), ("status", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("max_attempts", C.c_int32), ("kernel", C.c_int32),
                ("threads_per_block", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("blob_in_shared", C.c_int32), ("ws_in_shared", C.c_int32),
                ("schedule", C.c_int32), ("specialize", C.c_int32),
                ("t_end_zone", C.c_void_p), ("time_budget_s", C.c_double),
                ("zeta_zone", C.c_void_p), ("warps_per_zone", C.c_int32)]


def load(build_if_needed: bool = True):
    """The loaded library; builds it first when missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB
        lib = C.CDLL(path)
        P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        lib.nb_net_load.argtypes = [P, P, P]
        lib.nb_net_free.argtypes = [P]
        lib.nb_net_get_info.argtypes = [P, P]
        lib.nb_default_options.argtypes = [P]
        lib.nb_default_options.restype = None
        lib.nb_burn_batch.argtypes = [P, I64, P, P, P, D, D, D, P, I32, P, P, P,
                                      P, P, P, P, P]
        lib.nb_burn_batch_host.argtypes = [P, I64, P, P, P, D, D, D, P, I32, P,
                                           P, P, P, P, P, P]
        lib.nb_tape_alloc.argtypes = [P, I64, I32, I32, P]
        lib.nb_tape_read.argtypes = [P, I64, I32, P, P, P, P, P, P]
        lib.nb_tape_free.argtypes = [P]
        lib.nb_tape_steps.argtypes = [P, P]
        lib.nb_burn_adjoint.argtypes = [P, P, I32, P, P, P, P, P, P, P]
        lib.nb_burn_adjoint_ex.argtypes = [P, P, I32, P, P, P, P, P, P, P, P]
        lib.nb_burn_adjoint_ex.restype = C.c_int
        lib.nb_burn_batch_noalloc.argtypes = [P, I64, P, P, P, D, D, D, P, I32, P,
                                              P, P, P, P, P, P]
        lib.nb_burn_batch_noalloc.restype = C.c_int
        lib.nb_burn_multi.argtypes = [I32, P, D, D, D, P, P]
        lib.nb_burn_multi.restype = C.c_int
        lib.nb_net_specialize.argtypes = [P, I32, P, I64]
        lib.nb_net_specialize.restype = C.c_int
        lib.nb_specialize_source.argtypes = [P, P, I32, P, I64, P]
        lib.nb_specialize_source.restype = C.c_int
        lib.nb_specialize_compile.argtypes = [P, P, I32, P, I64]
        lib.nb_specialize_compile.restype = C.c_int
        lib.nb_exp_eval.argtypes = [P, P, P, I64, P]
        lib.nb_zone_costs.argtypes = [P, I64, P, P, P, D, D, D, P, P, P]
        lib.nb_zone_costs.restype = C.c_int
        lib.nb_exp_eval.restype = C.c_int
        lib.nb_strerror.argtypes = [C.c_int]
        lib.nb_strerror.restype = C.c_char_p
        for name in ("nb_net_load", "nb_net_free", "nb_net_get_info",
                     "nb_burn_batch", "nb_burn_batch_host", "nb_tape_alloc",
                     "nb_tape_free", "nb_tape_steps", "nb_tape_read", "nb_burn_adjoint"):
            getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


class NetburnError(RuntimeError):
    pass


def check(rc: int, what: str):
    if rc != NB_OK:
        lib = load(False)
        raise NetburnError(f"{what}: {ERRORS.get(rc, rc)} "
                           f"({lib.nb_strerror(rc).decode()})")
