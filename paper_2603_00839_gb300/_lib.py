"""ctypes declarations of the librtg C ABI (include/rtg.h).

Loading fails loudly when the compiled library is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librtg.so")

MAX_ORDER = 4
MAX_RADIUS = 32
MAX_KRYLOV = 256
MAX_MU = 32
MAX_SLOTS = 64
MAX_BATCH = 1024
MAX_QUEUE = 65536

# rtg_status
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_ALLOC, ERR_TIMEOUT, ERR_NONFINITE = range(7)
# rtg_dtype
F64, F32, BF16 = 0, 1, 2
# rtg_factor_kind
FACTOR_IDENTITY, FACTOR_BANDED_TOEPLITZ, FACTOR_DENSE = 0, 1, 2
FLAG_NO_GRAPH, FLAG_TRUE_RESIDUAL, FLAG_PHASE_TIMES, FLAG_BF16_BASIS = 1, 2, 4, 8
PHASES = ("setup", "init", "apply", "sketch", "gs", "update", "tikhonov", "assemble")
PHASE_COUNT = len(PHASES)


class Shape(C.Structure):
    _fields_ = [("order", C.c_int32), ("dims", C.c_int64 * MAX_ORDER)]


class Factor(C.Structure):
    _fields_ = [("mode", C.c_int32), ("kind", C.c_int32), ("n", C.c_int32), ("radius", C.c_int32),
                ("taps", C.POINTER(C.c_double)), ("dense", C.POINTER(C.c_double))]


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("mu_grid", C.POINTER(C.c_double)), ("n_mu", C.c_int32),
                ("max_restarts", C.c_int32), ("breakdown_tol", C.c_double), ("flags", C.c_int32),
                ("slot", C.c_int32), ("group_max", C.c_int32), ("queue_slots", C.c_int32)]


class Problem(C.Structure):
    _fields_ = [("A_factors", C.POINTER(Factor)), ("nA", C.c_int32), ("B_factors", C.POINTER(Factor)),
                ("nB", C.c_int32), ("shape", Shape), ("C", C.c_void_p), ("X0", C.c_void_p),
                ("X", C.c_void_p), ("m", C.c_int32), ("pad", C.c_int32),
                ("sketch_dims", C.c_int64 * MAX_ORDER), ("seed", C.c_uint64), ("lam", C.c_double),
                ("tol", C.c_double)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("breakdown", C.c_int32),
                ("converged", C.c_int32), ("beta", C.c_double), ("mu", C.c_double),
                ("rho_final", C.c_double), ("rho_hist", C.POINTER(C.c_double)),
                ("gcv", C.POINTER(C.c_double)), ("true_rel_resid", C.c_double),
                ("elapsed_ms", C.c_double), ("device_status", C.c_int32), ("launches", C.c_int32),
                ("tile_config", C.c_int32), ("phase_ms", C.c_double * PHASE_COUNT),
                ("phase_launches", C.c_int32 * PHASE_COUNT), ("true_rel_resid_theta", C.c_double)]


class WsResult(C.Structure):
    _fields_ = [("fell_back", C.c_int32), ("pad", C.c_int32), ("lam", C.c_double), ("tol", C.c_double),
                ("sketch_norm_C", C.c_double), ("sketch_norm_R0", C.c_double)]


class KrylovView(C.Structure):
    _fields_ = [("j", C.c_int32), ("m", C.c_int32), ("breakdown", C.c_int32),
                ("sketch_size", C.c_int32), ("n", C.c_int64), ("beta", C.c_double),
                ("rho", C.c_double), ("V", C.c_void_p), ("Q", C.c_void_p)]


# Every symbol include/rtg.h declares, with its ctypes signature.
_SIGS = {
    "rtg_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "rtg_destroy": (C.c_int, [C.c_void_p]),
    "rtg_last_error": (C.c_char_p, []),
    "rtg_status_string": (C.c_char_p, [C.c_int]),
    "rtg_version": (C.c_int32, []),
    "rtg_operator_apply": (C.c_int, [C.c_void_p, C.POINTER(Factor), C.c_int32, C.POINTER(Factor),
                                     C.c_int32, Shape, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rtg_sketch": (C.c_int, [C.c_void_p, Shape, C.c_int, C.POINTER(C.c_int64), C.c_uint64,
                             C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rtg_philox_words": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int64, C.c_void_p,
                                   C.c_void_p]),
    "rtg_krylov_create": (C.c_int, [C.c_void_p, C.POINTER(Factor), C.c_int32, C.POINTER(Factor),
                                    C.c_int32, Shape, C.c_int, C.c_int32, C.POINTER(C.c_int64),
                                    C.c_uint64, C.c_uint64, C.POINTER(C.c_void_p)]),
    "rtg_krylov_destroy": (C.c_int, [C.c_void_p]),
    "rtg_krylov_start": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rtg_arnoldi_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rtg_krylov_query": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(KrylovView),
                                   C.POINTER(C.c_double), C.c_void_p]),
    "rtg_gmres_solve": (C.c_int, [C.c_void_p, C.POINTER(Factor), C.c_int32, C.POINTER(Factor),
                                  C.c_int32, Shape, C.c_int, C.c_void_p, C.c_int32,
                                  C.POINTER(C.c_int64), C.c_uint64, C.c_double, C.c_void_p,
                                  C.c_void_p, C.POINTER(Opts), C.POINTER(Info), C.c_void_p]),
    "rtg_gmres_submit": (C.c_int, [C.c_void_p, C.POINTER(Factor), C.c_int32, C.POINTER(Factor),
                                   C.c_int32, Shape, C.c_int, C.c_void_p, C.c_int32,
                                   C.POINTER(C.c_int64), C.c_uint64, C.c_double, C.c_void_p,
                                   C.c_void_p, C.POINTER(Opts), C.c_void_p]),
    "rtg_gmres_wait": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Info)]),
    "rtg_gk_solve": (C.c_int, [C.c_void_p, C.POINTER(Factor), C.c_int32, C.POINTER(Factor),
                               C.c_int32, Shape, C.c_int, C.c_void_p, C.c_int32,
                               C.POINTER(C.c_int64), C.c_uint64, C.c_double, C.c_void_p,
                               C.c_void_p, C.POINTER(Opts), C.POINTER(Info), C.c_void_p]),
    "rtg_gmres_solve_batched": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Problem), C.c_int,
                                          C.POINTER(Opts), C.POINTER(Info), C.c_void_p]),
    "rtg_ws_create": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_void_p)]),
    "rtg_ws_destroy": (C.c_int, [C.c_void_p]),
    "rtg_ws_num_params": (C.c_int64, [C.c_void_p]),
    "rtg_ws_get": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "rtg_ws_predict": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "rtg_ws_train_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_float, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "rtg_nn_conv3x3": (C.c_int, [C.c_int32] * 7 + [C.c_void_p] * 8 + [C.c_void_p]),
    "rtg_selftest_bounded_wait": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "rtg_ws_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Factor), C.c_int32, C.POINTER(Factor),
                               C.c_int32, Shape, C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.c_uint64,
                               C.c_void_p, C.POINTER(Opts), C.POINTER(Info), C.POINTER(WsResult), C.c_void_p]),
    "rtg_sketch_noalloc": (C.c_int, [Shape, C.c_int, C.POINTER(C.c_int64), C.c_uint64, C.c_uint64,
                                     C.c_void_p, C.c_void_p, C.c_void_p]),
}

SYMBOLS = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load librtg; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librtg is not built ({path} missing): run __graft_entry__.build() "
                           "or python -m paper_2603_00839_gb300._build")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RtgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} [status {status}]")
        self.status = status


def check(status: int) -> None:
    if status != OK:
        lib = load()
        raise RtgError(status, lib.rtg_last_error().decode())
