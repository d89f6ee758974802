"""ctypes binding of libgenios.so (include/genios.h).  Argument marshalling only: every step
of the solver runs in the library's CUDA kernels.  Importing this module does not need a GPU;
loading the library does need it to be built (``python -m paper_2310_08333_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# GENIOS_LIB selects another build of the same library (the bounds-checked diagnostic build)
LIB_PATH = os.environ.get("GENIOS_LIB") or os.path.join(_HERE, "libgenios.so")

# enums (genios.h)
OK, EINVAL, ESTATE, ENOMEM, ECUDA, EMAXITER, ENUMERIC, ETIMEOUT, EUNSUPPORTED = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ESTATE", "ENOMEM", "ECUDA", "EMAXITER", "ENUMERIC", "ETIMEOUT",
                "EUNSUPPORTED"]
LOSS_SQUARED, LOSS_LOGISTIC, LOSS_HUBER = 0, 1, 2
LOSSES = {"squared": LOSS_SQUARED, "logistic": LOSS_LOGISTIC, "huber": LOSS_HUBER}
FP64, FP32, BF16, FP8_E4M3 = 0, 1, 2, 3
DT_F64, DT_F32, DT_BF16, DT_U8 = 0, 1, 2, 3
STOP_RESID, STOP_GAP, STOP_KKT = 1, 2, 4
NYS_REUSE_BASIS, NYS_WARM = 1, 2   # genios_op_nystrom flags

PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp8": FP8_E4M3}


class Options(C.Structure):
    _fields_ = [
        ("rho", C.c_double), ("sigma", C.c_double), ("alpha", C.c_double),
        ("eps_abs", C.c_double), ("eps_rel", C.c_double), ("eps_gap", C.c_double),
        ("eps_kkt", C.c_double), ("gamma", C.c_double), ("cg_tol_floor", C.c_double),
        ("cg_tol_first", C.c_double),
        ("sketch_rank", C.c_int32), ("resketch_every", C.c_int32),
        ("rho_update_every", C.c_int32), ("rho_update_max", C.c_int32),
        ("rho_update_until", C.c_int32),
        ("rho_tau", C.c_double), ("rho_mu", C.c_double),
        ("max_iter", C.c_int32), ("max_cg_iter", C.c_int32), ("stop_rule", C.c_int32),
        ("precision", C.c_int32), ("kkt_check_every", C.c_int32), ("use_graphs", C.c_int32),
        ("seed", C.c_uint64), ("device_wait_limit_us", C.c_int64),
        ("verbose", C.c_int32), ("profile", C.c_int32), ("tensor_sketch", C.c_int32),
        ("batch_lockstep", C.c_int32), ("persistent_cg", C.c_int32), ("box", C.c_int32),
        ("box_lo", C.c_double), ("box_hi", C.c_double), ("sketch_adaptive", C.c_int32),
        ("sketch_rank_max", C.c_int32), ("sketch_theta", C.c_double), ("device_loop", C.c_int32),
        ("batch_streams", C.c_int32),
        ("autotune", C.c_int32),
        ("fuse_gradient", C.c_int32),
    ]


class Info(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iters", C.c_int32), ("cg_iters_total", C.c_int32),
        ("sketches", C.c_int32), ("rho_updates", C.c_int32), ("nnz", C.c_int32),
        ("rho", C.c_double), ("lambda1", C.c_double), ("lambda2", C.c_double),
        ("r_p", C.c_double), ("r_d", C.c_double), ("rel_gap", C.c_double), ("rel_kkt", C.c_double),
        ("objective", C.c_double), ("t_setup_ms", C.c_double), ("t_sketch_ms", C.c_double),
        ("t_solve_ms", C.c_double), ("kernel_launches", C.c_int64), ("hv_launches", C.c_int64),
        ("hv_ms", C.c_double), ("grad_launches", C.c_int64), ("grad_ms", C.c_double),
        ("hv_bytes", C.c_double), ("sketch_rank_used", C.c_int32), ("fused_grad_passes", C.c_int32),
        ("sketch_bound", C.c_double), ("cg_launches", C.c_int64), ("cg_ms", C.c_double),
        ("cg_phase_ms", C.c_double * 6), ("fused_phase_ms", C.c_double * 2),
        ("cg_span_ms", C.c_double), ("cg_gap_ms", C.c_double),
        ("stage_kb", C.c_int32), ("tune_n", C.c_int32), ("tune_kb", C.c_int32 * 8), ("tune_us", C.c_double * 8),
        ("cg_tail_ms", C.c_double * 4),
    ]

    def as_dict(self) -> dict:
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if isinstance(v, C.Array) else v
        return out


_vp = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int
_d = C.c_double
_sz = C.c_size_t
_u32 = C.c_uint32

# name -> (restype, argtypes)
SIGNATURES = {
    "genios_default_options": (None, [C.POINTER(Options)]),
    "genios_create": (_i32, [C.POINTER(Options), _i32, _vp, C.POINTER(_vp)]),
    "genios_set_data": (_i32, [_vp, _i32, _i32, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_vp), _i32,
                               C.POINTER(_i64), C.POINTER(_vp), _i32]),
    "genios_lambda_max": (_i32, [_vp, C.POINTER(_d)]),
    "genios_solve": (_i32, [_vp, C.POINTER(_d), C.POINTER(_d), _vp, _i32, C.POINTER(Info), _i32]),
    "genios_grad": (_i32, [_vp, _vp, C.POINTER(_d), _vp, _vp]),
    "genios_last_error": (C.c_char_p, [_vp]),
    "genios_destroy": (None, [_vp]),
    "genios_op_workspace_bytes": (_sz, [_i32, _i64, _i64]),
    "genios_op_lda": (_i64, [_i32, _i64]),
    "genios_op_hv": (_i32, [_i32, _i64, _i64, _vp, _i64, _vp, _vp, _d, _vp, _vp, _vp, _sz, _vp]),
    "genios_op_gradient": (_i32, [_i32, _i32, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _d, _vp, _vp, _vp,
                                  _vp, _vp, _sz, _vp]),
    "genios_op_zu_update": (_i32, [_i32, _i64, _vp, _vp, _vp, _d, _d, _d, _vp, _vp, _sz, _vp]),
    "genios_op_nystrom_workspace_bytes": (_sz, [_i32, _i64, _i64, _i32]),
    "genios_op_nystrom": (_i32, [_i32, _i64, _i64, _i32, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                 _sz, _i32, _vp]),
    "genios_op_sketch_workspace_bytes": (_sz, [_i32, _i64, _i64, _i32]),
    "genios_op_sketch": (_i32, [_i32, _i64, _i64, _i32, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "genios_op_precond": (_i32, [_i32, _i64, _i32, _vp, _vp, _d, _vp, _vp, _vp, _sz, _vp]),
    "genios_op_omega": (_i32, [_i32, _i64, _i32, C.c_uint64, _u32, _vp, _vp]),
    "genios_op_philox": (_i32, [_u32, _u32, _u32, _u32, _u32, _u32, _i64, _vp, _vp]),
    "genios_op_quantize": (_i32, [_i32, _i64, _i64, _vp, _i64, _vp, _vp, _vp, _vp]),
    "genios_op_pcg": (_i32, [_i32, _i64, _i64, _vp, _i64, _vp, _vp, _d, _vp, _i32, _vp, _vp, _d, _i32,
                             _vp, C.POINTER(_i32), C.POINTER(_d), _vp]),
    "genios_op_hv_noalloc": (_i32, [_i32, _i64, _i64, _vp, _i64, _vp, _vp, _d, _vp, _vp, _vp]),
    "genios_op_status": (_i32, [_vp]),
}

_lib = None


def lib() -> C.CDLL:
    """Load libgenios.so (raises when it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not found: build it with "
                              "`python -m paper_2310_08333_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class GeniosError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")
        self.status = status


def check(status: int, ctx=None) -> int:
    if status not in (OK, EMAXITER):
        msg = lib().genios_last_error(ctx).decode()
        raise GeniosError(status, msg)
    return status


def default_options(**kw) -> Options:
    o = Options()
    lib().genios_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o
