"""GB300-native (sm_103a) GeNIOS x-subproblem engine.

The solver and its kernels live in ``libgenios.so`` (CUDA, C ABI in include/genios.h); this
package is the Python binding: ``_lib`` marshals arguments through ctypes, ``solver`` wraps a
context for torch tensors / NumPy arrays.  PyTorch is used only for device memory and streams.
"""
from . import _lib  # noqa: F401
from ._lib import (  # noqa: F401
    FP64, FP32, BF16, FP8_E4M3, LOSS_SQUARED, LOSS_LOGISTIC, LOSS_HUBER, STOP_RESID, STOP_GAP, STOP_KKT,
    GeniosError, Info, Options, default_options, lib,
)
from .solver import Solver, ops  # noqa: F401
try:
    from .solver import solve_differentiable  # noqa: F401
except ImportError:  # pragma: no cover - torch absent
    pass
