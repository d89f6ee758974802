"""CPU FP64 oracle for the GeNIOS hot path (test infrastructure).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import or run it.  The CUDA library and its
Python binding never import it, and it imports nothing from them.

Contents (each function cites the passage of the paper it follows):

* ``losses``     per-sample losses l, l', l'', l* (§3.3, §4.1, §4.2, App. A)
* ``prox``       soft-threshold prox of lambda||.||_1 (§3.1)
* ``linalg``     gradient pass, Hessian-vector product, x-step right-hand side, PCG,
                 randomized Nystrom approximation and preconditioner (§2.1, §2.2, §3.3)
* ``admm``       reference ADMM with an exact x-subproblem solve (§2, §2.5, §3.3), one
                 GeNIOS-style inexact step, residuals and the penalty update
* ``checks``     lambda_max, objective, KKT / relative KKT, duality gap (App. A),
                 brute-force support enumeration, FISTA cross-check
* ``quant``      BF16 hi/lo split and FP8-E4M3 per-row quantisation (round to nearest even)
* ``philox``     Philox4x32-10 counter-based generator and Box-Muller normals
* ``implicit``   dense implicit gradient of the solution on its support

Parity status of each part is listed in each module header.
"""

from . import losses, prox, linalg, admm, checks, quant, philox, implicit  # noqa: F401
