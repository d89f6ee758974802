"""Python front-end over the C ABI: a ``Solver`` context and kernel-level ``ops``.

Arrays may be torch tensors (CUDA or CPU) or NumPy arrays; device memory and streams come from
torch.  Nothing here computes: each call forwards pointers and sizes to libgenios.so.
"""
from __future__ import annotations

import ctypes as C
from types import SimpleNamespace

import numpy as np

from . import _lib as L

try:  # torch is the device-memory / stream provider; CPU-only use works without a GPU
    import torch
except ImportError:  # pragma: no cover
    torch = None


def _stream_ptr():
    if torch is not None and torch.cuda.is_available():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


def _ptr(a):
    if a is None:
        return None
    if torch is not None and isinstance(a, torch.Tensor):
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    raise TypeError(type(a))


def _rows(A):
    """A with unit stride along its rows (the C ABI reads row-major with a leading dimension):
    NumPy arrays and torch tensors laid out otherwise (a transpose, a column slice) are copied
    into row-major order."""
    if torch is not None and isinstance(A, torch.Tensor):
        if A.dim() != 2:
            raise ValueError("A must be a matrix")
        if A.stride(1) != 1 or A.stride(0) < A.shape[1]:
            A = A.contiguous()
        return A
    return np.ascontiguousarray(A)


def _vec(v, like):
    """v as a contiguous vector in the dtype of the matrix `like` (the C ABI reads b with A's
    dtype), on like's device when both are torch tensors.  A NumPy vector given with a torch
    matrix becomes a tensor on that matrix's device, and the reverse a NumPy array."""
    if torch is not None and isinstance(like, torch.Tensor):
        if not isinstance(v, torch.Tensor):
            v = torch.from_numpy(np.ascontiguousarray(v))
        return v.to(device=like.device, dtype=like.dtype).contiguous()
    if torch is not None and isinstance(v, torch.Tensor):
        v = v.detach().cpu().numpy()
    return np.ascontiguousarray(v, dtype=like.dtype)


def _lda(A) -> int:
    return A.stride(0) if torch is not None and isinstance(A, torch.Tensor) else A.strides[0] // A.itemsize


def _dt(a) -> int:
    if torch is not None and isinstance(a, torch.Tensor):
        return {torch.float64: L.DT_F64, torch.float32: L.DT_F32}[a.dtype]
    return {np.dtype(np.float64): L.DT_F64, np.dtype(np.float32): L.DT_F32}[a.dtype]


class Solver:
    """One GeNIOS context (one problem, one device, one stream)."""

    def __init__(self, options: L.Options | None = None, device: int = 0, **kw):
        self._lib = L.lib()
        self.options = options if options is not None else L.default_options(**kw)
        self._ctx = C.c_void_p()
        st = self._lib.genios_create(C.byref(self.options), device, _stream_ptr(), C.byref(self._ctx))
        L.check(st, None)
        self.n = 0
        self.m = 0
        self._keep = []

    # ------------------------------------------------------------------
    def set_data(self, A, b, loss: int | str = L.LOSS_SQUARED):
        if isinstance(loss, str):
            loss = L.LOSSES[loss]
        A = _rows(A)
        b = _vec(b, A)
        m, n = A.shape
        if tuple(b.shape) != (m,):
            raise ValueError("b must be a vector of m entries")
        mm, nn, ll = (C.c_int64 * 1)(m), (C.c_int64 * 1)(n), (C.c_int64 * 1)(_lda(A))
        Ap = (C.c_void_p * 1)(_ptr(A).value)
        bp = (C.c_void_p * 1)(_ptr(b).value)
        st = self._lib.genios_set_data(self._ctx, loss, 1, mm, nn, Ap, _dt(A), ll, bp, 0)
        L.check(st, self._ctx)
        self.m, self.n = m, n
        return self

    def set_batch(self, As, bs, loss: int | str = L.LOSS_SQUARED, path_size: int | None = None):
        """Load a batch.  path_size = K: one data set (As[0], bs[0]) shared by K problems that
        differ in lambda (a regularisation path).  Otherwise: len(As) independent problems."""
        if isinstance(loss, str):
            loss = L.LOSSES[loss]
        As = [_rows(a) for a in As]
        if any(_dt(a) != _dt(As[0]) for a in As):
            raise ValueError("every matrix of a batch must have the same dtype (float64 or float32)")
        bs = [_vec(b, a) for a, b in zip(As, bs)]
        if any(tuple(b.shape) != (a.shape[0],) for a, b in zip(As, bs)):
            raise ValueError("each b must be a vector of its matrix's m entries")
        K = path_size if path_size is not None else len(As)
        cnt = len(As)
        ms = (C.c_int64 * cnt)(*[a.shape[0] for a in As])
        ns = (C.c_int64 * cnt)(*[a.shape[1] for a in As])
        lds = (C.c_int64 * cnt)(*[_lda(a) for a in As])
        Ap = (C.c_void_p * cnt)(*[_ptr(a).value for a in As])
        bp = (C.c_void_p * cnt)(*[_ptr(b).value for b in bs])
        st = self._lib.genios_set_data(self._ctx, loss, K, ms, ns, Ap, _dt(As[0]), lds, bp,
                                       1 if path_size is not None else 0)
        L.check(st, self._ctx)
        self._keep = [As, bs]
        self.K = K
        self.ns = [As[0].shape[1]] * K if path_size is not None else [a.shape[1] for a in As]
        self.m, self.n = As[0].shape
        return self

    def lambda_max_batch(self) -> np.ndarray:
        out = (C.c_double * self.K)()
        L.check(self._lib.genios_lambda_max(self._ctx, out), self._ctx)
        return np.array(out[:])

    def solve_batch(self, lams1, lams2=None, warm_start: bool = False):
        """Returns (list of z arrays, list of info dicts) for the K problems of the batch."""
        K = self.K
        lams2 = np.zeros(K) if lams2 is None else lams2
        l1 = (C.c_double * K)(*[float(v) for v in lams1])
        l2 = (C.c_double * K)(*[float(v) for v in lams2])
        out = np.empty(int(sum(self.ns)), dtype=np.float64)
        infos = (L.Info * K)()
        st = self._lib.genios_solve(self._ctx, l1, l2, _ptr(out), L.DT_F64, infos, int(warm_start))
        L.check(st, self._ctx)
        zs, o = [], 0
        for nk in self.ns:
            zs.append(out[o:o + nk])
            o += nk
        ds = []
        for i in range(K):
            d = infos[i].as_dict()
            d["status_name"] = L.STATUS_NAMES[d["status"]]
            ds.append(d)
        return zs, ds

    def lambda_max(self) -> float:
        out = C.c_double()
        L.check(self._lib.genios_lambda_max(self._ctx, C.byref(out)), self._ctx)
        return out.value

    def solve(self, lam1: float, lam2: float = 0.0, out=None, warm_start: bool = False,
              out_dtype=np.float64):
        """Returns (z, info dict).  ``out`` (host ndarray or torch tensor) receives z if given."""
        if out is None:
            out = np.empty(self.n, dtype=out_dtype)
        elif tuple(out.shape) != (self.n,) or not (out.is_contiguous() if torch is not None and
                                                   isinstance(out, torch.Tensor) else out.flags.c_contiguous):
            raise ValueError("out must be a contiguous vector of n entries")
        info = L.Info()
        l1, l2 = (C.c_double * 1)(lam1), (C.c_double * 1)(lam2)
        st = self._lib.genios_solve(self._ctx, l1, l2, _ptr(out), _dt(out), C.byref(info),
                                    int(warm_start))
        L.check(st, self._ctx)
        d = info.as_dict()
        d["status_name"] = L.STATUS_NAMES[d["status"]]
        return out, d

    def grad(self, dL_dz, want_db: bool = True, want_dA: bool = False):
        """Implicit gradient at the last solve for a scalar loss with gradient dL_dz (n) w.r.t.
        the solution.  Returns dict(dL_dlambda1, dL_db (m) or None, dL_dA (m x n) or None, status)."""
        g = np.ascontiguousarray(np.asarray(dL_dz, dtype=np.float64).reshape(-1))
        if g.size != self.n:
            raise ValueError("dL_dz must have n entries")
        dlam = C.c_double()
        db = np.empty(self.m, dtype=np.float64) if want_db else None
        dA = np.empty((self.m, self.n), dtype=np.float64) if want_dA else None
        st = self._lib.genios_grad(self._ctx, _ptr(g), C.byref(dlam), _ptr(db), _ptr(dA))
        L.check(st, self._ctx)
        return {"dL_dlambda1": dlam.value, "dL_db": db, "dL_dA": dA, "status": L.STATUS_NAMES[st]}

    def last_error(self) -> str:
        return self._lib.genios_last_error(self._ctx).decode()

    def close(self):
        if self._ctx:
            self._lib.genios_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------------------
# kernel-level ops on torch CUDA tensors
# ----------------------------------------------------------------------------------------
def _vt(prec):
    return torch.float64 if prec == L.FP64 else torch.float32


def _chk(st):
    if st != L.OK:
        raise L.GeniosError(st, L.lib().genios_last_error(None).decode())


def lda(prec: int, n: int) -> int:
    return int(L.lib().genios_op_lda(prec, n))


def pad(A, prec: int):
    """Copy a 2-D tensor into a zero-padded device matrix with the kernels' leading dimension
    (storage dtype float64 / float32; BF16 / FP8 copies come from ``quantize``)."""
    m, n = A.shape
    ld = lda(prec, n)
    dt = torch.float64 if prec == L.FP64 else torch.float32
    out = torch.zeros((m, ld), dtype=dt, device="cuda")
    out[:, :n] = A.to(device="cuda", dtype=dt)
    return out


def _ws(prec, m, n):
    nb = int(L.lib().genios_op_workspace_bytes(prec, m, n))
    return torch.empty(nb, dtype=torch.uint8, device="cuda"), nb


def hv(prec, A, n, d, nu, v, row_scale=None):
    m = A.shape[0]
    y = torch.empty(n, dtype=_vt(prec), device="cuda")
    ws, nb = _ws(prec, m, n)
    _chk(L.lib().genios_op_hv(prec, m, n, _ptr(A), A.shape[1], _ptr(row_scale), _ptr(d), nu, _ptr(v),
                              _ptr(y), _ptr(ws), nb, _stream_ptr()))
    return y


def hv_noalloc(prec, A, n, d, nu, v, row_scale=None):
    """Same product as ``hv`` through the entry point that allocates nothing (fixed scratch)."""
    m = A.shape[0]
    y = torch.empty(n, dtype=_vt(prec), device="cuda")
    _chk(L.lib().genios_op_hv_noalloc(prec, m, n, _ptr(A), A.shape[1], _ptr(row_scale), _ptr(d), nu,
                                      _ptr(v), _ptr(y), _stream_ptr()))
    return y


def status():
    """Raises GeniosError(ETIMEOUT) if an op-level row pass on the current device ran out of its
    wait bound since the last check (synchronises the current stream)."""
    _chk(L.lib().genios_op_status(_stream_ptr()))


def gradient(loss, prec, A, A_lo, n, b, x, lam2):
    m = A.shape[0]
    g = torch.empty(n, dtype=_vt(prec), device="cuda")
    w = torch.empty(m, dtype=_vt(prec), device="cuda")
    D = torch.empty(m, dtype=_vt(prec), device="cuda")
    ls = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws, nb = _ws(prec, m, n)
    _chk(L.lib().genios_op_gradient(loss, prec, m, n, _ptr(A), _ptr(A_lo), A.shape[1], _ptr(b), _ptr(x),
                                    lam2, _ptr(g), _ptr(w), _ptr(D), _ptr(ls), _ptr(ws), nb,
                                    _stream_ptr()))
    return g, w, D, ls


def zu_update(prec, x, z, u, rho, lam1, alpha):
    n = x.numel()
    norms = torch.zeros(6, dtype=torch.float64, device="cuda")
    ws, nb = _ws(prec, 1, n)
    _chk(L.lib().genios_op_zu_update(prec, n, _ptr(x), _ptr(z), _ptr(u), rho, lam1, alpha, _ptr(norms),
                                     _ptr(ws), nb, _stream_ptr()))
    return norms


def nystrom_workspace(prec, m, n, s):
    nb = int(L.lib().genios_op_nystrom_workspace_bytes(prec, m, n, s))
    return torch.empty(nb, dtype=torch.uint8, device="cuda")


def nystrom(prec, A, n, s, d, Omega, row_scale=None, workspace=None, flags=0):
    """``workspace`` (from ``nystrom_workspace``) may be passed back in with ``flags`` =
    L.NYS_REUSE_BASIS | L.NYS_WARM to reuse the basis / eigenvectors of the previous call."""
    m = A.shape[0]
    U = torch.empty((n, s), dtype=_vt(prec), device="cuda")
    lam = torch.empty(s, dtype=torch.float64, device="cuda")
    eta = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = nystrom_workspace(prec, m, n, s) if workspace is None else workspace
    _chk(L.lib().genios_op_nystrom(prec, m, n, s, _ptr(A), A.shape[1], _ptr(row_scale), _ptr(d),
                                   _ptr(Omega), _ptr(U), _ptr(lam), _ptr(eta), _ptr(ws), ws.numel(),
                                   int(flags), _stream_ptr()))
    return U, lam, eta


def sketch(prec, A, n, s, d, Omega, row_scale=None):
    """Tensor-core sketch Y = A^T diag(d) A Omega; Omega (float32, n x s) is rounded to bf16 in
    place.  Returns Y (n x s float32)."""
    m = A.shape[0]
    Y = torch.empty((n, s), dtype=torch.float32, device="cuda")
    nb = int(L.lib().genios_op_sketch_workspace_bytes(prec, m, n, s))
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
    _chk(L.lib().genios_op_sketch(prec, m, n, s, _ptr(A), A.shape[1], _ptr(row_scale), _ptr(d), _ptr(Omega),
                                  _ptr(Y), _ptr(ws), nb, _stream_ptr()))
    return Y


def precond(prec, U, lam, nu, v):
    n, s = U.shape
    y = torch.empty(n, dtype=_vt(prec), device="cuda")
    ws, nb = _ws(prec, 1, n)
    _chk(L.lib().genios_op_precond(prec, n, s, _ptr(U), _ptr(lam), nu, _ptr(v), _ptr(y), _ptr(ws), nb,
                                   _stream_ptr()))
    return y


def omega(prec, n, s, seed, stream_id=0):
    Om = torch.empty((n, s), dtype=_vt(prec), device="cuda")
    _chk(L.lib().genios_op_omega(prec, n, s, seed, stream_id, _ptr(Om), _stream_ptr()))
    return Om


def philox(ctr, key, nblocks):
    out = torch.empty(4 * nblocks, dtype=torch.int32, device="cuda")
    _chk(L.lib().genios_op_philox(*[int(c) & 0xFFFFFFFF for c in ctr], *[int(k) & 0xFFFFFFFF for k in key],
                                  nblocks, _ptr(out), _stream_ptr()))
    return out.cpu().numpy().view(np.uint32).reshape(nblocks, 4)


def quantize(prec, A32):
    m, n = A32.shape
    A32 = A32.contiguous()
    ld = lda(prec, n)
    if prec == L.BF16:
        hi = torch.empty((m, ld), dtype=torch.bfloat16, device="cuda")
        lo = torch.empty((m, ld), dtype=torch.bfloat16, device="cuda")
        _chk(L.lib().genios_op_quantize(prec, m, n, _ptr(A32), A32.stride(0), _ptr(hi), _ptr(lo), None,
                                        _stream_ptr()))
        return hi, lo
    codes = torch.empty((m, ld), dtype=torch.uint8, device="cuda")
    sc = torch.empty(m, dtype=torch.float32, device="cuda")
    _chk(L.lib().genios_op_quantize(prec, m, n, _ptr(A32), A32.stride(0), _ptr(codes), None, _ptr(sc),
                                    _stream_ptr()))
    return codes, sc


def pcg(prec, A, n, d, nu, r, U=None, lam=None, rtol=1e-6, max_iter=100, row_scale=None):
    m = A.shape[0]
    s = 0 if U is None else U.shape[1]
    delta = torch.empty(n, dtype=_vt(prec), device="cuda")
    it = C.c_int()
    rel = C.c_double()
    _chk(L.lib().genios_op_pcg(prec, m, n, _ptr(A), A.shape[1], _ptr(row_scale), _ptr(d), nu, _ptr(r), s,
                               _ptr(U), _ptr(lam), rtol, max_iter, _ptr(delta), C.byref(it), C.byref(rel),
                               _stream_ptr()))
    return delta, it.value, rel.value


ops = SimpleNamespace(lda=lda, pad=pad, hv=hv, hv_noalloc=hv_noalloc, status=status, gradient=gradient, zu_update=zu_update, nystrom=nystrom,
                      nystrom_workspace=nystrom_workspace, sketch=sketch,
                      precond=precond, omega=omega, philox=philox, quantize=quantize, pcg=pcg)


# ----------------------------------------------------------------------------------------
# differentiable solve (torch autograd over genios_solve / genios_grad)
# ----------------------------------------------------------------------------------------
if torch is not None:
    class _SolveFn(torch.autograd.Function):
        """z*(lambda_1, b, A) with the implicit gradient of genios_grad in backward."""

        @staticmethod
        def forward(fctx, A, b, lam1, lam2, loss, options):
            s = Solver(options)
            s.set_data(A.detach(), b.detach(), loss)
            z, info = s.solve(float(lam1), float(lam2))
            fctx.solver = s
            fctx.info = info
            fctx.needs = (A.requires_grad, b.requires_grad, torch.is_tensor(lam1) and lam1.requires_grad)
            return torch.as_tensor(z, dtype=A.dtype, device=A.device)

        @staticmethod
        def backward(fctx, gz):
            s = fctx.solver
            need_A, need_b, need_lam = fctx.needs
            out = s.grad(gz.detach().double().cpu().numpy(), want_db=need_b, want_dA=need_A)
            s.close()
            dev, dt = gz.device, gz.dtype
            dA = torch.as_tensor(out["dL_dA"], dtype=dt, device=dev) if need_A else None
            db = torch.as_tensor(out["dL_db"], dtype=dt, device=dev) if need_b else None
            dlam = torch.tensor(out["dL_dlambda1"], dtype=dt, device=dev) if need_lam else None
            return dA, db, dlam, None, None, None

    def solve_differentiable(A, b, lam1, lam2: float = 0.0, loss: str = "squared", **opts):
        """Solution z of  min sum_i loss(a_i^T x - b_i) + lam1 ||x||_1 + lam2/2 ||x||^2  as a torch
        tensor that carries gradients to lam1 (0-d tensor), b and A through the implicit
        gradient at the solution (genios_grad).  opts: genios_options fields."""
        options = L.default_options(**opts)
        return _SolveFn.apply(A, b, lam1, lam2, loss, options)
