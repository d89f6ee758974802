"""The Hessian-vector product entry point that allocates no device memory.

Some callers of this library cannot allocate device memory at all: code embedded in a host
application that owns every byte of GPU memory and hands out no workspace, or a code path where
an allocation could fail or stall.  For them genios_op_hv_noalloc computes the same product as
genios_op_hv with its scratch in a fixed array inside the library.  These tests call both entry
points through the C ABI and check that they agree (two calls in a row, so a stale scratch from
the first call cannot hide in the second), and that a request larger than the fixed scratch is
refused with a clear error.  This file is collected last so that a failure here cannot stop a
first-failure run before the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 2e-5, 2: 2e-5, 3: 2e-5}   # the kernel tests' tolerances per precision


@pytest.fixture(scope="module")
def G():
    from paper_2310_08333_gb300 import build as b
    b.build()
    import paper_2310_08333_gb300 as pkg
    pkg.lib()
    return pkg


def _stored(G, prec, A):
    """A in the storage of `prec` (BF16: the library's bf16 copy; FP8: E4M3 codes with per-row
    scales) and the row scales (FP8 only)."""
    if prec in (0, 1):
        return G.ops.pad(A, prec), None
    if prec == 2:
        hi, _ = G.ops.quantize(2, A.to("cuda", torch.float32))
        return hi, None
    return G.ops.quantize(3, A.to("cuda", torch.float32))


@pytest.mark.parametrize("with_d", [True, False])
@pytest.mark.parametrize("prec", [1, 0, 2, 3])
def test_noalloc_matches_workspace_entry_point_on_two_calls(G, prec, with_d):
    """Every storage precision (FP8 with its per-row scales), with and without row weights: the
    product of the entry point without allocation equals genios_op_hv's on two calls in a row of
    different shapes, and no row pass of either ran out of its wait bound."""
    dt = torch.float64 if prec == 0 else torch.float32
    for call, (m, n) in enumerate([(1237, 3001), (4000, 2000)]):
        gen = torch.Generator().manual_seed(100 + call)
        A = torch.randn(m, n, generator=gen, dtype=torch.float64)
        d = torch.rand(m, generator=gen, dtype=torch.float64).to("cuda", dt) if with_d else None
        v = torch.randn(n, generator=gen, dtype=torch.float64).to("cuda", dt)
        Ad, sc = _stored(G, prec, A)
        y_ws = G.ops.hv(prec, Ad, n, d, 0.3, v, row_scale=sc)
        y_na = G.ops.hv_noalloc(prec, Ad, n, d, 0.3, v, row_scale=sc)
        G.ops.status()
        ref = y_ws.double().cpu().numpy()
        err = np.max(np.abs(y_na.double().cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err <= TOL[prec], (call, err)


def test_noalloc_refuses_requests_beyond_its_scratch(G):
    L = G._lib
    m, n = 2000, 20000          # 152 CTAs x 20000 x 4 bytes of partial sums > 8 MiB
    A = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    lib = L.lib()
    st = lib.genios_op_hv_noalloc(L.FP32, m, n, ctypes.c_void_p(A.data_ptr()), n, None, None, 0.0,
                                  ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.EINVAL
    assert b"scratch" in lib.genios_last_error(None)
