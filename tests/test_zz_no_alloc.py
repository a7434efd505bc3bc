"""tho_orth_noalloc: the allocation-free entry point, against tho_orth.

Some callers cannot allocate device memory (code running under a stream
capture with a no-allocation policy, latency-critical loops that cannot take
cudaMalloc's implicit synchronization, plugins whose host owns all device
memory).  tho_orth_noalloc serves them with a fixed static device scratch.
These tests call it through the C ABI twice in a row per case and compare
with the plan-based tho_orth, at the tolerance of the other parity tests.
The file is named to be collected last.
"""
import ctypes

import pytest
import torch

from paper_2602_14449_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_14449_gb300 import tho
    h = tho.load()
    f = h.tho_orth_noalloc
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [ctypes.POINTER(tho.Desc), vp, i64, vp, i64, vp, i64, vp, vp, vp]
    f.restype = ctypes.c_int
    return tho, f


def _empty(r, c, dt):
    return torch.empty_strided((r, c), (1, max(r, 1)), dtype=dt, device="cuda")


CASES = [
    (torch.float64, 4096, 16, 4),
    (torch.float64, 20000, 32, 8),
    (torch.complex128, 5000, 16, 8),
    (torch.float64, 3 * 256 + 17, 64, 30),
]


@pytest.mark.parametrize("dtype,n,k0,k", CASES)
def test_noalloc_matches_tho_orth(lib, dtype, n, k0, k):
    tho, f = lib
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=100 + n + k0 + k)
    V, A = p.V.cuda(), p.A.cuda()
    Qr, Rr, Sr = tho.orth(V, A)  # existing plan-based entry point
    desc = tho.Desc(n, k0, k, tho.THO_C128 if dtype.is_complex else tho.THO_F64, tho.THO_PREC_FP64, 0)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        Q, R, S = _empty(n, k, dtype), _empty(k, k, dtype), _empty(k0, k, dtype)
        Q.fill_(float("nan"))
        rc = f(ctypes.byref(desc), V.data_ptr(), n, A.data_ptr(), n, Q.data_ptr(), n, R.data_ptr(),
               S.data_ptr(), st)
        assert rc == tho.THO_OK, tho.status_string(rc)
        torch.cuda.synchronize()
        assert float((Q - Qr).abs().max()) <= TOL
        assert float((R - Rr).abs().max()) <= TOL * max(1.0, float(Rr.abs().max()))
        assert float((S - Sr).abs().max()) <= TOL * max(1.0, float(Sr.abs().max()))


def test_noalloc_rejects_problems_beyond_the_scratch(lib):
    tho, f = lib
    desc = tho.Desc(1 << 22, 128, 32, tho.THO_C128, tho.THO_PREC_FP64, 0)
    # The size check runs before any pointer is used; aligned placeholders suffice.
    rc = f(ctypes.byref(desc), 256, 1 << 22, 256, 1 << 22, 256, 1 << 22, None, None, None)
    assert rc == tho.THO_ERR_UNSUPPORTED
    bad = tho.Desc(100, 60, 50, tho.THO_F64, tho.THO_PREC_FP64, 0)
    assert f(ctypes.byref(bad), 256, 100, 256, 100, 256, 100, None, None, None) == tho.THO_ERR_SHAPE
