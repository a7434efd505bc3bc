"""tho_orth_noalloc: the allocation-free entry point.

Some callers cannot allocate device memory: latency-critical loops that cannot
take cudaMalloc's implicit synchronization, and plugins whose host application
owns all device memory.  tho_orth_noalloc serves them with a fixed static
device scratch.  These tests call it through the C ABI twice in a row per
case and check each result against the CPU oracle at the tolerance of the
other parity tests, and against the plan-based tho_orth (same partition and
kernels: the same bits).  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from metrics import loo as loo_np
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


def _noalloc(tho, f, V, A, k0, prec):
    n, k = A.shape
    dtype = A.dtype
    flags = tho.THO_FLAG_ALLOW_K0_ZERO if k0 == 0 else 0
    desc = tho.Desc(n, k0, k, tho.THO_C128 if dtype.is_complex else tho.THO_F64, prec, flags)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Q, R, S = _empty(n, k, dtype), _empty(k, k, dtype), _empty(k0, k, dtype)
    for X in (Q, R, S):
        X.fill_(float("nan"))
    rc = f(ctypes.byref(desc), V.data_ptr() if k0 else None, n, A.data_ptr(), n, Q.data_ptr(), n,
           R.data_ptr(), S.data_ptr() if k0 else None, st)
    assert rc == tho.THO_OK, tho.status_string(rc)
    torch.cuda.synchronize()
    return Q, R, S


def _plan_orth(tho, V, A, k0, prec):
    n, k = A.shape
    flags = tho.THO_FLAG_ALLOW_K0_ZERO if k0 == 0 else 0
    plan = tho.Plan([(n, k0, k)], A.dtype, prec, flags)
    Vd = V if k0 else torch.zeros((n, 0), dtype=A.dtype, device="cuda")
    Q, R, S = tho.orth(Vd, A, prec=prec, plan=plan)
    torch.cuda.synchronize()
    return Q, R, S


CASES = [
    (torch.float64, 4096, 16, 4, "THO_PREC_FP64"),
    (torch.float64, 20000, 32, 8, "THO_PREC_FP64"),
    (torch.complex128, 5000, 16, 8, "THO_PREC_FP64"),
    (torch.float64, 3 * 256 + 17, 64, 30, "THO_PREC_FP64"),
    (torch.float64, 3000, 0, 8, "THO_PREC_FP64"),
    (torch.complex128, 9000, 24, 12, "THO_PREC_FP32_BULK"),
]


@pytest.mark.parametrize("dtype,n,k0,k,prec_name", CASES)
def test_noalloc_matches_oracle_and_tho_orth(lib, dtype, n, k0, k, prec_name):
    tho, f = lib
    prec = getattr(tho, prec_name)
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=100 + n + k0 + k)
    V, A = (p.V.cuda() if k0 else None), p.A.cuda()
    if k0:
        Qo, Ro, So = oracle.two_stage(p.V.numpy(), p.A.numpy())
    else:
        Qo, Ro = oracle.householder_qr(p.A.numpy())
    Qp, Rp, Sp = _plan_orth(tho, V, A, k0, prec)
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        Q, R, S = _noalloc(tho, f, V, A, k0, prec)
        Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
        if prec == tho.THO_PREC_FP64:
            np.testing.assert_allclose(Qh, Qo, atol=TOL, rtol=0)
            np.testing.assert_allclose(Rh, Ro, atol=TOL * max(1.0, np.abs(Ro).max()), rtol=0)
            if k0:
                np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL * max(1.0, np.abs(So).max()), rtol=0)
        else:  # FP32-bulk: the variant's stated bound against the FP64 oracle
            assert loo_np(p.V.numpy(), Qh) < 1e-5
            assert np.abs(Qh - Qo).max() < 1e-3
        assert torch.equal(Q, Qp) and torch.equal(R, Rp)
        if k0:
            assert torch.equal(S, Sp)


def test_noalloc_larger_then_smaller(lib):
    """A large call leaves the scratch full of its partial sums and tree factors;
    a smaller call with another k that follows must not see any of it."""
    tho, f = lib
    big = inputs.random_problem(30000, 64, 24, dtype=torch.float64, seed=7)
    small = inputs.random_problem(5000, 8, 5, dtype=torch.float64, seed=8)
    _noalloc(tho, f, big.V.cuda(), big.A.cuda(), 64, tho.THO_PREC_FP64)
    Vs, As = small.V.cuda(), small.A.cuda()
    Q, R, S = _noalloc(tho, f, Vs, As, 8, tho.THO_PREC_FP64)
    Qo, Ro, So = oracle.two_stage(small.V.numpy(), small.A.numpy())
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL, rtol=0)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL * max(1.0, np.abs(Ro).max()), rtol=0)
    np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL * max(1.0, np.abs(So).max()), rtol=0)
    Qp, Rp, Sp = _plan_orth(tho, Vs, As, 8, tho.THO_PREC_FP64)
    assert torch.equal(Q, Qp) and torch.equal(R, Rp) and torch.equal(S, Sp)


def test_noalloc_rejects_problems_beyond_the_scratch(lib):
    tho, f = lib
    desc = tho.Desc(1 << 22, 128, 32, tho.THO_C128, tho.THO_PREC_FP64, 0)
    # The size check runs before any pointer is used; aligned placeholders suffice.
    rc = f(ctypes.byref(desc), 256, 1 << 22, 256, 1 << 22, 256, 1 << 22, None, None, None)
    assert rc == tho.THO_ERR_UNSUPPORTED
    bad = tho.Desc(100, 60, 50, tho.THO_F64, tho.THO_PREC_FP64, 0)
    assert f(ctypes.byref(bad), 256, 100, 256, 100, 256, 100, None, None, None) == tho.THO_ERR_SHAPE
    emu = tho.Desc(1000, 8, 4, tho.THO_F64, tho.THO_PREC_FP64_EMU, 0)
    assert f(ctypes.byref(emu), 256, 1000, 256, 1000, 256, 1000, None, None, None) == tho.THO_ERR_ARG
    chk = tho.Desc(1000, 8, 4, tho.THO_F64, tho.THO_PREC_FP64, tho.THO_FLAG_CHECK_ORTH)
    assert f(ctypes.byref(chk), 256, 1000, 256, 1000, 256, 1000, None, None, None) == tho.THO_ERR_ARG
