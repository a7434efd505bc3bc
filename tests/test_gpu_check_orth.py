"""THO_FLAG_CHECK_ORTH: the device estimate of delta_1 = ||V^* V - I||_2, the
precondition of Theorem 4 (Section 4).

Pinned to closed forms: for V with orthonormal columns and w a unit vector,
V (I + s w w^*) has V'^* V' - I = (2 s + s^2) w w^*, so delta_1 = 2 s + s^2
exactly (up to V's own rounding-level defect), and two power-iteration steps
recover it to rounding; for V M with a general M, delta_1 = ||M^* M - I||_2
(numpy's SVD of a k0 x k0 matrix), which the estimate never exceeds and, from
a random start, reaches within a small factor.  Orthonormal V stays below
THO_ORTH_TOL and leaves Q, R, S bitwise as without the flag; defects above it
latch THO_ERR_NOT_ORTH with Q, R, S still computed.
"""
import numpy as np
import pytest
import torch

from paper_2602_14449_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tho():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_14449_gb300 import tho as _tho
    _tho.load()
    return _tho


def _run(tho, V, A, prec, flags=0):
    n, k = A.shape
    k0 = V.shape[1] if V is not None else 0
    if k0 == 0:
        flags |= tho.THO_FLAG_ALLOW_K0_ZERO
    plan = tho.Plan([(n, k0, k)], A.dtype, prec, flags | tho.THO_FLAG_CHECK_ORTH)
    Q, R, S = tho.orth(V, A, prec=prec, plan=plan, flags=flags | tho.THO_FLAG_CHECK_ORTH)
    torch.cuda.synchronize()
    return plan, Q, R, S


def _unit(k0, dtype, seed):
    g = torch.Generator().manual_seed(seed)
    w = inputs.gaussian(k0, 1, dtype, g)
    return w / torch.linalg.vector_norm(w)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("prec_name", ["THO_PREC_FP64", "THO_PREC_FP64_EMU"])
@pytest.mark.parametrize("n,k0,k", [(20000, 64, 16), (4099, 7, 3), (3000, 128, 32)])
def test_orthonormal_v_passes_and_results_unchanged(tho, dtype, prec_name, n, k0, k):
    prec = getattr(tho, prec_name)
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=9100 + n + k0)
    V, A = p.V.cuda(), p.A.cuda()
    plan, Q, R, S = _run(tho, V, A, prec)
    d = plan.orth_defect()
    assert plan.status() == tho.THO_OK
    assert 0.0 <= d < 1e-13, d
    Q0, R0, S0 = tho.orth(V, A, prec=prec)
    torch.cuda.synchronize()
    assert torch.equal(Q, Q0) and torch.equal(R, R0) and torch.equal(S, S0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("s", [1e-8, 3e-5, 0.25])
def test_rank_one_defect_is_recovered(tho, dtype, s):
    n, k0, k = 30000, 48, 8
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=9200)
    w = _unit(k0, dtype, 9201)
    M = torch.eye(k0, dtype=dtype) + s * (w @ w.conj().T)
    V = inputs.colmajor(p.V @ M).cuda()
    plan, Q, R, S = _run(tho, V, p.A.cuda(), tho.THO_PREC_FP64)
    d = plan.orth_defect()
    exact = 2 * s + s * s
    assert plan.status() == tho.THO_ERR_NOT_ORTH
    assert abs(d - exact) <= 1e-6 * exact + 1e-14, (d, exact)
    assert torch.isfinite(torch.view_as_real(Q) if Q.is_complex() else Q).all()


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("eps", [1e-9, 1e-4])
def test_general_defect_is_bounded_by_delta1(tho, dtype, eps):
    n, k0, k = 25000, 96, 16
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=9300)
    g = torch.Generator().manual_seed(9301)
    M = torch.eye(k0, dtype=dtype) + eps * inputs.gaussian(k0, k0, dtype, g)
    V = inputs.colmajor(p.V @ M).cuda()
    plan, Q, R, S = _run(tho, V, p.A.cuda(), tho.THO_PREC_FP64)
    d = plan.orth_defect()
    Mn = M.numpy()
    delta1 = np.linalg.norm(Mn.conj().T @ Mn - np.eye(k0), 2)
    assert d <= delta1 * (1 + 1e-6) + 1e-14, (d, delta1)
    assert d >= 0.1 * delta1, (d, delta1)
    assert plan.status() == tho.THO_ERR_NOT_ORTH


def test_defect_below_tolerance_is_not_latched(tho):
    n, k0, k = 20000, 32, 8
    p = inputs.random_problem(n, k0, k, dtype=torch.float64, seed=9400)
    s = 5e-14
    w = _unit(k0, torch.float64, 9401)
    V = inputs.colmajor(p.V @ (torch.eye(k0, dtype=torch.float64) + s * (w @ w.T))).cuda()
    plan, Q, R, S = _run(tho, V, p.A.cuda(), tho.THO_PREC_FP64)
    d = plan.orth_defect()
    assert d < tho.THO_ORTH_TOL
    assert abs(d - 2 * s) < 5e-14, d
    assert plan.status() == tho.THO_OK


def test_nonfinite_v_gives_infinite_estimate(tho):
    n, k0, k = 5000, 16, 4
    p = inputs.random_problem(n, k0, k, dtype=torch.float64, seed=9500)
    V = p.V.clone()
    V[1234, 5] = float("nan")
    plan, Q, R, S = _run(tho, V.cuda(), p.A.cuda(), tho.THO_PREC_FP64)
    assert plan.orth_defect() == float("inf")
    assert plan.status() == tho.THO_ERR_NOT_ORTH


def test_k0_zero_has_nothing_to_check(tho):
    A = inputs.random_problem(3000, 0, 8, seed=9600).A.cuda()
    plan, Q, R, S = _run(tho, None, A, tho.THO_PREC_FP64)
    assert plan.orth_defect() == 0.0
    assert plan.status() == tho.THO_OK


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_b_inner_product_checks_the_scaled_basis(tho, dtype):
    """tho_orth_b checks D^{1/2} V, orthonormal when V^* B V = I."""
    n, k0, k = 6000, 24, 8
    pb = inputs.diag_b_problem(n, k0, k, kappa_b=1e5, dtype=dtype, seed=9700)
    flags = tho.THO_FLAG_CHECK_ORTH
    plan = tho.Plan([(n, k0, k)], dtype, tho.THO_PREC_FP64, flags)
    tho.orth_b(pb.d.cuda(), pb.V.cuda(), pb.A.cuda(), prec=tho.THO_PREC_FP64, flags=flags, plan=plan)
    torch.cuda.synchronize()
    assert plan.orth_defect() < 1e-13
    assert plan.status() == tho.THO_OK
    # The unscaled V is not orthonormal in the Euclidean product: the plain call flags it.
    plan2, *_ = _run(tho, pb.V.cuda(), pb.A.cuda(), tho.THO_PREC_FP64)
    assert plan2.orth_defect() > tho.THO_ORTH_TOL
    assert plan2.status() == tho.THO_ERR_NOT_ORTH


def test_check_orth_refusals(tho):
    with pytest.raises(RuntimeError, match="tho_plan"):
        tho.Plan([(5000, 8, 4), (6000, 8, 4)], torch.float64, tho.THO_PREC_FP64, tho.THO_FLAG_CHECK_ORTH)
    plan = tho.Plan([(5000, 8, 4)], torch.float64, tho.THO_PREC_FP64, 0)
    with pytest.raises(RuntimeError, match="tho_plan_orth_defect"):
        plan.orth_defect()
