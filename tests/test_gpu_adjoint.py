"""The hand-written adjoint (tho_orth_backward) on the GPU, real and complex.

Against: autograd through the oracle's torch-CPU restatement of Algorithm 1
(relative error <= 1e-10), and central finite differences (h = 1e-6) of the GPU
forward at the full differentiation workload (n = 2^20, k0 = 64, k = 16) on 32
random normalized directions (relative error <= 1e-6); complex128 the same
way, with torch's gradient convention for complex values and a real loss
Re sum(conj(dQ) Q).
"""
import numpy as np
import pytest
import torch

from oracle import autograd_ref
from paper_2602_14449_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tho():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_14449_gb300 import tho as _tho
    _tho.load()
    return _tho


def _ref_grads(V, A, dQ):
    Vr = V.clone().requires_grad_()
    Ar = A.clone().requires_grad_()
    Q = autograd_ref.two_stage(Vr, Ar)
    (Q * dQ).sum().backward()
    return Vr.grad, Ar.grad


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("n,k0,k", [(4096, 64, 16), (1000, 7, 3), (3000, 32, 32), (2000, 128, 8), (600, 1, 1)])
def test_adjoint_vs_oracle_autograd(tho, n, k0, k):
    p = inputs.config_problem(5, n=n) if (k0, k) == (64, 16) else inputs.random_problem(n, k0, k, seed=n + k0)
    dQ = p.dQ if p.dQ is not None else inputs.colmajor(torch.randn(n, k, dtype=torch.float64,
                                                                    generator=torch.Generator().manual_seed(7)))
    gV, gA = _ref_grads(p.V, p.A, dQ)
    V, A, dQd = p.V.cuda(), p.A.cuda(), inputs.colmajor(dQ).cuda()
    Q, _, _ = tho.orth(V, A)
    dV, dA = tho.orth_backward(V, A, Q, dQd)
    torch.cuda.synchronize()
    assert _rel(dA.cpu(), gA) <= 1e-10
    assert _rel(dV.cpu(), gV) <= 1e-10


@pytest.mark.parametrize("n,k0,k,eps", [(2000, 16, 8, 0.1), (3000, 64, 16, 0.02), (700, 5, 3, 0.3)])
def test_adjoint_at_non_orthonormal_v(tho, n, k0, k, eps):
    """The derivative of the algorithm's map at a V whose columns are not
    orthonormal (V = orthonormal + eps * Gaussian): the adjoint recovers Z2 and
    Qbar from the top rows of Q, which holds at any V, and must match autograd
    through the oracle's restatement."""
    p = inputs.random_problem(n, k0, k, seed=500 + n)
    g = torch.Generator().manual_seed(501 + n)
    V = inputs.colmajor(p.V + eps * torch.randn(n, k0, dtype=torch.float64, generator=g))
    assert float(torch.linalg.matrix_norm(V.T @ V - torch.eye(k0, dtype=torch.float64), 2)) > eps
    dQ = inputs.colmajor(torch.randn(n, k, dtype=torch.float64, generator=g))
    gV, gA = _ref_grads(V, p.A, dQ)
    Vd, Ad = V.cuda(), p.A.cuda()
    Q, _, _ = tho.orth(Vd, Ad)
    dV, dA = tho.orth_backward(Vd, Ad, Q, dQ.cuda())
    torch.cuda.synchronize()
    assert _rel(dA.cpu(), gA) <= 1e-10
    assert _rel(dV.cpu(), gV) <= 1e-10


def test_autograd_function(tho):
    from paper_2602_14449_gb300.autograd import two_stage_orth
    p = inputs.config_problem(5, n=5000)
    V = p.V.cuda().requires_grad_()
    A = p.A.cuda().requires_grad_()
    Q = two_stage_orth(V, A)
    W = p.dQ.cuda()
    (Q * W).sum().backward()
    gV, gA = _ref_grads(p.V, p.A, p.dQ)
    assert _rel(A.grad.cpu(), gA) <= 1e-10
    assert _rel(V.grad.cpu(), gV) <= 1e-10


def test_adjoint_full_size_finite_differences(tho):
    """C5: n = 2^20, k0 = 64, k = 16; 32 directions, central differences h = 1e-6."""
    p = inputs.config_problem(5, device="cuda")
    V, A, dQ = p.V, p.A, p.dQ
    Q, _, _ = tho.orth(V, A)
    dV, dA = tho.orth_backward(V, A, Q, dQ)
    g = torch.Generator(device="cuda").manual_seed(99)
    h = 1e-6
    worst = 0.0
    for _ in range(32):
        eV = torch.randn(V.shape[1], V.shape[0], dtype=torch.float64, device="cuda", generator=g).t()
        eA = torch.randn(A.shape[1], A.shape[0], dtype=torch.float64, device="cuda", generator=g).t()
        s = torch.sqrt((eV ** 2).sum() + (eA ** 2).sum())
        eV, eA = eV / s, eA / s
        Qp, _, _ = tho.orth(inputs.colmajor(V + h * eV), inputs.colmajor(A + h * eA), want_R=False, want_S=False)
        Qm, _, _ = tho.orth(inputs.colmajor(V - h * eV), inputs.colmajor(A - h * eA), want_R=False, want_S=False)
        fd = float((dQ * (Qp - Qm)).sum()) / (2 * h)
        ad = float((dV * eV).sum() + (dA * eA).sum())
        worst = max(worst, abs(fd - ad) / max(1.0, abs(fd)))
    assert worst <= 1e-6, worst


def _ref_grads_c(V, A, dQ):
    """Complex: gradients of the real loss Re sum(conj(dQ) Q) in torch's convention."""
    Vr = V.clone().requires_grad_()
    Ar = A.clone().requires_grad_()
    Q = autograd_ref.two_stage(Vr, Ar)
    (dQ.conj() * Q).real.sum().backward()
    return Vr.grad, Ar.grad


def _cgauss(n, k, g):
    return inputs.colmajor(torch.complex(torch.randn(n, k, dtype=torch.float64, generator=g),
                                         torch.randn(n, k, dtype=torch.float64, generator=g)))


@pytest.mark.parametrize("n,k0,k", [(1500, 16, 8), (700, 7, 3), (2000, 64, 32), (900, 128, 4), (300, 1, 2)])
def test_complex_adjoint_vs_oracle_autograd(tho, n, k0, k):
    """complex128 adjoint against autograd through the oracle's complex restatement."""
    p = inputs.random_problem(n, k0, k, dtype=torch.complex128, seed=600 + n + k0)
    dQ = _cgauss(n, k, torch.Generator().manual_seed(601 + n))
    gV, gA = _ref_grads_c(p.V, p.A, dQ)
    V, A = p.V.cuda(), p.A.cuda()
    Q, _, _ = tho.orth(V, A)
    dV, dA = tho.orth_backward(V, A, Q, dQ.cuda())
    torch.cuda.synchronize()
    assert _rel(dA.cpu(), gA) <= 1e-10
    assert _rel(dV.cpu(), gV) <= 1e-10


def test_complex_adjoint_at_non_orthonormal_v(tho):
    n, k0, k = 1200, 12, 6
    p = inputs.random_problem(n, k0, k, dtype=torch.complex128, seed=610)
    g = torch.Generator().manual_seed(611)
    V = inputs.colmajor(p.V + 0.1 * _cgauss(n, k0, g))
    dQ = _cgauss(n, k, g)
    gV, gA = _ref_grads_c(V, p.A, dQ)
    Vd, Ad = V.cuda(), p.A.cuda()
    Q, _, _ = tho.orth(Vd, Ad)
    dV, dA = tho.orth_backward(Vd, Ad, Q, dQ.cuda())
    torch.cuda.synchronize()
    assert _rel(dA.cpu(), gA) <= 1e-10
    assert _rel(dV.cpu(), gV) <= 1e-10


def test_complex_adjoint_finite_differences(tho):
    """complex128 at the headline shapes with fewer rows (n = 2^17, k0 = 128,
    k = 32): 16 random complex directions, central differences h = 1e-6 of the
    GPU forward; the directional derivative of L = Re sum(conj(dQ) Q) along
    (eV, eA) is Re sum(conj(dV) eV) + Re sum(conj(dA) eA)."""
    n, k0, k = 1 << 17, 128, 32
    p = inputs.random_problem(n, k0, k, dtype=torch.complex128, seed=620, device="cuda")
    V, A = p.V, p.A
    g = torch.Generator(device="cuda").manual_seed(621)
    cg = lambda r, c: torch.complex(torch.randn(c, r, dtype=torch.float64, device="cuda", generator=g),
                                    torch.randn(c, r, dtype=torch.float64, device="cuda", generator=g)).t()
    dQ = inputs.colmajor(cg(n, k))
    Q, _, _ = tho.orth(V, A)
    dV, dA = tho.orth_backward(V, A, Q, dQ)
    h = 1e-6
    worst = 0.0
    for _ in range(16):
        eV, eA = cg(n, k0), cg(n, k)
        s = torch.sqrt((eV.abs() ** 2).sum() + (eA.abs() ** 2).sum())
        eV, eA = eV / s, eA / s
        Qp, _, _ = tho.orth(inputs.colmajor(V + h * eV), inputs.colmajor(A + h * eA), want_R=False, want_S=False)
        Qm, _, _ = tho.orth(inputs.colmajor(V - h * eV), inputs.colmajor(A - h * eA), want_R=False, want_S=False)
        fd = float((dQ.conj() * (Qp - Qm)).real.sum()) / (2 * h)
        ad = float((dV.conj() * eV).real.sum() + (dA.conj() * eA).real.sum())
        worst = max(worst, abs(fd - ad) / max(1.0, abs(fd)))
    assert worst <= 1e-6, worst


def test_complex_autograd_function(tho):
    from paper_2602_14449_gb300.autograd import two_stage_orth
    p = inputs.random_problem(3000, 32, 16, dtype=torch.complex128, seed=630)
    dQ = _cgauss(3000, 16, torch.Generator().manual_seed(631))
    V = p.V.cuda().requires_grad_()
    A = p.A.cuda().requires_grad_()
    Q = two_stage_orth(V, A)
    (dQ.cuda().conj() * Q).real.sum().backward()
    gV, gA = _ref_grads_c(p.V, p.A, dQ)
    assert _rel(A.grad.cpu(), gA) <= 1e-10
    assert _rel(V.grad.cpu(), gV) <= 1e-10


def test_backward_rejects_unsupported(tho):
    """The adjoint covers THO_PREC_FP64 plans with the second choice of P and k0 >= 1."""
    p = inputs.random_problem(500, 8, 4, dtype=torch.complex128, seed=1)
    V, A = p.V.cuda(), p.A.cuda()
    Q, _, _ = tho.orth(V, A)
    plan = tho.Plan([(500, 8, 4)], torch.complex128, tho.THO_PREC_FP64_EMU)
    with pytest.raises(tho.ThoError) as ei:
        tho.orth_backward(V, A, Q, Q.clone(), plan=plan)
    assert ei.value.code == tho.THO_ERR_UNSUPPORTED
    plan = tho.Plan([(500, 8, 4)], torch.complex128, tho.THO_PREC_FP64, tho.THO_FLAG_P_POLAR)
    with pytest.raises(tho.ThoError) as ei:
        tho.orth_backward(V, A, Q, Q.clone(), plan=plan)
    assert ei.value.code == tho.THO_ERR_UNSUPPORTED
