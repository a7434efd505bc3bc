"""Pins of the differentiable oracle restatement (oracle/autograd_ref.py)."""
import numpy as np
import torch

import oracle
from metrics import qf
from oracle import autograd_ref
from paper_2602_14449_gb300 import inputs


def _dirs(n, k0, k, seed):
    g = torch.Generator().manual_seed(seed)
    dV = torch.randn(n, k0, generator=g, dtype=torch.float64)
    dA = torch.randn(n, k, generator=g, dtype=torch.float64)
    s = torch.sqrt((dV ** 2).sum() + (dA ** 2).sum())
    return dV / s, dA / s


def test_forward_matches_c_oracle():
    p = inputs.config_problem(5, n=300)
    Q = autograd_ref.two_stage(p.V, p.A).numpy()
    Qo, _, _ = oracle.two_stage(p.V.numpy(), p.A.numpy())
    np.testing.assert_allclose(Q, Qo, atol=1e-13)


def test_gradient_matches_finite_differences_of_c_oracle():
    """<dQ, Q'(V,A)[dV, dA]> by central differences (h = 1e-6) of the C oracle."""
    p = inputs.config_problem(5, n=200)
    n, k0, k = p.n, p.k0, p.k
    V = p.V.clone().requires_grad_()
    A = p.A.clone().requires_grad_()
    dQ = p.dQ
    Q = autograd_ref.two_stage(V, A)
    (Q * dQ).sum().backward()
    h = 1e-6
    for s in range(4):
        eV, eA = _dirs(n, k0, k, s)
        Qp, _, _ = oracle.two_stage((p.V + h * eV).numpy(), (p.A + h * eA).numpy())
        Qm, _, _ = oracle.two_stage((p.V - h * eV).numpy(), (p.A - h * eA).numpy())
        fd = float((dQ.numpy() * (Qp - Qm)).sum() / (2 * h))
        ad = float((V.grad * eV).sum() + (A.grad * eA).sum())
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(fd)), (s, fd, ad)


def test_tangent_directions_match_closed_form():
    """On the Stiefel manifold (V^T dV + dV^T V = 0) the map is qf((I - V V^T) A)."""
    p = inputs.config_problem(5, n=150)
    V0, A0 = p.V.numpy(), p.A.numpy()
    g = np.random.default_rng(3)
    Om = g.standard_normal((p.k0, p.k0))
    Om = Om - Om.T                                  # skew: V Om is tangent
    Xp = g.standard_normal((p.n, p.k0))
    Xp = Xp - V0 @ (V0.T @ Xp)                      # orthogonal complement part
    dV = V0 @ Om + Xp
    dV /= np.linalg.norm(dV)
    h = 1e-6

    def closed(V, A):
        Vq, _ = np.linalg.qr(V)                      # V + h dV re-orthonormalized to first order
        return qf(A - Vq @ (Vq.T @ A))[0]

    Vt = torch.tensor(V0, requires_grad=True)
    At = torch.tensor(A0)
    Q = autograd_ref.two_stage(Vt, At)
    W = torch.tensor(g.standard_normal(Q.shape))
    (Q * W).sum().backward()
    ad = float((Vt.grad.numpy() * dV).sum())
    fd = float((W.numpy() * (closed(V0 + h * dV, A0) - closed(V0 - h * dV, A0))).sum() / (2 * h))
    assert abs(fd - ad) <= 1e-6 * max(1.0, abs(fd)), (fd, ad)


# --- complex128: the same pins for the complex map (torch's gradient convention:
# for a real loss L, z.grad = dL/dRe z + i dL/dIm z, so the directional
# derivative along dz is Re sum(conj(z.grad) dz)) ---

def _cdirs(n, k0, k, seed):
    g = torch.Generator().manual_seed(seed)
    c = lambda r, s: torch.complex(torch.randn(r, s, generator=g, dtype=torch.float64),
                                   torch.randn(r, s, generator=g, dtype=torch.float64))
    dV, dA = c(n, k0), c(n, k)
    s = torch.sqrt((dV.abs() ** 2).sum() + (dA.abs() ** 2).sum())
    return dV / s, dA / s


def test_complex_forward_matches_c_oracle():
    p = inputs.random_problem(250, 12, 6, dtype=torch.complex128, seed=8)
    Q = autograd_ref.two_stage(p.V, p.A).numpy()
    Qo, _, _ = oracle.two_stage(p.V.numpy(), p.A.numpy())
    np.testing.assert_allclose(Q, Qo, atol=1e-13)


def test_complex_gradient_matches_finite_differences_of_c_oracle():
    """Re <dQ, Q'(V,A)[dV, dA]> by central differences (h = 1e-6) of the C oracle."""
    p = inputs.random_problem(200, 10, 6, dtype=torch.complex128, seed=9)
    n, k0, k = p.n, p.k0, p.k
    g = torch.Generator().manual_seed(10)
    dQ = torch.complex(torch.randn(n, k, generator=g, dtype=torch.float64),
                       torch.randn(n, k, generator=g, dtype=torch.float64))
    V = p.V.clone().requires_grad_()
    A = p.A.clone().requires_grad_()
    Q = autograd_ref.two_stage(V, A)
    (dQ.conj() * Q).real.sum().backward()
    h = 1e-6
    for s in range(4):
        eV, eA = _cdirs(n, k0, k, s)
        Qp, _, _ = oracle.two_stage((p.V + h * eV).numpy(), (p.A + h * eA).numpy())
        Qm, _, _ = oracle.two_stage((p.V - h * eV).numpy(), (p.A - h * eA).numpy())
        fd = float((np.conj(dQ.numpy()) * (Qp - Qm)).real.sum() / (2 * h))
        ad = float((V.grad.conj() * eV).real.sum() + (A.grad.conj() * eA).real.sum())
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(fd)), (s, fd, ad)


def test_complex_tangent_directions_match_closed_form():
    """On the complex Stiefel manifold (V^* dV + dV^* V = 0) the map is
    qf((I - V V^*) A) with diag(R) real >= 0."""
    p = inputs.random_problem(150, 8, 5, dtype=torch.complex128, seed=11)
    V0, A0 = p.V.numpy(), p.A.numpy()
    g = np.random.default_rng(4)
    cx = lambda r, s: g.standard_normal((r, s)) + 1j * g.standard_normal((r, s))
    Om = cx(p.k0, p.k0)
    Om = Om - Om.conj().T                            # skew-Hermitian: V Om is tangent
    Xp = cx(p.n, p.k0)
    Xp = Xp - V0 @ (V0.conj().T @ Xp)
    dV = V0 @ Om + Xp
    dV /= np.linalg.norm(dV)
    h = 1e-6

    def closed(V, A):
        Vq, _ = np.linalg.qr(V)
        return qf(A - Vq @ (Vq.conj().T @ A))[0]

    Vt = torch.tensor(V0, requires_grad=True)
    At = torch.tensor(A0)
    Q = autograd_ref.two_stage(Vt, At)
    Wt = torch.tensor(cx(*Q.shape))
    (Wt.conj() * Q).real.sum().backward()
    ad = float((np.conj(Vt.grad.numpy()) * dV).real.sum())
    fd = float((np.conj(Wt.numpy()) * (closed(V0 + h * dV, A0) - closed(V0 - h * dV, A0))).real.sum() / (2 * h))
    assert abs(fd - ad) <= 1e-6 * max(1.0, abs(fd)), (fd, ad)
