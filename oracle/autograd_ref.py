"""ORACLE — test infrastructure only.

Algorithm 1 (second choice of P, Section 3.2) restated in plain PyTorch CPU
float64 ops so that torch.autograd can differentiate the algorithm's own map
(V, A) -> Q at arbitrary V and A.  It follows the same steps and conventions
as tho_oracle.cpp (reflector v = x + sign(x_1)||x|| e_1, diag(R) >= 0, T-solves
by substitution) with explicit loops; it is the reference gradient for the
hand-written adjoint (real), and for complex inputs the reference of the
complex map's derivative (torch's convention: the gradient of a real loss L is
dL/dRe z + i dL/dIm z).

Pinned in tests/test_oracle_adjoint.py, real and complex: its Q equals the C
oracle's Q, and its gradients equal central finite differences of the C oracle
(an independent implementation) in random directions; in directions tangent to
the orthonormal V its derivative equals that of the closed form
qf((I - V V^*) A) (LAPACK).
"""
import torch


def _phase(z: torch.Tensor) -> torch.Tensor:
    """z / |z| for a complex scalar, 1 at z = 0 (differentiable away from 0)."""
    a = torch.sqrt(z.real * z.real + z.imag * z.imag)
    return z / a if float(a.detach()) > 0 else torch.ones((), dtype=z.dtype)


def householder_qr(X: torch.Tensor):
    """Unblocked Householder QR with diag(R) real >= 0 (differentiable): X = Q R.
    Reflector v = x + phase(x_1) ||x|| e_1, H = I - 2 v v^* / (v^* v).  For real
    X the sign is locally constant and taken as a constant; for complex X the
    phase stays in the graph (a fixed phase would not map the perturbed column
    onto e_1, and the derivative would be wrong)."""
    m, k = X.shape
    cplx = X.is_complex()
    R = X
    vs, betas = [], []
    for j in range(k):
        x = R[j:, j]
        alpha = torch.sqrt((x.conj() * x).real.sum()) if cplx else torch.sqrt((x * x).sum())
        s = _phase(x[0]) if cplx else (1.0 if float(x[0].detach()) >= 0 else -1.0)
        v = torch.cat([x[:1] + s * alpha, x[1:]])
        beta = 2.0 / ((v.conj() * v).real.sum() if cplx else (v * v).sum())
        R = torch.cat([R[:j], R[j:] - beta * torch.outer(v, v.conj() @ R[j:])], 0)
        vs.append(v)
        betas.append(beta)
    Q = torch.eye(m, k, dtype=X.dtype)
    for j in reversed(range(k)):
        Q = torch.cat([Q[:j], Q[j:] - betas[j] * torch.outer(vs[j], vs[j].conj() @ Q[j:])], 0)
    if cplx:
        d = torch.stack([_phase(R[i, i]) for i in range(k)])
        return Q * d, d.conj()[:, None] * torch.triu(R[:k])
    d = torch.where(torch.diagonal(R[:k]) < 0, -1.0, 1.0).to(X.dtype)
    return Q * d, d[:, None] * torch.triu(R[:k])


def _solve_upper(U, B):
    """U X = B by back substitution (U upper triangular)."""
    n = U.shape[0]
    rows = [None] * n
    for i in range(n - 1, -1, -1):
        s = B[i]
        for j in range(i + 1, n):
            s = s - U[i, j] * rows[j]
        rows[i] = s / U[i, i]
    return torch.stack(rows, 0)


def _solve_lower(L, B):
    """L X = B by forward substitution (L lower triangular)."""
    n = L.shape[0]
    rows = [None] * n
    for i in range(n):
        s = B[i]
        for j in range(i):
            s = s - L[i, j] * rows[j]
        rows[i] = s / L[i, i]
    return torch.stack(rows, 0)


def two_stage(V: torch.Tensor, A: torch.Tensor) -> torch.Tensor:
    """Algorithm 1 (choice 2 of P), returns Q; differentiable in V and A (real
    or complex; ^* is the conjugate transpose)."""
    n, k0 = V.shape
    h = lambda M: M.conj().T if M.is_complex() else M.T
    Q1, R1 = householder_qr(V[:k0])          # choice 2: V_{1:k0,:} = Q1 R1
    P = -Q1
    T = torch.eye(k0, dtype=V.dtype) + h(R1)  # T = I - V_{1:k0,:}^* P = I + R1^*
    W = torch.cat([P, torch.zeros(n - k0, k0, dtype=V.dtype)], 0) - V
    Z = _solve_upper(h(T), h(W) @ A)          # Z = T^{-*} W^* A
    Ap = A - W @ Z                            # A <- (I - W T^{-*} W^*) A
    Qb, _ = householder_qr(Ap[k0:])           # A_{k0+1:n,:} = Qbar R
    E = torch.cat([torch.zeros(k0, A.shape[1], dtype=A.dtype), Qb], 0)
    Z2 = _solve_lower(T, h(W) @ E)            # Z2 = T^{-1} W^* [0; Qbar]
    return E - W @ Z2                         # Q = (I - W T^{-1} W^*) [0; Qbar]
