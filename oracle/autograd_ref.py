"""ORACLE — test infrastructure only.

Algorithm 1 (second choice of P, Section 3.2) restated in plain PyTorch CPU
float64 ops so that torch.autograd can differentiate the algorithm's own map
(V, A) -> Q at arbitrary V and A.  It follows the same steps and conventions
as tho_oracle.cpp (reflector v = x + sign(x_1)||x|| e_1, diag(R) >= 0, T-solves
by substitution) with explicit loops; it is the reference gradient for the
hand-written adjoint.  Real only.

Pinned in tests/test_oracle_adjoint.py: its Q equals the C oracle's Q, and its
gradients equal central finite differences of the C oracle (an independent
implementation) in random directions; in directions tangent to the orthonormal
V its derivative equals that of the closed form qf((I - V V^T) A) (LAPACK).
"""
import torch


def householder_qr(X: torch.Tensor):
    """Unblocked Householder QR with diag(R) >= 0 (differentiable): X = Q R."""
    m, k = X.shape
    R = X
    vs, betas = [], []
    for j in range(k):
        x = R[j:, j]
        alpha = torch.sqrt((x * x).sum())
        s = 1.0 if float(x[0].detach()) >= 0 else -1.0
        v = torch.cat([x[:1] + s * alpha, x[1:]])
        beta = 2.0 / (v * v).sum()
        R = torch.cat([R[:j], R[j:] - beta * torch.outer(v, v @ R[j:])], 0)
        vs.append(v)
        betas.append(beta)
    Q = torch.eye(m, k, dtype=X.dtype)
    for j in reversed(range(k)):
        Q = torch.cat([Q[:j], Q[j:] - betas[j] * torch.outer(vs[j], vs[j] @ Q[j:])], 0)
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
    """Algorithm 1 (choice 2 of P), returns Q; differentiable in V and A."""
    n, k0 = V.shape
    Q1, R1 = householder_qr(V[:k0])          # choice 2: V_{1:k0,:} = Q1 R1
    P = -Q1
    T = torch.eye(k0, dtype=V.dtype) + R1.T   # T = I - V_{1:k0,:}^T P = I + R1^T
    W = torch.cat([P, torch.zeros(n - k0, k0, dtype=V.dtype)], 0) - V
    Z = _solve_upper(T.T, W.T @ A)            # Z = T^{-T} W^T A
    Ap = A - W @ Z                            # A <- (I - W T^{-T} W^T) A
    Qb, _ = householder_qr(Ap[k0:])           # A_{k0+1:n,:} = Qbar R
    E = torch.cat([torch.zeros(k0, A.shape[1], dtype=A.dtype), Qb], 0)
    Z2 = _solve_lower(T, W.T @ E)             # Z2 = T^{-1} W^T [0; Qbar]
    return E - W @ Z2                         # Q = (I - W T^{-1} W^T) [0; Qbar]
