"""Accuracy measures on CUDA tensors (test helpers, plain torch).

Long inner products over n rows are taken in row chunks (cuBLAS within a chunk)
and the chunk results are added pairwise, keeping the metrics' own rounding
far below the 1e-13 bounds being checked.
"""
import torch

CHUNK = 1 << 16


def _pairwise(parts):
    while len(parts) > 1:
        nxt = [parts[i] + parts[i + 1] for i in range(0, len(parts) - 1, 2)]
        if len(parts) % 2:
            nxt.append(parts[-1])
        parts = nxt
    return parts[0]


def gram(X, Y):
    """X^* Y over the rows, chunked + pairwise."""
    n = X.shape[0]
    parts = [X[r:r + CHUNK].conj().T @ Y[r:r + CHUNK] for r in range(0, n, CHUNK)]
    return _pairwise(parts)


def spec_norm(M):
    return float(torch.linalg.matrix_norm(M.cpu(), ord=2))


def loo(V, Q):
    """||[V,Q]^*[V,Q] - I||_2."""
    VQ = torch.cat([V, Q], dim=1) if V.shape[1] else Q
    G = gram(VQ, VQ)
    return spec_norm(G - torch.eye(G.shape[0], dtype=G.dtype, device=G.device))


def resid_fro(V, A, Q, R, S):
    """||[V,A] - [V,Q][[I,S],[0,R]]||_F / ||[V,A]||_F (the V block is exact)."""
    n = A.shape[0]
    num = torch.zeros((), dtype=torch.float64, device=A.device)
    den = torch.zeros((), dtype=torch.float64, device=A.device)
    for r in range(0, n, CHUNK):
        Ar, Vr, Qr = A[r:r + CHUNK], V[r:r + CHUNK], Q[r:r + CHUNK]
        E = Ar - Qr @ R
        if V.shape[1]:
            E = E - Vr @ S
        num += (E.abs() ** 2).sum()
        den += (Ar.abs() ** 2).sum() + ((Vr.abs() ** 2).sum() if V.shape[1] else 0)
    return float(torch.sqrt(num / den))


def assert_r_triangular(R):
    """R is upper triangular (exact zeros below the diagonal) with a real
    nonnegative diagonal: the normalization that makes Q unique (the trailing
    QR's sign convention), so a Q rotated inside its range cannot pass."""
    assert R.shape[0] == R.shape[1]
    below = torch.tril(R, -1)
    assert float(below.abs().max()) == 0.0
    d = torch.diagonal(R)
    if d.is_complex():
        assert float(d.imag.abs().max()) == 0.0
        d = d.real
    assert float(d.min()) >= 0.0
