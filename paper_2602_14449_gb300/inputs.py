"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the orthogonalization method: it only draws
random matrices.  Orthonormal V comes from a library QR (``torch.linalg.qr``, CPU)
or CholeskyQR2 (GPU) of a Gaussian matrix: input generation, not the method.

Workloads (the shapes of block Krylov orthogonalization, the paper's usage
mode in Section 1 and Algorithm 3):
  * ``worked``  — the 4 x 2 example of eq. (badbcg), Section 1.
  * ``C1``  real,    n=4096,   k0=16,  k=4,  A ~ N(0,1).
  * ``C2``  real,    n=2^20,   k0=64,  k=16, A = V C + 1e-10 G   (cond([V,A]) ~ 1e10).
  * ``C3``  complex, n=2^22,   k0=128, k=32, A = [V C1 + 1e-14 G1, G2]
            (16 columns numerically in Range(V), 16 independent).
  * ``C4``  256 real instances, n log-uniform in [16384, 262144],
            k0 in {8,16,32,64,128}, k in {4,8,16,32}, A ~ N(0,1).
  * ``C5``  real, n=2^20, k0=64, k=16, A ~ N(0,1), upstream gradient dQ ~ N(0,1).
Complex Gaussians are (N + iN)/sqrt(2).  Every config draws from
``torch.Generator().manual_seed(1449 + config_id)``; ``n`` may be overridden to
get a smaller matrix with the same structure.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

SEED_BASE = 1449
C4_K0 = (8, 16, 32, 64, 128)
C4_K = (4, 8, 16, 32)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def gaussian(rows: int, cols: int, dtype: torch.dtype, g: torch.Generator, device="cpu") -> torch.Tensor:
    """Column-major (Fortran-order) N(0,1) matrix; complex entries are (N + iN)/sqrt(2)."""
    if dtype.is_complex:
        re = torch.randn(cols, rows, dtype=torch.float64, generator=g, device=device)
        im = torch.randn(cols, rows, dtype=torch.float64, generator=g, device=device)
        x = torch.complex(re, im) / math.sqrt(2.0)
    else:
        x = torch.randn(cols, rows, dtype=dtype, generator=g, device=device)
    return x.t()  # (rows, cols) view with column stride 1 along rows: column-major


def colmajor(x: torch.Tensor) -> torch.Tensor:
    """Return a column-major copy/view of a 2-D tensor (stride (1, rows))."""
    return x.t().contiguous().t()


def orthonormal(n: int, k0: int, dtype: torch.dtype, g: torch.Generator, device="cpu") -> torch.Tensor:
    """V = Q factor of a seeded Gaussian n x k0 matrix, column-major.

    On the CPU: the library (LAPACK) QR.  On a GPU: CholeskyQR2 -- two rounds
    of X <- X L^{-*} with G = X^* X = L L^* (Gram by cuBLAS, the k0 x k0
    Cholesky and triangular inverse on the CPU) -- which for a Gaussian
    n x k0 matrix (condition ~ 1 + 2 sqrt(k0/n)) gives ||V^* V - I|| ~ u.
    """
    x = gaussian(n, k0, dtype, g, device)
    if torch.device(device).type == "cpu":
        q, _ = torch.linalg.qr(x, mode="reduced")
        return colmajor(q)
    x = colmajor(x)
    eye = torch.eye(k0, dtype=dtype)
    for _ in range(2):
        G = (x.conj().T @ x).cpu()
        G = 0.5 * (G + G.conj().T)
        L = torch.linalg.cholesky(G)
        Linv = torch.linalg.solve_triangular(L, eye, upper=False)
        x = colmajor(x @ Linv.conj().T.to(x.device))
    return x


def worked_example(dtype=torch.float64):
    """V and A of eq. (badbcg), Section 1."""
    s = math.sqrt(2.0) / 2.0
    V = torch.tensor([[s, s], [-s, s], [0.0, 0.0], [0.0, 0.0]], dtype=torch.float64)
    A = torch.tensor([[1.0, 1.0], [1.0, 1.0], [1e-30, 0.0], [0.0, 1e-30]], dtype=torch.float64)
    return colmajor(V.to(dtype)), colmajor(A.to(dtype))


@dataclass
class Problem:
    V: torch.Tensor
    A: torch.Tensor
    n: int
    k0: int
    k: int
    dQ: torch.Tensor | None = None


CONFIG_SHAPES = {
    1: (4096, 16, 4, torch.float64),
    2: (1 << 20, 64, 16, torch.float64),
    3: (1 << 22, 128, 32, torch.complex128),
    5: (1 << 20, 64, 16, torch.float64),
}


def config_problem(cid: int, n: int | None = None, device="cpu", dtype: torch.dtype | None = None) -> Problem:
    """Seeded inputs of config ``cid`` (1, 2, 3 or 5), optionally with fewer rows ``n``."""
    n0, k0, k, dt = CONFIG_SHAPES[cid]
    n = n0 if n is None else n
    dt = dt if dtype is None else dtype
    g = _gen(SEED_BASE + cid, device)
    V = orthonormal(n, k0, dt, g, device)
    dQ = None
    if cid in (1, 5):
        A = gaussian(n, k, dt, g, device)
        if cid == 5:
            dQ = colmajor(gaussian(n, k, dt, g, device))
    elif cid == 2:
        C = gaussian(k0, k, dt, g, device)
        G = gaussian(n, k, dt, g, device)
        A = V @ C + 1e-10 * G
    elif cid == 3:
        h = k // 2
        C1 = gaussian(k0, h, dt, g, device)
        G1 = gaussian(n, h, dt, g, device)
        G2 = gaussian(n, k - h, dt, g, device)
        A = torch.cat([V @ C1 + 1e-14 * G1, G2], dim=1)
    else:
        raise ValueError(f"unknown config {cid}")
    return Problem(V=colmajor(V), A=colmajor(A), n=n, k0=k0, k=k, dQ=dQ)


def batched_shapes(count: int = 256, seed: int = SEED_BASE + 4, n_lo: int = 16384, n_hi: int = 262144):
    """The seeded (n, k0, k) list of the batched workload: n log-uniform, k0 and k uniform."""
    g = _gen(seed, "cpu")
    u = torch.rand(count, dtype=torch.float64, generator=g)
    ns = torch.round(torch.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))).to(torch.int64)
    k0i = torch.randint(0, len(C4_K0), (count,), generator=g)
    ki = torch.randint(0, len(C4_K), (count,), generator=g)
    return [(int(ns[i]), C4_K0[int(k0i[i])], C4_K[int(ki[i])]) for i in range(count)]


def batched_problems(shapes, seed: int = SEED_BASE + 4, device="cpu", dtype=torch.float64):
    """One Problem per (n, k0, k): V orthonormal, A ~ N(0,1)."""
    g = _gen(seed + 1000, device)
    out = []
    for (n, k0, k) in shapes:
        V = orthonormal(n, k0, dtype, g, device)
        A = colmajor(gaussian(n, k, dtype, g, device))
        out.append(Problem(V=V, A=A, n=n, k0=k0, k=k))
    return out


def random_problem(n: int, k0: int, k: int, dtype=torch.float64, seed: int = 0, device="cpu") -> Problem:
    """Well-conditioned random case: V orthonormal, A ~ N(0,1)."""
    g = _gen(seed, device)
    V = orthonormal(n, k0, dtype, g, device) if k0 > 0 else torch.zeros(n, 0, dtype=dtype, device=device)
    A = colmajor(gaussian(n, k, dtype, g, device))
    return Problem(V=colmajor(V), A=A, n=n, k0=k0, k=k)
