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
  * ``table4``  real, n=1000, k0=100: V built as in Appendix A so that the
            modified LU of V_{1:k0,:} (Algorithm 2) yields U of eq. (badmlu)
            (kappa_2(U) ~ 1.1e7), A ~ N(0,1) (Example 4 and Table 4, Section 6).
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


def graded_problem(n: int, k0: int, k: int, dtype=torch.float64, seed: int = 0, decades: float = 12.0,
                   period: int = 256) -> Problem:
    """Rows graded over ``decades`` decades within every ``period`` rows:
    D = diag(10^(-decades (i mod period) / (period - 1))), V = Q factor of
    D G1 (so V's rows are graded too), A = D G2, G1 and G2 Gaussian.  Every
    leaf and every row chunk of the streaming sweeps then holds rows whose
    scales span all the decades.  Well conditioned: the rows near scale 1
    alone make A and [V, A] full rank with condition of order one."""
    g = _gen(seed, "cpu")
    i = torch.arange(n, dtype=torch.float64)
    d = torch.pow(10.0, -decades * torch.remainder(i, period) / (period - 1)).to(dtype)
    if k0 > 0:
        x = gaussian(n, k0, dtype, g) * d[:, None]
        q, _ = torch.linalg.qr(x, mode="reduced")
        V = colmajor(q)
    else:
        V = torch.zeros(n, 0, dtype=dtype)
    A = colmajor(gaussian(n, k, dtype, g) * d[:, None])
    return Problem(V=V, A=A, n=n, k0=k0, k=k)


def badmlu_u(k0: int, alpha: float = 0.1) -> torch.Tensor:
    """U of eq. (badmlu) (Section 3.2, first choice of P): with 0-based row i,
    U_ii = 1 + alpha / sqrt(k0 - i) and U_ij = -1 / sqrt(k0 - i) for j > i."""
    U = torch.zeros(k0, k0, dtype=torch.float64)
    for i in range(k0):
        s = 1.0 / math.sqrt(k0 - i)
        U[i, i] = 1.0 + alpha * s
        U[i, i + 1:] = -s
    return U


def appendix_a_v(n: int, k0: int, alpha: float = 0.1, seed: int = SEED_BASE + 7) -> torch.Tensor:
    """Real V (n x k0, orthonormal columns, column-major) whose top block
    Z = V_{1:k0,:} makes the modified LU factorization (Algorithm 2) return
    P = I and U of eq. (badmlu): the construction of Appendix A.

    With R = U - I (each row of 2-norm below one), V is built from the bottom
    of a Householder QR upward: the last trailing column is a unit vector with
    first entry b_1; then, one row of R at a time from the last, the Lemma of
    Appendix A extends an orthonormal m x j matrix W to an (m+1) x (j+1) one
    whose first row is the given b and whose first Householder step gives back
    [[-sign(b_1), 0], [0, W]]: with V_H that block matrix, a unit v orthogonal
    to Range(V_H), x = sqrt(1 - ||b||^2) v + V_H b and the reflector H taking x
    to e_1, the new matrix is H V_H.

    Two readings.  (1) The rows enter negated (b = -R_{i, i:k0}): Algorithm 2
    takes P_ii = -sign(Z_ii), so the rows of R themselves would give U = -(I + R);
    with the negated rows it gives I + R, eq. (badmlu) itself (kappa_2 is the
    same either way).  (2) H is formed as I - 2 w w^T / (w^T w) with w = x - e_1,
    which equals the Appendix's I - (1 - x_1) w' w'^T, w' = (x - e_1)/(x_1 - 1),
    when ||x|| = 1 exactly; the Appendix's form loses orthogonality geometrically
    (by 1e-1 at k0 = 100 in FP64) because rounding makes ||x|| != 1 step after
    step, while this one stays orthogonal to rounding (||V^T V - I|| ~ 1e-14).
    Inputs only: no step of the orthogonalization method is taken here."""
    if not (1 <= k0 <= n):
        raise ValueError("need 1 <= k0 <= n")
    g = _gen(seed, "cpu")
    R = badmlu_u(k0, alpha) - torch.eye(k0, dtype=torch.float64)
    m = n - k0 + 1
    x = torch.randn(m - 1, dtype=torch.float64, generator=g)
    x *= math.sqrt(1.0 - float(R[k0 - 1, k0 - 1]) ** 2) / float(torch.linalg.vector_norm(x))
    W = torch.cat([-R[k0 - 1, k0 - 1:], x]).reshape(m, 1)
    for i in range(1, k0):
        b = -R[k0 - 1 - i, k0 - 1 - i:]
        rows, j = W.shape
        VH = torch.zeros(rows + 1, j + 1, dtype=torch.float64)
        VH[0, 0] = -1.0 if float(b[0]) >= 0 else 1.0
        VH[1:, 1:] = W
        v = torch.randn(rows + 1, dtype=torch.float64, generator=g)
        v[0] = 0.0
        for _ in range(2):  # orthogonal to Range(V_H), twice for working accuracy
            v -= VH @ (VH.t() @ v)
        v /= torch.linalg.vector_norm(v)
        xv = math.sqrt(max(0.0, 1.0 - float(b @ b))) * v + VH @ b
        w = xv.clone()
        w[0] -= 1.0
        W = VH - (2.0 / float(w @ w)) * torch.outer(w, w @ VH)
    return colmajor(W)


def table4_problem(n: int = 1000, k0: int = 100, k: int = 100, alpha: float = 0.1,
                   seed: int = SEED_BASE + 7) -> Problem:
    """Example 4 / Table 4 (Section 6): V of Appendix A (eq. (badmlu) with
    alpha), A ~ N(0,1) n x k."""
    V = appendix_a_v(n, k0, alpha, seed)
    A = colmajor(gaussian(n, k, torch.float64, _gen(seed + 1, "cpu")))
    return Problem(V=V, A=A, n=n, k0=k0, k=k)


@dataclass
class BProblem:
    B: torch.Tensor
    V: torch.Tensor
    U: torch.Tensor
    A: torch.Tensor
    d: torch.Tensor | None = None  # the diagonal, when B is diagonal


def b_inner_problem(n: int, k0: int, k: int, kappa_b: float = 1e2, dtype=torch.float64,
                    seed: int = SEED_BASE + 8) -> BProblem:
    """Inputs of Algorithm 4 (Section 5): B = X diag(lambda) X^* Hermitian
    positive definite with eigenvalues log-spaced in [1, kappa_b] (X the Q factor
    of a Gaussian matrix), V with B-orthonormal columns (a Gaussian G times the
    inverse of the Cholesky factor of G^* B G), U = [L^{-*}; 0] from the Cholesky
    factor L of the leading (k0 + k) x (k0 + k) block of B (the initial
    B-orthonormal basis the method suggests), A ~ N(0,1).  Library steps only."""
    g = _gen(seed, "cpu")
    X = torch.linalg.qr(gaussian(n, n, dtype, g))[0]
    lam = torch.logspace(0.0, math.log10(kappa_b), n, dtype=torch.float64).to(dtype)
    B = (X * lam[None, :]) @ X.conj().T
    B = 0.5 * (B + B.conj().T)
    G = gaussian(n, k0, dtype, g)
    C = torch.linalg.cholesky(G.conj().T @ B @ G)
    V = torch.linalg.solve_triangular(C, G.conj().T, upper=False).conj().T  # G C^{-*}
    L = torch.linalg.cholesky(B[:k0 + k, :k0 + k])
    U = torch.zeros(n, k0 + k, dtype=dtype)
    U[:k0 + k] = torch.linalg.solve_triangular(L.conj().T, torch.eye(k0 + k, dtype=dtype), upper=True)
    A = gaussian(n, k, dtype, g)
    return BProblem(B=B, V=colmajor(V), U=colmajor(U), A=colmajor(A))


def diag_b_problem(n: int, k0: int, k: int, kappa_b: float = 1e5, dtype=torch.float64,
                   seed: int = SEED_BASE + 9) -> BProblem:
    """Inputs of Algorithm 4 (Section 5) with a diagonal B = diag(d): d
    log-spaced in [1, kappa_b] in a seeded random order, V = D^{-1/2} Q0 with Q0
    the Q factor of a Gaussian n x k0 matrix (so V^* B V = I), U = D^{-1/2} [I; 0]
    (the Cholesky construction of Section 5 for a diagonal B), A ~ N(0,1).
    ``B`` is the dense diag(d) for the CPU oracle; ``d`` is the diagonal."""
    g = _gen(seed, "cpu")
    d = torch.logspace(0.0, math.log10(kappa_b), n, dtype=torch.float64)[torch.randperm(n, generator=g)]
    isd = 1.0 / torch.sqrt(d)
    Q0 = orthonormal(n, k0, dtype, g) if k0 > 0 else torch.zeros(n, 0, dtype=dtype)
    V = Q0 * isd[:, None].to(dtype)
    U = torch.zeros(n, k0 + k, dtype=dtype)
    idx = torch.arange(k0 + k)
    U[idx, idx] = isd[:k0 + k].to(dtype)
    A = gaussian(n, k, dtype, g)
    return BProblem(B=torch.diag(d).to(dtype), V=colmajor(V), U=colmajor(U), A=colmajor(A), d=d)
