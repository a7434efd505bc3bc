"""ORACLE — test infrastructure only.

Plain, slow CPU reference for the two-stage Householder orthogonalization of
He & Shao (arXiv 2602.14449), Algorithm 1 with the second choice of P
(Section 3.2).  The arithmetic lives in ``tho_oracle.cpp`` (plain C++ loops,
FP64 / complex128, no BLAS); this module only builds it with g++ and marshals
numpy arrays through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never links or calls
it, and the two share no code.

Every function here is pinned in ``tests/test_oracle.py``:
  * ``two_stage``      — worked example eq. (badbcg) / Example 1; closed form
                         qf((I - V V^*) A); LAPACK QR of [V, A] (eq. vavq);
                         invariants of choice 2 (T = I + R_1^*, T + T^* = W^* W,
                         ||T||_2 <= 2, kappa_2(T) < 2 sqrt(2) k0); H [P; 0] = V;
                         special cases V = [I; 0], V_1 = 0, k0 = 0.
  * ``householder_qr`` — LAPACK QR after phase normalization.
  * ``bcgs``           — Table 1 first row (loss of orthogonality ~ 1) and the
                         three-projection rows (~ u) on the worked example.
  * ``modified_lu``, ``two_stage_mlu`` — Algorithm 2 and Algorithm 1 with the
                         first choice of P: P - V_1 = L U with |U_ii| >= 1,
                         T = (P - V_1)^* P; Q, R, S equal the closed form
                         (they do not depend on P) and the second choice's.
  * ``two_stage_polar`` — Algorithm 1 with the third choice of P: V_1 = Q2 M,
                         T = I + M Hermitian positive definite with
                         kappa_2(T) <= 2; Q, R, S equal the closed form.
  * ``block_hhqr``     — Algorithm 3: the unique QR with real nonnegative
                         diag(R) of a full-rank A by LAPACK (phase-normalized),
                         for several block splittings; Q^* Q = I, A = Q R.
  * ``two_stage_given_p`` (tests/test_oracle_figure1.py) — Algorithm 1 for a
                         given unitary P: the three choices' results when given
                         their P; Example 5's error laws against kappa_2(T).
  * ``two_stage_b``, ``block_hhqr_b`` (tests/test_oracle_b_inner.py) —
                         Algorithm 4 (B-inner product) and its block form
                         (Example 3): reduces to Algorithm 1 for B = I, U = [I; 0];
                         the closed-form B-orthogonal QR of (I - V V^* B) A;
                         [V, Q]^* B [V, Q] = I, eq. (vavqb), Theorem 5's HX = Y
                         and H^* B H = B.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tho_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (portable flags only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, dp = ctypes.c_int64, ctypes.c_void_p
            for name in ("oracle_two_stage_f64", "oracle_two_stage_c128"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64, dp, dp, dp]
                f.restype = ctypes.c_int
            for name in ("oracle_householder_qr_f64", "oracle_householder_qr_c128"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, dp, i64, dp, i64, dp]
                f.restype = ctypes.c_int
            for name in ("oracle_bcgs_f64", "oracle_bcgs_c128"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64, ctypes.c_char_p]
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _fortran(x, dtype):
    return np.asfortranarray(np.asarray(x, dtype=dtype))


def _dtype_of(*arrs):
    return np.complex128 if any(np.iscomplexobj(a) for a in arrs) else np.float64


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


def two_stage(V, A, return_aux: bool = False):
    """Algorithm 1 (second choice of P) on column-major copies of V (n x k0), A (n x k).

    Returns (Q, R, S) and, with ``return_aux``, a dict of the intermediate
    quantities Q1, R1, T, Wtop (k0 x k0), G, Z, Z2 (k0 x k) and Aprime (n x k).
    """
    dt = _dtype_of(V, A)
    V = _fortran(V, dt)
    A = _fortran(A, dt)
    n, k = A.shape
    k0 = V.shape[1] if V.ndim == 2 else 0
    if V.shape[0] != n and k0 > 0:
        raise ValueError("V and A must have the same number of rows")
    Q = np.zeros((n, k), dtype=dt, order="F")
    R = np.zeros((k, k), dtype=dt, order="F")
    S = np.zeros((k0, k), dtype=dt, order="F")
    aux = None
    if return_aux:
        aux = np.zeros(4 * k0 * k0 + 3 * k0 * k + n * k, dtype=dt)
    fn = _load().oracle_two_stage_c128 if dt == np.complex128 else _load().oracle_two_stage_f64
    rc = fn(n, k0, k, _ptr(V), max(n, 1), _ptr(A), n, _ptr(Q), n, _ptr(R), _ptr(S), _ptr(aux))
    if rc != 0:
        raise ValueError(f"oracle two_stage rejected shapes n={n} k0={k0} k={k}")
    if not return_aux:
        return Q, R, S
    out, o = {}, 0
    for name, r, c in (("Q1", k0, k0), ("R1", k0, k0), ("T", k0, k0), ("Wtop", k0, k0),
                       ("G", k0, k), ("Z", k0, k), ("Z2", k0, k), ("Aprime", n, k)):
        out[name] = aux[o:o + r * c].reshape((r, c), order="F")
        o += r * c
    return Q, R, S, out


def householder_qr(X):
    """Unblocked Householder QR with real nonnegative diag(R): X = Q R."""
    dt = _dtype_of(X)
    X = _fortran(X, dt)
    m, k = X.shape
    Q = np.zeros((m, k), dtype=dt, order="F")
    R = np.zeros((k, k), dtype=dt, order="F")
    fn = _load().oracle_householder_qr_c128 if dt == np.complex128 else _load().oracle_householder_qr_f64
    if fn(m, k, _ptr(X), m, _ptr(Q), m, _ptr(R)) != 0:
        raise ValueError("householder_qr needs m >= k >= 1")
    return Q, R


def modified_lu(Z):
    """Algorithm 2 (modified LU factorization): for Z (k x k, ||Z||_2 <= 1),
    a diagonal unitary P and the LU factorization P - Z = L U (L unit lower,
    U upper triangular) with P's entries chosen on the fly, P_ii = -sign(Z_ii)
    (sign(mu) = 1 if Re mu >= 0 else -1), so that |U_ii| >= 1 without pivoting.
    Plain loops in the algorithm's order.  Returns (P, L, U)."""
    Z = np.array(Z, dtype=np.result_type(Z, np.float64), copy=True)
    k = Z.shape[0]
    P = np.eye(k, dtype=Z.dtype)
    L = np.eye(k, dtype=Z.dtype)
    U = np.zeros((k, k), dtype=Z.dtype)
    for i in range(k):
        P[i, i] = -1.0 if Z[i, i].real >= 0 else 1.0
        U[i, i] = P[i, i] - Z[i, i]
        for j in range(i + 1, k):
            U[i, j] = -Z[i, j]
        for r in range(i + 1, k):
            L[r, i] = -Z[r, i] / U[i, i]
        for r in range(i + 1, k):
            for j in range(i + 1, k):
                Z[r, j] = Z[r, j] + L[r, i] * U[i, j]
    return P, L, U


def _tri(M, B, lower):
    """Substitution with the triangular M (plain loops, no explicit inverse)."""
    n = M.shape[0]
    X = np.zeros(B.shape, dtype=np.result_type(M, B))
    order = range(n) if lower else range(n - 1, -1, -1)
    for i in order:
        acc = B[i].astype(X.dtype)
        for j in (range(i) if lower else range(i + 1, n)):
            acc = acc - M[i, j] * X[j]
        X[i] = acc / M[i, i]
    return X


def two_stage_mlu(V, A):
    """Algorithm 1 with the first choice of P (Section 3.2): P diagonal from the
    modified LU factorization of P - V_{1:k0,:} (Algorithm 2), T = I - V_1^* P
    = (P - V_1)^* P = U^* L^* P, so T^{-*} G = U^{-1} L^{-1} (P G) and
    T^{-1} G_2 = P^* L^{-*} U^{-*} G_2 by triangular substitution.  The trailing
    QR is the oracle's Householder QR.  Returns (Q, R, S, aux) with aux the
    dict of P, L, U, T, Wtop, G, Z, Z2."""
    dt = _dtype_of(V, A)
    V = np.asarray(V, dtype=dt)
    A = np.asarray(A, dtype=dt)
    n, k = A.shape
    k0 = V.shape[1]
    V1, V2 = V[:k0], V[k0:]
    P, L, U = modified_lu(V1)
    Wtop = P - V1                      # W = [P; 0] - V
    T = np.eye(k0) - V1.conj().T @ P
    G = Wtop.conj().T @ A[:k0] - V2.conj().T @ A[k0:]
    Z = _tri(U, _tri(L, P @ G, lower=True), lower=False)       # T^{-*} G
    A1 = A[:k0] - Wtop @ Z                                       # A <- A - W T^{-*} W^* A
    A2 = A[k0:] + V2 @ Z
    S = P.conj().T @ A1
    Qb, R = householder_qr(A2)
    G2 = -V2.conj().T @ Qb                                       # W^* [0; Qbar]
    Z2 = P.conj().T @ _tri(L.conj().T, _tri(U.conj().T, G2, lower=True), lower=False)  # T^{-1} G2
    Q = np.vstack([-Wtop @ Z2, Qb + V2 @ Z2])
    return Q, R, S, {"P": P, "L": L, "U": U, "T": T, "Wtop": Wtop, "G": G, "Z": Z, "Z2": Z2}


def two_stage_polar(V, A):
    """Algorithm 1 with the third choice of P (Section 3.2): the polar
    decomposition V_{1:k0,:} = Q2 M (from the SVD, a library step: V_1 = X S Y^*,
    Q2 = X Y^*, M = Y S Y^*), P = -Q2, so T = I - V_1^* P = I + M is Hermitian
    positive definite with kappa_2(T) <= 2; T^{-*} = T^{-1} is applied through
    its Cholesky factor T = C C^* by triangular substitution.  Returns
    (Q, R, S, aux) with aux the dict of P, M, T, C, Wtop, G, Z, Z2."""
    dt = _dtype_of(V, A)
    V = np.asarray(V, dtype=dt)
    A = np.asarray(A, dtype=dt)
    n, k = A.shape
    k0 = V.shape[1]
    V1, V2 = V[:k0], V[k0:]
    X, sv, Yh = np.linalg.svd(V1)
    Q2 = X @ Yh
    M = Yh.conj().T @ np.diag(sv) @ Yh
    P = -Q2
    Wtop = P - V1
    T = np.eye(k0) - V1.conj().T @ P
    C = np.linalg.cholesky(0.5 * (T + T.conj().T))
    solve = lambda B: _tri(C.conj().T, _tri(C, B, lower=True), lower=False)  # T^{-1} B
    G = Wtop.conj().T @ A[:k0] - V2.conj().T @ A[k0:]
    Z = solve(G)                                                  # T^{-*} = T^{-1}
    A1 = A[:k0] - Wtop @ Z
    A2 = A[k0:] + V2 @ Z
    S = P.conj().T @ A1
    Qb, R = householder_qr(A2)
    Z2 = solve(-V2.conj().T @ Qb)
    Q = np.vstack([-Wtop @ Z2, Qb + V2 @ Z2])
    return Q, R, S, {"P": P, "M": M, "T": T, "C": C, "Wtop": Wtop, "G": G, "Z": Z, "Z2": Z2}


def two_stage_given_p(V, A, P):
    """Algorithm 1 for a given unitary P (k0 x k0): the generalized Householder
    transformation H = I - W T^{-1} W^* with W = [P; 0] - V and T = I - V_1^* P
    (Section 3.1), whatever the choice of P; Example 5 (Section 6) runs it with
    (V, P) built for a prescribed kappa_2(T).  T^{-*} G and T^{-1} G2 come from a
    library LU solve with partial pivoting (a backward stable solver, as the
    analysis of Section 4 assumes); the trailing QR is the oracle's Householder
    QR.  Returns (Q, R, S, aux) with aux the dict of T, Wtop, G, Z, Z2."""
    dt = _dtype_of(V, A)
    V = np.asarray(V, dtype=dt)
    A = np.asarray(A, dtype=dt)
    P = np.asarray(P, dtype=dt)
    n, k = A.shape
    k0 = V.shape[1]
    V1, V2 = V[:k0], V[k0:]
    Wtop = P - V1
    T = np.eye(k0) - V1.conj().T @ P
    G = Wtop.conj().T @ A[:k0] - V2.conj().T @ A[k0:]
    Z = np.linalg.solve(T.conj().T, G)                           # T^{-*} G
    A1 = A[:k0] - Wtop @ Z
    A2 = A[k0:] + V2 @ Z
    S = P.conj().T @ A1
    Qb, R = householder_qr(A2)
    Z2 = np.linalg.solve(T, -V2.conj().T @ Qb)                   # T^{-1} W^* [0; Qbar]
    Q = np.vstack([-Wtop @ Z2, Qb + V2 @ Z2])
    return Q, R, S, {"T": T, "Wtop": Wtop, "G": G, "Z": Z, "Z2": Z2}


def _phase(z):
    """z / |z|, with phase(0) = 1."""
    a = abs(z)
    return z / a if a != 0 else 1.0


def two_stage_b(B, V, U, A):
    """Algorithm 4 (Section 5): two-stage Householder-QR in the B-inner product
    <x, y>_B = y^* B x, B Hermitian positive definite (n x n).  V (n x k0) and
    U (n x (k0 + k)) have B-orthonormal columns; returns (Q, R, S, aux) with
    [V, A] = [V, Q] [[I, S], [0, R]] (eq. vavqb) and [V, Q]^* B [V, Q] = I.

    Steps in the algorithm's order, with Theorem 5's generalized reflector
    H = I - W T^{-1} W^* B (X = U_1 P, Y = V, W = X - Y, T = W^* B X = I - V^* B U_1 P):
      P       the second choice (Section 3.2) on the k0 x k0 matrix the method
              names, Z = U_1^* B V = Q1 R1 (diag(R1) >= 0), P = -Q1, so that
              T = I + R1^* as in Algorithm 1;
      A       <- H^{-1} A = (I - W T^{-*} W^* B) A (T^* solved by substitution);
      S       = U_1^* B A, then A <- A - U_1 S (the Gram-Schmidt step);
      Qbar R  the QR of A in the B-inner product with u_{k0+1}, ..., u_{k0+k} as
              the initial basis, column by column (left-looking): the current
              column x (earlier reflectors applied) loses its components r_ij
              along u_{k0+i}, i < j, and the rest x' is mapped by Theorem 5's
              reflector for one column (X = x', Y = y = -phase(u_{k0+j}^* B x')
              ||x'||_B u_{k0+j}) onto y.  The method recommends reorthogonalizing
              w = x' - y against [U_1 P, u_{k0+1}, ..., u_{k0+j-1}]; as y is
              B-orthogonal to that basis, this is done on x' itself (twice,
              before ||x'||_B and y are formed, the coefficients removed along
              u_{k0+i} added to r_ij), so that the reflector stays B-unitary
              when x' is at rounding level (a rank-deficient column);
              Qbar = H_1^{-1} ... H_k^{-1} [u_{k0+1}, ..., u_{k0+k}];
      Q       = H Qbar; finally diag(R) is made real >= 0 (column phases of Q).
    The inner QR is written from the method's description of it (Section 5);
    a column with x' = 0 takes H_j = I and R_jj = 0."""
    dt = _dtype_of(B, V, U, A)
    B = np.asarray(B, dtype=dt)
    V = np.asarray(V, dtype=dt)
    U = np.asarray(U, dtype=dt)
    A = np.array(A, dtype=dt, copy=True)
    n, k = A.shape
    k0 = V.shape[1]
    if U.shape != (n, k0 + k) or B.shape != (n, n):
        raise ValueError("need B n x n, V n x k0, U n x (k0 + k), A n x k")
    h = lambda M: M.conj().T
    Bip = lambda X, Y: h(X) @ (B @ Y)                      # X^* B Y
    U1, U2 = U[:, :k0], U[:, k0:]
    if k0 > 0:
        # Choice of P and the reflector of the first stage.
        Q1, R1 = householder_qr(Bip(U1, V))
        P = -Q1
        U1 = U1 @ P
        W = U1 - V
        T = np.eye(k0, dtype=dt) - Bip(V, U1)
        Z = _tri(h(T), Bip(W, A), lower=False)             # T^{-*} W^* B A (T^* upper)
        A = A - W @ Z                                      # H^{-1} A
        S = Bip(U1, A)
        A = A - U1 @ S
    else:                                                  # k0 = 0: the B-inner-product QR of A alone
        P = T = np.zeros((0, 0), dtype=dt)
        W = np.zeros((n, 0), dtype=dt)
        S = np.zeros((0, k), dtype=dt)
    # QR of A in the B-inner product, u_{k0+1..k0+k} as the initial basis.
    R = np.zeros((k, k), dtype=dt)
    ws, ts = [], []
    for j in range(k):
        x = A[:, j].copy()
        for w_i, t_i in zip(ws, ts):                        # x <- H_{j-1} ... H_1 a_j
            if t_i != 0:
                x = x - w_i * (np.vdot(w_i, B @ x) / t_i)
        R[:j, j] = h(U2[:, :j]) @ (B @ x)
        xp = x - U2[:, :j] @ R[:j, j]
        basis = np.concatenate([U1, U2[:, :j]], axis=1)
        for _ in range(2):                                  # reorthogonalization (of x', hence of w)
            cb = h(basis) @ (B @ xp)
            xp = xp - basis @ cb
            R[:j, j] += cb[k0:]
        rho = np.sqrt(max(np.vdot(xp, B @ xp).real, 0.0))
        c = np.vdot(U2[:, j], B @ xp)
        y = -_phase(c) * rho * U2[:, j]
        R[j, j] = -_phase(c) * rho
        w = xp - y
        t = np.vdot(w, B @ xp) if rho != 0 else 0.0
        ws.append(w)
        ts.append(t)
    Qb = U2.copy()
    for w_i, t_i in reversed(list(zip(ws, ts))):           # Qbar = H_1^{-1} ... H_k^{-1} U_2
        if t_i != 0:
            Qb = Qb - np.outer(w_i, (h(w_i) @ (B @ Qb)) / np.conj(t_i))
    Z2 = _tri(T, Bip(W, Qb), lower=True) if k0 > 0 else np.zeros((0, k), dtype=dt)  # T^{-1} W^* B Qbar
    Q = Qb - W @ Z2                                        # H Qbar
    d = np.array([_phase(R[j, j]) for j in range(k)], dtype=dt)
    Q = Q * d[None, :]
    R = np.conj(d)[:, None] * R
    return Q, R, S, {"P": P, "T": T, "W": W, "U1P": U1, "Qbar": Qb * d[None, :]}


def block_hhqr_b(B, A, kb):
    """Algorithm 3 in the B-inner product (Example 3, Section 6): the blocks
    A_i taken in order, step i = Algorithm 4 (``two_stage_b``) with
    V = [Q_1, ..., Q_{i-1}] (step 1: k0 = 0) and the initial B-orthonormal basis
    U = [L^{-*}; 0] from the Cholesky factor L of the leading (k0 + k_i) x
    (k0 + k_i) block of B (the construction the method suggests; a library
    Cholesky and triangular solve).  Returns (Q, R): A = Q R, Q^* B Q = I."""
    dt = _dtype_of(B, A)
    B = np.asarray(B, dtype=dt)
    A = np.asarray(A, dtype=dt)
    n, K = A.shape
    if sum(kb) != K:
        raise ValueError("block widths must add up to the columns of A")
    Q = np.zeros((n, K), dtype=dt)
    R = np.zeros((K, K), dtype=dt)
    o = 0
    for k in kb:
        L = np.linalg.cholesky(B[:o + k, :o + k])
        U = np.zeros((n, o + k), dtype=dt)
        U[:o + k] = np.linalg.solve(L.conj().T, np.eye(o + k, dtype=dt))
        Qi, Rii, S, _ = two_stage_b(B, Q[:, :o], U, A[:, o:o + k])
        Q[:, o:o + k] = Qi
        R[:o, o:o + k] = S
        R[o:o + k, o:o + k] = Rii
        o += k
    return Q, R


def block_hhqr(A, kb):
    """Algorithm 3 (Block Householder-QR, Section 5): the QR factorization of
    A = [A_1, ..., A_p] (block widths kb) taking the blocks in order.  Step 1
    is the Householder QR of A_1; step i >= 2 is Algorithm 1 with
    V = [Q_1, ..., Q_{i-1}] and A = A_i, whose Q, R and S give Q_i, the
    diagonal block R_ii and the block above it, R_{1:i-1, i}.  Returns (Q, R)."""
    dt = _dtype_of(A)
    A = _fortran(A, dt)
    n, K = A.shape
    if sum(kb) != K:
        raise ValueError("block widths must add up to the columns of A")
    Q = np.zeros((n, K), dtype=dt, order="F")
    R = np.zeros((K, K), dtype=dt, order="F")
    o = 0
    for i, k in enumerate(kb):
        if i == 0:
            Qi, Rii = householder_qr(A[:, :k])
        else:
            Qi, Rii, S = two_stage(Q[:, :o], A[:, o:o + k])
            R[:o, o:o + k] = S
        Q[:, o:o + k] = Qi
        R[o:o + k, o:o + k] = Rii
        o += k
    return Q, R


def bcgs(V, A, passes: str = "PQ"):
    """BCGS comparator, eq. (BQR): 'P' = projection (BQR-1), 'Q' = Householder QR (BQR-2)."""
    dt = _dtype_of(V, A)
    V = _fortran(V, dt)
    A = _fortran(A, dt)
    n, k = A.shape
    k0 = V.shape[1]
    Q = np.zeros((n, k), dtype=dt, order="F")
    fn = _load().oracle_bcgs_c128 if dt == np.complex128 else _load().oracle_bcgs_f64
    if fn(n, k0, k, _ptr(V), n, _ptr(A), n, _ptr(Q), n, passes.encode()) != 0:
        raise ValueError("bcgs: bad shapes or pass string")
    return Q
