"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is either
printed in the paper (tests/golden/), a closed form evaluated by a different
route (LAPACK QR through numpy, or mpmath in extended precision), an invariant
the paper proves, or a special case that reduces to a textbook routine.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from metrics import loo, orth, qf, resid_fro, resid_paper, vq
from paper_2602_14449_gb300 import inputs

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _np(t):
    return t.numpy() if isinstance(t, torch.Tensor) else t


def _worked():
    with open(os.path.join(GOLDEN, "worked_example_badbcg.json")) as f:
        gold = json.load(f)

    def val(x):
        if isinstance(x, str):
            return {"sqrt2/2": math.sqrt(2) / 2, "-sqrt2/2": -math.sqrt(2) / 2, "sqrt2": math.sqrt(2)}[x]
        return float(x)

    V = np.array([[val(x) for x in r] for r in gold["V_rows"]])
    A = np.array([[val(x) for x in r] for r in gold["A_rows"]])
    return gold, V, A, val


def test_worked_example_inputs_match_generator():
    gold, V, A, _ = _worked()
    Vg, Ag = inputs.worked_example()
    np.testing.assert_array_equal(V, Vg.numpy())
    np.testing.assert_array_equal(A, Ag.numpy())


def test_worked_example_algorithm1():
    """eq. (badbcg) + Example 1: Algorithm 1 reaches LOO ~ 2u; Q, R, S, T exact."""
    gold, V, A, val = _worked()
    Q, R, S, aux = oracle.two_stage(V, A, return_aux=True)
    d = gold["derived_by_hand"]
    np.testing.assert_allclose(Q, np.array(d["Q_rows"], float), atol=4 * U, rtol=0)
    np.testing.assert_allclose(R, np.array(d["R_rows"], float), rtol=1e-14, atol=0)
    np.testing.assert_allclose(S, np.array([[val(x) for x in r] for r in d["S_rows"]]), atol=4 * U)
    np.testing.assert_allclose(aux["T"], np.array(d["T_rows"], float), atol=4 * U)
    assert loo(V, Q) <= 10 * U  # paper: ~2u
    assert gold["paper_values"]["alg1_loo_approx"] < 1e-15


def test_worked_example_bcgs_table1():
    """Table 1: BCGS loses orthogonality completely; three projections recover it."""
    gold, V, A, _ = _worked()
    tab = gold["paper_values"]["table1_bcgs_loo"]
    got = {p: loo(V, oracle.bcgs(V, A, p)) for p in tab}
    # Rows 1-3 reproduce the printed two significant digits (1.0e0, 9.8e-2, 7.0e-2).
    for p in ("PQ", "PPQ", "PQPQ"):
        assert float(f"{got[p]:.1e}") == tab[p], (p, got[p], tab[p])
    # Rows 4-5 are printed as 2.2e-16, i.e. a couple of units of roundoff.
    assert got["PPPQ"] <= 4 * U and got["PQPQPQ"] <= 4 * U


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("n,k0,k", [(64, 8, 4), (300, 16, 5), (97, 1, 1), (40, 20, 20), (129, 7, 33)])
def test_closed_form_lapack(dtype, n, k0, k):
    """Q = qf((I - V V^*) A), R from the same QR, S = V^* A (eq. vavq, Section 3.1)."""
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=n * 131 + k0 * 7 + k)
    V, A = _np(p.V), _np(p.A)
    Q, R, S = oracle.two_stage(V, A)
    Qc, Rc = qf(A - V @ (V.conj().T @ A))
    np.testing.assert_allclose(Q, Qc, atol=1e-12, rtol=0)
    np.testing.assert_allclose(R, Rc, atol=1e-12 * np.abs(Rc).max(), rtol=0)
    np.testing.assert_allclose(S, V.conj().T @ A, atol=1e-12 * np.abs(S).max(), rtol=0)
    assert loo(V, Q) < 100 * U
    assert resid_fro(V, A, Q, R, S) < 100 * U


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_full_householder_qr_of_VA(dtype):
    """eq. (vavq): the QR of [V, A] with diag(R) >= 0 has blocks [[I, S], [0, R]] and Q-factor [V, Q]."""
    p = inputs.random_problem(200, 12, 6, dtype=dtype, seed=5)
    V, A = _np(p.V), _np(p.A)
    Q, R, S = oracle.two_stage(V, A)
    Qf, Rf = qf(np.concatenate([V, A], axis=1))
    k0 = V.shape[1]
    np.testing.assert_allclose(Qf[:, :k0], V, atol=1e-13)
    np.testing.assert_allclose(Rf[:k0, :k0], np.eye(k0), atol=1e-13)
    np.testing.assert_allclose(Rf[:k0, k0:], S, atol=1e-12)
    np.testing.assert_allclose(Rf[k0:, k0:], R, atol=1e-12)
    np.testing.assert_allclose(Qf[:, k0:], Q, atol=1e-12)


def _mp_closed_form(V, A, dps=60):
    """Closed form qf((I - V V^*) A) by modified Gram-Schmidt in mpmath (extended precision)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = dps
    n, k0 = V.shape
    k = A.shape[1]
    cplx = np.iscomplexobj(V) or np.iscomplexobj(A)
    conv = (lambda z: mpmath.mpc(z.real, z.imag)) if cplx else (lambda z: mpmath.mpf(float(z)))
    Vm = [[conv(V[i, j]) for j in range(k0)] for i in range(n)]
    cols = []
    for c in range(k):
        x = [conv(A[i, c]) for i in range(n)]
        for j in range(k0):  # project out V exactly (V^*V = I to ~1e-16 is corrected below)
            s = sum(mpmath.conj(Vm[i][j]) * x[i] for i in range(n))
            x = [x[i] - Vm[i][j] * s for i in range(n)]
        for q in cols:
            s = sum(mpmath.conj(q[i]) * x[i] for i in range(n))
            x = [x[i] - q[i] * s for i in range(n)]
        nr = mpmath.sqrt(sum(abs(xi) ** 2 for xi in x))
        cols.append([xi / nr for xi in x])
    out = np.array([[complex(cols[c][i]) if cplx else float(cols[c][i]) for c in range(k)] for i in range(n)])
    return out


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_closed_form_extended_precision(dtype):
    """Brute force on a tiny input: Gram-Schmidt in 60-digit arithmetic vs the oracle."""
    p = inputs.random_problem(9, 3, 2, dtype=dtype, seed=11)
    V, A = _np(p.V), _np(p.A)
    Q, _, _ = oracle.two_stage(V, A)
    np.testing.assert_allclose(Q, _mp_closed_form(V, A), atol=1e-14)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("k0", [1, 6, 24])
def test_choice2_invariants(dtype, k0):
    """Section 3.2, second choice: T = I + R1^* lower, diag >= 1, T + T^* = W^*W,
    ||w_i||^2 = 2 T_ii, ||T||_2 <= 2, kappa_2(T) < 2 sqrt(2) k0; P = -Q1 unitary;
    Section 3.1: H [P; 0] = V, H^* H = I, H^* A = [P V^* A; V_perp^* A]."""
    n, k = 60, 5
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=k0)
    V, A = _np(p.V), _np(p.A)
    Q, R, S, aux = oracle.two_stage(V, A, return_aux=True)
    T, Q1, R1, Wt = aux["T"], aux["Q1"], aux["R1"], aux["Wtop"]
    # QR of V_1 against LAPACK
    Q1c, R1c = qf(V[:k0])
    np.testing.assert_allclose(Q1, Q1c, atol=1e-13)
    np.testing.assert_allclose(R1, R1c, atol=1e-13)
    assert np.allclose(np.triu(T, 1), 0)
    assert np.all(np.real(np.diag(T)) >= 1 - 1e-15) and np.allclose(np.imag(np.diag(T)), 0)
    P = -Q1
    np.testing.assert_allclose(T, np.eye(k0) - V[:k0].conj().T @ P, atol=1e-13)  # Algorithm 1, T
    W = np.concatenate([Wt, -V[k0:]], axis=0)
    np.testing.assert_allclose(W, np.concatenate([P, np.zeros((n - k0, k0))]) - V, atol=1e-14)
    np.testing.assert_allclose(T + T.conj().T, W.conj().T @ W, atol=1e-13)
    np.testing.assert_allclose(np.sum(np.abs(W) ** 2, axis=0), 2 * np.real(np.diag(T)), atol=1e-13)
    assert np.linalg.norm(T, 2) <= 2 + 1e-13
    assert np.linalg.cond(T) < 2 * math.sqrt(2) * k0
    np.testing.assert_allclose(P.conj().T @ P, np.eye(k0), atol=1e-14)
    H = np.eye(n) - W @ np.linalg.solve(T, W.conj().T)
    np.testing.assert_allclose(H @ np.concatenate([P, np.zeros((n - k0, k0))]), V, atol=1e-13)
    np.testing.assert_allclose(H.conj().T @ H, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(aux["Aprime"], H.conj().T @ A, atol=1e-13)
    np.testing.assert_allclose(aux["Aprime"][:k0], P @ (V.conj().T @ A), atol=1e-13)
    np.testing.assert_allclose(Q, H @ np.concatenate([np.zeros((k0, k)), qf(aux["Aprime"][k0:])[0]]), atol=1e-13)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_special_case_V_identity(dtype):
    """V = [I; 0]: V_1 = I so R_1 = I, T = 2I, and Q = [0; qf(A_2)]."""
    n, k0, k = 50, 6, 4
    V = np.zeros((n, k0), dtype=np.complex128 if dtype.is_complex else np.float64)
    V[:k0, :k0] = np.eye(k0)
    A = _np(inputs.random_problem(n, 0, k, dtype=dtype, seed=3).A)
    Q, R, S, aux = oracle.two_stage(V, A, return_aux=True)
    np.testing.assert_allclose(aux["T"], 2 * np.eye(k0), atol=1e-15)
    Qc, Rc = qf(A[k0:])
    np.testing.assert_allclose(Q[:k0], 0, atol=1e-15)
    np.testing.assert_allclose(Q[k0:], Qc, atol=1e-13)
    np.testing.assert_allclose(R, Rc, atol=1e-13)
    np.testing.assert_allclose(S, A[:k0], atol=1e-15)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_special_case_V1_zero(dtype):
    """V_1 = 0: every reflector of the k0 x k0 QR is the identity, Q1 = I, R1 = 0, T = I."""
    n, k0, k = 70, 5, 3
    g = inputs.random_problem(n - k0, k0, k, dtype=dtype, seed=9)
    V = np.concatenate([np.zeros((k0, k0)), _np(g.V)], axis=0)
    A = _np(inputs.random_problem(n, 0, k, dtype=dtype, seed=10).A)
    Q, R, S, aux = oracle.two_stage(V, A, return_aux=True)
    np.testing.assert_allclose(aux["Q1"], np.eye(k0), atol=0)
    np.testing.assert_allclose(aux["R1"], 0, atol=0)
    np.testing.assert_allclose(aux["T"], np.eye(k0), atol=0)
    Qc, _ = qf(A - V @ (V.conj().T @ A))
    np.testing.assert_allclose(Q, Qc, atol=1e-13)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_special_case_k0_zero_is_householder_qr(dtype):
    """k0 = 0: the method is the textbook Householder QR of A."""
    p = inputs.random_problem(80, 0, 7, dtype=dtype, seed=21)
    A = _np(p.A)
    V = np.zeros((80, 0), dtype=A.dtype)
    Q, R, S = oracle.two_stage(V, A)
    Qc, Rc = qf(A)
    np.testing.assert_allclose(Q, Qc, atol=1e-13)
    np.testing.assert_allclose(R, Rc, atol=1e-13)
    Qh, Rh = oracle.householder_qr(A)
    np.testing.assert_allclose(Qh, Qc, atol=1e-13)
    np.testing.assert_allclose(Rh, Rc, atol=1e-13)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_rank_deficient_stability(dtype):
    """Theorem 4 / Remark: stability does not depend on kappa([V,A]).  The
    C3-like structure (half of A in Range(V) + 1e-14 noise) keeps LOO and the
    residual at O(u) while BCGS loses orthogonality."""
    p = inputs.config_problem(3, n=3000, dtype=dtype)
    V, A = _np(p.V), _np(p.A)
    Q, R, S = oracle.two_stage(V, A)
    assert loo(V, Q) < 1e-14
    assert resid_fro(V, A, Q, R, S) < 1e-14
    assert resid_paper(V, A, Q, R, S) < 1e-14
    assert loo(V, oracle.bcgs(V, A, "PQ")) > 1e-6


def test_ill_conditioned_c2_structure():
    """C2 structure: A = V C + 1e-10 G, cond([V,A]) ~ 1e10; Theorem 4 bounds hold at O(u)."""
    p = inputs.config_problem(2, n=5000)
    V, A = _np(p.V), _np(p.A)
    Q, R, S = oracle.two_stage(V, A)
    assert loo(V, Q) < 1e-14
    assert orth(Q) < 1e-14 and vq(V, Q) < 1e-14
    assert resid_fro(V, A, Q, R, S) < 1e-14


def test_householder_qr_rank_deficient_columns():
    """Exactly dependent and zero columns: Q stays orthonormal (tau = 0 convention)."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((30, 5))
    X[:, 2] = X[:, 0] + X[:, 1]
    X[:, 4] = 0
    Q, R = oracle.householder_qr(X)
    assert orth(Q) < 1e-14
    np.testing.assert_allclose(Q @ R, X, atol=1e-13)
    assert np.all(np.diag(R) >= 0)


def test_oracle_rejects_bad_shapes():
    with pytest.raises(ValueError):
        oracle.two_stage(np.zeros((4, 3)), np.zeros((4, 2)))  # k0 + k > n


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("kb", [[5], [3, 4], [4, 7, 1, 6], [1, 1, 1, 1, 1, 1]])
def test_block_hhqr_is_the_unique_qr(dtype, kb):
    """Algorithm 3 on a full-rank A: the unique QR with real nonnegative diag(R)
    (LAPACK, phase-normalized), whatever the block splitting."""
    p = inputs.random_problem(300, 0, sum(kb), dtype=dtype, seed=31 + len(kb))
    A = _np(p.A)
    Q, R = oracle.block_hhqr(A, kb)
    Qc, Rc = qf(A)
    np.testing.assert_allclose(Q, Qc, atol=1e-13)
    np.testing.assert_allclose(R, Rc, atol=1e-12)
    assert np.abs(np.tril(R, -1)).max() == 0.0
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(sum(kb)), atol=1e-14)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13 * np.abs(A).max())


def test_block_hhqr_ill_conditioned_krylov():
    """Block Krylov-style blocks A_{i+1} = D A_i (spread spectrum D): the whole
    matrix is ill-conditioned, and Algorithm 3 keeps orthogonality at the
    rounding level (the stability of Section 5's example)."""
    rng = np.random.default_rng(7)
    n, k, p = 400, 4, 6
    d = np.exp(np.linspace(0.0, 6.0, n))
    blocks = [rng.standard_normal((n, k))]
    for _ in range(p - 1):
        blocks.append(d[:, None] * blocks[-1])
    A = np.hstack(blocks)
    assert np.linalg.cond(A) > 1e8
    Q, R = oracle.block_hhqr(A, [k] * p)
    assert np.linalg.norm(Q.T @ Q - np.eye(k * p), 2) < 1e-14
    assert np.linalg.norm(A - Q @ R, "fro") / np.linalg.norm(A, "fro") < 1e-14


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("k0", [1, 6, 16])
def test_modified_lu_properties(dtype, k0):
    """Algorithm 2: P diagonal with entries -sign(.) = +-1, L unit lower, U upper,
    P - Z = L U, and |U_ii| >= 1 (no pivoting needed) for ||Z||_2 <= 1."""
    p = inputs.random_problem(3 * k0 + 5, k0, 1, dtype=dtype, seed=41 + k0)
    Z = _np(p.V)[:k0]
    assert np.linalg.norm(Z, 2) <= 1.0 + 1e-14
    P, L, U = oracle.modified_lu(Z)
    assert np.allclose(P, np.diag(np.diag(P))) and set(np.round(np.diag(P).real).tolist()) <= {-1.0, 1.0}
    assert np.allclose(np.diag(L), 1.0) and np.abs(np.triu(L, 1)).max() == 0.0
    assert np.abs(np.tril(U, -1)).max() == 0.0
    np.testing.assert_allclose(L @ U, P - Z, atol=1e-13)
    assert np.abs(np.diag(U)).min() >= 1.0 - 1e-15


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("n,k0,k", [(200, 6, 4), (500, 16, 7), (64, 1, 3)])
def test_first_choice_matches_closed_form(dtype, n, k0, k):
    """Algorithm 1 with the first choice of P: T = (P - V_1)^* P = I - V_1^* P,
    H^* H = I, H [P; 0] = V, and Q, R, S equal the closed form qf((I - V V^*) A),
    V^* A (independent of P) and the second choice's results."""
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=n + k0 + k)
    V, A = _np(p.V), _np(p.A)
    Q, R, S, aux = oracle.two_stage_mlu(V, A)
    P, T, Wtop = aux["P"], aux["T"], aux["Wtop"]
    np.testing.assert_allclose(T, Wtop.conj().T @ P, atol=1e-14)
    W = np.vstack([Wtop, -V[k0:]])
    H = np.eye(n) - W @ np.linalg.solve(T, W.conj().T)
    np.testing.assert_allclose(H.conj().T @ H, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(H @ np.vstack([P, np.zeros((n - k0, k0))]), V, atol=1e-12)
    Qc, Rc = qf(A - V @ (V.conj().T @ A))
    np.testing.assert_allclose(Q, Qc, atol=1e-12)
    np.testing.assert_allclose(R, Rc, atol=1e-12)
    np.testing.assert_allclose(S, V.conj().T @ A, atol=1e-12)
    Q2, R2, S2 = oracle.two_stage(V, A)
    np.testing.assert_allclose(Q, Q2, atol=1e-12)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("n,k0,k", [(200, 6, 4), (500, 16, 7), (64, 1, 3)])
def test_third_choice_matches_closed_form(dtype, n, k0, k):
    """Algorithm 1 with the third choice of P (polar factor): V_1 = Q2 M with Q2
    unitary and M Hermitian positive semidefinite, T = I + M with kappa_2(T) <= 2,
    H [P; 0] = V, and Q, R, S equal the closed form (independent of P)."""
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=7 * n + k0 + k)
    V, A = _np(p.V), _np(p.A)
    Q, R, S, aux = oracle.two_stage_polar(V, A)
    P, M, T, Wtop = aux["P"], aux["M"], aux["T"], aux["Wtop"]
    np.testing.assert_allclose((-P) @ M, V[:k0], atol=1e-13)
    np.testing.assert_allclose(P.conj().T @ P, np.eye(k0), atol=1e-13)
    np.testing.assert_allclose(M, M.conj().T, atol=1e-13)
    assert np.linalg.eigvalsh(M).min() > -1e-13
    np.testing.assert_allclose(T, np.eye(k0) + M, atol=1e-13)
    assert np.linalg.cond(T) <= 2.0 + 1e-12
    W = np.vstack([Wtop, -V[k0:]])
    H = np.eye(n) - W @ np.linalg.solve(T, W.conj().T)
    np.testing.assert_allclose(H @ np.vstack([P, np.zeros((n - k0, k0))]), V, atol=1e-12)
    Qc, Rc = qf(A - V @ (V.conj().T @ A))
    np.testing.assert_allclose(Q, Qc, atol=1e-12)
    np.testing.assert_allclose(R, Rc, atol=1e-12)
    np.testing.assert_allclose(S, V.conj().T @ A, atol=1e-12)
