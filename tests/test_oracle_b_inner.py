"""Pins of the oracle's Algorithm 4 (two-stage Householder-QR in the B-inner
product, Section 5), on the CPU.

* With B = I and U = [I; 0] the method is Algorithm 1 itself: same Q, R, S.
* For a Hermitian positive definite B the result is the unique B-orthogonal QR
  of (I - V V^* B) A with diag(R) real >= 0 (written out with a library
  Cholesky factorization), S = V^* B A, [V, Q]^* B [V, Q] = I and eq. (vavqb).
* Theorem 5: the reflector H = I - W T^{-1} W^* B of the first stage maps
  X = U_1 P onto Y = V and satisfies H^* B H = B.
* Rank-deficient and zero columns keep [V, Q] B-orthonormal.
Example 3's kappa(B) = 1e5 is among the cases (its matrices are not available).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_14449_gb300 import inputs


def _h(M):
    return M.conj().T


def _np(p):
    return p.B.numpy(), p.V.numpy(), p.U.numpy(), p.A.numpy()


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_identity_inner_product_is_algorithm_1(dtype):
    q = inputs.random_problem(300, 12, 7, dtype=dtype, seed=3)
    V, A = q.V.numpy(), q.A.numpy()
    U = np.eye(300, 19, dtype=V.dtype)
    Q4, R4, S4, _ = oracle.two_stage_b(np.eye(300, dtype=V.dtype), V, U, A)
    Q1, R1, S1 = oracle.two_stage(V, A)
    np.testing.assert_allclose(Q4, Q1, atol=1e-13, rtol=0)
    np.testing.assert_allclose(R4, R1, atol=1e-13 * np.abs(R1).max(), rtol=0)
    np.testing.assert_allclose(S4, S1, atol=1e-13 * np.abs(S1).max(), rtol=0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("kappa_b", [1e2, 1e5])
def test_closed_form_and_invariants(dtype, kappa_b):
    B, V, U, A = _np(inputs.b_inner_problem(400, 16, 8, kappa_b, dtype, seed=5))
    n, k0, k = 400, 16, 8
    Q, R, S, aux = oracle.two_stage_b(B, V, U, A)
    # Closed form: A' = (I - V V^* B) A = Q R with Q^* B Q = I and diag(R) > 0.
    Ap = A - V @ (_h(V) @ B @ A)
    Rc = _h(np.linalg.cholesky(_h(Ap) @ B @ Ap))
    Qc = np.linalg.solve(_h(Rc), _h(Ap)).conj().T  # Ap Rc^{-1}
    np.testing.assert_allclose(Q, Qc, atol=1e-12, rtol=0)
    np.testing.assert_allclose(R, Rc, atol=1e-12 * np.abs(Rc).max(), rtol=0)
    np.testing.assert_allclose(S, _h(V) @ B @ A, atol=1e-12 * np.abs(S).max(), rtol=0)
    assert np.allclose(np.tril(R, -1), 0) and (np.diag(R).real > 0).all() and np.allclose(np.diag(R).imag, 0)
    VQ = np.concatenate([V, Q], axis=1)
    assert np.linalg.norm(_h(VQ) @ B @ VQ - np.eye(k0 + k), 2) < 1e-13
    Rhat = np.block([[np.eye(k0), S], [np.zeros((k, k0)), R]])
    assert np.linalg.norm(np.concatenate([V, A], 1) - VQ @ Rhat) / np.linalg.norm(np.concatenate([V, A], 1)) < 1e-14
    # Theorem 5 for the first stage's reflector.
    H = np.eye(n) - aux["W"] @ np.linalg.solve(aux["T"], _h(aux["W"]) @ B)
    assert np.abs(H @ aux["U1P"] - V).max() < 1e-13
    assert np.linalg.norm(_h(H) @ B @ H - B, 2) / np.linalg.norm(B, 2) < 1e-13
    # The second choice of P (Section 3.2): T = I + R1^*, lower triangular with diag >= 1.
    T = aux["T"]
    assert np.abs(np.triu(T, 1)).max() < 1e-13 and (np.diag(T).real >= 1 - 1e-13).all()


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_rank_deficient_and_zero_columns(dtype):
    B, V, U, A = _np(inputs.b_inner_problem(400, 16, 8, 1e2, dtype, seed=6))
    A[:, 3] = 2 * A[:, 1] - A[:, 0] + V @ np.arange(16.0)  # in the span of V and earlier columns
    A[:, 6] = 0
    Q, R, S, _ = oracle.two_stage_b(B, V, U, A)
    assert abs(R[3, 3]) < 1e-12 * np.abs(R).max() and R[6, 6] == 0
    VQ = np.concatenate([V, Q], axis=1)
    assert np.linalg.norm(_h(VQ) @ B @ VQ - np.eye(24), 2) < 1e-13
    assert np.linalg.norm(A - V @ S - Q @ R) / np.linalg.norm(A) < 1e-14


def _krylov_blocks(n, k, nb, dtype, seed):
    """Block-Krylov stand-in: A_{i+1} = D A_i with a spread diagonal D, so the
    whole A is numerically rank deficient (cond > 1e14)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, k))
    if dtype.is_complex:
        X = X + 1j * rng.standard_normal((n, k))
    d = np.exp(np.linspace(0.0, 5.0, n))
    blocks = [X]
    for _ in range(nb - 1):
        blocks.append(d[:, None] * blocks[-1])
    return np.hstack(blocks)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_block_form_is_the_b_orthogonal_qr(dtype):
    """Algorithm 3 in the B-inner product on a full-rank A: the unique QR with
    Q^* B Q = I and diag(R) real > 0 (closed form by a library Cholesky)."""
    B = inputs.b_inner_problem(500, 1, 1, 1e2, dtype, seed=13).B.numpy()
    rng = np.random.default_rng(14)
    A = rng.standard_normal((500, 24)) + (1j * rng.standard_normal((500, 24)) if dtype.is_complex else 0)
    Q, R = oracle.block_hhqr_b(B, A, [5, 8, 11])
    Rc = _h(np.linalg.cholesky(_h(A) @ B @ A))
    np.testing.assert_allclose(R, Rc, atol=1e-12 * np.abs(Rc).max(), rtol=0)
    np.testing.assert_allclose(Q, np.linalg.solve(_h(Rc), _h(A)).conj().T, atol=1e-12, rtol=0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_example3_structure_keeps_b_orthogonality(dtype):
    """Example 3's setting (kappa_2(B) = 1e5, blocks of 10 columns) on an
    ill-conditioned block-Krylov stand-in: ||Q^* B Q - I||_2 and the residual
    stay below 10x Table 3's second-choice figures."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table3_b_inner.json")))
    B = inputs.b_inner_problem(1000, 1, 1, gold["kappa2_B"], dtype, seed=12).B.numpy()
    assert np.linalg.cond(B) == pytest.approx(gold["kappa2_B"], rel=1e-3)
    A = _krylov_blocks(1000, 10, 8, dtype, seed=3)
    assert np.linalg.cond(A) > 1e14
    Q, R = oracle.block_hhqr_b(B, A, [10] * 8)
    worst = max(gold["second_choice"].values(), key=lambda r: r["loo_B"])
    assert np.linalg.norm(_h(Q) @ B @ Q - np.eye(80), 2) < 10 * worst["loo_B"]
    assert np.linalg.norm(A - Q @ R, 2) / np.linalg.norm(A, 2) < 10 * worst["resid"]
    assert np.abs(np.tril(R, -1)).max() == 0
