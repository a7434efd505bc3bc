"""Algorithm 1 with a given P, and Example 5 / Figure 1 of Section 6.

oracle.two_stage_given_p runs Algorithm 1 for any unitary P.  It is pinned to
the three choices of P (Section 3.2), each of which has its own oracle function
pinned elsewhere: given their P it must return their Q, R and S.

Example 5 builds (V, P) pairs for a prescribed kappa_2(T) and shows (Figure 1,
whose data the paper text does not carry) that the errors grow as the rounding
error analysis predicts; the remark after Theorem 4 states the prediction:
||Q^*Q - I||_2 = O(kappa_2(T) u), ||V^*Q||_2 = O(sqrt(kappa_2(T)) u) and the
relative residual = O(kappa_2(T) u).  The test checks those three laws over
twelve orders of magnitude of kappa_2(T), from both sides: each ratio to its
prediction stays between 0.2 and 100 once the amplified term dominates.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_14449_gb300 import inputs

U_ROUND = 2.0 ** -53


@pytest.mark.parametrize("dtype", ["float64", "complex128"])
def test_given_p_reproduces_the_three_choices(dtype):
    import torch
    p = inputs.random_problem(600, 20, 8, dtype=getattr(torch, dtype), seed=21)
    V, A = p.V.numpy(), p.A.numpy()
    Q2, R2, S2, aux2 = oracle.two_stage(V, A, return_aux=True)
    Q1, R1, S1, aux1 = oracle.two_stage_mlu(V, A)
    Q3, R3, S3, aux3 = oracle.two_stage_polar(V, A)
    for (Q, R, S), P in (((Q2, R2, S2), -aux2["Q1"]), ((Q1, R1, S1), aux1["P"]), ((Q3, R3, S3), aux3["P"])):
        Qg, Rg, Sg, _ = oracle.two_stage_given_p(V, A, P)
        np.testing.assert_allclose(Qg, Q, atol=1e-12, rtol=0)
        np.testing.assert_allclose(Rg, R, atol=1e-12 * np.abs(R).max(), rtol=0)
        np.testing.assert_allclose(Sg, S, atol=1e-12 * np.abs(S).max(), rtol=0)


def _pair(n, k0, kappa, rng):
    """(V, P) with V^T V = I and T = I - V_1^T P of 2-norm condition number
    kappa: V_1 = Qa diag(sigma) Qb^T and P = Qa Qb^T give T = Qb diag(1 - sigma) Qb^T;
    the 1 - sigma_i run geometrically from 1 to 1/kappa, and
    V_2 = Y diag(sqrt(1 - sigma^2)) Qb^T completes the orthonormal columns."""
    Qa = np.linalg.qr(rng.standard_normal((k0, k0)))[0]
    Qb = np.linalg.qr(rng.standard_normal((k0, k0)))[0]
    sigma = 1.0 - np.logspace(0.0, -math.log10(kappa), k0)
    Y = np.linalg.qr(rng.standard_normal((n - k0, k0)))[0]
    V = np.vstack([Qa @ np.diag(sigma) @ Qb.T, Y @ np.diag(np.sqrt(1.0 - sigma ** 2)) @ Qb.T])
    return V, Qa @ Qb.T


@pytest.mark.parametrize("seed", [5, 6])
def test_figure1_errors_follow_kappa_of_T(seed):
    rng = np.random.default_rng(seed)
    n, k0, k = 1000, 100, 100  # the sizes of Example 5
    A = rng.standard_normal((n, k))
    for kappa in (1.0, 1e3, 1e6, 1e9, 1e12):
        V, P = _pair(n, k0, kappa, rng)
        assert np.linalg.norm(V.T @ V - np.eye(k0), 2) < 1e-14
        Q, R, S, aux = oracle.two_stage_given_p(V, A, P)
        assert abs(np.linalg.cond(aux["T"]) / kappa - 1) < 1e-3
        loo = np.linalg.norm(Q.T @ Q - np.eye(k), 2) / (kappa * U_ROUND)
        vq = np.linalg.norm(V.T @ Q, 2) / (math.sqrt(kappa) * U_ROUND)
        res = np.linalg.norm(A - V @ S - Q @ R, 2) / np.linalg.norm(A, 2) / (kappa * U_ROUND)
        for ratio in (loo, vq, res):
            assert ratio < 100, (kappa, loo, vq, res)
            if kappa >= 1e3:
                assert ratio > 0.2, (kappa, loo, vq, res)
