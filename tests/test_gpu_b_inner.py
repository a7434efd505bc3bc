"""Algorithm 4 (two-stage Householder QR in the B-inner product, Section 5)
on the device for a diagonal positive definite B, through tho_orth_b.

Against the oracle's Algorithm 4 (left-looking QR in the B-inner product with
Theorem 5's reflectors and reorthogonalization, on the dense B), entry by entry
at the parity tolerance, with the initial basis U = D^{-1/2} [I; 0] the method
builds from the Cholesky factor of B's leading block; kappa_2(B) = 1e2 and
Example 3's 1e5; both FP64-accurate modes; real and complex; k0 = 0 (the QR of
A in the B-inner product alone).  Also [V, Q]^* B [V, Q] = I and eq. (vavqb)
at the FP64 level, the residual in the B-norm.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_14449_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_Q = 1e-11


@pytest.fixture(scope="module")
def tho():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_14449_gb300 import tho as _tho
    _tho.load()
    return _tho


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("prec_name", ["THO_PREC_FP64", "THO_PREC_FP64_EMU"])
@pytest.mark.parametrize("n,k0,k,kappa", [(3000, 16, 8, 1e5), (2500, 64, 32, 1e2), (1500, 0, 12, 1e5), (777, 5, 3, 1e5)])
def test_algorithm4_diagonal_b_matches_oracle(tho, dtype, prec_name, n, k0, k, kappa):
    prec = getattr(tho, prec_name)
    p = inputs.diag_b_problem(n, k0, k, kappa_b=kappa, dtype=dtype, seed=1460 + n + k0)
    B, V, U, A = p.B.numpy(), p.V.numpy(), p.U.numpy(), p.A.numpy()
    Qo, Ro, So, _ = oracle.two_stage_b(B, V, U, A)
    Q, R, S = tho.orth_b(p.d.cuda(), p.V.cuda() if k0 else None, p.A.cuda(), prec=prec)
    torch.cuda.synchronize()
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    # Q's entries scale like d^{-1/2}; compare them in the B-weighted rows.
    sd = np.sqrt(p.d.numpy())[:, None]
    np.testing.assert_allclose(sd * Qh, sd * Qo, atol=TOL_Q, rtol=0)
    np.testing.assert_allclose(Rh, Ro, atol=TOL_Q * max(1.0, np.abs(Ro).max()), rtol=0)
    if k0:
        np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL_Q * max(1.0, np.abs(So).max()), rtol=0)
    VQ = np.concatenate([V, Qh], axis=1) if k0 else Qh
    G = VQ.conj().T @ (p.d.numpy()[:, None] * VQ)
    assert np.linalg.norm(G - np.eye(k0 + k), 2) < 1e-13
    # eq. (vavqb), measured in the B-norm of the setting (Section 5).
    Sh = S.cpu().numpy() if k0 else np.zeros((0, k))
    res = A - (V @ Sh if k0 else 0) - Qh @ Rh
    assert np.linalg.norm(sd * res) / np.linalg.norm(sd * A) < 1e-13


def test_algorithm4_rejects_a_non_positive_weight(tho):
    p = inputs.diag_b_problem(1000, 8, 4, seed=3)
    d = p.d.clone()
    d[17] = -1.0
    plan = tho.Plan([(1000, 8, 4)], torch.float64)
    tho.orth_b(d.cuda(), p.V.cuda(), p.A.cuda(), plan=plan)
    torch.cuda.synchronize()
    assert plan.status() == tho.THO_ERR_NONFINITE
