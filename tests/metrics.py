"""Accuracy measures of Section 6 (test helpers, numpy/LAPACK only).

* loss of orthogonality ||[V,Q]^*[V,Q] - I||_2 (Table 1, Example 1),
* ||Q^*Q - I||_2 and ||V^*Q||_2 (Table 4 columns),
* relative residual ||[V,A] - [V,Q] [[I,S],[0,R]]||_F / ||[V,A]||_F (eq. vavq),
* the paper's ||A - V S - Q R||_2 / ||A||_2 (Table 4),
* qf(X): the library (LAPACK) QR with diag(R) made real >= 0, used as an
  independent closed-form pin.
"""
import numpy as np


def _h(x):
    return x.conj().T


def loo(V, Q):
    VQ = np.concatenate([V, Q], axis=1)
    return float(np.linalg.norm(_h(VQ) @ VQ - np.eye(VQ.shape[1]), 2))


def orth(Q):
    return float(np.linalg.norm(_h(Q) @ Q - np.eye(Q.shape[1]), 2))


def vq(V, Q):
    return float(np.linalg.norm(_h(V) @ Q, 2))


def resid_fro(V, A, Q, R, S):
    k0, k = V.shape[1], A.shape[1]
    top = np.concatenate([np.eye(k0), S], axis=1)
    bot = np.concatenate([np.zeros((k, k0)), R], axis=1)
    Rhat = np.concatenate([top, bot], axis=0)
    VA = np.concatenate([V, A], axis=1)
    VQ = np.concatenate([V, Q], axis=1)
    return float(np.linalg.norm(VA - VQ @ Rhat) / np.linalg.norm(VA))


def resid_paper(V, A, Q, R, S):
    return float(np.linalg.norm(A - V @ S - Q @ R, 2) / np.linalg.norm(A, 2))


def qf(X):
    """LAPACK Householder QR with diag(R) real and >= 0: returns (Q, R)."""
    q, r = np.linalg.qr(X, mode="reduced")
    d = np.diag(r).copy()
    ph = np.where(np.abs(d) == 0, 1.0, d / np.where(np.abs(d) == 0, 1.0, np.abs(d)))
    return q * ph[None, :], (np.conj(ph)[:, None] * r)
