"""The accuracy measures themselves, on the CPU.

tests/gpu_metrics.py checks the full-size GPU runs (chunked, pairwise-summed
Gram products in torch); tests/metrics.py checks the small ones (numpy/LAPACK).
Both must agree with each other and with values known in closed form."""
import numpy as np
import pytest
import torch

import gpu_metrics
import metrics


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_chunked_metrics_match_the_plain_ones(dtype, monkeypatch):
    monkeypatch.setattr(gpu_metrics, "CHUNK", 1000)  # several chunks and a ragged tail
    g = torch.Generator().manual_seed(4)
    n, k0, k = 4321, 7, 5
    X = torch.randn(n, k0 + k, dtype=torch.float64, generator=g)
    if dtype.is_complex:
        X = torch.complex(X, torch.randn(n, k0 + k, dtype=torch.float64, generator=g))
    Qf, _ = torch.linalg.qr(X)
    V, Q = Qf[:, :k0], Qf[:, k0:] * (1 + 1e-9)  # a known departure from orthonormality
    A = V @ torch.randn(k0, k, dtype=torch.float64, generator=g).to(dtype) + Q
    R = torch.eye(k, dtype=dtype) * (1 + 1e-8)  # residual -1e-8 Q: well above rounding
    S = (V.conj().T @ A)
    assert gpu_metrics.loo(V, Q) == pytest.approx(metrics.loo(V.numpy(), Q.numpy()), rel=1e-6)
    assert gpu_metrics.loo(V, Q) == pytest.approx(2e-9, rel=1e-3)  # (1 + e)^2 - 1 on the Q block
    np.testing.assert_allclose(gpu_metrics.gram(V, Q).numpy(), (V.conj().T @ Q).numpy(), atol=1e-14)
    r_gpu = gpu_metrics.resid_fro(V, A, Q, R, S)
    r_np = metrics.resid_fro(V.numpy(), A.numpy(), Q.numpy(), R.numpy(), S.numpy())
    assert r_gpu == pytest.approx(r_np, rel=1e-6)
    VA = torch.cat([V, A], dim=1)
    expect = 1e-8 * float(torch.linalg.norm(Q)) / float(torch.linalg.norm(VA))
    assert r_gpu == pytest.approx(expect, rel=1e-4)


def test_residual_of_an_exact_factorization_is_rounding_level():
    g = np.random.default_rng(1)
    X = g.standard_normal((500, 9))
    q, r = metrics.qf(X)
    assert (np.diag(r) >= 0).all()
    V, Q = q[:, :4], q[:, 4:]
    A = X[:, 4:]
    S, R = r[:4, 4:], r[4:, 4:]
    assert metrics.resid_fro(V, A, Q, R, S) < 1e-15
    assert metrics.resid_paper(V, A, Q, R, S) < 1e-15
    assert metrics.loo(V, Q) < 1e-14 and metrics.orth(Q) < 1e-14 and metrics.vq(V, Q) < 1e-14
