"""Entrywise parity with the oracle on the code paths that only run at large n,
and on the edge cases of the FP64-accurate emulated products.

* Large n: with about 2^12 leaves the widest TSQR levels have at least
  8 nodes per SM, where the downward pass runs one warp per node (a kernel the
  small parity cases never reach), and the streaming sweeps run the default
  split of two chunks per SM less one.  Real n = 2^20, k0 = 64, k = 16 (the
  differentiation workload's inputs) and complex n = 2^19, k0 = 128, k = 32
  (the shapes of the headline workload), A ~ N(0,1): Q, R, S against the
  oracle entry by entry at 1e-11, in FP64 arithmetic and with the emulated
  products, plus R upper triangular with a real nonnegative diagonal.
* The worked example of eq. (badbcg) with the emulated products (entries of
  1e-30 beside 1).
* Rows graded over 12 decades inside every leaf and every row chunk (the
  emulated products cut each value to 56-bit fixed point relative to the
  largest entry of its column in the chunk): entrywise at 1e-11 and the
  normwise bounds.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_metrics import assert_r_triangular, loo, resid_fro
from paper_2602_14449_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_Q = 1e-11
TOL_LOO = 1e-13
PRECS = ["THO_PREC_FP64", "THO_PREC_FP64_EMU"]

_cache = {}


@pytest.fixture(scope="module")
def tho():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_14449_gb300 import tho as _tho
    _tho.load()
    return _tho


def _problem(name):
    if name not in _cache:
        if name == "real_2^20":
            p = inputs.config_problem(5)
        elif name == "complex_2^19":
            p = inputs.random_problem(1 << 19, 128, 32, dtype=torch.complex128, seed=1455)
        elif name == "graded_real":
            p = inputs.graded_problem(1 << 18, 32, 16, dtype=torch.float64, seed=1456)
        elif name == "graded_complex":
            p = inputs.graded_problem(1 << 18, 32, 32, dtype=torch.complex128, seed=1457)
        else:
            raise KeyError(name)
        _cache[name] = (p, oracle.two_stage(p.V.numpy(), p.A.numpy()))
    return _cache[name]


def _check(tho, name, prec_name, wide_tree):
    p, (Qo, Ro, So) = _problem(name)
    prec = getattr(tho, prec_name)
    plan = tho.Plan([(p.n, p.k0, p.k)], p.A.dtype, prec, 0)
    if wide_tree:
        # The widest tree level must reach the one-warp-per-node downward pass.
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        nb = -(-(p.n - p.k0) // plan.leaf_rows)
        assert (nb + 1) // 2 >= 8 * sms, (nb, sms)
    V, A = p.V.cuda(), p.A.cuda()
    Q, R, S = tho.orth(V, A, prec=prec, plan=plan)
    torch.cuda.synchronize()
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q, rtol=0)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * max(1.0, np.abs(Ro).max()), rtol=0)
    np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL_Q * max(1.0, np.abs(So).max()), rtol=0)
    assert_r_triangular(R)
    assert loo(V, Q) < TOL_LOO
    assert resid_fro(V, A, Q, R, S) < TOL_LOO


@pytest.mark.parametrize("prec_name", PRECS)
def test_real_2p20_wide_tree(tho, prec_name):
    _check(tho, "real_2^20", prec_name, wide_tree=True)


@pytest.mark.parametrize("prec_name", PRECS)
def test_complex_2p19_wide_tree(tho, prec_name):
    _check(tho, "complex_2^19", prec_name, wide_tree=True)


@pytest.mark.parametrize("name", ["graded_real", "graded_complex"])
@pytest.mark.parametrize("prec_name", PRECS)
def test_rows_graded_over_12_decades(tho, name, prec_name):
    _check(tho, name, prec_name, wide_tree=False)


def test_worked_example_emulated(tho):
    """eq. (badbcg) with the emulated products: Q = [e3, e4], R = 1e-30 I, LOO ~ u."""
    from metrics import loo as loo_np
    V, A = inputs.worked_example()
    Q, R, S = tho.orth(V.cuda(), A.cuda(), prec=tho.THO_PREC_FP64_EMU)
    torch.cuda.synchronize()
    Qh = Q.cpu().numpy()
    np.testing.assert_allclose(Qh, np.array([[0, 0], [0, 0], [1, 0], [0, 1.0]]), atol=1e-15)
    np.testing.assert_allclose(R.cpu().numpy(), 1e-30 * np.eye(2), rtol=1e-14, atol=0)
    s = np.sqrt(2.0)
    np.testing.assert_allclose(S.cpu().numpy(), np.array([[0, 0], [s, s]]), atol=1e-15)
    assert loo_np(V.numpy(), Qh) < 1e-15
