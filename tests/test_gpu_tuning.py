"""Tuned plans and the autotuner on the GPU, through the C ABI.

Every partition a tuned plan can take (TSQR leaf height, split-n factor) must
give the oracle's result to the parity tolerance: the partition changes only
the order of the partial sums.  The autotuner must return a partition that
plans accept, record it in its cache and answer from the cache the second time.
"""
import json

import numpy as np
import pytest
import torch

import oracle
from metrics import loo as loo_np
from paper_2602_14449_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_Q = 1e-11
TOL_LOO = 1e-13


@pytest.fixture(scope="module")
def tho():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_14449_gb300 import tho as _tho
    _tho.load()
    return _tho


@pytest.fixture(scope="module")
def sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


_ORACLE = {}


def _oracle(p, key):
    if key not in _ORACLE:
        _ORACLE[key] = oracle.two_stage(p.V.numpy(), p.A.numpy())
    return _ORACLE[key]


CASES = [  # (dtype, precision name, n, k0, k)
    (torch.float64, "THO_PREC_FP64", 20000, 32, 8),
    (torch.float64, "THO_PREC_FP64_EMU", 30000, 64, 16),
    (torch.complex128, "THO_PREC_FP64", 9000, 16, 12),
    (torch.complex128, "THO_PREC_FP64_EMU", 40000, 64, 32),  # tensor-core leaf QR (k >= 24)
    (torch.float64, "THO_PREC_FP64_EMU", 3 * 256 + 17, 7, 30),
]


@pytest.mark.parametrize("dtype,prec_name,n,k0,k", CASES)
def test_tuned_plans_match_oracle(tho, sms, dtype, prec_name, n, k0, k):
    prec = getattr(tho, prec_name)
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=900 + n + k0 + k)
    Qo, Ro, So = _oracle(p, (dtype, n, k0, k))
    V, A = p.V.cuda(), p.A.cuda()
    ran = 0
    for leaf in (64, 128, 256):
        for split in (1, sms // 2, 4 * sms, 16 * sms):
            try:
                plan = tho.Plan([(n, k0, k)], dtype, prec, tuning=(leaf, split))
            except tho.ThoError as e:
                assert e.code == tho.THO_ERR_UNSUPPORTED, (leaf, split, e)
                continue
            assert plan.tuning == (leaf, split, 0)
            assert plan.leaf_rows == leaf
            Q, R, S = tho.orth(V, A, prec=prec, plan=plan)
            torch.cuda.synchronize()
            assert plan.status() == tho.THO_OK
            Q = Q.cpu().numpy()
            np.testing.assert_allclose(Q, Qo, atol=TOL_Q, rtol=0, err_msg=f"leaf {leaf} split {split}")
            np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * max(1.0, np.abs(Ro).max()), rtol=0)
            np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL_Q * max(1.0, np.abs(So).max()), rtol=0)
            assert loo_np(p.V.numpy(), Q) < TOL_LOO
            plan.close()
            ran += 1
    assert ran >= 4  # at least the default-sized panels at every split


BATCH_SHAPES = [(300, 8, 4), (1000, 16, 8), (5000, 32, 16), (777, 1, 1), (4096, 64, 32), (2000, 128, 8),
                (50000, 16, 4), (33, 16, 17), (70001, 5, 9)]


@pytest.mark.parametrize("prec_name", ["THO_PREC_FP64", "THO_PREC_FP64_EMU"])
def test_tuned_batch_matches_oracle(tho, sms, prec_name):
    prec = getattr(tho, prec_name)
    probs = [inputs.random_problem(n, k0, k, dtype=torch.float64, seed=300 + i)
             for i, (n, k0, k) in enumerate(BATCH_SHAPES)]
    pairs = [(p.V.cuda(), p.A.cuda()) for p in probs]
    ref = [_oracle(p, ("batch", i)) for i, p in enumerate(probs)]
    for tuning in ((64, len(BATCH_SHAPES), 0), (128, sms, 1), (0, 32 * sms, 1), (0, 0, 1)):
        plan = tho.Plan(BATCH_SHAPES, torch.float64, prec, tuning=tuning)
        res = tho.orth_batched(pairs, prec=prec, plan=plan)
        torch.cuda.synchronize()
        for (Qo, Ro, So), (Q, R, S) in zip(ref, res):
            np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q, err_msg=str(tuning))
            np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * max(1, np.abs(Ro).max()))
            np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL_Q * max(1, np.abs(So).max()))
        plan.close()


def test_autotune_single_problem_and_cache(tho, tmp_path):
    shape, dtype, prec = (1 << 18, 64, 16), torch.float64, tho.THO_PREC_FP64_EMU
    cache = str(tmp_path / "tune.jsonl")
    t, ms = tho.autotune([shape], dtype, prec, cache=cache)
    assert ms > 0
    plan = tho.Plan([shape], dtype, prec, tuning=t)
    assert plan.tuning == t
    rows = [json.loads(line) for line in open(cache)]
    name = torch.cuda.get_device_name(0)
    assert len(rows) == 1 and rows[0]["key"] == tho.tune_key([shape], dtype, prec, 0, name)
    assert (rows[0]["leaf_rows"], rows[0]["split_chunks"], rows[0]["balance"]) == t
    # The tuned plan computes what the default plan computes.
    p = inputs.random_problem(*shape, dtype=dtype, seed=77)
    V, A = p.V.cuda(), p.A.cuda()
    Qd, Rd, Sd = tho.orth(V, A, prec=prec)
    Qt, Rt, St = tho.orth(V, A, prec=prec, plan=plan)
    torch.cuda.synchronize()
    assert float((Qt - Qd).abs().max()) <= TOL_Q
    assert float((Rt - Rd).abs().max()) <= TOL_Q * max(1.0, float(Rd.abs().max()))
    # Second call: answered from the cache (ms stored with 6 decimals), nothing appended.
    t2, ms2 = tho.autotune([shape], dtype, prec, cache=cache)
    assert t2 == t and ms2 == pytest.approx(ms, abs=1e-6)
    assert len(open(cache).readlines()) == 1


def test_autotune_batch_via_environment(tho, tmp_path, monkeypatch):
    cache = str(tmp_path / "env.jsonl")
    monkeypatch.setenv("THO_TUNE_CACHE", cache)
    t, ms = tho.autotune(BATCH_SHAPES, torch.float64, tho.THO_PREC_FP64)
    assert ms > 0 and len(open(cache).readlines()) == 1
    probs = [inputs.random_problem(n, k0, k, dtype=torch.float64, seed=300 + i)
             for i, (n, k0, k) in enumerate(BATCH_SHAPES)]
    pairs = [(p.V.cuda(), p.A.cuda()) for p in probs]
    plan = tho.Plan(BATCH_SHAPES, torch.float64, tho.THO_PREC_FP64, tuning=t)
    res = tho.orth_batched(pairs, plan=plan)
    torch.cuda.synchronize()
    for i, (p, (Q, R, S)) in enumerate(zip(probs, res)):
        Qo, Ro, So = _oracle(p, ("batch", i))
        np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q)
