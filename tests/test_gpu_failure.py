"""Device-side failure detection without a GPU fault.

The tcgen05 kernels never wait without a bound: a wait that runs out makes the
kernel leave its loop, latch THO_ERR_TIMEOUT in the plan's status word and
return.  tho_plan_expire_wait runs that same bounded wait, cut short, on an
mbarrier that nothing completes; the host must read THO_ERR_TIMEOUT through
tho_plan_status, and the context must stay usable for the next calls.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_14449_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tho():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_14449_gb300 import tho as _tho
    _tho.load()
    return _tho


@pytest.mark.parametrize("spins", [1, 4096, 1 << 16])
def test_expired_wait_is_reported_and_the_context_stays_usable(tho, spins):
    n, k0, k = 5000, 16, 8
    p = inputs.random_problem(n, k0, k, dtype=torch.float64, seed=5)
    V, A = p.V.cuda(), p.A.cuda()
    emu = tho.THO_PREC_FP64_EMU
    plan = tho.Plan([(n, k0, k)], torch.float64, emu)
    assert plan.status() == tho.THO_OK
    plan.expire_wait(spins)
    assert plan.status() == tho.THO_ERR_TIMEOUT
    assert plan.status() == tho.THO_OK  # reading clears the word
    # The same plan (tcgen05 Gram and updates) still gives the oracle's result,
    # also with an expired wait queued between two calls on the stream.
    Qo, Ro, So = oracle.two_stage(p.V.numpy(), p.A.numpy())
    for _ in range(2):
        Q, R, S = tho.orth(V, A, prec=emu, plan=plan)
        plan.expire_wait(spins)
        torch.cuda.synchronize()
        np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=1e-11, rtol=0)
        assert plan.status() == tho.THO_ERR_TIMEOUT
    Q, R, S = tho.orth(V, A, prec=emu, plan=plan)
    torch.cuda.synchronize()
    assert plan.status() == tho.THO_OK
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=1e-11, rtol=0)


def test_expire_wait_bounds(tho):
    plan = tho.Plan([(300, 4, 4)], torch.float64, tho.THO_PREC_FP64)
    lib = tho.load()
    for bad in (0, -5, (1 << 20) + 1):
        assert lib.tho_plan_expire_wait(plan.handle, bad, None) == tho.THO_ERR_ARG
    assert plan.status() == tho.THO_OK


def test_injected_allocation_failure_leaves_the_library_usable(tho, monkeypatch):
    monkeypatch.setenv("THO_INJECT_NOMEM", "1")
    with pytest.raises(tho.ThoError) as e:
        tho.Plan([(4096, 16, 4)], torch.float64, tho.THO_PREC_FP64)
    assert e.value.code == tho.THO_ERR_NOMEM
    monkeypatch.setenv("THO_INJECT_NOMEM", "0")
    plan = tho.Plan([(4096, 16, 4)], torch.float64, tho.THO_PREC_FP64)
    p = inputs.random_problem(4096, 16, 4, dtype=torch.float64, seed=9)
    Q, _, _ = tho.orth(p.V.cuda(), p.A.cuda(), plan=plan)
    torch.cuda.synchronize()
    Qo, _, _ = oracle.two_stage(p.V.numpy(), p.A.numpy())
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=1e-11, rtol=0)


def test_log_prints_the_plan_choices(tho, monkeypatch, capfd):
    monkeypatch.setenv("THO_LOG", "1")
    plan = tho.Plan([(20000, 64, 32)], torch.complex128, tho.THO_PREC_FP64_EMU, tuning=(128, 77))
    err = capfd.readouterr().err
    line = [x for x in err.splitlines() if x.startswith("[tho] plan:")][-1]
    assert "leaf_rows=128" in line and "split_chunks=77" in line and "dtype=c128" in line
    assert f"launches={plan.kernel_launches}" in line
    assert "leaf=k_leaf_emu" in line  # complex k >= 24 in the emulated mode
