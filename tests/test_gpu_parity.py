"""CUDA path against the CPU oracle (through the C ABI), element by element.

Tolerances: entrywise |Q - Q_oracle| <= 1e-11 on well-conditioned inputs, loss
of orthogonality and relative residual <= 1e-13 in FP64 (the bounds stated for
the method), <= 1e-5 loss of orthogonality for the FP32-bulk variant.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_metrics import assert_r_triangular
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


def _run(tho, p, prec=0):
    dev = torch.device("cuda")
    V = p.V.to(dev)
    A = p.A.to(dev)
    Q, R, S = tho.orth(V, A, prec=prec)
    torch.cuda.synchronize()
    return Q.cpu().numpy(), R.cpu().numpy(), (S.cpu().numpy() if S is not None else None)


def _cmp(tho, p, tol=TOL_Q):
    Q, R, S = _run(tho, p)
    Qo, Ro, So = oracle.two_stage(p.V.numpy(), p.A.numpy())
    np.testing.assert_allclose(Q, Qo, atol=tol, rtol=0)
    np.testing.assert_allclose(R, Ro, atol=tol * max(1.0, np.abs(Ro).max()), rtol=0)
    if p.k0:
        np.testing.assert_allclose(S, So, atol=tol * max(1.0, np.abs(So).max()), rtol=0)
    assert loo_np(p.V.numpy(), Q) < TOL_LOO
    return Q


def test_config1_full_size(tho):
    """real FP64, n=4096, k0=16, k=4 (C1), entrywise against the oracle."""
    _cmp(tho, inputs.config_problem(1))


def test_worked_example(tho):
    """eq. (badbcg): Q = [e3, e4] and LOO ~ u on the GPU too (Example 1)."""
    V, A = inputs.worked_example()
    dev = torch.device("cuda")
    Q, R, S = tho.orth(V.to(dev), A.to(dev))
    Q = Q.cpu().numpy()
    np.testing.assert_allclose(Q, np.array([[0, 0], [0, 0], [1, 0], [0, 1.0]]), atol=1e-15)
    np.testing.assert_allclose(R.cpu().numpy(), 1e-30 * np.eye(2), rtol=1e-14, atol=0)
    assert loo_np(V.numpy(), Q) < 1e-15


SHAPES = [
    (64, 1, 1), (33, 16, 17), (97, 8, 4), (1000, 7, 3), (4095, 16, 4), (5000, 32, 32),
    (12345, 64, 16), (40000, 128, 32), (70001, 5, 9), (3 * 256 + 17, 64, 30),
]


@pytest.mark.parametrize("n,k0,k", SHAPES)
def test_random_real(tho, n, k0, k):
    _cmp(tho, inputs.random_problem(n, k0, k, dtype=torch.float64, seed=n + 7 * k0 + 31 * k))


@pytest.mark.parametrize("n,k0,k", [(64, 1, 1), (300, 8, 5), (5000, 32, 32), (20001, 128, 32), (777, 13, 2)])
def test_random_complex(tho, n, k0, k):
    _cmp(tho, inputs.random_problem(n, k0, k, dtype=torch.complex128, seed=n + k0 + k))


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_k0_zero_is_householder_qr(tho, dtype):
    p = inputs.random_problem(3000, 0, 8, dtype=dtype, seed=2)
    dev = torch.device("cuda")
    A = p.A.to(dev)
    V = torch.zeros((3000, 0), dtype=dtype, device=dev)
    Q, R, _ = tho.orth(V, A)
    Qo, Ro = oracle.householder_qr(p.A.numpy())
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * np.abs(Ro).max())


def test_minimal_rows(tho):
    """n = k0 + k: a single leaf holding exactly k rows."""
    _cmp(tho, inputs.random_problem(48, 16, 32, seed=4))


def test_deterministic(tho):
    p = inputs.random_problem(50000, 32, 8, seed=8)
    a = _run(tho, p)[0]
    b = _run(tho, p)[0]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_rank_deficient_small(tho, dtype):
    """C3 structure (half of A in Range(V) + 1e-14 noise), oracle-size: invariants."""
    from gpu_metrics import loo, resid_fro
    p = inputs.config_problem(3, n=20000, dtype=dtype)
    dev = torch.device("cuda")
    V, A = p.V.to(dev), p.A.to(dev)
    Q, R, S = tho.orth(V, A)
    assert loo(V, Q) < TOL_LOO
    assert resid_fro(V, A, Q, R, S) < TOL_LOO


def test_config2_full_size(tho):
    """C2: n=2^20, k0=64, k=16, cond([V,A]) ~ 1e10: LOO and residual <= 1e-13;
    S = V^*A matches the oracle (Q itself is only defined to ~u*cond)."""
    from gpu_metrics import loo, resid_fro
    p = inputs.config_problem(2, device="cuda")
    Q, R, S = tho.orth(p.V, p.A)
    assert loo(p.V, Q) < TOL_LOO
    assert resid_fro(p.V, p.A, Q, R, S) < TOL_LOO
    assert_r_triangular(R)
    Sref = (p.V.conj().T @ p.A)
    assert float((S - Sref).abs().max()) < 1e-12 * float(Sref.abs().max())


def test_config3_full_size_fp64(tho):
    """C3: complex128, n=2^22, k0=128, k=32, numerically rank deficient."""
    from gpu_metrics import loo, resid_fro
    p = inputs.config_problem(3, device="cuda")
    Q, R, S = tho.orth(p.V, p.A)
    assert loo(p.V, Q) < TOL_LOO
    assert resid_fro(p.V, p.A, Q, R, S) < TOL_LOO
    assert_r_triangular(R)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_fp32_bulk_variant(tho, dtype):
    """FP32-bulk: loss of orthogonality <= 1e-5 against the FP64 oracle's bound."""
    p = inputs.random_problem(30000, 32, 16, dtype=dtype, seed=12)
    Q, R, S = _run(tho, p, prec=tho.THO_PREC_FP32_BULK)
    Qo, _, _ = oracle.two_stage(p.V.numpy(), p.A.numpy())
    assert loo_np(p.V.numpy(), Q) < 1e-5
    assert np.abs(Q - Qo).max() < 1e-3


def test_interleaved_plans(tho):
    """A plan built after another (smaller panels) must not break the first one."""
    big = inputs.random_problem(9000, 128, 32, dtype=torch.complex128, seed=21)
    small = inputs.random_problem(600, 8, 4, seed=22)
    dev = torch.device("cuda")
    Vb, Ab = big.V.to(dev), big.A.to(dev)
    Qb1, _, _ = tho.orth(Vb, Ab)
    Qs, _, _ = tho.orth(small.V.to(dev), small.A.to(dev))
    Qb2, _, _ = tho.orth(Vb, Ab)
    torch.cuda.synchronize()
    assert torch.equal(Qb1, Qb2)
    Qso, _, _ = oracle.two_stage(small.V.numpy(), small.A.numpy())
    np.testing.assert_allclose(Qs.cpu().numpy(), Qso, atol=TOL_Q)


BATCH_SHAPES = [(300, 8, 4), (1000, 16, 8), (5000, 32, 16), (777, 1, 1), (4096, 64, 32), (2000, 128, 8),
                (50000, 16, 4), (33, 16, 17), (70001, 5, 9)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_batched_matches_oracle(tho, dtype):
    """tho_orth_batched (one graph replay for the whole batch) against the oracle, per problem."""
    probs = [inputs.random_problem(n, k0, k, dtype=dtype, seed=40 + i) for i, (n, k0, k) in enumerate(BATCH_SHAPES)]
    pairs = [(p.V.cuda(), p.A.cuda()) for p in probs]
    res = tho.orth_batched(pairs)
    torch.cuda.synchronize()
    for p, (Q, R, S) in zip(probs, res):
        Qo, Ro, So = oracle.two_stage(p.V.numpy(), p.A.numpy())
        np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q)
        np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * max(1, np.abs(Ro).max()))
        np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL_Q * max(1, np.abs(So).max()))
    # A second call replays the same graph with new output buffers: same bits.
    res2 = tho.orth_batched(pairs)
    torch.cuda.synchronize()
    for (Q, _, _), (Q2, _, _) in zip(res, res2):
        assert torch.equal(Q, Q2)


@pytest.mark.parametrize("prec_name", ["THO_PREC_FP64", "THO_PREC_FP64_EMU"])
def test_batched_c4_workload(tho, prec_name):
    """The 256-problem batched workload (n log-uniform in [16384, 262144]), in
    both FP64-accurate modes: every problem meets LOO and residual <= 1e-13 and
    matches the looped tho_orth."""
    from gpu_metrics import loo, resid_fro
    prec = getattr(tho, prec_name)
    shapes = inputs.batched_shapes()
    probs = inputs.batched_problems(shapes, device="cuda")
    pairs = [(p.V, p.A) for p in probs]
    res = tho.orth_batched(pairs, prec=prec)
    torch.cuda.synchronize()
    worst = 0.0
    for i, (p, (Q, R, S)) in enumerate(zip(probs, res)):
        assert loo(p.V, Q) < TOL_LOO, i
        assert resid_fro(p.V, p.A, Q, R, S) < TOL_LOO, i
        assert_r_triangular(R)
        if i % 16 == 0:
            Ql, _, _ = tho.orth(p.V, p.A, prec=prec)
            worst = max(worst, float((Ql - Q).abs().max()))
    assert worst < TOL_Q


# --- FP64-accurate emulated products (bf16 tensor cores): same tolerances as FP64 ---

@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("n,k0,k", [(4096, 16, 4), (33, 16, 17), (12345, 64, 16), (40000, 128, 32), (3 * 256 + 17, 7, 30)])
def test_emulated_matches_oracle(tho, dtype, n, k0, k):
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=n + 3 * k0 + k)
    Q, R, S = _run(tho, p, prec=tho.THO_PREC_FP64_EMU)
    Qo, Ro, So = oracle.two_stage(p.V.numpy(), p.A.numpy())
    np.testing.assert_allclose(Q, Qo, atol=TOL_Q, rtol=0)
    np.testing.assert_allclose(R, Ro, atol=TOL_Q * max(1.0, np.abs(Ro).max()), rtol=0)
    np.testing.assert_allclose(S, So, atol=TOL_Q * max(1.0, np.abs(So).max()), rtol=0)
    assert loo_np(p.V.numpy(), Q) < TOL_LOO


@pytest.mark.parametrize("cid", [2, 3])
def test_emulated_full_size(tho, cid):
    """C2 (cond 1e10) and C3 (rank deficient) at full size: LOO, residual <= 1e-13."""
    from gpu_metrics import loo, resid_fro
    p = inputs.config_problem(cid, device="cuda")
    Q, R, S = tho.orth(p.V, p.A, prec=tho.THO_PREC_FP64_EMU)
    assert loo(p.V, Q) < TOL_LOO
    assert resid_fro(p.V, p.A, Q, R, S) < TOL_LOO
    assert_r_triangular(R)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_emulated_k0_zero(tho, dtype):
    """k0 = 0 in the emulated mode: the leaf QR reads A itself (complex k = 32 takes
    the tensor-core trailing updates) and the apply forms Q from the compact WY form."""
    n, k = 5000, 32
    p = inputs.random_problem(n, 0, k, dtype=dtype, seed=12)
    A = p.A.cuda()
    V = torch.zeros((n, 0), dtype=dtype, device="cuda")
    Q, R, _ = tho.orth(V, A, prec=tho.THO_PREC_FP64_EMU)
    Qo, Ro = oracle.householder_qr(p.A.numpy())
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * np.abs(Ro).max())


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
def test_emulated_batched_matches_oracle(tho, dtype):
    """Batched plans in the emulated mode (mixed k0 and k in one graph: tcgen05 Gram and
    update per instance, one leaf kernel for all) against the oracle, per problem."""
    probs = [inputs.random_problem(n, k0, k, dtype=dtype, seed=60 + i) for i, (n, k0, k) in enumerate(BATCH_SHAPES)]
    pairs = [(p.V.cuda(), p.A.cuda()) for p in probs]
    res = tho.orth_batched(pairs, prec=tho.THO_PREC_FP64_EMU)
    torch.cuda.synchronize()
    for p, (Q, R, S) in zip(probs, res):
        Qo, Ro, So = oracle.two_stage(p.V.numpy(), p.A.numpy())
        np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q)
        np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * max(1, np.abs(Ro).max()))
        np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL_Q * max(1, np.abs(So).max()))
    res2 = tho.orth_batched(pairs, prec=tho.THO_PREC_FP64_EMU)
    torch.cuda.synchronize()
    for (Q, _, _), (Q2, _, _) in zip(res, res2):
        assert torch.equal(Q, Q2)


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("prec_name", ["THO_PREC_FP64", "THO_PREC_FP64_EMU"])
def test_orth_host_matches_device(tho, dtype, prec_name):
    """tho_orth_host: five different problems back to back through the two
    staging sets (copies overlapping the previous computation), pinned and
    pageable host buffers, each bitwise equal to tho_orth on the device."""
    prec = getattr(tho, prec_name)
    n, k0, k = 6000, 24, 12
    plan = tho.Plan([(n, k0, k)], dtype, prec, 0)
    probs = [inputs.random_problem(n, k0, k, dtype=dtype, seed=80 + i) for i in range(5)]
    outs = []
    for i, p in enumerate(probs):
        pin = i % 2 == 0
        hV = p.V.clone().pin_memory() if pin else p.V.clone()
        hA = p.A.clone().pin_memory() if pin else p.A.clone()
        hQ = torch.empty_strided((n, k), (1, n), dtype=dtype)
        hR = torch.empty_strided((k, k), (1, k), dtype=dtype)
        hS = torch.empty_strided((k0, k), (1, k0), dtype=dtype)
        if pin:
            hQ, hR, hS = hQ.pin_memory(), hR.pin_memory(), hS.pin_memory()
        tho.orth_host(hV, hA, hQ, hR, hS, prec=prec, plan=plan)
        outs.append((hV, hA, hQ, hR, hS))
    tho.orth_host_wait(plan)
    torch.cuda.synchronize()
    for p, (_, _, hQ, hR, hS) in zip(probs, outs):
        Q, R, S = tho.orth(p.V.cuda(), p.A.cuda(), prec=prec, plan=plan)
        torch.cuda.synchronize()
        assert torch.equal(hQ, Q.cpu()) and torch.equal(hR, R.cpu()) and torch.equal(hS, S.cpu())
    Qo, _, _ = oracle.two_stage(probs[-1].V.numpy(), probs[-1].A.numpy())
    np.testing.assert_allclose(outs[-1][2].numpy(), Qo, atol=TOL_Q)


def test_orth_host_k0_zero(tho):
    """tho_orth_host with k0 = 0 (V absent): the Householder QR of A."""
    n, k = 3000, 8
    p = inputs.random_problem(n, 0, k, dtype=torch.float64, seed=7)
    plan = tho.Plan([(n, 0, k)], torch.float64, tho.THO_PREC_FP64, tho.THO_FLAG_ALLOW_K0_ZERO)
    hQ = torch.empty_strided((n, k), (1, n), dtype=torch.float64)
    hR = torch.empty_strided((k, k), (1, k), dtype=torch.float64)
    tho.orth_host(None, p.A.clone(), hQ, hR, None, plan=plan)
    tho.orth_host_wait(plan)
    torch.cuda.synchronize()
    Qo, Ro = oracle.householder_qr(p.A.numpy())
    np.testing.assert_allclose(hQ.numpy(), Qo, atol=TOL_Q)
    np.testing.assert_allclose(hR.numpy(), Ro, atol=TOL_Q * np.abs(Ro).max())


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("prec_name", ["THO_PREC_FP64", "THO_PREC_FP64_EMU"])
@pytest.mark.parametrize("kb", [[4, 7, 16, 3], [32, 32, 32, 32, 32]])
def test_blocks_match_oracle(tho, dtype, prec_name, kb):
    """Algorithm 3 (tho_orth_blocks): ragged block widths, and five blocks of 32
    (the last step at k0 = THO_MAX_K0), against the oracle's Algorithm 3."""
    n = 3000
    p = inputs.random_problem(n, 0, sum(kb), dtype=dtype, seed=90 + len(kb))
    blk = tho.Blocks(n, kb, dtype, getattr(tho, prec_name))
    Q, R = blk.orth(p.A.cuda())
    torch.cuda.synchronize()
    Qo, Ro = oracle.block_hhqr(p.A.numpy(), kb)
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * np.abs(Ro).max())


@pytest.mark.parametrize("prec_name", ["THO_PREC_FP64", "THO_PREC_FP64_EMU"])
def test_blocks_ill_conditioned_krylov(tho, prec_name):
    """Block Krylov-style A (A_{i+1} = D A_i, cond far beyond 1e10) at n = 2^18,
    eight blocks of 16: orthogonality and residual at the rounding level."""
    n, k, nb = 1 << 18, 16, 8
    g = torch.Generator().manual_seed(5)
    d = torch.exp(torch.linspace(0.0, 4.0, n, dtype=torch.float64))
    blocks = [torch.randn(n, k, generator=g, dtype=torch.float64)]
    for _ in range(nb - 1):
        blocks.append(d[:, None] * blocks[-1])
    A = inputs.colmajor(torch.cat(blocks, dim=1)).cuda()
    blk = tho.Blocks(n, [k] * nb, torch.float64, getattr(tho, prec_name))
    Q, R = blk.orth(A)
    torch.cuda.synchronize()
    K = k * nb
    I = torch.eye(K, dtype=torch.float64, device="cuda")
    assert float(torch.linalg.matrix_norm(Q.T @ Q - I, ord=2)) < TOL_LOO
    assert float(torch.linalg.norm(A - Q @ R) / torch.linalg.norm(A)) < TOL_LOO
    assert float(torch.tril(R, -1).abs().max()) == 0.0


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("prec_name", ["THO_PREC_FP64", "THO_PREC_FP64_EMU"])
@pytest.mark.parametrize("n,k0,k", [(3000, 16, 8), (20000, 128, 32), (785, 7, 30)])
def test_first_choice_of_P_matches_oracle(tho, dtype, prec_name, n, k0, k):
    """The first choice of P (THO_FLAG_P_MLU: Algorithm 2's modified LU) against
    the oracle's Algorithm 1 with that choice; Q, R, S agree with the second
    choice's too (they do not depend on P)."""
    prec = getattr(tho, prec_name)
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=n + 5 * k0 + k)
    plan = tho.Plan([(n, k0, k)], dtype, prec, tho.THO_FLAG_P_MLU)
    Q, R, S = tho.orth(p.V.cuda(), p.A.cuda(), prec=prec, plan=plan)
    torch.cuda.synchronize()
    Qo, Ro, So, _ = oracle.two_stage_mlu(p.V.numpy(), p.A.numpy())
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * max(1, np.abs(Ro).max()))
    np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL_Q * max(1, np.abs(So).max()))
    Q2, _, _ = tho.orth(p.V.cuda(), p.A.cuda(), prec=prec)
    assert float((Q2 - Q).abs().max()) < TOL_Q


@pytest.mark.parametrize("dtype", [torch.float64, torch.complex128])
@pytest.mark.parametrize("prec_name", ["THO_PREC_FP64", "THO_PREC_FP64_EMU"])
@pytest.mark.parametrize("n,k0,k", [(3000, 16, 8), (20000, 128, 32), (785, 7, 30), (500, 1, 3)])
def test_third_choice_of_P_matches_oracle(tho, dtype, prec_name, n, k0, k):
    """The third choice of P (THO_FLAG_P_POLAR: polar factor of V_{1:k0,:} by the
    Newton-Schulz iteration, T = I + M through its Cholesky factor) against the
    oracle's Algorithm 1 with that choice (polar factor from an SVD)."""
    prec = getattr(tho, prec_name)
    p = inputs.random_problem(n, k0, k, dtype=dtype, seed=n + 9 * k0 + k)
    plan = tho.Plan([(n, k0, k)], dtype, prec, tho.THO_FLAG_P_POLAR)
    Q, R, S = tho.orth(p.V.cuda(), p.A.cuda(), prec=prec, plan=plan)
    torch.cuda.synchronize()
    assert plan.status() == tho.THO_OK
    Qo, Ro, So, _ = oracle.two_stage_polar(p.V.numpy(), p.A.numpy())
    np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=TOL_Q * max(1, np.abs(Ro).max()))
    np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL_Q * max(1, np.abs(So).max()))
    assert loo_np(p.V.numpy(), Q.cpu().numpy()) < TOL_LOO


def test_third_choice_batched(tho):
    """The polar iteration over a batch (one launch per step for all problems,
    each stopping on its own) against the oracle per problem."""
    probs = [inputs.random_problem(n, k0, k, seed=70 + i) for i, (n, k0, k) in enumerate(BATCH_SHAPES)]
    pairs = [(p.V.cuda(), p.A.cuda()) for p in probs]
    res = tho.orth_batched(pairs, flags=tho.THO_FLAG_P_POLAR)
    torch.cuda.synchronize()
    for p, (Q, R, S) in zip(probs, res):
        Qo, _, So, _ = oracle.two_stage_polar(p.V.numpy(), p.A.numpy())
        np.testing.assert_allclose(Q.cpu().numpy(), Qo, atol=TOL_Q)
        np.testing.assert_allclose(S.cpu().numpy(), So, atol=TOL_Q * max(1, np.abs(So).max()))


def test_third_choice_singular_v1_latches_noconv(tho):
    """V_{1:k0,:} exactly singular (a zero row): the polar factor is not unique
    and the iteration cannot reach a unitary matrix; the plan latches
    THO_ERR_NOCONV instead of returning silently."""
    n, k0, k = 2000, 8, 4
    p = inputs.random_problem(n, k0, k, seed=77)
    X = p.V.clone()
    X[3, :] = 0.0
    V = inputs.colmajor(torch.linalg.qr(X, mode="reduced")[0])
    V[3, :] = 0.0  # the QR leaves rounding-level entries in the zero row; clear them
    plan = tho.Plan([(n, k0, k)], torch.float64, tho.THO_PREC_FP64, tho.THO_FLAG_P_POLAR)
    tho.orth(V.cuda(), p.A.cuda(), plan=plan)
    torch.cuda.synchronize()
    assert plan.status() == tho.THO_ERR_NOCONV


def test_first_choice_refused_by_the_adjoint(tho):
    n, k0, k = 2000, 8, 4
    p = inputs.random_problem(n, k0, k, dtype=torch.float64, seed=3)
    plan = tho.Plan([(n, k0, k)], torch.float64, tho.THO_PREC_FP64, tho.THO_FLAG_P_MLU)
    V, A = p.V.cuda(), p.A.cuda()
    Q, _, _ = tho.orth(V, A, plan=plan)
    dV, dA = torch.empty_like(V), torch.empty_like(A)
    import ctypes
    rc = tho.load().tho_orth_backward(plan.handle, V.data_ptr(), n, A.data_ptr(), n, Q.data_ptr(), n,
                                      Q.data_ptr(), n, dV.data_ptr(), n, dA.data_ptr(), n,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == tho.THO_ERR_UNSUPPORTED
