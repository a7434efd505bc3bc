"""The row-sharded form of Algorithm 1 on CPU ranks over gloo, against the
unsharded oracle.

P ranks own contiguous row blocks of V, A and Q; rank 0 also owns rows
1..k0.  One orthogonalization needs three small exchanges (Section 3.1's
three global reductions, in this order): an allreduce of G = W^*A (k0 x k),
an allgather of the ranks' leaf R factors for the top of the TSQR tree
(k x k each) and an allreduce of G2 = W^*[0; Qbar] (k0 x k).  Rank 0's QR of
V_{1:k0,:} (Section 3.2, second choice of P) is broadcast first.  The library
runs on one GPU; this checks the arithmetic of the sharded design, with the
oracle's Householder QR as the local factorization, for real and complex data.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _t(x):  # numpy -> torch, complex carried as (re, im) pairs for gloo
    t = torch.from_numpy(np.ascontiguousarray(x))
    return torch.view_as_real(t).contiguous() if t.is_complex() else t


def _n(t, cplx):
    return torch.view_as_complex(t).numpy() if cplx else t.numpy()


def _allreduce(x):
    t = _t(x)
    dist.all_reduce(t)
    return _n(t, np.iscomplexobj(x))


def _tri_solve(M, B, lower):
    """Plain substitution with the triangular M (no explicit inverse)."""
    n = M.shape[0]
    X = np.zeros_like(B)
    order = range(n) if lower else range(n - 1, -1, -1)
    for i in order:
        js = range(i) if lower else range(i + 1, n)
        acc = B[i].copy()
        for j in js:
            acc = acc - M[i, j] * X[j]
        X[i] = acc / M[i, i]
    return X


def _problem(n, k0, k, cplx):
    rng = np.random.default_rng(20260214 + n + k0 + k + cplx)
    def g(r, c):
        x = rng.standard_normal((r, c))
        return (x + 1j * rng.standard_normal((r, c))) / np.sqrt(2) if cplx else x
    V, _ = np.linalg.qr(g(n, k0))
    return V, g(n, k)


def _worker(rank, world, port, n, k0, k, cplx, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        V, A = _problem(n, k0, k, cplx)
        bounds = np.linspace(0, n, world + 1).astype(int)
        lo, hi = int(bounds[rank]), int(bounds[rank + 1])
        t0 = max(lo, k0)  # first trailing row of this rank
        # a1-a2: QR of V_{1:k0,:} on rank 0 (diag(R1) >= 0), broadcast.
        if rank == 0:
            Q1, R1 = oracle.householder_qr(V[:k0])
        else:
            Q1 = np.zeros((k0, k0), V.dtype)
            R1 = np.zeros((k0, k0), V.dtype)
        tq, tr = _t(Q1), _t(R1)
        dist.broadcast(tq, 0)
        dist.broadcast(tr, 0)
        Q1, R1 = _n(tq, cplx), _n(tr, cplx)
        P = -Q1
        T = np.eye(k0) + R1.conj().T  # lower triangular
        Wtop = P - V[:k0] if rank == 0 else None
        V2, A2 = V[t0:hi], A[t0:hi]
        # a3: G = Wtop^* A_1 - V_2^* A_2, one allreduce.
        Gp = -V2.conj().T @ A2
        if rank == 0:
            Gp = Gp + Wtop.conj().T @ A[:k0]
        G = _allreduce(Gp)
        # a4-a6.
        Z = _tri_solve(T.conj().T, G, lower=False)
        A2p = A2 + V2 @ Z
        S = P.conj().T @ (A[:k0] - Wtop @ Z) if rank == 0 else None
        # a7: local Householder QR, allgather of the R's, QR of the stack.
        Qr, Rr = oracle.householder_qr(A2p)
        parts = [torch.zeros_like(_t(Rr)) for _ in range(world)]
        dist.all_gather(parts, _t(Rr))
        stack = np.vstack([_n(x, cplx) for x in parts])
        Qt, R = oracle.householder_qr(stack)
        Qbar = Qr @ Qt[rank * k:(rank + 1) * k]
        # a8: G2 = -V_2^* Qbar, one allreduce; Z2 = T^-1 G2.
        G2 = _allreduce(-V2.conj().T @ Qbar)
        Z2 = _tri_solve(T, G2, lower=True)
        # a9.
        Qrows = np.zeros((hi - lo, k), V.dtype)
        if rank == 0:
            Qrows[:k0] = -Wtop @ Z2
        Qrows[t0 - lo:] = Qbar + V2 @ Z2
        # Gather Q on every rank (fixed-size blocks).
        mx = int(max(bounds[i + 1] - bounds[i] for i in range(world)))
        blk = np.zeros((mx, k), V.dtype)
        blk[:hi - lo] = Qrows
        got = [torch.zeros_like(_t(blk)) for _ in range(world)]
        dist.all_gather(got, _t(blk))
        if rank == 0:
            Q = np.vstack([_n(got[i], cplx)[:bounds[i + 1] - bounds[i]] for i in range(world)])
            Qo, Ro, So = oracle.two_stage(V, A)
            out["dQ"] = float(np.abs(Q - Qo).max())
            out["dR"] = float(np.abs(R - Ro).max())
            out["dS"] = float(np.abs(S - So).max())
            out["loo"] = float(np.linalg.norm(np.hstack([V, Q]).conj().T @ np.hstack([V, Q]) - np.eye(k0 + k), 2))
            out["resid"] = float(np.linalg.norm(np.hstack([V, A]) - np.hstack([V, Q]) @ np.block(
                [[np.eye(k0), So], [np.zeros((k, k0)), R]]), "fro") / np.linalg.norm(np.hstack([V, A]), "fro"))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("world", [2, 3])
def test_row_sharded_matches_unsharded_oracle(cplx, world):
    n, k0, k = 1500, 16, 6
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, n, k0, k, cplx, out)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    assert out["dQ"] < 1e-12 and out["dR"] < 1e-12 and out["dS"] < 1e-12, dict(out)
    assert out["loo"] < 1e-13 and out["resid"] < 1e-14, dict(out)
