"""ORACLE — test infrastructure only.

Plain, slow CPU reference for the two-stage Householder orthogonalization of
He & Shao (arXiv 2602.14449), Algorithm 1 with the second choice of P
(Section 3.2).  The arithmetic lives in ``tho_oracle.cpp`` (plain C++ loops,
FP64 / complex128, no BLAS); this module only builds it with g++ and marshals
numpy arrays through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never links or calls
it, and the two share no code.

Every function here is pinned in ``tests/test_oracle.py``:
  * ``two_stage``      — worked example eq. (badbcg) / Example 1; closed form
                         qf((I - V V^*) A); LAPACK QR of [V, A] (eq. vavq);
                         invariants of choice 2 (T = I + R_1^*, T + T^* = W^* W,
                         ||T||_2 <= 2, kappa_2(T) < 2 sqrt(2) k0); H [P; 0] = V;
                         special cases V = [I; 0], V_1 = 0, k0 = 0.
  * ``householder_qr`` — LAPACK QR after phase normalization.
  * ``bcgs``           — Table 1 first row (loss of orthogonality ~ 1) and the
                         three-projection rows (~ u) on the worked example.
  * ``block_hhqr``     — Algorithm 3: the unique QR with real nonnegative
                         diag(R) of a full-rank A by LAPACK (phase-normalized),
                         for several block splittings; Q^* Q = I, A = Q R.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tho_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (portable flags only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, dp = ctypes.c_int64, ctypes.c_void_p
            for name in ("oracle_two_stage_f64", "oracle_two_stage_c128"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64, dp, dp, dp]
                f.restype = ctypes.c_int
            for name in ("oracle_householder_qr_f64", "oracle_householder_qr_c128"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, dp, i64, dp, i64, dp]
                f.restype = ctypes.c_int
            for name in ("oracle_bcgs_f64", "oracle_bcgs_c128"):
                f = getattr(lib, name)
                f.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64, ctypes.c_char_p]
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _fortran(x, dtype):
    return np.asfortranarray(np.asarray(x, dtype=dtype))


def _dtype_of(*arrs):
    return np.complex128 if any(np.iscomplexobj(a) for a in arrs) else np.float64


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


def two_stage(V, A, return_aux: bool = False):
    """Algorithm 1 (second choice of P) on column-major copies of V (n x k0), A (n x k).

    Returns (Q, R, S) and, with ``return_aux``, a dict of the intermediate
    quantities Q1, R1, T, Wtop (k0 x k0), G, Z, Z2 (k0 x k) and Aprime (n x k).
    """
    dt = _dtype_of(V, A)
    V = _fortran(V, dt)
    A = _fortran(A, dt)
    n, k = A.shape
    k0 = V.shape[1] if V.ndim == 2 else 0
    if V.shape[0] != n and k0 > 0:
        raise ValueError("V and A must have the same number of rows")
    Q = np.zeros((n, k), dtype=dt, order="F")
    R = np.zeros((k, k), dtype=dt, order="F")
    S = np.zeros((k0, k), dtype=dt, order="F")
    aux = None
    if return_aux:
        aux = np.zeros(4 * k0 * k0 + 3 * k0 * k + n * k, dtype=dt)
    fn = _load().oracle_two_stage_c128 if dt == np.complex128 else _load().oracle_two_stage_f64
    rc = fn(n, k0, k, _ptr(V), max(n, 1), _ptr(A), n, _ptr(Q), n, _ptr(R), _ptr(S), _ptr(aux))
    if rc != 0:
        raise ValueError(f"oracle two_stage rejected shapes n={n} k0={k0} k={k}")
    if not return_aux:
        return Q, R, S
    out, o = {}, 0
    for name, r, c in (("Q1", k0, k0), ("R1", k0, k0), ("T", k0, k0), ("Wtop", k0, k0),
                       ("G", k0, k), ("Z", k0, k), ("Z2", k0, k), ("Aprime", n, k)):
        out[name] = aux[o:o + r * c].reshape((r, c), order="F")
        o += r * c
    return Q, R, S, out


def householder_qr(X):
    """Unblocked Householder QR with real nonnegative diag(R): X = Q R."""
    dt = _dtype_of(X)
    X = _fortran(X, dt)
    m, k = X.shape
    Q = np.zeros((m, k), dtype=dt, order="F")
    R = np.zeros((k, k), dtype=dt, order="F")
    fn = _load().oracle_householder_qr_c128 if dt == np.complex128 else _load().oracle_householder_qr_f64
    if fn(m, k, _ptr(X), m, _ptr(Q), m, _ptr(R)) != 0:
        raise ValueError("householder_qr needs m >= k >= 1")
    return Q, R


def block_hhqr(A, kb):
    """Algorithm 3 (Block Householder-QR, Section 5): the QR factorization of
    A = [A_1, ..., A_p] (block widths kb) taking the blocks in order.  Step 1
    is the Householder QR of A_1; step i >= 2 is Algorithm 1 with
    V = [Q_1, ..., Q_{i-1}] and A = A_i, whose Q, R and S give Q_i, the
    diagonal block R_ii and the block above it, R_{1:i-1, i}.  Returns (Q, R)."""
    dt = _dtype_of(A)
    A = _fortran(A, dt)
    n, K = A.shape
    if sum(kb) != K:
        raise ValueError("block widths must add up to the columns of A")
    Q = np.zeros((n, K), dtype=dt, order="F")
    R = np.zeros((K, K), dtype=dt, order="F")
    o = 0
    for i, k in enumerate(kb):
        if i == 0:
            Qi, Rii = householder_qr(A[:, :k])
        else:
            Qi, Rii, S = two_stage(Q[:, :o], A[:, o:o + k])
            R[:o, o:o + k] = S
        Q[:, o:o + k] = Qi
        R[o:o + k, o:o + k] = Rii
        o += k
    return Q, R


def bcgs(V, A, passes: str = "PQ"):
    """BCGS comparator, eq. (BQR): 'P' = projection (BQR-1), 'Q' = Householder QR (BQR-2)."""
    dt = _dtype_of(V, A)
    V = _fortran(V, dt)
    A = _fortran(A, dt)
    n, k = A.shape
    k0 = V.shape[1]
    Q = np.zeros((n, k), dtype=dt, order="F")
    fn = _load().oracle_bcgs_c128 if dt == np.complex128 else _load().oracle_bcgs_f64
    if fn(n, k0, k, _ptr(V), n, _ptr(A), n, _ptr(Q), n, passes.encode()) != 0:
        raise ValueError("bcgs: bad shapes or pass string")
    return Q
