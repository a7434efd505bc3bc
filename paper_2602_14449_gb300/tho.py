"""Thin Python binding of libtho (include/tho.h) over ctypes.

Argument marshalling only: every step of the orthogonalization runs in the
CUDA kernels of ``libtho.so``.  PyTorch provides device memory and the current
stream.  There is no CPU or PyTorch fallback: if the library is missing the
calls raise.

Matrices are column-major torch CUDA tensors: shape (rows, cols) with
stride (1, ld), ld >= rows -- the layout of ``x.t().contiguous().t()`` or
``torch.empty_strided((r, c), (1, r))``.  ``colmajor`` converts explicitly.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtho.so")

THO_OK, THO_ERR_ARG, THO_ERR_SHAPE, THO_ERR_ALIGN, THO_ERR_NOMEM = 0, 1, 2, 3, 4
THO_ERR_CUDA, THO_ERR_TIMEOUT, THO_ERR_NONFINITE, THO_ERR_UNSUPPORTED, THO_ERR_NOCONV = 5, 6, 7, 8, 9
THO_ERR_NOT_ORTH = 10
THO_F64, THO_C128 = 0, 1
THO_PREC_FP64, THO_PREC_FP32_BULK, THO_PREC_FP64_EMU = 0, 1, 2
THO_FLAG_ALLOW_K0_ZERO, THO_FLAG_CHECK_FINITE, THO_FLAG_P_MLU, THO_FLAG_P_POLAR = 0x1, 0x2, 0x4, 0x8
THO_FLAG_CHECK_ORTH = 0x10
THO_ORTH_TOL = 1e-12
THO_MAX_K0, THO_MAX_K = 128, 32
THO_TUNE_MAX_SPLIT = 1 << 20

EXPORTED = ("tho_plan", "tho_plan_destroy", "tho_plan_workspace_bytes", "tho_plan_kernel_launches",
            "tho_plan_leaf_rows", "tho_orth_host", "tho_orth_host_wait",
            "tho_blocks_plan", "tho_blocks_destroy", "tho_orth_blocks", "tho_blocks_kernel_launches",
            "tho_orth", "tho_orth_batched", "tho_orth_backward", "tho_plan_status", "tho_status_string",
            "tho_plan_set_phase_timing", "tho_plan_read_phase_timing", "tho_phase_name",
            "tho_orth_noalloc", "tho_plan_tuned", "tho_plan_tuning", "tho_autotune", "tho_tune_key",
            "tho_tune_cache_get", "tho_tune_cache_put", "tho_plan_expire_wait", "tho_orth_b",
            "tho_plan_orth_defect")
THO_NUM_PHASES = 11


class ThoError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} (status {code})")


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("k0", ctypes.c_int64), ("k", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("prec", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    """tho_tuning_t: TSQR leaf height, split-n factor (0 = library default) and
    how a batch shares the chunks (0 = by rows, 1 = by streaming work)."""
    _fields_ = [("leaf_rows", ctypes.c_int32), ("split_chunks", ctypes.c_int32), ("balance", ctypes.c_int32)]

    def as_tuple(self):
        return (self.leaf_rows, self.split_chunks, self.balance)


class Instance(ctypes.Structure):
    _fields_ = [("V", ctypes.c_void_p), ("A", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("R", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("ldv", ctypes.c_int64), ("lda", ctypes.c_int64), ("ldq", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libtho.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libtho.so not found at {p}; build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.tho_plan.argtypes = [ctypes.POINTER(Desc), i32, ctypes.POINTER(vp)]
        lib.tho_plan.restype = ctypes.c_int
        lib.tho_plan_tuned.argtypes = [ctypes.POINTER(Desc), i32, ctypes.POINTER(Tuning), ctypes.POINTER(vp)]
        lib.tho_plan_tuned.restype = ctypes.c_int
        lib.tho_plan_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        lib.tho_plan_tuning.restype = ctypes.c_int
        lib.tho_autotune.argtypes = [ctypes.POINTER(Desc), i32, ctypes.c_char_p, vp, ctypes.POINTER(Tuning),
                                     ctypes.POINTER(ctypes.c_double)]
        lib.tho_autotune.restype = ctypes.c_int
        lib.tho_tune_key.argtypes = [ctypes.POINTER(Desc), i32, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_size_t]
        lib.tho_tune_key.restype = ctypes.c_int
        lib.tho_tune_cache_get.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(Tuning),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        lib.tho_tune_cache_get.restype = ctypes.c_int
        lib.tho_tune_cache_put.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(Tuning), ctypes.c_double]
        lib.tho_tune_cache_put.restype = ctypes.c_int
        lib.tho_plan_destroy.argtypes = [vp]
        lib.tho_plan_destroy.restype = ctypes.c_int
        lib.tho_plan_workspace_bytes.argtypes = [vp]
        lib.tho_plan_workspace_bytes.restype = ctypes.c_size_t
        lib.tho_plan_kernel_launches.argtypes = [vp]
        lib.tho_plan_kernel_launches.restype = ctypes.c_int32
        lib.tho_plan_leaf_rows.argtypes = [vp]
        lib.tho_plan_leaf_rows.restype = ctypes.c_int32
        lib.tho_orth.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp, vp, vp]
        lib.tho_orth.restype = ctypes.c_int
        lib.tho_orth_host.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp, vp, vp]
        lib.tho_orth_b.argtypes = [vp, vp, vp, i64, vp, i64, vp, i64, vp, vp, vp]
        lib.tho_orth_b.restype = ctypes.c_int
        lib.tho_orth_host.restype = ctypes.c_int
        lib.tho_orth_host_wait.argtypes = [vp, vp]
        lib.tho_orth_host_wait.restype = ctypes.c_int
        lib.tho_blocks_plan.argtypes = [i64, ctypes.POINTER(i32), i32, i32, i32, ctypes.POINTER(vp)]
        lib.tho_blocks_plan.restype = ctypes.c_int
        lib.tho_blocks_destroy.argtypes = [vp]
        lib.tho_blocks_destroy.restype = ctypes.c_int
        lib.tho_orth_blocks.argtypes = [vp, vp, i64, vp, i64, vp, vp]
        lib.tho_orth_blocks.restype = ctypes.c_int
        lib.tho_blocks_kernel_launches.argtypes = [vp]
        lib.tho_blocks_kernel_launches.restype = ctypes.c_int32
        lib.tho_orth_batched.argtypes = [vp, ctypes.POINTER(Instance), i32, vp]
        lib.tho_orth_batched.restype = ctypes.c_int
        lib.tho_orth_backward.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp]
        lib.tho_orth_backward.restype = ctypes.c_int
        lib.tho_plan_expire_wait.argtypes = [vp, i32, vp]
        lib.tho_plan_expire_wait.restype = ctypes.c_int
        lib.tho_plan_status.argtypes = [vp]
        lib.tho_plan_status.restype = ctypes.c_int
        lib.tho_plan_orth_defect.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.tho_plan_orth_defect.restype = ctypes.c_int
        lib.tho_status_string.argtypes = [ctypes.c_int]
        lib.tho_status_string.restype = ctypes.c_char_p
        lib.tho_plan_set_phase_timing.argtypes = [vp, i32]
        lib.tho_plan_set_phase_timing.restype = ctypes.c_int
        lib.tho_plan_read_phase_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        lib.tho_plan_read_phase_timing.restype = ctypes.c_int
        lib.tho_phase_name.argtypes = [i32]
        lib.tho_phase_name.restype = ctypes.c_char_p
        _lib = lib
        return lib


def status_string(code: int) -> str:
    return load().tho_status_string(code).decode()


def _check(code: int, what: str):
    if code != THO_OK:
        raise ThoError(code, what)


def colmajor(x: torch.Tensor) -> torch.Tensor:
    """Column-major copy of a 2-D tensor (explicit layout conversion for callers)."""
    return x.t().contiguous().t()


def _ld(x: torch.Tensor, name: str, host: bool = False) -> int:
    if x.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if x.is_cuda == host:
        raise ValueError(f"{name} must be a {'host (CPU)' if host else 'CUDA'} tensor")
    rows, cols = x.shape
    if cols > 1 and x.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride (1, ld)); use tho.colmajor()")
    return max(x.stride(1), rows) if cols > 1 else max(rows, 1)


def _dtype_code(t: torch.dtype) -> int:
    if t == torch.float64:
        return THO_F64
    if t == torch.complex128:
        return THO_C128
    raise ValueError(f"unsupported dtype {t}; use float64 or complex128")


def _descs(shapes, dtype, prec, flags):
    shapes = list(shapes)
    arr = (Desc * len(shapes))()
    code = _dtype_code(dtype)
    for i, (n, k0, k) in enumerate(shapes):
        arr[i] = Desc(n, k0, k, code, prec, flags)
    return arr


def autotune(shapes, dtype=torch.float64, prec: int = THO_PREC_FP64, flags: int = 0, cache: str | None = None):
    """tho_autotune: time candidate partitions for these problem shapes on the
    current device (synthetic operands) and return ((leaf_rows, split_chunks,
    balance), median ms per call).  ``cache``: JSON-lines file (None: $THO_TUNE_CACHE if
    set); a cached entry is returned without measuring."""
    shapes = list(shapes)
    t = Tuning()
    ms = ctypes.c_double()
    st = torch.cuda.current_stream().cuda_stream
    _check(load().tho_autotune(_descs(shapes, dtype, prec, flags), len(shapes),
                               cache.encode() if cache else None, ctypes.c_void_p(st), ctypes.byref(t),
                               ctypes.byref(ms)), "tho_autotune")
    return t.as_tuple(), ms.value


def tune_key(shapes, dtype, prec: int, flags: int, device_name: str) -> str:
    """tho_tune_key: the autotuner's cache key for these shapes on a device named ``device_name``."""
    shapes = list(shapes)
    buf = ctypes.create_string_buffer(4096)
    _check(load().tho_tune_key(_descs(shapes, dtype, prec, flags), len(shapes), device_name.encode(), buf,
                               len(buf)), "tho_tune_key")
    return buf.value.decode()


def tune_cache_get(path: str, key: str):
    """tho_tune_cache_get: ((leaf_rows, split_chunks, balance), ms) of the last entry for ``key``, or None."""
    t = Tuning()
    ms = ctypes.c_double()
    found = ctypes.c_int32()
    _check(load().tho_tune_cache_get(path.encode(), key.encode(), ctypes.byref(t), ctypes.byref(ms),
                                     ctypes.byref(found)), "tho_tune_cache_get")
    return (t.as_tuple(), ms.value) if found.value else None


def tune_cache_put(path: str, key: str, tuning, ms: float):
    """tho_tune_cache_put: append one entry to the cache file."""
    t = Tuning(*tuning)
    _check(load().tho_tune_cache_put(path.encode(), key.encode(), ctypes.byref(t), float(ms)), "tho_tune_cache_put")


def _empty_cm(rows: int, cols: int, dtype, device) -> torch.Tensor:
    return torch.empty_strided((rows, cols), (1, max(rows, 1)), dtype=dtype, device=device)


class Plan:
    """Owns one tho_plan_t (workspace, launch tables, batched graph)."""

    def __init__(self, shapes, dtype=torch.float64, prec: int = THO_PREC_FP64, flags: int = 0, tuning=None):
        """``tuning``: None (library defaults) or (leaf_rows, split_chunks[, balance]),
        e.g. from ``autotune``; 0 keeps the default."""
        lib = load()
        shapes = list(shapes)
        arr = _descs(shapes, dtype, prec, flags)
        h = ctypes.c_void_p()
        if tuning is None:
            _check(lib.tho_plan(arr, len(shapes), ctypes.byref(h)), "tho_plan")
        else:
            t = Tuning(*tuning)
            _check(lib.tho_plan_tuned(arr, len(shapes), ctypes.byref(t), ctypes.byref(h)), "tho_plan_tuned")
        self.handle = h
        self.shapes = shapes
        self.dtype = dtype
        self.prec = prec
        self.flags = flags

    @property
    def workspace_bytes(self) -> int:
        return load().tho_plan_workspace_bytes(self.handle)

    @property
    def kernel_launches(self) -> int:
        return load().tho_plan_kernel_launches(self.handle)

    @property
    def leaf_rows(self) -> int:
        return load().tho_plan_leaf_rows(self.handle)

    @property
    def tuning(self):
        """(leaf_rows, split_chunks, balance) the plan was built with."""
        t = Tuning()
        _check(load().tho_plan_tuning(self.handle, ctypes.byref(t)), "tho_plan_tuning")
        return t.as_tuple()

    def status(self) -> int:
        return load().tho_plan_status(self.handle)

    def orth_defect(self) -> float:
        """tho_plan_orth_defect: the last estimate of ||V^* V - I||_2 of a plan
        made with THO_FLAG_CHECK_ORTH (synchronizes the device)."""
        d = ctypes.c_double(0.0)
        _check(load().tho_plan_orth_defect(self.handle, ctypes.byref(d)), "tho_plan_orth_defect")
        return d.value

    def expire_wait(self, spins: int = 4096):
        """tho_plan_expire_wait: on the current stream, a bounded device wait that
        runs out and latches THO_ERR_TIMEOUT (read it with ``status()``)."""
        st = torch.cuda.current_stream().cuda_stream
        _check(load().tho_plan_expire_wait(self.handle, int(spins), ctypes.c_void_p(st)), "tho_plan_expire_wait")

    def set_phase_timing(self, enable: bool = True):
        _check(load().tho_plan_set_phase_timing(self.handle, int(enable)), "tho_plan_set_phase_timing")

    def read_phase_timing(self):
        """{phase name: (ms summed over traced calls, launch groups)} since the last read."""
        lib = load()
        ms = (ctypes.c_double * THO_NUM_PHASES)()
        gr = (ctypes.c_int32 * THO_NUM_PHASES)()
        _check(lib.tho_plan_read_phase_timing(self.handle, ms, gr), "tho_plan_read_phase_timing")
        return {lib.tho_phase_name(i).decode(): (ms[i], gr[i]) for i in range(THO_NUM_PHASES)}

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.tho_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_plan_cache: dict = {}


def get_plan(shapes, dtype, prec=THO_PREC_FP64, flags=0) -> Plan:
    """Plan cached per (shapes, dtype, prec, flags, device, stream): calls on one
    plan share its workspace, so concurrent streams get separate plans."""
    dev = torch.cuda.current_device()
    st = torch.cuda.current_stream().cuda_stream
    key = (tuple(shapes), dtype, prec, flags, dev, st)
    p = _plan_cache.get(key)
    if p is None:
        p = Plan(shapes, dtype, prec, flags)
        _plan_cache[key] = p
    return p


def _ptr(x):
    return ctypes.c_void_p(x.data_ptr()) if x is not None else None


def orth(V: torch.Tensor, A: torch.Tensor, prec: int = THO_PREC_FP64, want_R: bool = True,
         want_S: bool = True, flags: int = 0, plan: Plan | None = None, Q: torch.Tensor | None = None,
         R: torch.Tensor | None = None, S: torch.Tensor | None = None):
    """Algorithm 1 (second choice of P) on the GPU: returns (Q, R, S).

    V: n x k0 (orthonormal columns), A: n x k, column-major CUDA tensors of
    dtype float64 or complex128.  R (k x k) and S (k0 x k) are None unless
    requested.  Q, R, S may be passed preallocated (column-major, R with
    ld = k, S with ld = k0).  Runs on the current torch stream.
    """
    n, k = A.shape
    k0 = V.shape[1] if V is not None else 0
    if k0 == 0:
        flags |= THO_FLAG_ALLOW_K0_ZERO
    dt = A.dtype
    if V is not None and k0 > 0 and (V.dtype != dt or V.shape[0] != n or V.device != A.device):
        raise ValueError("V and A must share dtype, device and row count")
    ldv = _ld(V, "V") if k0 > 0 else n
    lda = _ld(A, "A")
    if Q is None:
        Q = _empty_cm(n, k, dt, A.device)
    ldq = _ld(Q, "Q")
    if R is None and want_R:
        R = _empty_cm(k, k, dt, A.device)
    if S is None and want_S and k0 > 0:
        S = _empty_cm(k0, k, dt, A.device)
    for x, nm, ld in ((R, "R", k), (S, "S", k0)):
        if x is not None and (x.stride(0) != 1 or (x.shape[1] > 1 and x.stride(1) != ld)):
            raise ValueError(f"{nm} must be column-major with ld = {ld}")
    p = plan or get_plan([(n, k0, k)], dt, prec, flags)
    st = torch.cuda.current_stream().cuda_stream
    _check(load().tho_orth(p.handle, _ptr(V) if k0 > 0 else None, ldv, _ptr(A), lda, _ptr(Q), ldq,
                           _ptr(R), _ptr(S), ctypes.c_void_p(st)), "tho_orth")
    return Q, R, S


def orth_host(V: torch.Tensor, A: torch.Tensor, Q: torch.Tensor, R: torch.Tensor | None = None,
              S: torch.Tensor | None = None, prec: int = THO_PREC_FP64, plan: Plan | None = None):
    """tho_orth_host: Algorithm 1 with V, A and the outputs Q, R, S in host memory.

    V (n x k0), A (n x k) and Q (n x k) are column-major CPU tensors (pinned for
    full copy bandwidth); R (k x k) and S (k0 x k) are optional outputs with
    ld = k and k0.  Asynchronous on the current torch stream: the inputs must
    not change until their copy is done, and the outputs are complete after
    orth_host_wait(plan) and a synchronization of that stream.  Consecutive
    calls overlap their copies with the previous computation.
    """
    n, k = A.shape
    k0 = V.shape[1] if V is not None else 0
    flags = THO_FLAG_ALLOW_K0_ZERO if k0 == 0 else 0
    for x, nm in ((R, "R"), (S, "S")):
        if x is not None and x.is_cuda:
            raise ValueError(f"{nm} must be a host (CPU) tensor")
    for x, nm, ld in ((R, "R", k), (S, "S", k0)):
        if x is not None and (x.stride(0) != 1 or (x.shape[1] > 1 and x.stride(1) != ld)):
            raise ValueError(f"{nm} must be column-major with ld = {ld}")
    p = plan or get_plan([(n, k0, k)], A.dtype, prec, flags)
    st = torch.cuda.current_stream().cuda_stream
    _check(load().tho_orth_host(p.handle, _ptr(V) if k0 > 0 else None, _ld(V, "V", True) if k0 > 0 else n,
                                _ptr(A), _ld(A, "A", True), _ptr(Q), _ld(Q, "Q", True), _ptr(R), _ptr(S),
                                ctypes.c_void_p(st)),
           "tho_orth_host")
    return Q, R, S


def orth_b(d: torch.Tensor, V: torch.Tensor, A: torch.Tensor, prec: int = THO_PREC_FP64, flags: int = 0,
           plan: Plan | None = None):
    """tho_orth_b: Algorithm 4 (B-inner product) for B = diag(d), with the
    initial basis U = D^{-1/2} [I; 0].  d: n positive float64 CUDA values;
    V (n x k0, V^* B V = I) and A (n x k) column-major CUDA tensors.
    Returns (Q, R, S) with [V, Q]^* B [V, Q] = I."""
    n, k = A.shape
    k0 = V.shape[1] if V is not None else 0
    if k0 == 0:
        flags |= THO_FLAG_ALLOW_K0_ZERO
    if d.dtype != torch.float64 or d.numel() != n or not d.is_cuda or not d.is_contiguous():
        raise ValueError("d must be a contiguous float64 CUDA vector of n entries")
    dt = A.dtype
    Q = _empty_cm(n, k, dt, A.device)
    R = _empty_cm(k, k, dt, A.device)
    S = _empty_cm(k0, k, dt, A.device) if k0 > 0 else None
    p = plan or get_plan([(n, k0, k)], dt, prec, flags)
    st = torch.cuda.current_stream().cuda_stream
    _check(load().tho_orth_b(p.handle, _ptr(d), _ptr(V) if k0 > 0 else None, _ld(V, "V") if k0 > 0 else n,
                             _ptr(A), _ld(A, "A"), _ptr(Q), _ld(Q, "Q"), _ptr(R), _ptr(S), ctypes.c_void_p(st)),
           "tho_orth_b")
    return Q, R, S


def orth_host_wait(plan: Plan):
    """Make the current torch stream wait for every orth_host output copy of ``plan``."""
    st = torch.cuda.current_stream().cuda_stream
    _check(load().tho_orth_host_wait(plan.handle, ctypes.c_void_p(st)), "tho_orth_host_wait")


class Blocks:
    """tho_blocks_t: Block Householder-QR (Algorithm 3) of n x K matrices whose
    columns come in blocks of widths ``kb`` (one Algorithm 1 plan per block)."""

    def __init__(self, n: int, kb, dtype: torch.dtype, prec: int = THO_PREC_FP64):
        lib = load()
        self.n, self.kb, self.dtype, self.prec = n, list(kb), dtype, prec
        self.K = sum(self.kb)
        arr = (ctypes.c_int32 * len(self.kb))(*self.kb)
        h = ctypes.c_void_p()
        _check(lib.tho_blocks_plan(n, arr, len(self.kb), _dtype_code(dtype), prec, ctypes.byref(h)), "tho_blocks_plan")
        self.handle = h

    @property
    def kernel_launches(self) -> int:
        return load().tho_blocks_kernel_launches(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.tho_blocks_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def orth(self, A: torch.Tensor, Q: torch.Tensor | None = None, R: torch.Tensor | None = None):
        """Q (n x K) and R (K x K, upper block triangular) with A = Q R, on the current stream."""
        n, K = A.shape
        if n != self.n or K != self.K or A.dtype != self.dtype:
            raise ValueError("A does not match the block plan")
        if Q is None:
            Q = _empty_cm(n, K, A.dtype, A.device)
        if R is None:
            R = _empty_cm(K, K, A.dtype, A.device)
        if R.stride(0) != 1 or (K > 1 and R.stride(1) != K):
            raise ValueError("R must be column-major with ld = K")
        st = torch.cuda.current_stream().cuda_stream
        _check(load().tho_orth_blocks(self.handle, _ptr(A), _ld(A, "A"), _ptr(Q), _ld(Q, "Q"), _ptr(R),
                                      ctypes.c_void_p(st)), "tho_orth_blocks")
        return Q, R


def orth_batched(pairs, prec: int = THO_PREC_FP64, plan: Plan | None = None, outs=None, flags: int = 0):
    """Batched Algorithm 1 over a list of (V, A): one CUDA-graph replay.

    Returns a list of (Q, R, S).  ``outs`` may pass preallocated (Q, R, S) triples.
    """
    shapes = [(A.shape[0], V.shape[1], A.shape[1]) for V, A in pairs]
    dt = pairs[0][1].dtype
    p = plan or get_plan(shapes, dt, prec, flags)
    arr = (Instance * len(pairs))()
    res = []
    for i, (V, A) in enumerate(pairs):
        n, k = A.shape
        k0 = V.shape[1]
        if outs is None:
            Q = _empty_cm(n, k, dt, A.device)
            R = _empty_cm(k, k, dt, A.device)
            S = _empty_cm(k0, k, dt, A.device)
        else:
            Q, R, S = outs[i]
        arr[i] = Instance(V.data_ptr(), A.data_ptr(), Q.data_ptr(), R.data_ptr(), S.data_ptr(),
                          _ld(V, "V"), _ld(A, "A"), _ld(Q, "Q"))
        res.append((Q, R, S))
    st = torch.cuda.current_stream().cuda_stream
    _check(load().tho_orth_batched(p.handle, arr, len(pairs), ctypes.c_void_p(st)), "tho_orth_batched")
    return res


def orth_backward(V, A, Q, dQ, plan: Plan | None = None):
    """Reverse-mode derivative of (V, A) -> Q (FP64, real or complex): returns
    (dV, dA); for complex tensors the gradients of a real loss in torch's
    convention (dL/dRe z + i dL/dIm z)."""
    n, k = A.shape
    k0 = V.shape[1]
    dV = _empty_cm(n, k0, V.dtype, V.device)
    dA = _empty_cm(n, k, A.dtype, A.device)
    p = plan or get_plan([(n, k0, k)], A.dtype, THO_PREC_FP64, 0)
    st = torch.cuda.current_stream().cuda_stream
    _check(load().tho_orth_backward(p.handle, _ptr(V), _ld(V, "V"), _ptr(A), _ld(A, "A"), _ptr(Q), _ld(Q, "Q"),
                                    _ptr(dQ), _ld(dQ, "dQ"), _ptr(dV), _ld(dV, "dV"), _ptr(dA), _ld(dA, "dA"),
                                    ctypes.c_void_p(st)), "tho_orth_backward")
    return dV, dA
