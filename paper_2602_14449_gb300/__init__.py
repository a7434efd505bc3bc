"""GB300-native two-stage Householder orthogonalization (He & Shao, arXiv 2602.14449).

Given V (n x k0, orthonormal columns) and A (n x k), Algorithm 1 with the
second choice of P (Section 3.2) returns Q (n x k) with Q^* Q = I,
Range([V, A]) within Range([V, Q]) and Range(Q) orthogonal to Range(V), plus
the factors R (k x k) and S = V^* A (k0 x k) of eq. (vavq).

The work runs in hand-written sm_103a CUDA kernels behind the C ABI declared
in ``include/tho.h`` (``libtho.so``); ``paper_2602_14449_gb300.tho`` is the thin
ctypes binding and ``paper_2602_14449_gb300.autograd`` the autograd wrapper.
"""

__all__ = ["tho", "inputs", "autograd"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
