"""torch.autograd.Function over the C ABI: forward tho_orth, backward tho_orth_backward.

The backward is the hand-written adjoint of the map (V, A) -> Q of Algorithm 1
(second choice of P); it recomputes (W, T) and the small solves from V, A and
the saved Q instead of storing per-panel reflectors.  FP64, real or complex
(torch's gradient convention for complex tensors).
"""
import torch

from . import tho


class TwoStageOrth(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, A):
        Q, _, _ = tho.orth(V, A, want_R=False, want_S=False)
        ctx.save_for_backward(V, A, Q)
        return Q

    @staticmethod
    def backward(ctx, dQ):
        V, A, Q = ctx.saved_tensors
        dV, dA = tho.orth_backward(V, A, Q, tho.colmajor(dQ))
        return dV, dA


def two_stage_orth(V: torch.Tensor, A: torch.Tensor) -> torch.Tensor:
    """Q of Algorithm 1 (column-major float64 or complex128 CUDA tensors), differentiable in V and A."""
    return TwoStageOrth.apply(V, A)
