"""The bias as a differentiable torch function: V(pos) with a hand-written adjoint.

The paper computes CVs, bias and bias forces with PyTorch tensor operations
and automatic differentiation (Section "Frameworks of GPU-MetaD").  Here the
forward pass is the library's neighbour build, CV and bias kernels and the
backward pass is its adjoint kernels (metad_bias_forces with scale -dL/dV),
so autograd never records the per-pair graph.

Only the positions are saved for backward.  The per-atom CV state (q_m,
qbar_m, the adjoint seeds) lives once inside the context; if the context ran
another frame between this forward and its backward, backward recomputes
that state from the saved positions instead of having stored a copy per
call, which keeps memory flat at the largest system sizes.
"""
from __future__ import annotations

import numpy as np
import torch

from . import metad as _m


class BiasContext(_m.Metad):
    """A Metad context that counts its forward evaluations (generation)."""

    def __init__(self, params):
        super().__init__(params)
        self.generation = 0
        self.last_pos_ptr = None

    def evaluate(self, pos: torch.Tensor):
        """Neighbours, CVs and bias for pos (float32 [N, 4] on the device)."""
        self.build_neighbors(pos)
        self.cv_forward(want_host=False)
        self.bias_eval(want_host=False)
        self.generation += 1
        self.last_pos_ptr = pos.data_ptr()
        return self.generation


class MetadBias(torch.autograd.Function):
    """V = MetadBias.apply(pos, ctx): scalar float64 bias of the positions.

    pos: float32 [N, 4] on the context's device (x, y, z, species); the
    gradient with respect to the species column is zero.
    """

    @staticmethod
    def forward(fctx, pos: torch.Tensor, bias_ctx: BiasContext):
        if pos.dtype != torch.float32 or pos.dim() != 2 or pos.shape[1] != 4:
            raise ValueError("pos must be float32 [N, 4]")
        pos = pos.contiguous()
        gen = bias_ctx.evaluate(pos)
        cv, V, dV = bias_ctx.read_results()
        fctx.save_for_backward(pos)
        fctx.bias_ctx = bias_ctx
        fctx.gen = gen
        fctx.cv = cv
        return torch.tensor(V, dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(fctx, grad_V: torch.Tensor):
        (pos,) = fctx.saved_tensors
        bctx: BiasContext = fctx.bias_ctx
        if bctx.generation != fctx.gen or bctx.last_pos_ptr != pos.data_ptr():
            # the context moved on: recompute the per-atom state of this frame
            bctx.evaluate(pos)
            fctx.gen = bctx.generation
        g = float(grad_V.detach().cpu())
        n = pos.shape[0]
        dVdx = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        # forces are -dV/dx: scale by -g to get g * dV/dx
        bctx.bias_forces(dVdx, accumulate=False, scale=-g)
        grad = torch.zeros_like(pos)
        grad[:, :3] = dVdx
        return grad, None


def bias(pos: torch.Tensor, bias_ctx: BiasContext) -> torch.Tensor:
    return MetadBias.apply(pos, bias_ctx)

