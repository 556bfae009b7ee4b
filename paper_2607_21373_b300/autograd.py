"""torch.autograd wrappers of the forward map (the backward passes are the
library's transposed-step kernels; no PyTorch arithmetic on the path)."""
from __future__ import annotations

import torch


class WaveForward(torch.autograd.Function):
    """Y = G p0 with dL/dp0 = G^T dL/dY (Section 5.1's exact transpose)."""

    @staticmethod
    def forward(ctx, p0, mesh):
        ctx.mesh = mesh
        return mesh.forward(p0.contiguous())

    @staticmethod
    def backward(ctx, gY):
        return ctx.mesh.adjoint(gY.contiguous()), None


class WaveForwardC2(torch.autograd.Function):
    """Y = G(c2) p0 with gradients for p0 and the per-tetrahedron c^2.

    The backward pass runs pat_grad_c2: a checkpointed recomputation of the
    forward trajectory and the transposed recursion, giving dL/dc2 (summed over
    stacked samples) and dL/dp0 together.  c2 is a float64 tensor of length
    n_tets; changing it rebuilds the mesh's operators.
    """

    @staticmethod
    def forward(ctx, p0, c2, mesh):
        c2h = c2.detach().to("cpu", torch.float64)
        if getattr(mesh, "_c2_cache", None) is None or not torch.equal(mesh._c2_cache, c2h):
            mesh.set_c2(c2h)
            mesh._c2_cache = c2h.clone()
        p0c = p0.contiguous()
        ctx.save_for_backward(p0c)
        ctx.mesh = mesh
        ctx.c2_meta = (c2.dtype, c2.device)
        return mesh.forward(p0c)

    @staticmethod
    def backward(ctx, gY):
        (p0,) = ctx.saved_tensors
        g, pg = ctx.mesh.grad_c2(p0, gY.contiguous(), want_p0_grad=ctx.needs_input_grad[0])
        dtype, device = ctx.c2_meta
        return pg, g.to(device=device, dtype=dtype), None


def wave_forward(p0, mesh, c2=None):
    """Differentiable G p0 (and G(c2) p0 when c2 is given)."""
    if c2 is None:
        return WaveForward.apply(p0, mesh)
    return WaveForwardC2.apply(p0, c2, mesh)
