"""torch.autograd wrappers of the marching-cubes adjoint and the distance
loss (both hand-written CUDA in libchr), and the attribution of isosurface
error to grid points and 8^3 CHR bricks.

    tris = Isosurface.apply(field, k, cap)        # (T, 3, 3) vertex positions
    loss = DistanceLoss.apply(tris, orig, k)      # mean distance to orig's surface
    loss.backward()                               # field.grad = dloss/dfield

The forward passes return what isosurface_extract and
isosurface_distance_loss compute; the backward passes call
isosurface_backward (deterministic fixed-point sums) and use the loss
gradient the loss kernel produced in the same launch.
"""
from __future__ import annotations

import torch

from . import chr


class Isosurface(torch.autograd.Function):
    @staticmethod
    def forward(ctx, field: torch.Tensor, isovalue: float, cap: int):
        tris, counts, err = chr.isosurface_extract(field, [isovalue], cap)
        n = int(counts[0].item())
        if int(err.item()) != 0 or n > cap:
            raise RuntimeError(f"isosurface_extract: {n} triangles do not fit cap {cap}")
        ctx.save_for_backward(field)
        ctx.isovalue, ctx.cap, ctx.n = float(isovalue), int(cap), n
        return tris[0, :n]

    @staticmethod
    def backward(ctx, grad_tris):
        (field,) = ctx.saved_tensors
        g = torch.zeros((1, ctx.cap, 3, 3), dtype=torch.float32, device=field.device)
        g[0, :ctx.n] = grad_tris
        return chr.isosurface_backward(field, [ctx.isovalue], g, ctx.cap), None, None


class DistanceLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tris: torch.Tensor, orig: torch.Tensor, isovalue: float):
        loss, grad = chr.isosurface_distance_loss(orig, isovalue, tris.contiguous())
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (grad,) = ctx.saved_tensors
        return (grad * grad_loss.to(grad.dtype)).view(-1, 3, 3), None, None


def brick_attribution(grad_field: torch.Tensor) -> torch.Tensor:
    """Sum of |dL/dfield| over every 8^3 brick (x-fastest brick order, the
    CHR's brick order), by the library (chr_brick_abs_sum): the bricks with
    the largest values are the ones whose refinement moves the loss most."""
    return chr.chr_brick_abs_sum(grad_field.contiguous())
