"""Autograd wrapper of the differentiable relaxation of the render.

The relaxed render (exact bilinear motion-compensation weights, YCoCg-R
inverse with /2, no clamp) is linear in the dequantised coefficients and
root images for the stream's fixed motion vectors and signs.  Its forward
and adjoint are library kernels (hmlfc_render_views_relaxed,
hmlfc_render_backward); the adjoint recomputes every ray's samples instead
of storing anything from the forward.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import Stream, render_backward, render_views_relaxed, requantize


class RelaxedRender(torch.autograd.Function):
    """out = render(coeff, root) for one stream; views is a numpy array of
    96-byte view records (lf = 0).  bias adds the expected rounding of the
    integer decode (constant terms: the same adjoint)."""

    @staticmethod
    def forward(ctx, coeff: torch.Tensor, root: torch.Tensor, stream: Stream, views, bias: bool = False):
        coeff = coeff.contiguous()
        root = root.contiguous()
        out = render_views_relaxed([stream], [coeff], [root], views, bias=bias)
        ctx.stream = stream
        ctx.views = views
        ctx.shapes = (coeff.shape, root.shape)
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        gc = torch.zeros(ctx.shapes[0], dtype=torch.float32, device=grad_out.device)
        gr = torch.zeros(ctx.shapes[1], dtype=torch.float32, device=grad_out.device)
        render_backward([ctx.stream], ctx.views, grad_out.contiguous().float(), [gc], [gr])
        return gc, gr, None, None, None


def relaxed_render(coeff, root, stream, views, bias: bool = False):
    return RelaxedRender.apply(coeff, root, stream, views, bias)


def _ste_round(x: torch.Tensor, step: float) -> torch.Tensor:
    """step * round(x / step) in the forward pass, identity gradient."""
    return x + (torch.round(x / step) * step - x).detach()


def refine(stream: Stream, views, target: torch.Tensor, steps: int = 200, lr: float | None = None,
           refine_roots: bool = True, log_every: int = 0, quantise_aware: bool = False, bias: bool = False):
    """Adam on the dequantised coefficients (and roots) of a stream so that
    its relaxed render approaches `target`; returns (coeff, root, losses).

    With quantise_aware the forward pass renders the coefficients rounded to
    the stream's quantiser step (and the roots to integers) while the
    gradient passes straight through, so that the optimum survives the
    re-quantisation.  With bias the relaxed render carries the integer
    decode's expected rounding, so that its optimum is not offset from the
    integer render's."""
    coeff, root = stream.dequant()
    coeff = coeff.clone().requires_grad_(True)
    root = root.clone().requires_grad_(refine_roots)
    q = stream.info["qstep"]
    lr = 0.25 * q if lr is None else lr
    params = [coeff] + ([root] if refine_roots else [])
    opt = torch.optim.Adam(params, lr=lr)
    losses = []
    for it in range(steps):
        opt.zero_grad(set_to_none=True)
        if quantise_aware:
            out = relaxed_render(_ste_round(coeff, float(q)), _ste_round(root, 1.0), stream, views, bias)
        else:
            out = relaxed_render(coeff, root, stream, views, bias)
        loss = torch.mean((out - target) ** 2)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
        if log_every and it % log_every == 0:
            print(f"step {it}: loss {losses[-1]:.6e}")
    return coeff.detach(), root.detach(), losses


def requantized_stream(stream: Stream, coeff: torch.Tensor, root: torch.Tensor) -> bytes:
    """Write a stream from refined coefficients at the same quantiser step,
    motion vectors and signs."""
    return requantize(stream, coeff.cpu().numpy(), root.cpu().numpy())


def psnr(a: torch.Tensor, b: torch.Tensor, peak: float = 1.0) -> float:
    mse = float(torch.mean((a.double() - b.double()) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(peak * peak / mse)
