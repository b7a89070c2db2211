"""torch.autograd.Function over lodgs_render / lodgs_render_backward.

The differentiable input is the scene's record tensor (n_nodes x stride,
render-row order); only the rows of the view's LoD cut receive gradients, as in
the paper's training, where optimisation touches the cut set only (appendix,
Implementation Details).  The backward recomputes each pixel's transmittance
from the sorted per-tile lists, front to back, and takes the colour behind
each Gaussian from the rendered image (saved for backward); nothing else per
pixel is stored by the forward.
"""
from __future__ import annotations

import torch

from . import api


class LodRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rows: torch.Tensor, scene: api.Scene, frame: api.Frame, bg: tuple):
        rows_c = rows.detach().contiguous()
        img = api.render(scene, frame, rows=rows_c, bg=bg)
        ctx.scene, ctx.frame = scene, frame
        ctx.save_for_backward(rows_c, img)
        return img

    @staticmethod
    def backward(ctx, grad_img: torch.Tensor):
        rows_c, img = ctx.saved_tensors
        grad = torch.zeros_like(rows_c)
        api.render_backward(ctx.scene, ctx.frame, grad_img.contiguous(), rows=rows_c, grad=grad, dense=True,
                            image=img)
        return grad, None, None, None


def render(rows: torch.Tensor, scene: api.Scene, camera, frame: api.Frame | None = None,
           bg=(0.0, 0.0, 0.0)) -> torch.Tensor:
    """Differentiable LoD render of `camera`: select the cut, render it, and on
    backward return dense record gradients (zero outside the cut).  A frame holds
    one view's state until its backward has run, so pass a distinct frame (or
    none) for every render whose backward is still pending."""
    fr = api.select_lod(scene, camera, frame)
    return LodRender.apply(rows, scene, fr, tuple(float(b) for b in bg))
