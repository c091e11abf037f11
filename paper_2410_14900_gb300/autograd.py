"""Differentiable Defrise-Clack reconstruction (Ye et al., DRACO, Sec. 2.3).

The network of Eq. 12 with the redundancy weight (Eq. 10) as its only
trainable layer:

    f = ReLU(A3d^T w_d A2d^T D_b (W K) w_sino D_f A2d w_cos g)

forward  -> dc_filter, dc_backproject (optional ReLU)
backward -> dc_backproject_adjoint (masked by the ReLU), dc_filter_adjoint

Between the passes the forward keeps Grangeat's function S (cache_s, the
default: the backward then skips the line-sum pass that would recompute
it), or only g (cache_s=False: S is recomputed view-chunk by view-chunk),
plus W and, with ReLU, the output volume.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import api


class DefriseClackFunction(torch.autograd.Function):
    """f = A3d^T filter(g, W) with gradients for g and W.

    cache_s keeps Grangeat's function S from the forward pass (B*V*n_mu*n_s
    floats) so that the backward skips the line-sum pass that recomputes it;
    without it only g is kept."""

    @staticmethod
    def forward(ctx, g: torch.Tensor, W: Optional[torch.Tensor], geom: api.Geometry,
                relu: bool = False, view_chunk: int = 0, cache_s: bool = True):
        g = g.contiguous()
        Wc = None if W is None else W.contiguous()
        need_grad = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        S = None
        if cache_s and need_grad:
            S = torch.empty((g.shape[0], geom.V) + geom.sino_shape, device=g.device,
                            dtype=torch.float32)
        gF, _ = api.dc_filter(geom, g, Wc, S_out=S)
        vol = api.dc_backproject(geom, gF, relu=relu)
        del gF
        ctx.geom = geom
        ctx.relu = relu
        ctx.view_chunk = view_chunk
        ctx.has_W = W is not None
        ctx.has_S = S is not None
        ctx.save_for_backward(S if S is not None else g,
                              Wc if Wc is not None else g.new_empty(0),
                              vol if relu else g.new_empty(0))
        return vol

    @staticmethod
    def backward(ctx, grad_vol: torch.Tensor):
        kept, W, vol = ctx.saved_tensors
        W = W if ctx.has_W else None
        relu_vol = vol if ctx.relu else None
        need_g, need_W = ctx.needs_input_grad[0], ctx.needs_input_grad[1] and ctx.has_W
        if not (need_g or need_W):
            return None, None, None, None, None, None
        grad_gF = api.dc_backproject_adjoint(ctx.geom, grad_vol.contiguous(), relu_vol)
        if ctx.has_S:
            gg, gW = api.dc_filter_adjoint(ctx.geom, grad_gF, None, W, want_grad_g=need_g,
                                           want_grad_W=need_W, view_chunk=ctx.view_chunk,
                                           S=kept)
        else:
            gg, gW = api.dc_filter_adjoint(ctx.geom, grad_gF, kept, W, want_grad_g=need_g,
                                           want_grad_W=need_W, view_chunk=ctx.view_chunk)
        return gg, gW, None, None, None, None


def reconstruct(g: torch.Tensor, W: Optional[torch.Tensor], geom: api.Geometry,
                relu: bool = False, view_chunk: int = 0, cache_s: bool = True) -> torch.Tensor:
    """Differentiable Eq. 12 (see DefriseClackFunction)."""
    return DefriseClackFunction.apply(g, W, geom, relu, view_chunk, cache_s)


class GaussSmoothFunction(torch.autograd.Function):
    """The Gaussian filter layer on W (Sec. 3.1); backward is its transpose."""

    @staticmethod
    def forward(ctx, W: torch.Tensor, sigma: float, radius: int):
        ctx.sigma, ctx.radius = sigma, radius
        return api.dc_gauss_smooth(W.contiguous(), sigma, radius)

    @staticmethod
    def backward(ctx, grad: torch.Tensor):
        gW = api.dc_gauss_smooth(grad.contiguous(), ctx.sigma, ctx.radius, adjoint=True)
        return gW, None, None


def gauss_smooth(W: torch.Tensor, sigma: float = 20.0, radius: int = 60) -> torch.Tensor:
    """Differentiable Gaussian filter layer on the redundancy weight."""
    return GaussSmoothFunction.apply(W, sigma, radius)


class DefriseClackNet(torch.nn.Module):
    """The reconstruction network with a learnable redundancy weight W.

    W has shape [V, n_mu, n_s] (entry k on the half grid s_{k+1/2}) and is
    multiplied by K = -(1/4pi^2)|v.theta|/sqrt(s^2+D^2) inside the library,
    so W = 1/2 is the exact full-circle value (Eq. 14).  With `smooth` =
    (sigma, radius) the Gaussian filter layer of Sec. 3.1 (sigma 20, kernel
    121: (20.0, 60)) acts on W before the filter.  `init` is a constant or
    "uniform" (U[0, 1]: the paper's U[-1, 0] initialisation of its w_red,
    whose sign K carries here).
    """

    def __init__(self, geom: api.Geometry, init=0.5, relu: bool = True,
                 view_chunk: int = 0, device=None, smooth=None, seed: int = 0,
                 cache_s: bool = True):
        super().__init__()
        self.geom = geom
        self.relu = relu
        self.view_chunk = view_chunk
        self.smooth = smooth
        self.cache_s = cache_s
        shape = (geom.V,) + geom.sino_shape
        if init == "uniform":
            gen = torch.Generator(device="cpu").manual_seed(seed)
            W0 = torch.rand(shape, generator=gen, dtype=torch.float32).to(device)
        else:
            W0 = torch.full(shape, float(init), device=device, dtype=torch.float32)
        self.W = torch.nn.Parameter(W0)

    def weights(self) -> torch.Tensor:
        """The redundancy weight the filter uses (after smoothing, if any)."""
        return gauss_smooth(self.W, *self.smooth) if self.smooth else self.W

    def forward(self, g: torch.Tensor) -> torch.Tensor:
        return reconstruct(g, self.weights(), self.geom, self.relu, self.view_chunk,
                           self.cache_s)
