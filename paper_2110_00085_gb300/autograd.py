"""torch.autograd.Function mapping cloud extinction to multi-view images.

forward:  stored paths reweighted to the given extinction (Eq. 19/20,
          paths_reweight); with paths stored under the same extinction this
          is the plain estimator of Alg. 1.
backward: render_grad with grad_output as dL/dI (Eq. 21 with the path score
          function of Sec. 4.4).  The stored paths are the checkpoint: the
          backward pass re-traverses them (or reads the per-event
          contributions cached by the forward pass) instead of holding a tape.

The gradient is of the estimator with the paths held fixed, which is what
the paper's recycled gradient estimator computes.
"""
from __future__ import annotations

import torch

from . import native as N


class RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beta: torch.Tensor, paths: N.Paths, cache: bool = True):
        b = beta.detach().contiguous()
        if b.dtype != torch.float32:
            raise TypeError("RenderFn: extinction must be float32")
        images = paths.reweight(b.reshape(-1), cache=cache)
        ctx.paths = paths
        ctx.cache = cache
        ctx.token = paths.cache_token() if cache else 0
        ctx.shape = beta.shape
        ctx.save_for_backward(b)
        return images

    @staticmethod
    def backward(ctx, grad_images: torch.Tensor):
        (b,) = ctx.saved_tensors
        gi = grad_images.detach().to(torch.float64).contiguous()
        # the cache serves only if it still holds this forward's contributions
        # (another forward on the same paths replaces it): else re-trace
        use_cache = ctx.cache and ctx.paths.cache_token() == ctx.token
        g = ctx.paths.grad(b.reshape(-1), gi, cache=use_cache)
        return g.to(torch.float32).reshape(ctx.shape), None, None


def render(beta: torch.Tensor, paths: N.Paths, cache: bool = True) -> torch.Tensor:
    """Differentiable multi-view images (float64) of extinction ``beta``."""
    return RenderFn.apply(beta, paths, cache)
