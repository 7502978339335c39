"""Optimisation drivers: Alg. 1 (resample every step) and Alg. 2 (path
recycling with resampling every N_r steps), built on the C-ABI calls.

One step of Alg. 2 (t = 0, 1, ...):
  if t mod N_r == 0: paths_store(beta_t)     sample + sort, M_ref <- M_t
  paths_reweight(beta_t)                     F(M_t | M_ref)         (Eq. 19/20)
  loss_residual(F, I_gt)                     dL/dI = F - I_gt       (Eq. 7/8)
  render_grad(beta_t, dL/dI)                 recycled PSF gradient  (Eq. 21)
  adam_step(beta_t, grad)                    Adam + projection beta >= 0
Alg. 1 is the same step with N_r = 1 (a fresh, independently seeded path set
every step).  Every call is asynchronous on the current stream; the loss
stays on the device unless read.
"""
from __future__ import annotations

import torch

from . import native as N

# kernels launched per call (for launch accounting)
LAUNCHES = {"store": 5, "reweight": 2, "residual": 1, "grad_cache": 1, "grad": 2, "adam": 1}


class Reconstruction:
    def __init__(self, scene: N.Scene, gt_images: torch.Tensor, beta0: torch.Tensor, n_paths: int,
                 n_r: int = 10, lr: float = 1.0, seed: int = 1234, cache: bool = True,
                 b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.scene = scene
        self.gt = gt_images
        self.beta = beta0.clone().contiguous()
        self.m = torch.zeros_like(self.beta)
        self.v = torch.zeros_like(self.beta)
        self.n_paths = int(n_paths)
        self.n_r = int(n_r)
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.seed = int(seed)
        self.cache = cache
        self.paths = N.Paths(scene)
        self.images = scene.new_images()
        self.dldi = torch.zeros_like(self.images)
        self.grad = torch.zeros(scene.n_voxels, dtype=torch.float64, device=self.beta.device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.beta.device)
        self.t = 0
        self.epoch = 0
        self.launches = 0

    def resample(self):
        self.paths.store(self.beta, self.n_paths, self.seed, epoch=self.epoch)
        self.epoch += 1
        self.launches += LAUNCHES["store"]

    def step(self, timers=None):
        """One Adam step; ``timers`` (optional dict name -> list) receives
        CUDA-event pairs around each call, on the current stream."""
        def ev():
            e = torch.cuda.Event(enable_timing=True)
            e.record()
            return e

        if self.t % self.n_r == 0:
            a = ev() if timers is not None else None
            self.resample()
            if timers is not None:
                timers.setdefault("paths_store", []).append((a, ev()))
        a = ev() if timers is not None else None
        self.paths.reweight(self.beta, self.images, cache=self.cache)
        if timers is not None:
            timers.setdefault("paths_reweight", []).append((a, ev()))
        N.loss_residual(self.images, self.gt, self.dldi, self.loss)
        a = ev() if timers is not None else None
        self.paths.grad(self.beta, self.dldi, self.grad, cache=self.cache)
        if timers is not None:
            timers.setdefault("render_grad", []).append((a, ev()))
        N.adam_step(self.beta, self.m, self.v, self.grad, self.t + 1, self.lr, self.b1, self.b2, self.eps)
        self.launches += LAUNCHES["reweight"] + LAUNCHES["residual"] + LAUNCHES["adam"] + (
            LAUNCHES["grad_cache"] if self.cache else LAUNCHES["grad"])
        self.t += 1
