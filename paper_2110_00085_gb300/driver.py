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

# kernels of this library launched per call (for launch accounting; memsets
# are not counted): store = extinction check + sample + 6 path-sort kernels
# (keys, three-level scan, bucket table, scatter) + 5 event-binning kernels,
# reweight = delta + path weights + event forward, cached gradient = event
# gradient + path gradient, uncached = delta + per-path gradient, counted
# Adam = step counter + update (batched passes: native.Batch.kernels_per_step)
LAUNCHES = {"store": 13, "reweight": 3, "residual": 1, "grad_cache": 2, "grad": 2, "adam": 1,
            "adam_counted": 2}


MAX_CHUNK = 1 << 26   # paths per stored-path handle in ChunkedPaths


class ChunkedPaths:
    """A path set too large for one stored-path handle, kept as handles over
    contiguous ranges of path ids, each normalised by the total count; the
    calls of native.Paths run chunk after chunk, the first writing the
    images / gradient and the others accumulating into them.  The Philox
    streams depend on the path id only, so the result is the single-handle
    result up to the order of the FP64 additions.

    lean=True keeps one chunk's contribution cache at a time: a cached
    reweight computes the images without the cache, and the gradient
    reweights each chunk again with the cache (the same contributions),
    takes its gradient and drops the cache -- one more forward pass per
    step for a cache of one chunk instead of all (at workload 5: about
    35 GB instead of 142 GB)."""

    def __init__(self, scene: N.Scene, chunk: int = MAX_CHUNK, lean: bool = False):
        self.scene = scene
        self.chunk = int(chunk)
        self.lean = bool(lean)
        self.parts = []
        self._scratch = None

    def store(self, beta, n_paths: int, seed: int, epoch: int = 0, images_ref=None, tallies=None,
              fingerprints=None, first: int = 0, n_norm=None):
        """Paths [first, first + n_paths), normalised by n_norm (default n_paths)."""
        n = int(n_paths)
        norm = n if n_norm is None else n_norm
        k = (n + self.chunk - 1) // self.chunk
        while len(self.parts) < k:
            self.parts.append(N.Paths(self.scene))
        while len(self.parts) > k:
            self.parts.pop().close()
        for i, p in enumerate(self.parts):
            off = i * self.chunk
            m = min(self.chunk, n - off)
            p.store(beta, m, seed, first=int(first) + off, n_norm=norm, epoch=epoch, images_ref=images_ref,
                    accumulate=i > 0, tallies=tallies,
                    fingerprints=None if fingerprints is None else fingerprints[off:off + m])
        return self

    def reweight(self, beta_t, images=None, cache: bool = False, accumulate: bool = False):
        if images is None:
            images = self.scene.new_images()
        for i, p in enumerate(self.parts):
            p.reweight(beta_t, images, cache=cache and not self.lean, accumulate=accumulate or i > 0)
        return images

    def grad(self, beta_t, dldi, grad=None, cache: bool = False, accumulate: bool = False):
        if grad is None:
            grad = torch.zeros(self.scene.n_voxels, dtype=torch.float64, device=dldi.device)
        if cache and self.lean:
            if self._scratch is None:
                self._scratch = self.scene.new_images()
            for i, p in enumerate(self.parts):
                p.reweight(beta_t, self._scratch, cache=True)
                p.grad(beta_t, dldi, grad, cache=True, accumulate=accumulate or i > 0)
                p.drop_cache()
            return grad
        for i, p in enumerate(self.parts):
            p.grad(beta_t, dldi, grad, cache=cache, accumulate=accumulate or i > 0)
        return grad

    def info(self) -> dict:
        out = None
        for p in self.parts:
            d = p.info()
            if out is None:
                out = d
            else:
                for key in ("n_paths", "n_stored", "n_records", "bytes_device"):
                    out[key] += d[key]
                out["bucket"] = [a + b for a, b in zip(out["bucket"], d["bucket"])]
        return out

    def close(self):
        for p in self.parts:
            p.close()
        self.parts = []


class Reconstruction:
    """Alg. 2 (Alg. 1 with n_r = 1) on one scene.

    decorrelate=False is the paper's estimator: the residual F - I_gt and the
    image derivative come from the same paths, so the expected gradient is
    the loss gradient plus the gradient of half the summed variance of the
    image estimates, a bias of order 1/N.  decorrelate=True splits the path
    budget into two independent halves A and B (path ids [0, N/2) and
    [N/2, N), each its own estimator) and uses
        g = dF_A/dbeta (F_B - I_gt) + dF_B/dbeta (F_A - I_gt),
    unbiased (each product pairs independent sets) for the same work: two
    reweights and two gradients of N/2 paths.  (g is twice the loss gradient;
    Adam does not see the scale.)  The reported loss is then the mean of the
    two halves' losses.
    """

    def __init__(self, scene: N.Scene, gt_images: torch.Tensor, beta0: torch.Tensor, n_paths: int,
                 n_r: int = 10, lr: float = 1.0, seed: int = 1234, cache: bool = True,
                 b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8, decorrelate: bool = False,
                 lean: bool = False):
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
        self.decorrelate = bool(decorrelate)
        # one handle up to MAX_CHUNK paths, chunked handles above
        per_set = max(count for _, count, _ in self._sets())
        make = (lambda: N.Paths(scene)) if per_set <= MAX_CHUNK else (lambda: ChunkedPaths(scene, lean=lean))
        self.paths = make()
        self.paths_b = make() if self.decorrelate else None
        self.images = scene.new_images()
        self.dldi = torch.zeros_like(self.images)
        self.images_b = scene.new_images() if self.decorrelate else None
        self.dldi_b = torch.zeros_like(self.images) if self.decorrelate else None
        self.loss_b = torch.zeros(1, dtype=torch.float64, device=self.beta.device)
        self.grad = torch.zeros(scene.n_voxels, dtype=torch.float64, device=self.beta.device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.beta.device)
        self.t = 0
        self.epoch = 0
        self._need_store = False
        self.launches = 0
        self.mask = None     # optional uint8 voxel mask: voxels with 0 are not optimised

    def _sets(self):
        """(first id, count, normaliser) of each path set this process stores:
        the whole budget, or its halves A and B when decorrelated."""
        if self.decorrelate:
            h = self.n_paths // 2
            return [(0, h, h), (h, h, h)]
        return [(0, self.n_paths, self.n_paths)]

    def resample(self):
        for handle, (first, count, norm) in zip((self.paths, self.paths_b), self._sets()):
            handle.store(self.beta, count, self.seed, first=first, n_norm=norm, epoch=self.epoch)
        self.epoch += 1
        self.launches += LAUNCHES["store"] * self._parts()

    # the images and the gradient of this process's paths are the whole
    # estimate here; ShardedReconstruction sums them over its ranks
    def _combine_images(self):
        pass

    def _combine_grad(self):
        pass

    def _parts(self) -> int:
        k = len(self.paths.parts) if isinstance(self.paths, ChunkedPaths) else 1
        return 2 * k if self.decorrelate else k

    def step(self, timers=None):
        """One Adam step; ``timers`` (optional dict name -> list) receives
        CUDA-event pairs around each call, on the current stream."""
        def ev():
            e = torch.cuda.Event(enable_timing=True)
            e.record()
            return e

        if self.t % self.n_r == 0 or self._need_store:
            self._need_store = False
            a = ev() if timers is not None else None
            self.resample()
            if timers is not None:
                timers.setdefault("paths_store", []).append((a, ev()))
        a = ev() if timers is not None else None
        self.paths.reweight(self.beta, self.images, cache=self.cache)
        if self.decorrelate:
            self.paths_b.reweight(self.beta, self.images_b, cache=self.cache)
        self._combine_images()
        if timers is not None:
            timers.setdefault("paths_reweight", []).append((a, ev()))
        N.loss_residual(self.images, self.gt, self.dldi, self.loss)
        if self.decorrelate:
            N.loss_residual(self.images_b, self.gt, self.dldi_b, self.loss_b)
        a = ev() if timers is not None else None
        if self.decorrelate:
            # each half's derivative against the other half's residual
            self.paths.grad(self.beta, self.dldi_b, self.grad, cache=self.cache)
            self.paths_b.grad(self.beta, self.dldi, self.grad, cache=self.cache, accumulate=True)
            self.loss.add_(self.loss_b).mul_(0.5)
        else:
            self.paths.grad(self.beta, self.dldi, self.grad, cache=self.cache)
        self._combine_grad()
        if timers is not None:
            timers.setdefault("render_grad", []).append((a, ev()))
        N.adam_step(self.beta, self.m, self.v, self.grad, self.t + 1, self.lr, self.b1, self.b2, self.eps,
                    mask=self.mask)
        lean = isinstance(self.paths, ChunkedPaths) and self.paths.lean and self.cache
        self.launches += self._parts() * ((2 if lean else 1) * LAUNCHES["reweight"] + (
            LAUNCHES["grad_cache"] if self.cache else LAUNCHES["grad"])) + LAUNCHES["residual"] * (
            2 if self.decorrelate else 1) + LAUNCHES["adam"]
        self.t += 1

    def snapshot(self) -> dict:
        """Optimisation state (extinction, Adam moments, step and resample
        counters), for checkpoint / resume."""
        return {"beta": self.beta.clone(), "m": self.m.clone(), "v": self.v.clone(), "t": self.t,
                "epoch": self.epoch}

    def restore(self, snap: dict):
        """Back to a snapshot (tensors copied in place).  From a snapshot
        taken at a resample boundary (t mod N_r == 0) the next steps repeat
        exactly: the resample draws the same paths (same seeds and epoch)."""
        self.beta.copy_(snap["beta"])
        self.m.copy_(snap["m"])
        self.v.copy_(snap["v"])
        self.t = snap["t"]
        self.epoch = snap["epoch"]

    def save(self, path: str):
        """Checkpoint to a file: the snapshot, the voxel mask (the carved hull,
        or None) and the settings that define the path sets and the steps
        (path budget, N_r, seed, estimator, step size)."""
        snap = {k: (v.cpu() if torch.is_tensor(v) else v) for k, v in self.snapshot().items()}
        snap.update(n_paths=self.n_paths, n_r=self.n_r, seed=self.seed, decorrelate=self.decorrelate,
                    lr=float(self.lr), mask=None if self.mask is None else self.mask.to(torch.uint8).cpu())
        torch.save(snap, path)

    def load(self, path: str):
        """Resume from save(): exact from a resample boundary (t mod N_r == 0,
        the same paths are drawn again); elsewhere the next step draws paths
        at the loaded extinction, as its stored paths are not in the file.
        The voxel mask is restored; a checkpoint of another path budget, N_r,
        seed, estimator or step size is refused."""
        snap = torch.load(path, map_location="cpu")
        for k in ("n_paths", "n_r", "seed", "decorrelate", "lr"):
            if snap[k] != getattr(self, k):
                raise ValueError(f"checkpoint {k} = {snap[k]} differs from this run's {getattr(self, k)}")
        self.restore(snap)
        m = snap.get("mask")
        self.mask = None if m is None else m.to(device=self.beta.device, dtype=torch.uint8).contiguous()
        self._need_store = self.t % self.n_r != 0

    def close(self):
        self.paths.close()
        if self.paths_b is not None:
            self.paths_b.close()


def shard_range(n_paths: int, rank: int, world: int):
    """The contiguous path ids [first, first + count) of one rank when a set of
    n_paths paths is split over `world` ranks: shares differ by at most one
    path, the first n_paths mod world ranks take the larger ones, and the
    ranges tile [0, n_paths) in rank order.  Paths are independent (Sec. 5.3),
    and each path's random stream depends on its id only, so the union of the
    shards is the same path set as one process's."""
    n, r, w = int(n_paths), int(rank), int(world)
    if w < 1 or not 0 <= r < w or n < 0:
        raise ValueError(f"shard_range: rank {r} of world {w}, {n} paths")
    base, extra = divmod(n, w)
    return r * base + min(r, extra), base + (1 if r < extra else 0)


def allreduce_sum(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sum a tensor over the ranks of a process group, in place (NCCL on GPUs;
    gloo also takes CUDA tensors).  Every rank receives the same bits."""
    import torch.distributed as td
    td.all_reduce(t, op=td.ReduceOp.SUM, group=group)
    return t


class ShardedReconstruction(Reconstruction):
    """Alg. 2 with the path budget split over the ranks of a process group,
    one GPU per rank.  Each rank stores the ids shard_range gives it of every
    path set, normalised by the set's total, so its images and gradient are
    its part of the sums over paths (Eq. 19 and Eq. 21 are sums over
    independent paths).  A step is then:
      paths_reweight on the rank's paths       partial images
      all-reduce of the FP64 images            the whole estimate F
      loss_residual(F, I_gt)                   the same dL/dI on every rank
      render_grad on the rank's paths          partial gradient
      all-reduce of the FP64 gradient          the whole gradient
      adam_step                                the same extinction on every rank
    The two all-reduces are the only exchange: the extinction, the Adam
    moments and the residual stay replicated, and every rank applies the same
    update to the same bits.  With one rank it is Reconstruction."""

    def __init__(self, scene: N.Scene, gt_images: torch.Tensor, beta0: torch.Tensor, n_paths: int, group=None,
                 **kw):
        import torch.distributed as td
        self.group = group
        self.rank = td.get_rank(group) if td.is_initialized() else 0
        self.world = td.get_world_size(group) if td.is_initialized() else 1
        half = int(n_paths) // 2 if kw.get("decorrelate") else int(n_paths)
        if half < self.world:
            raise ValueError(f"ShardedReconstruction: {half} paths per set cannot give each of {self.world} "
                             "ranks at least one")
        super().__init__(scene, gt_images, beta0, n_paths, **kw)

    def _sets(self):
        out = []
        for first, count, norm in super()._sets():
            f, c = shard_range(count, self.rank, self.world)
            out.append((first + f, c, norm))
        return out

    def _combine_images(self):
        if self.world > 1:
            allreduce_sum(self.images, self.group)
            if self.decorrelate:
                allreduce_sum(self.images_b, self.group)

    def _combine_grad(self):
        if self.world > 1:
            allreduce_sum(self.grad, self.group)


class BatchReconstruction:
    """Alg. 2 on many scenes at once: every pass of a step is one persistent
    launch over all scenes (``native.Batch``).  The step after the optional
    resample (reweight, residuals, gradient, Adam) has fixed buffers and a
    device-side Adam step counter, so it can be captured once in a CUDA graph
    and replayed every step."""

    def __init__(self, scenes, gts, beta0s, n_paths, n_r: int = 10, lrs=None, seeds=None,
                 b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.scenes = list(scenes)
        n = len(self.scenes)
        self.gts = list(gts)
        self.beta = [b.clone().contiguous() for b in beta0s]
        self.m = [torch.zeros_like(b) for b in self.beta]
        self.v = [torch.zeros_like(b) for b in self.beta]
        dev = self.beta[0].device
        self.steps = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in range(n)]
        self.scratch = [torch.zeros(2, dtype=torch.float32, device=dev) for _ in range(n)]
        self.n_paths = [int(k) for k in n_paths]
        self.n_r = int(n_r)
        self.lrs = list(lrs) if lrs is not None else [1.0] * n
        self.seeds = list(seeds) if seeds is not None else [1234 + i for i in range(n)]
        self.b1, self.b2, self.eps = b1, b2, eps
        self.paths = [N.Paths(sc) for sc in self.scenes]
        self.images = [sc.new_images() for sc in self.scenes]
        self.dldi = [torch.zeros_like(im) for im in self.images]
        self.grad = [torch.zeros(sc.n_voxels, dtype=torch.float64, device=dev) for sc in self.scenes]
        self.loss = [torch.zeros(1, dtype=torch.float64, device=dev) for _ in range(n)]
        self.t = 0
        self.epoch = 0
        self.batch = None
        self.graph = None
        self.launches = 0

    def resample(self):
        for p, b, n, s in zip(self.paths, self.beta, self.n_paths, self.seeds):
            p.store(b, n, s, epoch=self.epoch)
        self.epoch += 1
        if self.batch is None:
            self.batch = N.Batch(self.paths)
        self.batch.bind(self.beta, self.images, self.dldi, self.grad)
        # the grouped schedule passes the scene table by value: a graph
        # captured before this bind may hold stale descriptors
        self.graph = None
        self.launches += LAUNCHES["store"] * len(self.scenes)

    def snapshot(self) -> dict:
        """Optimisation state (extinction, Adam moments and step counters,
        step and resample counters), for checkpoint / resume."""
        return {"beta": [b.clone() for b in self.beta], "m": [x.clone() for x in self.m],
                "v": [x.clone() for x in self.v], "steps": [x.clone() for x in self.steps],
                "t": self.t, "epoch": self.epoch}

    def restore(self, snap: dict):
        """Back to a snapshot; tensors are copied in place (the bound batch
        and any captured graph point at them).  From a snapshot taken at a
        resample boundary (t mod N_r == 0) the next steps repeat exactly:
        the resample draws the same paths (same seeds and epoch)."""
        for name in ("beta", "m", "v", "steps"):
            for dst, src in zip(getattr(self, name), snap[name]):
                dst.copy_(src)
        self.t = snap["t"]
        self.epoch = snap["epoch"]
        self.graph = None

    def set_launch(self, reg_cap: int, blocks_per_sm: int):
        """Launch shape of the batched passes (see native.Batch.set_launch);
        the step graph is captured again with it."""
        self.batch.set_launch(reg_cap, blocks_per_sm)
        self.graph = None

    def _body(self, batched: bool = True):
        if batched:
            self.batch.reweight(cache=True)
        else:
            for p, b, im in zip(self.paths, self.beta, self.images):
                p.reweight(b, im, cache=True)
        for im, gt, d, l in zip(self.images, self.gts, self.dldi, self.loss):
            N.loss_residual(im, gt, d, l)
        if batched:
            self.batch.grad(cache=True)
        else:
            for p, b, d, g in zip(self.paths, self.beta, self.dldi, self.grad):
                p.grad(b, d, g, cache=True)
        for b, m, v, g, st, sc, lr in zip(self.beta, self.m, self.v, self.grad, self.steps, self.scratch, self.lrs):
            N.adam_step_counted(b, m, v, g, st, sc, lr, self.b1, self.b2, self.eps)

    def step(self, use_graph: bool = False, batched: bool = True):
        """One Adam step on every scene.  ``batched=False`` issues the
        per-scene calls one scene after another on the same state (the
        comparison the batched launch is measured against)."""
        if self.t % self.n_r == 0:
            self.resample()
        if not batched:
            self._body(batched=False)
            n = len(self.scenes)
            self.launches += n * (LAUNCHES["reweight"] + LAUNCHES["residual"] + LAUNCHES["grad_cache"]
                                  + LAUNCHES["adam_counted"])
            self.t += 1
            return
        if use_graph:
            if self.graph is None:
                # capture after each resample / launch-shape change; buffers,
                # the batch table and the Adam counters are fixed in between,
                # so the same graph serves the steps until the next one
                torch.cuda.synchronize()
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph):
                    self._body()
            self.graph.replay()
        else:
            self._body()
        n = len(self.scenes)
        self.launches += n * (LAUNCHES["residual"] + LAUNCHES["adam_counted"]) + sum(self.batch.kernels_per_step())
        self.t += 1


def recon_errors(beta_true: torch.Tensor, beta: torch.Tensor):
    """Reconstruction quality of Sec. 6: relative L1 distance
    eps = |b* - b|_1 / |b*|_1 and relative mass bias
    delta = (|b*|_1 - |b|_1) / |b*|_1."""
    t = beta_true.double()
    b = beta.double()
    m = float(t.abs().sum())
    return float((t - b).abs().sum()) / m, (m - float(b.abs().sum())) / m


class CoarseToFine:
    """The reconstruction schedule of Sec. 6 on a synthetic scene: the true
    field renders the ground-truth images, space carving of the first
    level's images gives the photo-hull, which starts at the cloud's mean
    extinction, and Alg. 2 runs at increasing image resolution and path
    budget, moving on when the loss saturates.

    Readings (the paper gives the method, not its constants):
    - clear pixel: radiance at or below ``carve_frac`` of the mean lit
      pixel of the first level's ground truth;
    - the hull's starting value: the true field's mean over its cloud
      voxels, those above 5% of its maximum (the cloud's average
      extinction; smooth fields have long thin tails);
    - saturation: the mean loss of the last ``window`` steps is less than
      ``min_gain`` below that of the ``window`` steps before;
    - Adam restarts at each level; each level's ground truth is rendered
      at its resolution from the true field with an independent seed and
      ``gt_factor`` times its path budget;
    - only the photo-hull is optimised (the other voxels stay at 0), and by
      default with the decorrelated (unbiased) gradient of Reconstruction;
    - the step size decays as lr / (1 + k / lr_decay) over the run's steps k
      (lr_decay 0: constant), one reading of the paper's "modified Adam": at
      a fixed budget, late gradients are dominated by noise, and a constant
      step lets voxels outside the cloud random-walk upward against the
      projection beta >= 0.
    """

    def __init__(self, spec, beta_true, levels, n_r: int = 10, lr: float = None, seed: int = 1234,
                 gt_factor: int = 4, carve_frac: float = 0.05, window: int = 5, min_gain: float = 0.01,
                 max_steps_per_level: int = 40, decorrelate: bool = True, lr_decay: float = 0.0):
        import dataclasses
        self._replace = dataclasses.replace
        self.spec = spec
        self.beta_true = beta_true.contiguous()
        self.levels = [(int(px), int(n)) for px, n in levels]
        self.n_r, self.seed, self.gt_factor = int(n_r), int(seed), int(gt_factor)
        self.lr = float(lr) if lr is not None else float(beta_true.max()) / 50.0
        self.carve_frac, self.window, self.min_gain = carve_frac, int(window), float(min_gain)
        self.max_steps_per_level = int(max_steps_per_level)
        self.decorrelate = bool(decorrelate)
        self.lr_decay = float(lr_decay)
        self.level = -1
        self.history = []
        self.rec = None
        self.beta = None
        self.hull = None

    @staticmethod
    def cloud_mean(beta_true: torch.Tensor) -> float:
        cloud = beta_true[beta_true > 0.05 * float(beta_true.max())]
        return float(cloud.mean()) if cloud.numel() else 0.0

    def _level(self, k):
        px, n = self.levels[k]
        cams = [self._replace(c, width=px, height=px) for c in self.spec.cameras]
        scene = N.Scene(self.spec.replace(cameras=cams, n_paths=n))
        gt = scene.new_images()
        m = self.gt_factor
        for j in range(m):   # independent seed, m x the level's budget, in chunks of n
            scene.render_forward(self.beta_true, n, self.seed + 7919, first=j * n, n_norm=m * n, images=gt,
                                 accumulate=j > 0)
        return scene, gt

    def _start_level(self, k):
        scene, gt = self._level(k)
        if k == 0:
            lit = gt[gt > 0]
            thr = self.carve_frac * float(lit.mean()) if lit.numel() else 0.0
            self.hull = scene.space_carve(gt, thr)
            start = self.cloud_mean(self.beta_true)
            self.beta = self.hull.to(torch.float32) * start
        n = self.levels[k][1]
        self.rec = Reconstruction(scene, gt, self.beta, n, n_r=self.n_r, lr=self.lr, seed=self.seed + 101 * k,
                                  decorrelate=self.decorrelate)
        self.rec.mask = self.hull     # only the photo-hull is optimised
        self.level = k
        self.level_losses = []

    def saturated(self) -> bool:
        w = self.window
        L = self.level_losses
        if len(L) >= self.max_steps_per_level:
            return True
        if len(L) < 2 * w:
            return False
        prev, last = sum(L[-2 * w:-w]) / w, sum(L[-w:]) / w
        return (prev - last) < self.min_gain * prev

    def step(self):
        """One Adam step (starting the first or next level when due);
        returns False when the last level has saturated."""
        if self.level < 0:
            self._start_level(0)
        elif self.saturated():
            if self.level + 1 >= len(self.levels):
                return False
            self.beta = self.rec.beta.clone()
            self.rec.close()
            self._start_level(self.level + 1)
        if self.lr_decay > 0:
            self.rec.lr = self.lr / (1.0 + len(self.history) / self.lr_decay)
        e = torch.cuda.Event(enable_timing=True)
        f = torch.cuda.Event(enable_timing=True)
        e.record()
        self.rec.step()
        f.record()
        torch.cuda.synchronize()
        loss = float(self.rec.loss)
        self.level_losses.append(loss)
        eps, delta = recon_errors(self.beta_true, self.rec.beta)
        self.history.append({"level": self.level, "px": self.levels[self.level][0],
                             "paths": self.levels[self.level][1], "loss": loss, "eps": eps, "delta": delta,
                             "ms": e.elapsed_time(f)})
        return True

    def run(self, max_steps: int):
        for _ in range(max_steps):
            if not self.step():
                break
        return self.history


class SurfReconstruction:
    """Recovery of the Phong parameters of the central sphere (Sec. 6,
    reflectometry) by Adam on the image loss, the stored paths re-evaluated
    for n_r steps between re-tracings (n_r = 1: a new path set every step).

    (kappa, gamma) live on the device: the re-evaluation, the gradient and
    the Adam step (on (kappa, gamma / gamma_scale), so one step size suits
    both, step size lr / (1 + (t - 1) / lr_decay), projected onto
    0 <= kappa <= 1, gamma >= 0) read and write them there, so a step needs no host round trip and the steps between
    re-tracings replay one CUDA graph.  The path pdf does not depend on the
    parameters, so re-evaluated paths add no importance-weight variance;
    only re-tracing costs.  ``trace`` steps of (kappa, gamma) are recorded
    on the device.  The parameter error is
    eps = (|kappa - kappa*| / kappa* + |gamma - gamma*| / gamma*) / 2
    (a reading: the paper gives no eps for this scene).

    decorrelate: the paths are stored as two halves A and B, and the
    gradient is dF_A (F_B - y) + dF_B (F_A - y) (twice the gradient, in
    expectation exactly the gradient of the expected loss).  With one set,
    the expectation of dF (F - y) adds half the gradient of the image
    variance, which pulls gamma, whose loss curvature is weak, off the
    truth."""

    def __init__(self, scene, gt_images: torch.Tensor, kappa0: float, gamma0: float, n_paths: int,
                 n_r: int = 30, lr: float = 0.05, gamma_scale: float = 50.0, seed: int = 1234,
                 b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8, trace: int = 0,
                 decorrelate: bool = True, lr_decay: float = 0.0):
        self.scene = scene
        self.gt = gt_images
        self.scale = float(gamma_scale)
        self.decorrelate = bool(decorrelate)
        self.theta = torch.tensor([kappa0, gamma0], dtype=torch.float32, device="cuda")
        self.m = torch.zeros(2, dtype=torch.float32, device="cuda")
        self.v = torch.zeros_like(self.m)
        self.counter = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.trace = torch.zeros(2 * trace, dtype=torch.float32, device="cuda") if trace > 0 else None
        self.n_paths, self.n_r, self.lr, self.seed = int(n_paths), int(n_r), float(lr), int(seed)
        self.lr_decay = float(lr_decay)
        self.b1, self.b2, self.eps = b1, b2, eps
        self.paths = N.SurfPaths(scene)
        self.images = scene.new_images()
        self.dldi = torch.zeros_like(self.images)
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        if self.decorrelate:
            self.paths_b = N.SurfPaths(scene)
            self.images_b = scene.new_images()
            self.dldi_b = torch.zeros_like(self.images)
            self.loss_b = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.g = torch.zeros(2, dtype=torch.float64, device="cuda")
        self.graph = None
        self.t = 0
        self.epoch = 0
        self.launches = 0

    @property
    def params(self):
        k, g = self.theta.tolist()
        return k, g

    def _store(self):
        n = self.n_paths
        sort = self.n_r > 1        # sorting events by pixel pays off only for re-used paths
        if self.decorrelate:
            h = n // 2
            self.paths.store(h, self.seed, first=0, epoch=self.epoch, sort=sort)
            self.paths_b.store(n - h, self.seed, first=h, epoch=self.epoch, sort=sort)
        else:
            self.paths.store(n, self.seed, epoch=self.epoch, sort=sort)

    def _body(self):
        self.paths.reweight_dev(self.theta, self.images)
        N.loss_residual(self.images, self.gt, self.dldi, self.loss)
        if self.decorrelate:
            self.paths_b.reweight_dev(self.theta, self.images_b)
            N.loss_residual(self.images_b, self.gt, self.dldi_b, self.loss_b)
            self.paths.grad_dev(self.theta, self.dldi_b, self.g)
            self.paths_b.grad_dev(self.theta, self.dldi, self.g, accumulate=True)
        else:
            self.paths.grad_dev(self.theta, self.dldi, self.g)
        N.surf_adam_step(self.theta, self.m, self.v, self.g, self.counter, self.lr, self.scale, self.b1, self.b2,
                         self.eps, trace=self.trace, lr_decay=self.lr_decay)

    def prepare(self):
        """Allocate the stored-path buffers and capture the step graph
        without taking a step (the first step traces the paths again)."""
        if self.graph is None:
            self._store()
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._body()

    def step(self, use_graph: bool = False):
        if self.t % self.n_r == 0:
            self._store()
            self.epoch += 1
            self.launches += (4 if self.n_r > 1 else 1) * (2 if self.decorrelate else 1)   # trace (+ sort)
        if use_graph:
            if self.graph is None:
                # the stored-path buffers keep their addresses across
                # re-tracings of the same size (this driver's n_paths is
                # fixed), so one capture serves the run; a store that grew a
                # handle would need a new capture
                torch.cuda.synchronize()
                self.graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph):
                    self._body()
            self.graph.replay()
        else:
            self._body()
        self.launches += 7 if self.decorrelate else 4
        self.t += 1

    def error(self, kappa_true: float, gamma_true: float) -> float:
        k, g = self.params
        return surf_error(k, g, kappa_true, gamma_true)

    def close(self):
        self.graph = None
        self.paths.close()
        if self.decorrelate:
            self.paths_b.close()


def surf_error(kappa, gamma, kappa_true: float, gamma_true: float):
    """Mean relative error of the Phong parameters (scalars or arrays)."""
    return 0.5 * (abs(kappa - kappa_true) / kappa_true + abs(gamma - gamma_true) / gamma_true)
