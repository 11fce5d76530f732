"""The coarse-to-fine optimisation loop (Sec. 3.4 "Coarse to Fine", Supp. B.1) on libplenoxel.

Training starts from a dense low-resolution grid; at fixed steps the grid is pruned and then
upsampled to twice the resolution by trilinear interpolation, and optimisation continues on the
new grid with fresh RMSProp state.  Pruning drops a node when neither it nor any node of its 3x3x3
neighbourhood is hot; hot means a density of at least `prune_tau` (prune_by="density"), or a
largest sample weight over every pixel ray of every training view of at least `weight_tau`
(prune_by="weight", the form the paper uses on synthetic scenes with threshold 0.256).

Every step is Trainer.step (ray generation, training march, MSE gradient, adjoint, TV on a random
1% of the nodes in contiguous segments, sparse RMSProp); the weights are plx_max_weight, prune
and upsample are plx_grid_prune_* / plx_grid_upsample_*.

The training images are the ground-truth grid rendered by plx_render for every training view, copied
once to the device; each step's 5000 pixels and its TV segments are drawn on the device with a seeded
generator, 256 steps at a time, and the pixels' target colours gathered from the device images (the
role a data loader plays).
The paper does not give the steps at which it upsamples for a 128^3 start; `upsample_at` defaults to
thirds of the run.  `paper_synthetic()` is the paper's own synthetic schedule (Supp. B.2).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from .grid import Grid, RenderOpts, gen_rays
from .train import StepConfig, Trainer, lr_sh, lr_sigma


@dataclass
class C2FConfig:
    steps: int = 12800
    start_reso: int = 128
    upsample_at: Sequence[int] = (4266, 8533)
    prune_by: str = "density"  # or "weight"
    prune_tau: float = 5.0
    weight_tau: float = 0.256
    batch: int = 5000
    lambda_tv_sigma: float = 5e-4
    lambda_tv_sh: float = 1e-3
    tv_fraction: float = 0.01
    tv_segment: int = 4096
    tv_until: Optional[int] = None  # steps from which TV is off (Supp. B.2: synthetic scenes keep it for stage 1)
    init_sigma: float = 0.1
    opts: RenderOpts = field(default_factory=lambda: RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0))
    chunk: int = 256  # steps whose pixel batches are prepared and uploaded together
    seed: int = 0
    # record the fraction of rows that receive a gradient at every step (Sec. 3.8: the gradient becomes
    # sparse within the first minutes); each stage's log entry then holds it every `touched_every` steps
    track_touched: bool = False
    touched_every: int = 100
    lr_scale: float = 1.0  # multiplies both learning-rate schedules (0 keeps the grid's values fixed)


def paper_synthetic() -> C2FConfig:
    """The paper's schedule for synthetic scenes (Supp. B.2): a 256^3 start, weight-threshold prune (0.256)
    and upsample to 512^3 after 38400 steps, 128000 steps in all, TV (1e-5 density, 1e-3 SH) during the
    first stage only."""
    return C2FConfig(steps=128000, start_reso=256, upsample_at=(38400,), prune_by="weight", weight_tau=0.256,
                     lambda_tv_sigma=1e-5, lambda_tv_sh=1e-3, tv_until=38400)


def dense_grid(R: int, sigma: float, device="cuda") -> Grid:
    """Every node occupied, density `sigma`, SH zero."""
    idx = torch.arange(R ** 3, dtype=torch.int32, device=device)
    rows = torch.zeros((R ** 3, 32), dtype=torch.float32, device=device)
    rows[:, 0] = sigma
    return Grid(R, idx, rows)


def render_views(grid: Grid, cams: torch.Tensor, W: int, H: int, opts: RenderOpts) -> np.ndarray:
    """All views of `cams` rendered by plx_render, float32 [V, H, W, 3] on the host."""
    V = cams.shape[0]
    out = np.empty((V, H, W, 3), np.float32)
    rgb = torch.empty((W * H, 3), dtype=torch.float32, device=cams.device)
    for v in range(V):
        pix = torch.arange(v * W * H, (v + 1) * W * H, dtype=torch.int64, device=cams.device)
        o, d = gen_rays(cams, pix, W, H)
        grid.render(o, d, opts, rgb)
        out[v] = rgb.view(H, W, 3).cpu().numpy()
    return out


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = float(np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2))
    return float("inf") if mse == 0 else -10.0 * np.log10(mse)


class _Batches:
    """Pixel ids, targets and TV segments for `chunk` steps at a time, drawn on the device with a seeded
    generator, so that a step issues no host work beyond slicing and no copy of its own: pixel ids
    uniform over all pixels of all training views, their target colours gathered from the images on the
    device, and each step's TV segments as a uniformly random set of whole `tv_segment`-node slots of
    the node order (the same distribution as synth.tv_segments), sorted."""

    def __init__(self, images: np.ndarray, cfg: C2FConfig, device):
        self.flat = torch.from_numpy(np.ascontiguousarray(images.reshape(-1, 3), np.float32)).to(device)
        self.n_pix = self.flat.shape[0]
        self.cfg = cfg
        self.dev = device
        self.gen = torch.Generator(device=device)
        self.gen.manual_seed(cfg.seed)
        self.step0 = -1
        self.R = -1
        self.pix = self.tgt = self.ss = self.sl = None

    def get(self, step: int, R: int):
        c = self.cfg
        if self.pix is None or R != self.R or step >= self.step0 + c.chunk or step < self.step0:
            self.step0, self.R = step, R
            self.pix = torch.randint(0, self.n_pix, (c.chunk, c.batch), generator=self.gen, device=self.dev,
                                     dtype=torch.int64)
            self.tgt = self.flat.index_select(0, self.pix.view(-1)).view(c.chunk, c.batch, 3)
            N = R ** 3
            seg = min(c.tv_segment, N)
            n_slots = max(1, N // seg)  # whole slots only, so every segment has `seg` nodes
            n_seg = max(1, min(n_slots, int(round(c.tv_fraction * N / seg))))
            keys = torch.rand((c.chunk, n_slots), generator=self.gen, device=self.dev)
            slots = keys.topk(n_seg, dim=1, sorted=False).indices.sort(dim=1).values
            self.ss = slots.to(torch.int64) * seg
            self.sl = torch.full((c.chunk, n_seg), seg, dtype=torch.int64, device=self.dev)
            self.n_sel = n_seg * seg
        k = step - self.step0
        return self.pix[k], self.tgt[k], self.ss[k], self.sl[k], self.n_sel


def train(train_images: np.ndarray, cams: torch.Tensor, W: int, H: int, cfg: C2FConfig = C2FConfig(),
          log: Optional[List[dict]] = None, start: Optional[Grid] = None) -> Grid:
    """Runs the coarse-to-fine schedule and returns the final grid.  `log` receives one record per stage.
    The run starts from `start` (updated in place) or, by default, a dense cfg.start_reso grid of density
    cfg.init_sigma."""
    dev = cams.device
    grid = start if start is not None else dense_grid(cfg.start_reso, cfg.init_sigma, dev)
    sc = StepConfig(batch=cfg.batch, opts=cfg.opts, lambda_tv_sigma=cfg.lambda_tv_sigma,
                    lambda_tv_sh=cfg.lambda_tv_sh, track_touched=cfg.track_touched)
    tr = Trainer(grid, cams, W, H, sc)
    batches = _Batches(train_images, cfg, dev)
    ups = sorted(int(s) for s in cfg.upsample_at)
    t_stage = time.perf_counter()
    stage_start = 0
    for step in range(cfg.steps):
        if ups and step == ups[0]:
            ups.pop(0)
            tr.finish()
            torch.cuda.synchronize()
            touched = _touched_curve(tr, grid.M, stage_start, cfg)
            before = (grid.reso, grid.M)
            if cfg.prune_by == "weight":
                key = grid.max_weight_views(cams, W, H, cfg.opts)
                pruned = grid.prune(cfg.weight_tau, True, key=key)
                del key
            elif cfg.prune_by == "density":
                pruned = grid.prune(cfg.prune_tau, True)
            else:
                raise ValueError(f"prune_by must be 'density' or 'weight', not {cfg.prune_by!r}")
            grid = pruned.upsample(2 * grid.reso)
            del pruned, tr
            torch.cuda.empty_cache()
            tr = Trainer(grid, cams, W, H, sc)
            torch.cuda.synchronize()
            if log is not None:
                log.append({"step": step, "from": before, "to": (grid.reso, grid.M),
                            "stage_s": time.perf_counter() - t_stage, **touched})
            t_stage = time.perf_counter()
            stage_start = step
        pix, tgt, ss, sl, nsel = batches.get(step, grid.reso)
        if cfg.tv_until is not None and step >= cfg.tv_until:
            ss = sl = None
        # the next batch is planned during this step, unless a prune and upsample come first
        nxt = None
        if step + 1 < cfg.steps and not (ups and step + 1 == ups[0]):
            nxt = batches.get(step + 1, grid.reso)[0]
        tr.step(pix, tgt, ss, sl, nsel, cfg.lr_scale * lr_sigma(step), cfg.lr_scale * lr_sh(step), next_pix=nxt)
    tr.finish()
    torch.cuda.synchronize()
    grid.check()
    if log is not None:
        log.append({"step": cfg.steps, "final": (grid.reso, grid.M), "stage_s": time.perf_counter() - t_stage,
                    **_touched_curve(tr, grid.M, stage_start, cfg)})
    return grid


def _touched_curve(tr: Trainer, M: int, stage_start: int, cfg: C2FConfig) -> dict:
    """The stage's fraction of rows with a gradient, every `touched_every` steps and at its last step."""
    if not cfg.track_touched:
        return {}
    frac = tr.touched_counts() / max(M, 1)
    if frac.size == 0:
        return {}
    keep = list(range(0, frac.size, cfg.touched_every)) + [frac.size - 1]
    return {"touched_frac": {int(stage_start + k): float(frac[k]) for k in keep}}
