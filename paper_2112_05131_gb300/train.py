"""The optimisation step of Sec. 3.4 as a sequence of library calls, and the learning-rate schedules.

One step (Supp. A.1: 5000-ray batches, RMSProp, stochastic TV on contiguous segments):
  plx_gen_rays -> plx_render_train -> plx_mse_grad -> plx_render_backward_train -> plx_tv_grad
  -> plx_rmsprop_step
all libplenoxel calls enqueued on one stream with no host synchronisation.  The training march
(plx_render_train: header, plan, chunks, combine; plx_render_backward_train: chunks) splits rays
into chunk work items and hands the march state from the forward to the adjoint.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import torch

from .grid import ROW, Grid, RenderOpts, gen_rays, mse_grad

# kernels one step enqueues with stop_thresh = 0: gen_rays, render_train (header, plan, chunks,
# combine), mse, backward_train, tv, rmsprop (compact, apply; sparse mode)
LAUNCHES_PER_STEP = 11


def lr_sigma(step: int, init: float = 30.0, final: float = 0.05, max_steps: int = 250000, delay_steps: int = 15000,
             delay_mult: float = 0.01) -> float:
    """Delayed exponential decay for density (Supp. A.1, the Mip-NeRF schedule): log-linear from
    `init` to `final` over `max_steps`, scaled during the first `delay_steps` by
    delay_mult + (1 - delay_mult) sin(pi/2 clip(step/delay_steps, 0, 1)).  The paper does not print the
    delay multiplier; 0.01 is this implementation's choice."""
    if delay_steps > 0:
        d = delay_mult + (1.0 - delay_mult) * math.sin(0.5 * math.pi * min(max(step / delay_steps, 0.0), 1.0))
    else:
        d = 1.0
    t = min(max(step / max_steps, 0.0), 1.0)
    return d * math.exp((1.0 - t) * math.log(init) + t * math.log(final))


def lr_sh(step: int, init: float = 1e-2, final: float = 5e-6, max_steps: int = 250000) -> float:
    """Pure exponential decay for the SH coefficients (Supp. A.1)."""
    t = min(max(step / max_steps, 0.0), 1.0)
    return math.exp((1.0 - t) * math.log(init) + t * math.log(final))


@dataclass
class StepConfig:
    batch: int = 5000
    opts: RenderOpts = field(default_factory=lambda: RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0))
    lambda_tv_sigma: float = 1e-5
    lambda_tv_sh: float = 1e-3
    beta: float = 0.95
    eps: float = 1e-8
    sparse_rmsprop: bool = True
    # TV on a second stream, concurrent with ray generation, forward, MSE and adjoint: it reads only
    # rows (unchanged until RMSProp) and adds to the gradient with atomics; RMSProp waits for both
    overlap_tv: bool = True


class Trainer:
    """Holds the optimiser state (gradient rows, RMSProp running average) and the step's scratch buffers."""

    def __init__(self, grid: Grid, cams: torch.Tensor, W: int, H: int, cfg: StepConfig = StepConfig()):
        dev = grid.idx.device
        self.grid = grid
        self.cams = cams
        self.W, self.H = int(W), int(H)
        self.cfg = cfg
        self.grad = torch.zeros((grid.M, ROW), dtype=torch.float32, device=dev)
        self.v = torch.zeros((grid.M, ROW), dtype=torch.float32, device=dev)
        n = cfg.batch
        self.o = torch.empty((n, 3), dtype=torch.float32, device=dev)
        self.d = torch.empty((n, 3), dtype=torch.float32, device=dev)
        self.rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
        self.grad_rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.state = grid.new_march_state(n, cfg.opts)  # fits every batch of up to n rays
        self.side = torch.cuda.Stream(device=dev) if cfg.overlap_tv else None
        self._ev_start = torch.cuda.Event()
        self._ev_tv = torch.cuda.Event()

    def step(self, pix: torch.Tensor, target: torch.Tensor, seg_start: Optional[torch.Tensor],
             seg_len: Optional[torch.Tensor], n_selected: int, lr_s: float, lr_h: float,
             events: Optional[List[torch.cuda.Event]] = None, stream=None):
        """One optimisation step; `events`, if given, must hold 7 events recorded at the stage boundaries of
        the main stream (with overlap_tv the TV stage there is only the wait for the side stream)."""
        g, c = self.grid, self.cfg
        n = pix.shape[0]
        o, d, rgb, grgb = self.o[:n], self.d[:n], self.rgb[:n], self.grad_rgb[:n]
        main = stream if stream is not None else torch.cuda.current_stream()
        do_tv = seg_start is not None and n_selected > 0
        side = self.side if (do_tv and self.side is not None) else None

        def mark(i):
            if events is not None:
                events[i].record(main)

        if side is not None:  # TV starts after everything enqueued so far (the last RMSProp, the inputs)
            self._ev_start.record(main)
            side.wait_event(self._ev_start)
            g.tv_grad(seg_start, seg_len, n_selected, c.lambda_tv_sigma, c.lambda_tv_sh, self.grad, stream=side)
            self._ev_tv.record(side)
        mark(0)
        gen_rays(self.cams, pix, self.W, self.H, o, d, stream=main)
        mark(1)
        g.render_train(o, d, c.opts, self.state, rgb, stream=main)
        mark(2)
        mse_grad(rgb, target, grgb, self.loss, stream=main)
        mark(3)
        g.render_backward_train(o, d, grgb, c.opts, self.state, self.grad, stream=main)
        mark(4)
        if side is not None:
            main.wait_event(self._ev_tv)
        elif do_tv:
            g.tv_grad(seg_start, seg_len, n_selected, c.lambda_tv_sigma, c.lambda_tv_sh, self.grad, stream=main)
        mark(5)
        g.rmsprop_step(self.grad, self.v, lr_s, lr_h, c.beta, c.eps, sparse=c.sparse_rmsprop, stream=main)
        mark(6)
        return rgb

    STAGES = ("gen_rays", "render", "mse_grad", "render_backward", "tv_grad", "rmsprop_step")
