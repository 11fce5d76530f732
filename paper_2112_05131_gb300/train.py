"""The optimisation step of Sec. 3.5 as a sequence of library calls, and the learning-rate schedules.

One step (Supp. B.1: 5000-ray batches, RMSProp, stochastic TV on contiguous segments):
  plx_gen_rays -> plx_march_plan -> plx_render_planned_mse (forward and MSE gradient)
  -> plx_render_backward_train (with the Cauchy sparsity prior when configured) -> plx_tv_grad
  -> plx_rmsprop_step
all libplenoxel calls with no host synchronisation.  The training march splits rays into chunk work
items and hands the march state from the forward to the adjoint.

With overlap (the default) the calls use three streams and RMSProp is deferred to the start of the next
step (or to finish()): ray generation and the plan read no rows, so the next batch's are computed while
the previous update runs; TV reads rows only and adds to the gradient with atomics, so it runs beside
the forward and adjoint.  Every step computes exactly what the serial order computes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import torch

from .grid import ROW, Grid, RenderOpts, gen_rays

# kernels one step enqueues with stop_thresh = 0: gen_rays, march_plan (header, setup, plan),
# render_planned_mse (chunks, combine with the MSE gradient), backward_train, tv, rmsprop (compact, apply)
LAUNCHES_PER_STEP = 10


def lr_sigma(step: int, init: float = 30.0, final: float = 0.05, max_steps: int = 250000, delay_steps: int = 15000,
             delay_mult: float = 0.01) -> float:
    """Delayed exponential decay for density (Supp. B.1, the Mip-NeRF schedule): log-linear from
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
    """Pure exponential decay for the SH coefficients (Supp. B.1)."""
    t = min(max(step / max_steps, 0.0), 1.0)
    return math.exp((1.0 - t) * math.log(init) + t * math.log(final))


@dataclass
class StepConfig:
    batch: int = 5000
    opts: RenderOpts = field(default_factory=lambda: RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0))
    lambda_tv_sigma: float = 1e-5
    lambda_tv_sh: float = 1e-3
    # Cauchy sparsity prior on the samples' densities (Sec. 3.7; the paper uses 1e-12 on forward-facing and
    # 1e-11 on 360-degree scenes, none on synthetic ones), fused into the adjoint; its value accumulates in
    # Trainer.loss_sparsity
    lambda_sparsity: float = 0.0
    beta: float = 0.95
    eps: float = 1e-8
    sparse_rmsprop: bool = True
    # three streams and a deferred RMSProp (see the module docstring); False: one stream, in order
    overlap: bool = True
    # record, every step, how many rows received a gradient (plx_count_touched; Sec. 3.8's gradient
    # sparsity), into Trainer.touched_counts()
    track_touched: bool = False


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
        self.loss_sparsity = torch.zeros(1, dtype=torch.float32, device=dev)
        self.state = grid.new_march_state(n, cfg.opts)  # fits every batch of up to n rays
        if cfg.overlap:
            # the march (update, forward, MSE, adjoint) and the plan on high-priority streams, TV on a
            # low-priority one: when both have blocks waiting, the scheduler starts the march's first
            # and TV fills what is left
            self.march_stream = torch.cuda.Stream(device=dev, priority=-1)
            self.plan_stream = torch.cuda.Stream(device=dev, priority=-1)
            self.tv_stream = torch.cuda.Stream(device=dev, priority=0)
        self._ev = {k: torch.cuda.Event() for k in ("start", "plan", "rms", "tv", "bwd", "end")}
        self._bwd_recorded = False
        self.pending = None  # (lr_sigma, lr_sh) of an update not yet applied
        self._touched = torch.zeros(1 << 16 if cfg.track_touched else 0, dtype=torch.int64, device=dev)
        self._n_touched = 0

    def _count_touched(self, stream):
        """Appends this step's touched-row count (before the update clears the mask) to the log."""
        if not self.cfg.track_touched:
            return
        if self._n_touched == self._touched.numel():  # grow the log; ordered on `stream` like its writes
            with torch.cuda.stream(stream):
                grown = torch.zeros(2 * self._touched.numel(), dtype=torch.int64, device=self._touched.device)
                grown[: self._n_touched].copy_(self._touched)
            self._touched.record_stream(stream)  # its memory is not reused before `stream` is past the copy
            self._touched = grown
        self.grid.count_touched(self._touched[self._n_touched:self._n_touched + 1], stream=stream)
        self._n_touched += 1

    def touched_counts(self):
        """Rows that received a gradient in each recorded step (host int64 array; synchronises)."""
        torch.cuda.synchronize(self._touched.device)
        return self._touched[: self._n_touched].cpu().numpy()

    def _update(self, main, lrs):
        c = self.cfg
        self.grid.rmsprop_step(self.grad, self.v, lrs[0], lrs[1], c.beta, c.eps, sparse=c.sparse_rmsprop, stream=main)

    def finish(self, stream=None):
        """Applies the pending RMSProp update (overlap mode defers each step's update to the next call)."""
        if self.pending is not None:
            main = stream if stream is not None else torch.cuda.current_stream()
            self._update(main, self.pending)
            self.pending = None

    def step(self, pix: torch.Tensor, target: torch.Tensor, seg_start: Optional[torch.Tensor],
             seg_len: Optional[torch.Tensor], n_selected: int, lr_s: float, lr_h: float,
             events: Optional[List[torch.cuda.Event]] = None, stream=None):
        """One optimisation step.  `events`, if given, holds 8 events recorded on the main stream; the 7
        intervals between them are the stages named in STAGES (serial mode: rays and plan, -, forward with
        the MSE gradient, -, adjoint, TV, update; overlap mode: the previous step's update, the wait for this
        step's plan, forward with the MSE gradient, -, adjoint, the wait for TV, -).  In overlap mode call finish() after the last step."""
        g, c = self.grid, self.cfg
        n = pix.shape[0]
        o, d, rgb, grgb = self.o[:n], self.d[:n], self.rgb[:n], self.grad_rgb[:n]
        main = stream if stream is not None else torch.cuda.current_stream()
        do_tv = seg_start is not None and n_selected > 0
        ev = self._ev

        def mark(i):
            if events is not None:
                events[i].record(main)

        if not c.overlap:
            mark(0)
            gen_rays(self.cams, pix, self.W, self.H, o, d, stream=main)
            g.march_plan(o, d, c.opts, self.state, stream=main)
            mark(1)
            mark(2)
            g.render_planned_mse(o, d, c.opts, self.state, target, rgb, grgb, self.loss, stream=main)
            mark(3)
            mark(4)
            g.render_backward_train(o, d, grgb, c.opts, self.state, self.grad, c.lambda_sparsity,
                                    self.loss_sparsity if c.lambda_sparsity > 0 else None, stream=main)
            mark(5)
            if do_tv:
                g.tv_grad(seg_start, seg_len, n_selected, c.lambda_tv_sigma, c.lambda_tv_sh, self.grad, stream=main)
            self._count_touched(main)
            mark(6)
            self._update(main, (lr_s, lr_h))
            mark(7)
            return rgb

        # the march stream starts after everything the caller enqueued (inputs, the loss reset)
        caller = main
        ms = self.march_stream
        ev["start"].record(caller)
        ms.wait_event(ev["start"])
        main = ms  # the stage events follow the march stream
        # rays and plan of this batch on the plan stream, once the last adjoint is done with rays and state
        ps = self.plan_stream
        ps.wait_event(ev["start"])
        if self._bwd_recorded:
            ps.wait_event(ev["bwd"])
        gen_rays(self.cams, pix, self.W, self.H, o, d, stream=ps)
        g.march_plan(o, d, c.opts, self.state, stream=ps)
        ev["plan"].record(ps)
        # the previous step's update, concurrently
        mark(0)
        if self.pending is not None:
            self._update(ms, self.pending)
            self.pending = None
        mark(1)
        # TV of this step after that update, beside the march
        if do_tv:
            ev["rms"].record(ms)
            self.tv_stream.wait_event(ev["rms"])
            g.tv_grad(seg_start, seg_len, n_selected, c.lambda_tv_sigma, c.lambda_tv_sh, self.grad,
                      stream=self.tv_stream)
            ev["tv"].record(self.tv_stream)
        ms.wait_event(ev["plan"])
        mark(2)
        g.render_planned_mse(o, d, c.opts, self.state, target, rgb, grgb, self.loss, stream=ms)
        mark(3)
        mark(4)
        g.render_backward_train(o, d, grgb, c.opts, self.state, self.grad, c.lambda_sparsity,
                                self.loss_sparsity if c.lambda_sparsity > 0 else None, stream=ms)
        ev["bwd"].record(ms)
        self._bwd_recorded = True
        mark(5)
        if do_tv:
            ms.wait_event(ev["tv"])
        self._count_touched(ms)
        self.pending = (lr_s, lr_h)
        mark(6)
        mark(7)
        # the caller's stream resumes after the step (colours, loss and gradient are then complete)
        ev["end"].record(ms)
        caller.wait_event(ev["end"])
        return rgb

    # the 7 intervals between step()'s 8 events: serial mode | overlap mode
    STAGES = ("rays_plan|prev_update", "-|plan_wait", "render", "-", "render_backward", "tv_grad|tv_wait",
              "rmsprop_step|-")
