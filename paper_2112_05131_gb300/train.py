"""The optimisation step of Sec. 3.5 as a sequence of library calls, and the learning-rate schedules.

One step (Supp. B.1: 5000-ray batches, RMSProp, stochastic TV on contiguous segments):
  plx_gen_rays -> plx_march_plan -> plx_render_planned_mse (forward and MSE gradient)
  -> plx_render_backward_train (with the Cauchy sparsity prior when configured) -> plx_tv_grad
  -> plx_rmsprop_step
all libplenoxel calls with no host synchronisation.  The training march splits rays into chunk work
items and hands the march state from the forward to the adjoint.

With overlap (the default) a step is one native call, plx_trainer_step, which orders the same calls on
three streams and defers RMSProp to the start of the next step (or to finish()): ray generation and
the plan read no rows, so they run beside the previous update, or during the previous step when its
call was given this batch as `next_pix`; TV reads rows only and adds to the gradient with atomics, so it
runs beside the forward and adjoint.  Every step computes what the serial order computes.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import List, Optional

import torch

from . import _lib as L
from .grid import ROW, Grid, RenderOpts, _need, _p, _stream, gen_rays

# kernels one step of up to 32768 rays enqueues with stop_thresh = 0: gen_rays, march_plan (header, setup,
# plan), render_planned_mse (chunks, each ray combined with the MSE gradient by the warp that finishes it;
# larger batches launch the combine separately), backward_train, tv, rmsprop (compact, apply)
LAUNCHES_PER_STEP = 9


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
    # most TV segments of a step fed from host memory (step_host)
    max_segments: int = 0


class Trainer:
    """Holds the optimiser state (gradient rows, RMSProp running average) and the step's scratch buffers.

    Overlap mode (the default) is one native call per step, plx_trainer_step (three streams, deferred
    update, the next batch planned ahead: see include/plenoxel.h); serial mode issues the same library
    calls from here, in order, on one stream."""

    def __init__(self, grid: Grid, cams: torch.Tensor, W: int, H: int, cfg: StepConfig = StepConfig()):
        dev = grid.idx.device
        self.grid = grid
        self.cams = cams
        self.W, self.H = int(W), int(H)
        self.cfg = cfg
        self.grad = torch.zeros((grid.M, ROW), dtype=torch.float32, device=dev)
        self.v = torch.zeros((grid.M, ROW), dtype=torch.float32, device=dev)
        n = cfg.batch
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.loss_sparsity = torch.zeros(1, dtype=torch.float32, device=dev)
        self._touched = torch.zeros(1 << 16 if cfg.track_touched else 0, dtype=torch.int64, device=dev)
        self._n_touched = 0
        self._native = None
        if cfg.overlap:
            _need(cams, torch.float32, "cams")
            desc = L.plx_trainer_desc()
            desc.batch = n
            desc.opts = cfg.opts.c()
            desc.lambda_tv_sigma, desc.lambda_tv_sh = float(cfg.lambda_tv_sigma), float(cfg.lambda_tv_sh)
            desc.lambda_sparsity = float(cfg.lambda_sparsity)
            desc.beta, desc.eps = float(cfg.beta), float(cfg.eps)
            desc.sparse_rmsprop = 1 if cfg.sparse_rmsprop else 0
            desc.max_segments = int(cfg.max_segments)
            nbytes = int(L.load().plx_trainer_workspace_bytes(grid.handle, ctypes.byref(desc)))
            if nbytes == 0:
                raise ValueError("no trainer workspace for this grid and batch")
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            handle = ctypes.c_void_p()
            L.call("plx_trainer_create", grid.handle, ctypes.byref(desc), _p(cams), cams.shape[0], self.W, self.H,
                   _p(self.grad), _p(self.v), _p(self._ws), nbytes, ctypes.byref(handle))
            self._native = handle
            # views of the two sets of rays and march state inside the workspace
            self._o, self._d, self._state = [], [], []
            base = self._ws.data_ptr()
            for k in range(2):
                po, pd, prgb, pst = (ctypes.c_void_p() for _ in range(4))
                sb = ctypes.c_size_t()
                L.call("plx_trainer_buffers", handle, k, ctypes.byref(po), ctypes.byref(pd), ctypes.byref(prgb),
                       ctypes.byref(pst), ctypes.byref(sb))
                view = lambda ptr, size: self._ws[ptr.value - base: ptr.value - base + size]
                self._o.append(view(po, 12 * n).view(torch.float32).view(n, 3))
                self._d.append(view(pd, 12 * n).view(torch.float32).view(n, 3))
                self._state.append(view(pst, sb.value))
                self.rgb = view(prgb, 12 * n).view(torch.float32).view(n, 3)
            self._ahead = None  # (key, tensor) of the batch planned ahead
        else:
            self._o = [torch.empty((n, 3), dtype=torch.float32, device=dev)]
            self._d = [torch.empty((n, 3), dtype=torch.float32, device=dev)]
            self._state = [grid.new_march_state(n, cfg.opts)]  # fits every batch of up to n rays
            self.rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
            self.grad_rgb = torch.empty((n, 3), dtype=torch.float32, device=dev)
        self.o, self.d, self.state = self._o[0], self._d[0], self._state[0]

    def close(self):
        """Destroys the native trainer (its streams and events); the buffers stay with this object."""
        if getattr(self, "_native", None) is not None:
            L.load().plx_trainer_destroy(self._native)
            self._native = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # interpreter shutdown: the binding may already be gone
            pass

    def _touched_slot(self, stream) -> Optional[torch.Tensor]:
        """The log entry for this step's touched-row count (plx_count_touched), growing the log on `stream`."""
        if not self.cfg.track_touched:
            return None
        if self._n_touched == self._touched.numel():
            with torch.cuda.stream(stream):
                grown = torch.zeros(2 * self._touched.numel(), dtype=torch.int64, device=self._touched.device)
                grown[: self._n_touched].copy_(self._touched)
            self._touched = grown
        self._n_touched += 1
        return self._touched[self._n_touched - 1:self._n_touched]

    def touched_counts(self):
        """Rows that received a gradient in each recorded step (host int64 array; synchronises)."""
        torch.cuda.synchronize(self._touched.device)
        return self._touched[: self._n_touched].cpu().numpy()

    def _update(self, main, lrs):
        c = self.cfg
        self.grid.rmsprop_step(self.grad, self.v, lrs[0], lrs[1], c.beta, c.eps, sparse=c.sparse_rmsprop, stream=main)

    @staticmethod
    def host_batch(pix: torch.Tensor, target: torch.Tensor, seg_start: Optional[torch.Tensor] = None,
                   seg_len: Optional[torch.Tensor] = None, n_selected: int = 0):
        """A batch in (page-locked) host memory for step_host: the tensors are referenced, not copied."""
        for t, dt, name in ((pix, torch.int64, "pix"), (target, torch.float32, "target")):
            if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous():
                raise ValueError(f"{name}: a contiguous host tensor of {dt} is required")
        b = L.plx_host_batch()
        b.pix, b.target = pix.data_ptr(), target.data_ptr()
        b.n = pix.shape[0]
        if seg_start is not None and n_selected > 0:
            b.seg_start, b.seg_len = seg_start.data_ptr(), seg_len.data_ptr()
            b.n_seg, b.n_selected = seg_start.shape[0], int(n_selected)
        b._keep = (pix, target, seg_start, seg_len)
        return b

    def step_host(self, batch, lr_s: float, lr_h: float, next_batch=None, loss_out: Optional[torch.Tensor] = None,
                  stream=None):
        """One overlapped step fed from host memory (plx_trainer_step_host): `batch` and `next_batch` come from
        host_batch; the step's MSE lands in `loss_out` (a page-locked float32 host tensor of one element)
        once `stream` (default: the current stream) has reached the step's end."""
        if self._native is None:
            raise RuntimeError("host-fed steps need the native (overlap) trainer")
        if loss_out is not None and (loss_out.device.type != "cpu" or loss_out.dtype != torch.float32):
            raise ValueError("loss_out: a float32 host tensor is required")
        main = stream if stream is not None else torch.cuda.current_stream()
        L.call("plx_trainer_step_host", self._native, ctypes.byref(batch),
               ctypes.byref(next_batch) if next_batch is not None else None, float(lr_s), float(lr_h),
               _p(loss_out) if loss_out is not None else None, _stream(main))
        self._ahead = None

    def finish(self, stream=None):
        """Applies the pending RMSProp update (overlap mode defers each step's update to the next call)."""
        if self.cfg.overlap:
            if self._native is None:
                raise RuntimeError("the trainer is closed")
            L.call("plx_trainer_finish", self._native, _stream(stream))

    @staticmethod
    def _key(pix: torch.Tensor):
        # identifies a pixel batch and its contents: views of the same memory compare equal, and an
        # in-place change through any of them bumps the shared version (the planned-ahead tensor is kept
        # referenced, so its memory cannot be reused by another tensor meanwhile)
        return (pix.data_ptr(), tuple(pix.shape), tuple(pix.stride()), pix._version)

    def step(self, pix: torch.Tensor, target: torch.Tensor, seg_start: Optional[torch.Tensor],
             seg_len: Optional[torch.Tensor], n_selected: int, lr_s: float, lr_h: float,
             events: Optional[List[torch.cuda.Event]] = None, stream=None, next_pix: Optional[torch.Tensor] = None):
        """One optimisation step.  `events`, if given, holds 8 events recorded on the march (serial mode:
        the only) stream; the 7 intervals between them are the stages named in STAGES (serial mode: rays and
        plan, -, forward with the MSE gradient, -, adjoint, TV, update; overlap mode: the previous step's
        update, the wait for this step's plan, forward with the MSE gradient, -, adjoint, the wait for TV,
        -).  In overlap mode call finish() after the last step.

        `next_pix` (overlap mode): the pixel batch of the next call, whose rays and plan are then computed
        during this step, beside its march, and used by the next call if it passes the same, unchanged
        tensor as `pix` (otherwise they are computed again)."""
        g, c = self.grid, self.cfg
        n = pix.shape[0]
        main = stream if stream is not None else torch.cuda.current_stream()
        do_tv = seg_start is not None and n_selected > 0

        if c.overlap:
            if self._native is None:
                raise RuntimeError("the trainer is closed")
            _need(pix, torch.int64, "pix", (n,))
            _need(target, torch.float32, "target", (n, 3))
            if next_pix is not None:
                _need(next_pix, torch.int64, "next_pix", (n,))
            if do_tv:
                _need(seg_start, torch.int64, "seg_start")
                _need(seg_len, torch.int64, "seg_len", tuple(seg_start.shape))
            ahead = self._ahead is not None and self._ahead[0] == self._key(pix)
            ev = None
            if events is not None:
                for e in events:  # the native call records them; each must exist first
                    if not e.cuda_event:
                        e.record(main)
                ev = ctypes.cast((ctypes.c_void_p * 8)(*[e.cuda_event for e in events]), ctypes.c_void_p)
            touched = self._touched_slot(main)
            used = ctypes.c_int32()
            L.call("plx_trainer_step", self._native, _p(pix), n, _p(target),
                   _p(seg_start) if do_tv else None, _p(seg_len) if do_tv else None,
                   seg_start.shape[0] if do_tv else 0, int(n_selected) if do_tv else 0, float(lr_s), float(lr_h),
                   _p(next_pix), 1 if ahead else 0, _p(self.loss),
                   _p(self.loss_sparsity) if c.lambda_sparsity > 0 else None, _p(touched), ev, ctypes.byref(used),
                   _stream(main))
            self._ahead = (self._key(next_pix), next_pix) if next_pix is not None else None
            k = used.value
            self.o, self.d, self.state = self._o[k], self._d[k], self._state[k]
            return self.rgb[:n]

        o, d, rgb, grgb = self.o[:n], self.d[:n], self.rgb[:n], self.grad_rgb[:n]

        def mark(i):
            if events is not None:
                events[i].record(main)

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
        touched = self._touched_slot(main)
        if touched is not None:
            g.count_touched(touched, stream=main)
        mark(6)
        self._update(main, (lr_s, lr_h))
        mark(7)
        return rgb

    # the 7 intervals between step()'s 8 events: serial mode | overlap mode
    STAGES = ("rays_plan|prev_update", "-|plan_wait", "render", "-", "render_backward", "tv_grad|tv_wait",
              "rmsprop_step|-")
