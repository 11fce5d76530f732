"""Python face of libplenoxel: device buffers from PyTorch, every computation in the CUDA library.

``Grid`` owns the caller-side device buffers a grid needs (index volume, F32
rows, optional BF16-SH rows, workspace) and the library handle.  Its methods
call the C ABI one to one; ``PlenoxelRender`` wraps render/render_backward as
a ``torch.autograd.Function``.  No method computes anything itself.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L

ROW = 32  # floats per padded F32 row
NV = 28   # density + 27 SH values per row


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream] = None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t: torch.Tensor, dtype, name: str, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


@dataclass
class RenderOpts:
    step_vox: float = 0.5
    bg: Sequence[float] = (1.0, 1.0, 1.0)
    stop_thresh: float = 0.0

    def c(self) -> L.plx_render_opts:
        o = L.plx_render_opts()
        o.step_vox = float(self.step_vox)
        for i in range(3):
            o.bg[i] = float(self.bg[i])
        o.stop_thresh = float(self.stop_thresh)
        return o


def pad_rows(rows28: np.ndarray) -> np.ndarray:
    """[M, 28] float32 -> the padded [M, 32] row layout (pad = 0)."""
    out = np.zeros((rows28.shape[0], ROW), np.float32)
    out[:, :NV] = rows28
    return out


class Grid:
    """A sparse grid on the device: int32 index volume + padded rows (+ BF16-SH shadow)."""

    def __init__(self, reso: int, idx: torch.Tensor, rows: Optional[torch.Tensor], sh_form: int = L.PLX_SH_F32,
                 aabb=((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)), rows_h: Optional[torch.Tensor] = None,
                 n_rows: Optional[int] = None, stream=None):
        lib = L.load()
        self.reso = int(reso)
        self.sh_form = int(sh_form)
        self.aabb = (tuple(float(x) for x in aabb[0]), tuple(float(x) for x in aabb[1]))
        _need(idx, torch.int32, "idx", (self.reso ** 3,))
        self.idx = idx
        if rows is not None:
            _need(rows, torch.float32, "rows")
            if rows.dim() != 2 or rows.shape[1] != ROW:
                raise ValueError("rows must be [M, 32]")
        self.rows = rows
        M = int(rows.shape[0]) if rows is not None else int(n_rows if n_rows is not None else rows_h.shape[0])
        self.n_rows = M
        if self.sh_form == L.PLX_SH_BF16 and rows_h is None:
            rows_h = torch.zeros((M, ROW), dtype=torch.int16, device=idx.device)
        if rows_h is not None:
            _need(rows_h, torch.int16, "rows_h", (M, ROW))
        self.rows_h = rows_h if self.sh_form == L.PLX_SH_BF16 else None
        self.desc = L.plx_grid_desc()
        self.desc.reso = self.reso
        for a in range(3):
            self.desc.aabb_min[a] = self.aabb[0][a]
            self.desc.aabb_max[a] = self.aabb[1][a]
        self.desc.n_rows = M
        self.desc.sh_form = self.sh_form
        nbytes = lib.plx_grid_workspace_bytes(ctypes.byref(self.desc))
        if nbytes == 0:
            L.check(L.load().plx_grid_create(ctypes.byref(self.desc), None, None, None, None, None,
                                             ctypes.byref(ctypes.c_void_p())), "plx_grid_create")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=idx.device)
        handle = ctypes.c_void_p()
        L.call("plx_grid_create", ctypes.byref(self.desc), _p(idx), _p(rows), _p(self.rows_h), _p(self.workspace),
               _stream(stream), ctypes.byref(handle))
        self.handle = handle
        if self.sh_form == L.PLX_SH_BF16 and rows is not None:
            self.pack_bf16(stream)

    # ------------------------------------------------------------------ construction helpers
    @classmethod
    def from_host(cls, reso: int, idx: np.ndarray, rows28: np.ndarray, sh_form: int = L.PLX_SH_F32,
                  device="cuda", aabb=((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))) -> "Grid":
        idx_t = torch.from_numpy(np.ascontiguousarray(idx, np.int32)).to(device)
        rows_t = torch.from_numpy(pad_rows(np.asarray(rows28, np.float32))).to(device)
        return cls(reso, idx_t, rows_t, sh_form, aabb)

    @classmethod
    def render_only_bf16(cls, reso: int, idx: np.ndarray, rows28: np.ndarray, device="cuda",
                         aabb=((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))) -> "Grid":
        """A BF16-SH grid that keeps only its 64-byte rows on the device (serving): the F32 rows are
        packed by plx_pack_bf16 and then released."""
        full = cls.from_host(reso, idx, rows28, sh_form=L.PLX_SH_BF16, device=device, aabb=aabb)
        g = cls(reso, full.idx, None, L.PLX_SH_BF16, aabb, rows_h=full.rows_h, n_rows=full.M)
        full.close()
        del full
        return g

    def device_bytes(self) -> int:
        """Device memory this grid holds (index volume, rows, workspace)."""
        n = self.idx.numel() * 4 + self.workspace.numel()
        if self.rows is not None:
            n += self.rows.numel() * 4
        if self.rows_h is not None:
            n += self.rows_h.numel() * 2
        return n

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            L.load().plx_grid_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def M(self) -> int:
        return self.n_rows

    def values(self) -> torch.Tensor:
        """The 28 values of every row, [M, 28] (a view of the F32 rows)."""
        return self.rows[:, :NV]

    # ------------------------------------------------------------------ calls
    def pack_bf16(self, stream=None):
        L.call("plx_pack_bf16", self.handle, _stream(stream))

    def check(self, stream=None):
        L.call("plx_check", self.handle, _stream(stream))

    def render(self, origins: torch.Tensor, dirs: torch.Tensor, opts: RenderOpts = RenderOpts(),
               rgb: Optional[torch.Tensor] = None, T_end: Optional[torch.Tensor] = None, stream=None):
        n = origins.shape[0]
        _need(origins, torch.float32, "origins", (n, 3))
        _need(dirs, torch.float32, "dirs", (n, 3))
        if rgb is None:
            rgb = torch.empty((n, 3), dtype=torch.float32, device=origins.device)
        L.call("plx_render", self.handle, _p(origins), _p(dirs), n, ctypes.byref(opts.c()), _p(rgb), _p(T_end),
               _stream(stream))
        return rgb

    def render_backward(self, origins, dirs, grad_rgb, opts: RenderOpts = RenderOpts(),
                        grad_rows: Optional[torch.Tensor] = None, lambda_sparsity: float = 0.0,
                        loss_sparsity: Optional[torch.Tensor] = None, stream=None):
        """plx_render_backward; lambda_sparsity > 0 adds the Cauchy sparsity prior (its value is added to
        loss_sparsity, a float32 [1] device tensor, when given)."""
        n = origins.shape[0]
        _need(grad_rgb, torch.float32, "grad_rgb", (n, 3))
        if grad_rows is None:
            grad_rows = torch.zeros((self.M, ROW), dtype=torch.float32, device=origins.device)
        _need(grad_rows, torch.float32, "grad_rows", (self.M, ROW))
        if loss_sparsity is not None:
            _need(loss_sparsity, torch.float32, "loss_sparsity", (1,))
        L.call("plx_render_backward", self.handle, _p(origins), _p(dirs), n, ctypes.byref(opts.c()), _p(grad_rgb),
               _p(grad_rows), float(lambda_sparsity), _p(loss_sparsity), _stream(stream))
        return grad_rows

    def march_state_bytes(self, n: int, opts: RenderOpts = RenderOpts()) -> int:
        return int(L.load().plx_march_state_bytes(self.handle, int(n), ctypes.byref(opts.c())))

    def new_march_state(self, n: int, opts: RenderOpts = RenderOpts()) -> torch.Tensor:
        """A device buffer for the march state of n rays (plx_render_train / plx_render_backward_train)."""
        nbytes = self.march_state_bytes(n, opts)
        if nbytes == 0:
            raise ValueError("invalid arguments for a march state")
        return torch.empty(nbytes, dtype=torch.uint8, device=self.idx.device)

    def render_train(self, origins: torch.Tensor, dirs: torch.Tensor, opts: RenderOpts, state: torch.Tensor,
                     rgb: Optional[torch.Tensor] = None, T_end: Optional[torch.Tensor] = None, stream=None):
        """plx_render_train: the forward of a training batch, leaving the march state in `state`."""
        n = origins.shape[0]
        _need(origins, torch.float32, "origins", (n, 3))
        _need(dirs, torch.float32, "dirs", (n, 3))
        _need(state, torch.uint8, "state")
        if rgb is None:
            rgb = torch.empty((n, 3), dtype=torch.float32, device=origins.device)
        L.call("plx_render_train", self.handle, _p(origins), _p(dirs), n, ctypes.byref(opts.c()), _p(rgb), _p(T_end),
               _p(state), state.numel(), _stream(stream))
        return rgb

    def march_plan(self, origins: torch.Tensor, dirs: torch.Tensor, opts: RenderOpts, state: torch.Tensor,
                   stream=None):
        """plx_march_plan: the plan of a training batch (reads no rows)."""
        n = origins.shape[0]
        _need(origins, torch.float32, "origins", (n, 3))
        _need(dirs, torch.float32, "dirs", (n, 3))
        _need(state, torch.uint8, "state")
        L.call("plx_march_plan", self.handle, _p(origins), _p(dirs), n, ctypes.byref(opts.c()), _p(state),
               state.numel(), _stream(stream))

    def render_planned(self, origins: torch.Tensor, dirs: torch.Tensor, opts: RenderOpts, state: torch.Tensor,
                       rgb: Optional[torch.Tensor] = None, T_end: Optional[torch.Tensor] = None, stream=None):
        """plx_render_planned: the forward of a planned training batch."""
        n = origins.shape[0]
        _need(origins, torch.float32, "origins", (n, 3))
        _need(dirs, torch.float32, "dirs", (n, 3))
        _need(state, torch.uint8, "state")
        if rgb is None:
            rgb = torch.empty((n, 3), dtype=torch.float32, device=origins.device)
        L.call("plx_render_planned", self.handle, _p(origins), _p(dirs), n, ctypes.byref(opts.c()), _p(rgb),
               _p(T_end), _p(state), state.numel(), _stream(stream))
        return rgb

    def render_planned_mse(self, origins: torch.Tensor, dirs: torch.Tensor, opts: RenderOpts, state: torch.Tensor,
                           target: torch.Tensor, rgb: torch.Tensor, grad_rgb: torch.Tensor,
                           loss: Optional[torch.Tensor] = None, stream=None):
        """plx_render_planned_mse: colours, the MSE gradient and the loss of a planned training batch."""
        n = origins.shape[0]
        _need(target, torch.float32, "target", (n, 3))
        _need(rgb, torch.float32, "rgb", (n, 3))
        _need(grad_rgb, torch.float32, "grad_rgb", (n, 3))
        _need(state, torch.uint8, "state")
        L.call("plx_render_planned_mse", self.handle, _p(origins), _p(dirs), n, ctypes.byref(opts.c()), _p(target),
               _p(rgb), _p(grad_rgb), _p(loss), _p(state), state.numel(), _stream(stream))
        return rgb

    def render_backward_train(self, origins, dirs, grad_rgb, opts: RenderOpts, state: torch.Tensor,
                              grad_rows: Optional[torch.Tensor] = None, lambda_sparsity: float = 0.0,
                              loss_sparsity: Optional[torch.Tensor] = None, stream=None):
        """plx_render_backward_train: the adjoint of the last render_train on these rays, from its state
        (with the Cauchy sparsity prior when lambda_sparsity > 0, as render_backward)."""
        n = origins.shape[0]
        _need(grad_rgb, torch.float32, "grad_rgb", (n, 3))
        _need(state, torch.uint8, "state")
        if grad_rows is None:
            grad_rows = torch.zeros((self.M, ROW), dtype=torch.float32, device=origins.device)
        _need(grad_rows, torch.float32, "grad_rows", (self.M, ROW))
        if loss_sparsity is not None:
            _need(loss_sparsity, torch.float32, "loss_sparsity", (1,))
        L.call("plx_render_backward_train", self.handle, _p(origins), _p(dirs), n, ctypes.byref(opts.c()),
               _p(grad_rgb), _p(state), state.numel(), _p(grad_rows), float(lambda_sparsity), _p(loss_sparsity),
               _stream(stream))
        return grad_rows

    def count_nodes(self, origins, dirs, opts: RenderOpts = RenderOpts(), stream=None) -> torch.Tensor:
        """Per ray (distinct nodes of sampled non-empty cells, occupied ones among them, marched samples),
        int64 [n, 3]."""
        n = origins.shape[0]
        out = torch.empty((n, 3), dtype=torch.int64, device=origins.device)
        L.call("plx_count_nodes", self.handle, _p(origins), _p(dirs), n, ctypes.byref(opts.c()), _p(out),
               _stream(stream))
        return out

    def count_touched(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """plx_count_touched: rows that received a gradient since the last RMSProp step (int64 [1], device)."""
        if out is None:
            out = torch.empty(1, dtype=torch.int64, device=self.idx.device)
        _need(out, torch.int64, "out", (1,))
        L.call("plx_count_touched", self.handle, _p(out), _stream(stream))
        return out

    def max_weight(self, origins, dirs, opts: RenderOpts = RenderOpts(), wmax: Optional[torch.Tensor] = None,
                   stream=None) -> torch.Tensor:
        """plx_max_weight: per row, the largest weight of the samples crediting it over these rays, float32
        [M] (max-updated in place when given; start from zeros)."""
        n = origins.shape[0]
        if wmax is None:
            wmax = torch.zeros(self.M, dtype=torch.float32, device=self.idx.device)
        _need(wmax, torch.float32, "wmax", (self.M,))
        L.call("plx_max_weight", self.handle, _p(origins), _p(dirs), n, ctypes.byref(opts.c()), _p(wmax),
               _stream(stream))
        return wmax

    def max_weight_views(self, cams: torch.Tensor, W: int, H: int, opts: RenderOpts = RenderOpts(),
                         views: Optional[Sequence[int]] = None, wmax: Optional[torch.Tensor] = None,
                         stream=None) -> torch.Tensor:
        """plx_max_weight over every pixel ray of the given views (all views of `cams` by default), one
        view per launch; the rays of a view are generated by plx_gen_rays into a reused buffer."""
        dev = self.idx.device
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        with torch.cuda.stream(s):
            if wmax is None:
                wmax = torch.zeros(self.M, dtype=torch.float32, device=dev)
            n = W * H
            o = torch.empty((n, 3), dtype=torch.float32, device=dev)
            d = torch.empty((n, 3), dtype=torch.float32, device=dev)
            base = torch.arange(n, dtype=torch.int64, device=dev)
            pix = torch.empty_like(base)
            for v in (range(cams.shape[0]) if views is None else views):
                torch.add(base, int(v) * n, out=pix)
                gen_rays(cams, pix, W, H, o, d, stream=s)
                self.max_weight(o, d, opts, wmax, stream=s)
        return wmax

    def tv_grad(self, seg_start: torch.Tensor, seg_len: torch.Tensor, n_selected: int, lambda_sigma: float,
                lambda_sh: float, grad_rows: torch.Tensor, loss: Optional[torch.Tensor] = None, stream=None):
        _need(seg_start, torch.int64, "seg_start")
        _need(seg_len, torch.int64, "seg_len", tuple(seg_start.shape))
        L.call("plx_tv_grad", self.handle, _p(seg_start), _p(seg_len), seg_start.shape[0], int(n_selected),
               float(lambda_sigma), float(lambda_sh), _p(grad_rows), _p(loss), _stream(stream))
        return grad_rows

    def rmsprop_step(self, grad_rows: torch.Tensor, v: torch.Tensor, lr_sigma: float, lr_sh: float,
                     beta: float = 0.95, eps: float = 1e-8, sparse: bool = True, stream=None):
        _need(grad_rows, torch.float32, "grad_rows", (self.M, ROW))
        _need(v, torch.float32, "v", (self.M, ROW))
        L.call("plx_rmsprop_step", self.handle, _p(grad_rows), _p(v), float(lr_sigma), float(lr_sh), float(beta),
               float(eps), 1 if sparse else 0, _stream(stream))

    def prune(self, tau: float, dilate: bool = True, key: Optional[torch.Tensor] = None, stream=None) -> "Grid":
        """Density-threshold prune (key None), or weight-threshold prune on a per-row key (float32 [M], e.g.
        max_weight_views), with 3x3x3 dilation."""
        lib = L.load()
        ws = torch.empty(lib.plx_prune_workspace_bytes(self.reso), dtype=torch.uint8, device=self.idx.device)
        n_keep = ctypes.c_int64()
        if key is None:
            L.call("plx_grid_prune_count", self.handle, float(tau), 1 if dilate else 0, _p(ws), ctypes.byref(n_keep),
                   _stream(stream))
        else:
            _need(key, torch.float32, "key", (self.M,))
            L.call("plx_grid_prune_count_key", self.handle, _p(key), float(tau), 1 if dilate else 0, _p(ws),
                   ctypes.byref(n_keep), _stream(stream))
        idx_new = torch.empty(self.reso ** 3, dtype=torch.int32, device=self.idx.device)
        rows_new = torch.empty((n_keep.value, ROW), dtype=torch.float32, device=self.idx.device)
        L.call("plx_grid_prune_apply", self.handle, _p(ws), n_keep.value, _p(idx_new),
               _p(rows_new) if n_keep.value > 0 else None, _stream(stream))
        return Grid(self.reso, idx_new, rows_new, self.sh_form, self.aabb, stream=stream)

    def upsample(self, new_reso: int, stream=None) -> "Grid":
        lib = L.load()
        ws = torch.empty(lib.plx_upsample_workspace_bytes(int(new_reso)), dtype=torch.uint8, device=self.idx.device)
        n_new = ctypes.c_int64()
        L.call("plx_grid_upsample_count", self.handle, int(new_reso), _p(ws), ctypes.byref(n_new), _stream(stream))
        idx_new = torch.empty(int(new_reso) ** 3, dtype=torch.int32, device=self.idx.device)
        rows_new = torch.empty((n_new.value, ROW), dtype=torch.float32, device=self.idx.device)
        L.call("plx_grid_upsample_apply", self.handle, int(new_reso), _p(ws), n_new.value, _p(idx_new),
               _p(rows_new) if n_new.value > 0 else None, _stream(stream))
        return Grid(int(new_reso), idx_new, rows_new, self.sh_form, self.aabb, stream=stream)


def gen_rays(cams: torch.Tensor, pix: torch.Tensor, W: int, H: int, origins=None, dirs=None, stream=None):
    """Pixel-centre rays for pixel ids view*H*W + v*W + u (cams: float32 [V, 18] on the device)."""
    _need(cams, torch.float32, "cams")
    _need(pix, torch.int64, "pix")
    n = pix.shape[0]
    if origins is None:
        origins = torch.empty((n, 3), dtype=torch.float32, device=pix.device)
    if dirs is None:
        dirs = torch.empty((n, 3), dtype=torch.float32, device=pix.device)
    L.call("plx_gen_rays", _p(cams), cams.shape[0], int(W), int(H), _p(pix), n, _p(origins), _p(dirs),
           _stream(stream))
    return origins, dirs


TILE_W = 16
TILE_H = 16
MAX_TILE_SCENES = 8
# plx_tile: scene, camera, x0, y0, W, H (int32), d_rgb (device pointer)
TILE_DTYPE = np.dtype([("scene", "<i4"), ("camera", "<i4"), ("x0", "<i4"), ("y0", "<i4"), ("W", "<i4"),
                       ("H", "<i4"), ("d_rgb", "<u8")])
assert TILE_DTYPE.itemsize == 32


def render_tiles(grids: Sequence[Grid], cams: torch.Tensor, tiles: torch.Tensor, n_tiles: int,
                 opts: RenderOpts = RenderOpts(), stream=None):
    """plx_render_tiles: `tiles` is a device byte tensor holding n_tiles TILE_DTYPE records."""
    _need(cams, torch.float32, "cams")
    _need(tiles, torch.uint8, "tiles")
    if tiles.numel() < n_tiles * TILE_DTYPE.itemsize:
        raise ValueError("tiles holds fewer than n_tiles records")
    handles = (ctypes.c_void_p * len(grids))(*[g.handle.value for g in grids])
    L.call("plx_render_tiles", handles, len(grids), _p(cams), cams.shape[0], _p(tiles), int(n_tiles),
           ctypes.byref(opts.c()), _stream(stream))


def mse_grad(rgb: torch.Tensor, target: torch.Tensor, grad_rgb=None, loss=None, stream=None):
    n = rgb.shape[0]
    _need(rgb, torch.float32, "rgb", (n, 3))
    _need(target, torch.float32, "target", (n, 3))
    if grad_rgb is None:
        grad_rgb = torch.empty_like(rgb)
    L.call("plx_mse_grad", _p(rgb), _p(target), n, _p(grad_rgb), _p(loss), _stream(stream))
    return grad_rgb


class PlenoxelRender(torch.autograd.Function):
    """C = render(rows; rays): forward = plx_render, backward = plx_render_backward (Eq. 1 and its adjoint)."""

    @staticmethod
    def forward(ctx, rows, origins, dirs, grid: Grid, opts: RenderOpts):
        if rows.data_ptr() != grid.rows.data_ptr():
            raise ValueError("rows must be the grid's own F32 row tensor")
        ctx.grid = grid
        ctx.opts = opts
        ctx.save_for_backward(origins, dirs)
        return grid.render(origins, dirs, opts)

    @staticmethod
    def backward(ctx, grad_rgb):
        origins, dirs = ctx.saved_tensors
        grad_rows = ctx.grid.render_backward(origins, dirs, grad_rgb.contiguous(), ctx.opts)
        return grad_rows, None, None, None, None


def render(grid: Grid, origins, dirs, opts: RenderOpts = RenderOpts()):
    """Differentiable render: gradients flow to ``grid.rows`` (which must require grad)."""
    return PlenoxelRender.apply(grid.rows, origins, dirs, grid, opts)
