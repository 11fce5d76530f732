"""FP64 CPU oracle for the Plenoxels renderer (arXiv 2112.05131) -- test infrastructure.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``plx_oracle.c`` (plain C,
FP64) through ctypes and shares no code with the CUDA library.  Every function
takes NumPy arrays and returns NumPy arrays; see the C file for the definition
each one follows (Eq. 1, Sec. 3.2-3.4, Supp. B.1) and the pin that checks it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

NV = 28  # density + 27 SH coefficients (Sec. 3.2)


def build(force: bool = False) -> str:
    """Compile plx_oracle.c with gcc into oracle/_build/liborc.so.

    -ffp-contract=off keeps FP64 results identical on x86_64 and aarch64 (no
    fused multiply-add contraction); OpenMP parallelises over rays only.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        sig = {
            "orc_sh_basis": (None, [P, P]),
            "orc_interp": (None, [I64, P, P, I64, P, P, I64, P]),
            "orc_gen_rays": (None, [P, P, I64, P, P]),
            "orc_clip": (None, [P, P, I64, P, P]),
            "orc_render": (None, [I64, P, P, I64, P, P, P, I64, P, P, P]),
            "orc_render_backward": (None, [I64, P, P, I64, P, P, P, I64, P, P, P]),
            "orc_render_backward_abs": (None, [I64, P, P, I64, P, P, P, I64, P, P, P]),
            "orc_render_backward_mag": (None, [I64, P, P, I64, P, P, P, I64, P, P, P]),
            "orc_mse": (D, [P, P, I64, P]),
            "orc_tv": (D, [I64, P, P, I64, P, P, I64, D, D, P]),
            "orc_rmsprop": (None, [I64, P, P, P, D, D, D, D]),
            "orc_max_weight": (None, [I64, P, P, I64, P, P, P, I64, P, P]),
            "orc_sparsity": (D, [I64, P, P, I64, P, P, P, I64, P, D, P]),
            "orc_prune": (I64, [I64, P, P, I64, D, ctypes.c_int, P, P]),
            "orc_prune_key": (I64, [I64, P, P, I64, P, D, ctypes.c_int, P, P]),
            "orc_upsample": (I64, [I64, P, P, I64, I64, P, P]),
            "orc_round_bf16": (None, [P, I64]),
            "orc_num_threads": (ctypes.c_int, []),
            "orc_set_num_threads": (None, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _aabb(aabb):
    if aabb is None:
        aabb = (-1.0, -1.0, -1.0, 1.0, 1.0, 1.0)
    return _c(np.asarray(aabb, dtype=np.float64).reshape(6), np.float64)


def _rows(rows):
    rows = _c(rows, np.float64)
    assert rows.ndim == 2 and rows.shape[1] >= NV
    return rows


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the OpenMP regions from now on (the default is every host core)."""
    _load().orc_set_num_threads(int(n))


def sh_basis(dirs):
    """Real SH degree 2 at unit directions [n,3] -> [n,9] (Sec. 3.2)."""
    lib = _load()
    dirs = _c(np.atleast_2d(dirs), np.float64)
    out = np.zeros((dirs.shape[0], 9), np.float64)
    for q in range(dirs.shape[0]):
        lib.orc_sh_basis(_p(dirs[q]), _p(out[q]))
    return out


def interp(R, idx, rows, pts, aabb=None):
    """Trilinear interpolation of all 28 values at world points [n,3] (Sec. 3.3)."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    pts = _c(np.atleast_2d(pts), np.float64)
    out = np.zeros((pts.shape[0], NV), np.float64)
    lib.orc_interp(R, _p(idx), _p(rows), rows.shape[1], _p(_aabb(aabb)), _p(pts), pts.shape[0], _p(out))
    return out


def gen_rays(cams, pix):
    """Pixel-centre pinhole rays: cams [V,18], pix [n] int64 -> (o [n,3], d [n,3])."""
    lib = _load()
    cams = _c(cams, np.float64)
    pix = _c(pix, np.int64)
    n = pix.shape[0]
    o = np.zeros((n, 3), np.float64)
    d = np.zeros((n, 3), np.float64)
    lib.orc_gen_rays(_p(cams), _p(pix), n, _p(o), _p(d))
    return o, d


def clip(o, d, aabb=None):
    """Slab clip -> [n,3] = (t_near, t_far, hit)."""
    lib = _load()
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    out = np.zeros((o.shape[0], 3), np.float64)
    lib.orc_clip(_p(o), _p(d), o.shape[0], _p(_aabb(aabb)), _p(out))
    return out


def _opts(step_vox, bg, stop_thresh):
    bg = np.broadcast_to(np.asarray(bg, np.float64), (3,))
    return _c([step_vox, bg[0], bg[1], bg[2], stop_thresh], np.float64)


def render(R, idx, rows, o, d, step_vox=0.5, bg=(1.0, 1.0, 1.0), stop_thresh=0.0, aabb=None):
    """Forward render (Eq. 1).  Returns (rgb [n,3], aux [n,4] = T_end, n_samples, ratio, hit)."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    n = o.shape[0]
    rgb = np.zeros((n, 3), np.float64)
    aux = np.zeros((n, 4), np.float64)
    lib.orc_render(R, _p(idx), _p(rows), rows.shape[1], _p(_aabb(aabb)), _p(o), _p(d), n,
                   _p(_opts(step_vox, bg, stop_thresh)), _p(rgb), _p(aux))
    return rgb, aux


def render_backward(R, idx, rows, o, d, grad_rgb, step_vox=0.5, bg=(1.0, 1.0, 1.0),
                    stop_thresh=0.0, aabb=None, grad_rows=None):
    """Adjoint of ``render``: returns dL/d(rows) [M,28] FP64 (accumulated into grad_rows if given)."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    g = _c(grad_rgb, np.float64)
    if grad_rows is None:
        grad_rows = np.zeros((rows.shape[0], NV), np.float64)
    assert grad_rows.dtype == np.float64 and grad_rows.flags.c_contiguous
    lib.orc_render_backward(R, _p(idx), _p(rows), rows.shape[1], _p(_aabb(aabb)), _p(o), _p(d),
                            o.shape[0], _p(_opts(step_vox, bg, stop_thresh)), _p(g), _p(grad_rows))
    return grad_rows


def render_backward_abs(R, idx, rows, o, d, grad_rgb, step_vox=0.5, bg=(1.0, 1.0, 1.0), stop_thresh=0.0,
                        aabb=None):
    """The adjoint with every per-sample, per-corner term taken in absolute value (grad_rgb >= 0): an
    entrywise bound on |render_backward(g')| for all |g'| <= grad_rgb, used to propagate uncertainty."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    g = _c(grad_rgb, np.float64)
    assert np.all(g >= 0)
    out = np.zeros((rows.shape[0], NV), np.float64)
    lib.orc_render_backward_abs(R, _p(idx), _p(rows), rows.shape[1], _p(_aabb(aabb)), _p(o), _p(d),
                                o.shape[0], _p(_opts(step_vox, bg, stop_thresh)), _p(g), _p(out))
    return out


def render_backward_mag(R, idx, rows, o, d, grad_rgb, step_vox=0.5, bg=(1.0, 1.0, 1.0), stop_thresh=0.0,
                        aabb=None):
    """The magnitude adjoint: as render_backward_abs, but the density term takes |g| delta (T_{s+1} |c| + |R_s|),
    the size of the two numbers the adjoint subtracts.  Times a unit roundoff it bounds the rounding error
    of an implementation that forms T_{s+1} c - R_s in lower precision."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    g = _c(np.abs(np.asarray(grad_rgb, np.float64)), np.float64)
    out = np.zeros((rows.shape[0], NV), np.float64)
    lib.orc_render_backward_mag(R, _p(idx), _p(rows), rows.shape[1], _p(_aabb(aabb)), _p(o), _p(d),
                                o.shape[0], _p(_opts(step_vox, bg, stop_thresh)), _p(g), _p(out))
    return out


def mse(pred, target):
    """(L, dL/dpred) for the reconstruction term of Eq. 3."""
    lib = _load()
    pred = _c(pred, np.float64)
    target = _c(target, np.float64)
    grad = np.zeros_like(pred)
    L = lib.orc_mse(_p(pred), _p(target), pred.shape[0], _p(grad))
    return float(L), grad


def tv(R, idx, rows, seg_start, seg_len, lambda_sigma, lambda_sh, grad_rows=None):
    """TV loss and gradient (Sec. 3.5, Supp. B.1).  Returns (L, grad_rows [M,28])."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    ss = _c(seg_start, np.int64)
    sl = _c(seg_len, np.int64)
    if grad_rows is None:
        grad_rows = np.zeros((rows.shape[0], NV), np.float64)
    L = lib.orc_tv(R, _p(idx), _p(rows), rows.shape[1], _p(ss), _p(sl), ss.shape[0],
                   float(lambda_sigma), float(lambda_sh), _p(grad_rows))
    return float(L), grad_rows


def rmsprop(x, v, grad, lr_sigma, lr_sh, beta=0.95, eps=1e-8):
    """RMSProp on entries with non-zero gradient (Sec. 3.5).  Returns new (x, v, grad) FP64."""
    lib = _load()
    x = np.array(x, np.float64, order="C", copy=True)
    v = np.array(v, np.float64, order="C", copy=True)
    grad = np.array(grad, np.float64, order="C", copy=True)
    assert x.shape == v.shape == grad.shape and x.shape[1] == NV
    lib.orc_rmsprop(x.shape[0], _p(x), _p(v), _p(grad), float(lr_sigma), float(lr_sh), float(beta), float(eps))
    return x, v, grad


def prune(R, idx, rows, tau, dilate=True):
    """Density-threshold prune with 3x3x3 dilation.  Returns (idx', rows' [M',stride])."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    idx_out = np.empty(R ** 3, np.int32)
    m = lib.orc_prune(R, _p(idx), _p(rows), rows.shape[1], float(tau), int(bool(dilate)), _p(idx_out), None)
    rows_out = np.empty((m, rows.shape[1]), np.float64)
    lib.orc_prune(R, _p(idx), _p(rows), rows.shape[1], float(tau), int(bool(dilate)), _p(idx_out), _p(rows_out))
    return idx_out, rows_out


def max_weight(R, idx, rows, o, d, step_vox=0.5, stop_thresh=0.0, aabb=None, wmax=None):
    """Largest sample weight T_s alpha_s crediting each row over the rays (the weight-threshold prune's
    key, Sec. 3.4): a sample credits the 8 corner nodes of its cell.  Returns wmax [M] FP64 (max-updated
    in place when given)."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    if wmax is None:
        wmax = np.zeros(rows.shape[0], np.float64)
    assert wmax.dtype == np.float64 and wmax.flags.c_contiguous and wmax.shape == (rows.shape[0],)
    lib.orc_max_weight(R, _p(idx), _p(rows), rows.shape[1], _p(_aabb(aabb)), _p(o), _p(d), o.shape[0],
                       _p(_opts(step_vox, 0.0, stop_thresh)), _p(wmax))
    return wmax


def sparsity(R, idx, rows, o, d, lambda_s, step_vox=0.5, stop_thresh=0.0, aabb=None, grad_rows=None):
    """Cauchy sparsity prior lambda_s sum log(1 + 2 sigma^2) over every marched sample (Sec. 3.7, Eq. 4).
    Returns (L, grad_rows [M,28] FP64, density column accumulated)."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    if grad_rows is None:
        grad_rows = np.zeros((rows.shape[0], NV), np.float64)
    assert grad_rows.dtype == np.float64 and grad_rows.flags.c_contiguous and grad_rows.shape == (rows.shape[0], NV)
    L = lib.orc_sparsity(R, _p(idx), _p(rows), rows.shape[1], _p(_aabb(aabb)), _p(o), _p(d), o.shape[0],
                         _p(_opts(step_vox, 0.0, stop_thresh)), float(lambda_s), _p(grad_rows))
    return float(L), grad_rows


def prune_key(R, idx, rows, key, tau, dilate=True):
    """Prune with dilation on a per-row key (hot = key >= tau).  Returns (idx', rows' [M',stride])."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    key = _c(key, np.float64)
    assert key.shape == (rows.shape[0],)
    idx_out = np.empty(R ** 3, np.int32)
    args = (R, _p(idx), _p(rows), rows.shape[1], _p(key), float(tau), int(bool(dilate)), _p(idx_out))
    m = lib.orc_prune_key(*args, None)
    rows_out = np.empty((m, rows.shape[1]), np.float64)
    lib.orc_prune_key(*args, _p(rows_out))
    return idx_out, rows_out


def upsample(R, idx, rows, R2):
    """Trilinear resample R -> R2.  Returns (idx' [R2^3] int32, rows' [M',28] FP64)."""
    lib = _load()
    idx = _c(idx, np.int32)
    rows = _rows(rows)
    idx_out = np.empty(R2 ** 3, np.int32)
    m = lib.orc_upsample(R, _p(idx), _p(rows), rows.shape[1], R2, _p(idx_out), None)
    rows_out = np.zeros((m, NV), np.float64)
    lib.orc_upsample(R, _p(idx), _p(rows), rows.shape[1], R2, _p(idx_out), _p(rows_out))
    return idx_out, rows_out


def round_bf16(x):
    """FP32 -> BF16 (round to nearest even), returned as FP32 values."""
    lib = _load()
    y = np.array(x, np.float32, order="C", copy=True)
    lib.orc_round_bf16(_p(y), y.size)
    return y
