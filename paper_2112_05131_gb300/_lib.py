"""ctypes binding of libplenoxel (include/plenoxel.h): the same names, argument marshalling only.

``load()`` builds the library in-tree with nvcc if it is missing or stale and
returns the ``ctypes.CDLL``.  There is no fallback: if the library cannot be
built or loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import threading

from . import _build

_lock = threading.Lock()
_lib = None

c_void_p = ctypes.c_void_p
c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_float = ctypes.c_float
c_size_t = ctypes.c_size_t

PLX_OK = 0
PLX_SH_F32 = 0
PLX_SH_BF16 = 1
STATUS_NAMES = {0: "PLX_OK", 1: "PLX_EINVAL", 2: "PLX_ENOMEM", 3: "PLX_ECUDA", 4: "PLX_ETIMEOUT",
                5: "PLX_EBUSY", 6: "PLX_EUNSUPPORTED", 7: "PLX_EDEVICE"}


class plx_grid_desc(ctypes.Structure):
    _fields_ = [("reso", c_int32), ("aabb_min", c_float * 3), ("aabb_max", c_float * 3),
                ("n_rows", c_int64), ("sh_form", c_int32)]


class plx_render_opts(ctypes.Structure):
    _fields_ = [("step_vox", c_float), ("bg", c_float * 3), ("stop_thresh", c_float)]


class plx_trainer_desc(ctypes.Structure):
    _fields_ = [("batch", c_int32), ("opts", plx_render_opts), ("lambda_tv_sigma", c_float), ("lambda_tv_sh", c_float),
                ("lambda_sparsity", c_float), ("beta", c_float), ("eps", c_float), ("sparse_rmsprop", c_int32),
                ("max_segments", c_int32)]


class plx_host_batch(ctypes.Structure):
    _fields_ = [("pix", c_void_p), ("target", c_void_p), ("seg_start", c_void_p), ("seg_len", c_void_p),
                ("n", c_int64), ("n_seg", c_int64), ("n_selected", c_int64)]


# name -> (restype, argtypes); every name here is declared in include/plenoxel.h
SIGNATURES = {
    "plx_status_str": (ctypes.c_char_p, [c_int32]),
    "plx_last_error": (ctypes.c_char_p, []),
    "plx_version": (ctypes.c_char_p, []),
    "plx_grid_workspace_bytes": (c_size_t, [ctypes.POINTER(plx_grid_desc)]),
    "plx_grid_create": (c_int32, [ctypes.POINTER(plx_grid_desc), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  ctypes.POINTER(c_void_p)]),
    "plx_grid_destroy": (c_int32, [c_void_p]),
    "plx_grid_get_desc": (c_int32, [c_void_p, ctypes.POINTER(plx_grid_desc)]),
    "plx_pack_bf16": (c_int32, [c_void_p, c_void_p]),
    "plx_check": (c_int32, [c_void_p, c_void_p]),
    "plx_gen_rays": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "plx_render": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(plx_render_opts), c_void_p,
                             c_void_p, c_void_p]),
    "plx_render_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(plx_render_opts),
                                      c_void_p, c_void_p, c_float, c_void_p, c_void_p]),
    "plx_march_state_bytes": (c_size_t, [c_void_p, c_int64, ctypes.POINTER(plx_render_opts)]),
    "plx_render_train": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(plx_render_opts), c_void_p,
                                   c_void_p, c_void_p, c_size_t, c_void_p]),
    "plx_march_plan": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(plx_render_opts), c_void_p,
                                 c_size_t, c_void_p]),
    "plx_render_planned": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(plx_render_opts),
                                     c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "plx_render_planned_mse": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(plx_render_opts),
                                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "plx_render_backward_train": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(plx_render_opts),
                                            c_void_p, c_void_p, c_size_t, c_void_p, c_float, c_void_p, c_void_p]),
    "plx_render_tiles": (c_int32, [ctypes.POINTER(c_void_p), c_int32, c_void_p, c_int32, c_void_p, c_int64,
                                   ctypes.POINTER(plx_render_opts), c_void_p]),
    "plx_count_nodes": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(plx_render_opts), c_void_p,
                                  c_void_p]),
    "plx_count_touched": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "plx_trainer_workspace_bytes": (c_size_t, [c_void_p, ctypes.POINTER(plx_trainer_desc)]),
    "plx_trainer_create": (c_int32, [c_void_p, ctypes.POINTER(plx_trainer_desc), c_void_p, c_int32, c_int32, c_int32,
                                     c_void_p, c_void_p, c_void_p, c_size_t, ctypes.POINTER(c_void_p)]),
    "plx_trainer_destroy": (c_int32, [c_void_p]),
    "plx_trainer_step": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_float,
                                   c_float, c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                   ctypes.POINTER(c_int32), c_void_p]),
    "plx_trainer_step_host": (c_int32, [c_void_p, ctypes.POINTER(plx_host_batch), ctypes.POINTER(plx_host_batch),
                                        c_float, c_float, c_void_p, c_void_p]),
    "plx_trainer_finish": (c_int32, [c_void_p, c_void_p]),
    "plx_trainer_buffers": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                      ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), ctypes.POINTER(c_size_t)]),
    "plx_max_weight": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, ctypes.POINTER(plx_render_opts), c_void_p,
                                 c_void_p]),
    "plx_mse_grad": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "plx_tv_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_float, c_float, c_void_p, c_void_p,
                              c_void_p]),
    "plx_rmsprop_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_float, c_float, c_float, c_float, c_int32,
                                   c_void_p]),
    "plx_prune_workspace_bytes": (c_size_t, [c_int32]),
    "plx_grid_prune_count": (c_int32, [c_void_p, c_float, c_int32, c_void_p, ctypes.POINTER(c_int64), c_void_p]),
    "plx_grid_prune_count_key": (c_int32, [c_void_p, c_void_p, c_float, c_int32, c_void_p, ctypes.POINTER(c_int64),
                                           c_void_p]),
    "plx_grid_prune_apply": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "plx_grid_prune_noalloc": (c_int32, [c_void_p, c_float, c_int32, c_void_p, c_void_p, ctypes.POINTER(c_int64),
                                         c_void_p]),
    "plx_upsample_workspace_bytes": (c_size_t, [c_int32]),
    "plx_grid_upsample_count": (c_int32, [c_void_p, c_int32, c_void_p, ctypes.POINTER(c_int64), c_void_p]),
    "plx_grid_upsample_apply": (c_int32, [c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
}


class PlxError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def load(build: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) libplenoxel.so and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.LIB
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, where: str) -> None:
    if status != PLX_OK:
        msg = load().plx_last_error()
        raise PlxError(status, where, msg.decode() if msg else "")


def call(name: str, *args):
    """Call entry point `name` and raise PlxError unless it returns PLX_OK."""
    fn = getattr(load(), name)
    check(fn(*args), name)
