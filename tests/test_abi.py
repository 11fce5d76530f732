"""The C-ABI library builds, loads without a GPU, exports every function that
include/*.h declares, and rejects bad arguments on the host before any launch."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(plx_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2112_05131_gb300 import _lib

    return _lib.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ["plx_grid_create", "plx_render", "plx_render_backward", "plx_tv_grad", "plx_rmsprop_step",
              "plx_grid_prune_count", "plx_grid_upsample_apply", "plx_gen_rays", "plx_check"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2112_05131_gb300 import _lib

    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a signature for every exported entry point, under the same name
    assert names == set(_lib.SIGNATURES), names.symmetric_difference(set(_lib.SIGNATURES))


def test_status_strings_and_version(lib):
    assert lib.plx_status_str(0) == b"ok"
    assert lib.plx_status_str(1) == b"invalid argument"
    assert lib.plx_status_str(7).startswith(b"device")
    assert b"sm_103a" in lib.plx_version()


def test_workspace_sizes(lib):
    from paper_2112_05131_gb300 import _lib

    d = _lib.plx_grid_desc()
    d.reso = 512
    for a in range(3):
        d.aabb_min[a] = -1.0
        d.aabb_max[a] = 1.0
    d.n_rows = 4_000_000
    d.sh_form = 0
    ws = lib.plx_grid_workspace_bytes(ctypes.byref(d))
    # status block + one bit per node + one bit per 8^3-cell block (64 blocks per axis: cells 0..510) + one
    # bit per row + a 4-byte list entry per row, each rounded to 256 bytes

    def up(b):
        return (b + 255) // 256 * 256

    nb = (512 - 2) // 8 + 1
    assert ws == 256 + up(512 ** 3 // 8) + up((nb ** 3 + 31) // 32 * 4) + up(((4_000_000 + 31) // 32 + 1) * 4) \
        + up(4_000_000 * 4)
    assert ws % 256 == 0
    d.reso = 1
    assert lib.plx_grid_workspace_bytes(ctypes.byref(d)) == 0
    assert lib.plx_prune_workspace_bytes(1) == 0
    assert lib.plx_prune_workspace_bytes(64) > 2 * 64 ** 3 // 8
    assert lib.plx_upsample_workspace_bytes(128) > 128 ** 3 // 8


def _einval(lib, status):
    from paper_2112_05131_gb300 import _lib

    assert status == 1, status
    assert lib.plx_last_error() != b""


def test_host_validation_rejects_bad_arguments(lib):
    """Every check below fails before the library touches CUDA, so it runs without a GPU."""
    from paper_2112_05131_gb300 import _lib

    null = None
    opts = _lib.plx_render_opts()
    opts.step_vox = 0.5
    _einval(lib, lib.plx_render(null, null, null, 10, ctypes.byref(opts), null, null, null))
    _einval(lib, lib.plx_render_backward(null, null, null, 10, ctypes.byref(opts), null, null, 0.0, null, null))
    _einval(lib, lib.plx_gen_rays(null, 0, 8, 8, null, 4, null, null, null))
    _einval(lib, lib.plx_gen_rays(null, 1, 8, 8, null, 4, null, null, null))
    _einval(lib, lib.plx_mse_grad(null, null, 3, null, null, null))
    _einval(lib, lib.plx_mse_grad(null, null, -1, null, null, null))
    d = _lib.plx_grid_desc()
    d.reso = 8
    for a in range(3):
        d.aabb_min[a] = -1.0
        d.aabb_max[a] = 1.0
    d.n_rows = 10
    d.sh_form = 0
    out = ctypes.c_void_p()
    _einval(lib, lib.plx_grid_create(ctypes.byref(d), null, null, null, null, null, ctypes.byref(out)))
    # misaligned workspace
    _einval(lib, lib.plx_grid_create(ctypes.byref(d), ctypes.c_void_p(256), ctypes.c_void_p(256), null,
                                     ctypes.c_void_p(256 + 8), null, ctypes.byref(out)))
    # F32 form given BF16 rows
    _einval(lib, lib.plx_grid_create(ctypes.byref(d), ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(512),
                                     ctypes.c_void_p(1024), null, ctypes.byref(out)))
    d.sh_form = 5
    _einval(lib, lib.plx_grid_create(ctypes.byref(d), ctypes.c_void_p(256), ctypes.c_void_p(256), null,
                                     ctypes.c_void_p(1024), null, ctypes.byref(out)))
    d.sh_form = 0
    d.aabb_max[1] = -2.0
    _einval(lib, lib.plx_grid_create(ctypes.byref(d), ctypes.c_void_p(256), ctypes.c_void_p(256), null,
                                     ctypes.c_void_p(1024), null, ctypes.byref(out)))
    assert out.value is None
    _einval(lib, lib.plx_tv_grad(null, null, null, 1, 1, 1.0, 1.0, null, null, null))
    _einval(lib, lib.plx_rmsprop_step(null, null, null, 1.0, 1.0, 0.9, 1e-8, 1, null))
    n = ctypes.c_int64()
    _einval(lib, lib.plx_grid_prune_count(null, 5.0, 1, null, ctypes.byref(n), null))
    _einval(lib, lib.plx_grid_upsample_count(null, 64, null, ctypes.byref(n), null))
    # the trainer: no grid, no handle, bad descriptor
    td = _lib.plx_trainer_desc()
    td.batch, td.opts, td.beta, td.eps, td.sparse_rmsprop = 5000, opts, 0.95, 1e-8, 1
    assert lib.plx_trainer_workspace_bytes(null, ctypes.byref(td)) == 0
    tr = ctypes.c_void_p()
    _einval(lib, lib.plx_trainer_create(null, ctypes.byref(td), null, 1, 8, 8, null, null, null, 0, ctypes.byref(tr)))
    _einval(lib, lib.plx_trainer_create(null, ctypes.byref(td), null, 1, 8, 8, null, null, null, 0, null))
    assert tr.value is None
    used = ctypes.c_int32()
    _einval(lib, lib.plx_trainer_step(null, null, 10, null, null, null, 0, 0, 1.0, 1.0, null, 0, null, null, null,
                                      null, ctypes.byref(used), null))
    _einval(lib, lib.plx_trainer_finish(null, null))
    assert lib.plx_trainer_destroy(null) == 0
    _einval(lib, lib.plx_check(null, null))
    _einval(lib, lib.plx_grid_get_desc(null, null))
