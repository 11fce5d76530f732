"""plx_grid_prune_noalloc: pruning for callers that cannot allocate device memory while they run.

Such a caller (an embedder with a fixed memory budget and no allocator to lend, or a real-time loop
that cannot afford an allocation's device-wide synchronisation) calls this one entry point, which
keeps its scratch in a fixed device array inside the library.  These tests call it through the C ABI
and check that it returns exactly what the two-phase plx_grid_prune_count/apply returns, on two
calls in a row (the fixed array keeps the previous call's contents), and that it refuses grids beyond
its fixed size.  This file is collected last, so a stop at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _grid(R, frac, seed):
    from paper_2112_05131_gb300.grid import Grid

    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=R ** 3) < frac
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    rows = rng.normal(0, 1.0, size=(int(occ.sum()), 28)).astype(np.float32)
    rows[:, 0] = rng.uniform(0, 10, size=rows.shape[0]).astype(np.float32)
    return Grid.from_host(R, idx, rows)


def _noalloc(lib, g, tau, dilate):
    idx_new = torch.full((g.reso ** 3,), -7, dtype=torch.int32, device="cuda")
    rows_new = torch.full((max(g.M, 1), 32), float("nan"), dtype=torch.float32, device="cuda")
    n = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.plx_grid_prune_noalloc(g.handle, ctypes.c_float(tau), 1 if dilate else 0,
                                    ctypes.c_void_p(idx_new.data_ptr()), ctypes.c_void_p(rows_new.data_ptr()),
                                    ctypes.byref(n), stream)
    assert st == 0, lib.plx_last_error()
    return idx_new.cpu().numpy(), rows_new[: n.value].cpu().numpy(), n.value


def _check_against_workspace_prune(lib, calls):
    for g, tau, dilate in calls:
        idx_a, rows_a, n_a = _noalloc(lib, g, tau, dilate)
        ref = g.prune(tau, dilate)  # plx_grid_prune_count + plx_grid_prune_apply with a workspace
        torch.cuda.synchronize()
        assert n_a == ref.M
        assert np.array_equal(idx_a, ref.idx.cpu().numpy())
        assert np.array_equal(rows_a, ref.rows.cpu().numpy())
        g.check()


@pytest.mark.parametrize("R,frac", [(40, 0.2), (64, 0.05)])
def test_prune_noalloc_matches_prune_with_workspace(cuda_lib, R, frac):
    calls = [(_grid(R, frac, 1), 6.0, True), (_grid(R, frac * 2, 2), 3.5, False)]  # two calls in a row
    _check_against_workspace_prune(cuda_lib, calls)


def test_prune_noalloc_at_its_limit_then_smaller(cuda_lib):
    """A 256^3 grid, whose scratch layout fills the whole fixed array, then smaller grids: each later call
    reads only what it wrote itself, so the larger call's leftovers beyond the small layouts change
    nothing."""
    calls = [(_grid(256, 0.01, 3), 6.0, True), (_grid(64, 0.05, 4), 5.0, True), (_grid(40, 0.2, 5), 3.5, False)]
    _check_against_workspace_prune(cuda_lib, calls)


def test_prune_noalloc_refuses_grids_beyond_its_fixed_scratch(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid

    lib = cuda_lib
    R = 257  # one node per axis beyond the fixed scratch's 256
    idx = torch.full((R ** 3,), -1, dtype=torch.int32, device="cuda")
    g = Grid(R, idx, torch.zeros((0, 32), dtype=torch.float32, device="cuda"))
    n = ctypes.c_int64(-1)
    st = lib.plx_grid_prune_noalloc(g.handle, ctypes.c_float(1.0), 1, ctypes.c_void_p(idx.data_ptr()), None,
                                    ctypes.byref(n), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 6  # PLX_EUNSUPPORTED, nothing launched
    assert b"256" in lib.plx_last_error()
    assert n.value == -1
