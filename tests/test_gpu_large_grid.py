"""A grid past the size where a node's linear id leaves 32 bits in the march's cheap candidate test
(R = 1300: ids up to 2.2e9; the test switches to 64-bit ids above R = 1290), with the FP32 margin,
the coarse block mask and the occupancy build at that size: forward, the recomputing adjoint and the
training march against the oracle on rays through a blob of occupied nodes, and TV on runs of nodes
through it.  The index volume is
8.8 GB, on the host for the oracle and on the device; the test is skipped where either lacks room."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from parity import check_colours, check_grads, delta_of, tie_flags

pytestmark = pytest.mark.gpu

R = 1300
BG = (1.0, 1.0, 1.0)


def _host_free_bytes():
    try:
        with open("/proc/meminfo") as f:
            info = dict(line.split(":", 1) for line in f)
        return int(info["MemAvailable"].split()[0]) * 1024
    except (OSError, KeyError, ValueError):
        return 0


@pytest.fixture(scope="module")
def big_scene():
    need = 4 * R ** 3
    if _host_free_bytes() < 3 * need:
        pytest.skip("not enough host memory for a 1300^3 index volume")
    if torch.cuda.mem_get_info()[0] < 3 * need:
        pytest.skip("not enough device memory for a 1300^3 index volume")
    rng = np.random.default_rng(1300)
    idx = np.full(R ** 3, -1, np.int32)
    # a blob of nodes around (1275, 650, 200) in grid units: linear ids from 2.12e9 to 2.19e9, on both
    # sides of 2^31
    c = np.array([1275, 650, 200])
    ijk = np.stack(np.meshgrid(*[np.arange(-20, 21)] * 3, indexing="ij"), -1).reshape(-1, 3)
    ijk = ijk[(ijk ** 2).sum(1) <= 20 ** 2] + c
    ijk = ijk[rng.uniform(size=ijk.shape[0]) < 0.6]
    n = (ijk[:, 0].astype(np.int64) * R + ijk[:, 1]) * R + ijk[:, 2]
    idx[n] = np.arange(n.size, dtype=np.int32)
    rows = rng.normal(0, 0.4, size=(n.size, 28)).astype(np.float32)
    rows[:, 0] = rng.uniform(0.0, 400.0, size=n.size).astype(np.float32)
    assert n.min() < 2 ** 31 < n.max()
    return synth.Scene(R, idx, rows), c


def test_large_grid_render_and_adjoints(cuda_lib, big_scene):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc, c = big_scene
    h = 2.0 / (R - 1)
    centre = -1.0 + h * c.astype(np.float64)
    rng = np.random.default_rng(7)
    dirs = rng.normal(size=(400, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    o = (centre[None, :] - 3.0 * dirs + rng.normal(0, 12 * h, size=(400, 3))).astype(np.float32)
    d = dirs.astype(np.float32)
    delta = delta_of(R, 0.5)
    ref, aux = oracle.render(R, sc.idx, sc.rows, o.astype(float), d.astype(float), bg=BG)
    keep = ~tie_flags(aux, delta)
    o, d, ref, aux = o[keep], d[keep], ref[keep], aux[keep]
    n = o.shape[0]
    gw = (rng.normal(size=(n, 3)) * 1e-3).astype(np.float32)
    gref = oracle.render_backward(R, sc.idx, sc.rows, o.astype(float), d.astype(float), gw.astype(float), bg=BG)

    g = Grid.from_host(R, sc.idx, sc.rows)
    opts = RenderOpts(0.5, BG, 0.0)
    ot, dt, gwt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(gw).cuda()
    rgb = g.render(ot, dt, opts).cpu().numpy()
    grad = g.render_backward(ot, dt, gwt, opts).cpu().numpy()
    state = g.new_march_state(n, opts)
    g.march_plan(ot, dt, opts, state)
    rgb_t = g.render_planned(ot, dt, opts, state).cpu().numpy()
    grad_t = g.render_backward_train(ot, dt, gwt, opts, state).cpu().numpy()
    g.check()
    w1, _ = check_colours(rgb, ref, aux, sc.rows, delta, BG)
    check_colours(rgb_t, ref, aux, sc.rows, delta, BG)
    w2 = check_grads(grad, gref)
    check_grads(grad_t, gref)
    assert np.sum(np.abs(ref - 1.0).max(1) > 1e-2) > n // 2  # most rays cross the blob
    print(f"R = {R}: {sc.M} rows, colour err/tol {w1:.3f}, grad err/tol {w2:.3f} on {n} rays")


def test_large_grid_tv(cuda_lib, big_scene):
    """TV on runs of nodes through the blob, whose linear ids straddle 2^31 (the kernel's 32-bit
    coordinate division covers ids below 2^32): gradients and loss against the oracle."""
    from paper_2112_05131_gb300.grid import Grid

    sc, c = big_scene
    di, dj = np.meshgrid(np.arange(-20, 21, 2), np.arange(-20, 21, 2), indexing="ij")
    starts = (((c[0] + di.ravel()).astype(np.int64) * R + (c[1] + dj.ravel())) * R + (c[2] - 30)).astype(np.int64)
    starts = np.sort(starts)
    lens = np.full(starts.shape, 61, np.int64)
    assert starts.min() < 2 ** 31 < starts.max()
    g = Grid.from_host(R, sc.idx, sc.rows)
    grad = torch.zeros((sc.M, 32), device="cuda")
    loss = torch.zeros(1, device="cuda")
    g.tv_grad(torch.from_numpy(starts).cuda(), torch.from_numpy(lens).cuda(), int(lens.sum()), 1e-2, 3e-3, grad, loss)
    g.check()
    L_ref, g_ref = oracle.tv(R, sc.idx, sc.rows, starts, lens, 1e-2, 3e-3)
    w = check_grads(grad.cpu().numpy(), g_ref)
    assert abs(loss.item() - L_ref) <= 1e-5 * abs(L_ref) + 1e-12
    assert int((g_ref != 0).any(1).sum()) > 1000
    print(f"R = {R} TV: {starts.shape[0]} runs, grad err/tol {w:.3f}")
