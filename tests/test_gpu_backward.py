"""Adjoint parity: plx_render_backward (through the C ABI) vs the FP64 oracle's adjoint."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import FP32_SUM_U, bf16_grid_rows, check_grads, dense32_step_case

pytestmark = pytest.mark.gpu

Y00 = 0.28209479177387814


def _scene(R, frac_occ, seed, neg_frac=0.0, dc=0.0):
    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=R ** 3) < frac_occ
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    M = int(occ.sum())
    rows = np.empty((M, 28), np.float32)
    rows[:, 0] = rng.uniform(0.0, 25.0, size=M)
    if neg_frac:
        neg = rng.uniform(size=M) < neg_frac
        rows[neg, 0] *= -1
    rows[:, 1:] = rng.normal(0, 0.4, size=(M, 27))
    rows[:, [1, 10, 19]] += np.float32(dc / Y00)
    return synth.Scene(R, idx, rows)


def _backward_both(sc, o, d, gw, opts, form=0):
    from paper_2112_05131_gb300.grid import Grid

    g = Grid.from_host(sc.R, sc.idx, sc.rows, sh_form=form)
    grad = g.render_backward(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                             torch.from_numpy(gw.astype(np.float32)).cuda(), opts)
    g.check()
    rows = sc.rows if form == 0 else bf16_grid_rows(sc.rows)
    ref = oracle.render_backward(sc.R, sc.idx, rows, o.astype(float), d.astype(float), gw.astype(np.float32).astype(float),
                                 step_vox=opts.step_vox, bg=opts.bg, stop_thresh=opts.stop_thresh)
    return grad.cpu().numpy(), ref, g


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("stop", [0.0, 1e-4])
def test_backward_dense32(cuda_lib, form, stop):
    """The dense 32^3 workload's step: the adjoint of the perturbed grid fed the MSE gradient against the
    ground truth's colours (random-sign dL/dC is exercised by the sparse cases below)."""
    from paper_2112_05131_gb300.grid import RenderOpts

    sc, o, d, gw = dense32_step_case(2048, 31, stop_thresh=stop)
    grad, ref, _ = _backward_both(sc, o, d, gw, RenderOpts(0.5, (1.0, 1.0, 1.0), stop), form)
    rows = sc.rows if form == 0 else bf16_grid_rows(sc.rows)
    mag = oracle.render_backward_mag(sc.R, sc.idx, rows, o.astype(float), d.astype(float), gw.astype(float),
                                     step_vox=0.5, bg=(1.0, 1.0, 1.0), stop_thresh=stop)
    worst = check_grads(grad, ref, extra_abs=FP32_SUM_U * mag)
    assert np.all(grad[:, 28:] == 0.0)  # padding columns are never written
    print(f"dense32 form={form} stop={stop}: worst err/tol {worst:.3f}")


@pytest.mark.parametrize("R,n", [(40, 999), (57, 2500)])
def test_backward_sparse_with_negative_density(cuda_lib, R, n):
    from paper_2112_05131_gb300.grid import RenderOpts

    sc = _scene(R, 0.2, 200 + R, neg_frac=0.3, dc=0.0)
    o, d = synth.random_rays(n, seed=R + 1, spread=0.9)
    gw = np.random.default_rng(R).normal(size=(n, 3))
    grad, ref, _ = _backward_both(sc, o, d, gw, RenderOpts(0.5, (0.5, 0.7, 1.0), 0.0))
    worst = check_grads(grad, ref)
    # rows whose node lies farther than one cell diagonal from every ray cannot be a corner of a
    # sampled cell: exactly zero on the GPU (FP32 may give a corner on a cell face a 1e-8 weight where
    # FP64 gives 0, so rows merely untouched by the oracle are covered by the tolerance above)
    print(f"sparse R={R}: worst err/tol {worst:.3f}")
    from paper_2112_05131_gb300.grid import Grid

    few = 8
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    g8 = g.render_backward(torch.from_numpy(o[:few]).cuda(), torch.from_numpy(d[:few]).cuda(),
                           torch.ones((few, 3), device="cuda"), RenderOpts(0.5, (0.5, 0.7, 1.0), 0.0)).cpu().numpy()
    h = 2.0 / (R - 1)
    node_rows = np.flatnonzero(sc.idx >= 0)
    pos = -1.0 + h * np.stack(np.unravel_index(node_rows, (R, R, R)), 1)
    far = np.ones(node_rows.shape[0], bool)
    o64, d64 = o[:few].astype(np.float64), d[:few].astype(np.float64)
    for r in range(few):
        rel = pos - o64[r]
        dist = np.linalg.norm(rel - (rel @ d64[r])[:, None] * d64[r][None, :], axis=1)
        far &= dist > np.sqrt(3.0) * h * 1.001
    far_rows = sc.idx[node_rows[far]]
    assert far_rows.size > 0 and np.all(g8[far_rows] == 0.0)
    assert np.any(g8 != 0.0)


def test_autograd_function_matches_direct_backward(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts, render

    sc = _scene(24, 0.3, 7, dc=1.0)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    g.rows.requires_grad_(True)
    o, d = synth.random_rays(777, seed=8)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    target = torch.rand(777, 3, device="cuda")
    rgb = render(g, ot, dt, RenderOpts())
    loss = ((rgb - target) ** 2).sum()
    loss.backward()
    gw = (2 * (rgb.detach() - target)).contiguous()
    direct = g.render_backward(ot, dt, gw, RenderOpts())
    a, b = g.rows.grad.cpu().numpy(), direct.cpu().numpy()
    check_grads(a, b.astype(np.float64))


def test_backward_zero_rays_and_missing_rays(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _scene(16, 0.5, 3)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    e = torch.empty((0, 3), device="cuda")
    grad = g.render_backward(e, e, e, RenderOpts())
    assert torch.all(grad == 0)
    o = torch.tensor([[3.0, 3.0, 3.0]], device="cuda")
    dd = torch.tensor([[1.0, 0.0, 0.0]], device="cuda")
    grad = g.render_backward(o, dd, torch.ones(1, 3, device="cuda"), RenderOpts())
    assert torch.all(grad == 0)
