"""The Cauchy sparsity prior (Sec. 3.7, Eq. 4), fused into both adjoints: plx_render_backward and
plx_render_backward_train with lambda_sparsity > 0 against the oracle's adjoint plus the oracle's
sparsity gradient, and the prior's value against the oracle's.

Tolerances: gradients as every adjoint test (tests/parity.py).  The value is a sum of FP32
log1p terms, each within a few ulp, added in warps of 32 and then by one atomic per warp and chunk;
its relative error stays far below 1e-4, the bound asserted.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import bf16_grid_rows, check_grads, delta_of, tie_flags

pytestmark = pytest.mark.gpu

BG = (1.0, 1.0, 1.0)
LOSS_RTOL = 1e-4


def _scene(R, frac, seed):
    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=R ** 3) < frac
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    M = int(occ.sum())
    rows = rng.normal(0, 0.4, size=(M, 28)).astype(np.float32)
    rows[:, 0] = rng.uniform(-3.0, 25.0, size=M).astype(np.float32)  # some negative: no prior there
    return synth.Scene(R, idx, rows)


def _gpu_adjoint(g, path, o, d, gw, opts, lam):
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    gwt = torch.from_numpy(gw.astype(np.float32)).cuda()
    loss = torch.zeros(1, device="cuda")
    if path == "recompute":
        grad = g.render_backward(ot, dt, gwt, opts, lambda_sparsity=lam, loss_sparsity=loss)
    else:
        state = g.new_march_state(o.shape[0], opts)
        g.render_train(ot, dt, opts, state)
        grad = g.render_backward_train(ot, dt, gwt, opts, state, lambda_sparsity=lam, loss_sparsity=loss)
    g.check()
    return grad.cpu().numpy(), float(loss.item())


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("path", ["recompute", "train"])
@pytest.mark.parametrize("stop,photometric", [(0.0, False), (0.0, True), (1e-3, True)])
def test_sparsity_adjoint_matches_oracle(cuda_lib, form, path, stop, photometric):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _scene(40, 0.15, 11 + form)
    rows = sc.rows if form == 0 else bf16_grid_rows(sc.rows)
    o, d = synth.random_rays(1500, seed=12)
    _, aux = oracle.render(sc.R, sc.idx, rows, o.astype(float), d.astype(float), bg=BG, stop_thresh=stop)
    keep = ~tie_flags(aux, delta_of(sc.R, 0.5))
    o, d = o[keep], d[keep]
    n = o.shape[0]
    gw = np.random.default_rng(13).normal(size=(n, 3)) / n if photometric else np.zeros((n, 3))
    lam = 1e-4
    ref = oracle.render_backward(sc.R, sc.idx, rows, o.astype(float), d.astype(float),
                                 gw.astype(np.float32).astype(float), bg=BG, stop_thresh=stop)
    L_ref, ref = oracle.sparsity(sc.R, sc.idx, rows, o.astype(float), d.astype(float), lam, stop_thresh=stop,
                                 grad_rows=ref)
    g = Grid.from_host(sc.R, sc.idx, sc.rows, sh_form=form)
    grad, L = _gpu_adjoint(g, path, o, d, gw, RenderOpts(0.5, BG, stop), lam)
    worst = check_grads(grad, ref)
    if not photometric:
        assert np.all(grad[:, 1:] == 0.0)  # the prior reaches the density column only
    assert L_ref > 0 and abs(L - L_ref) <= LOSS_RTOL * L_ref, (L, L_ref)
    print(f"sparsity form {form} {path} stop {stop} photometric {photometric}: grad err/tol {worst:.3f}, "
          f"loss rel err {abs(L - L_ref) / L_ref:.2e}")


def test_sparsity_zero_lambda_changes_nothing(cuda_lib):
    """lambda 0 with a loss buffer: the adjoint equals the one without the prior, the loss stays 0."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _scene(24, 0.3, 21)
    o, d = synth.random_rays(700, seed=22)
    gw = torch.from_numpy(np.random.default_rng(23).normal(size=(700, 3)).astype(np.float32) * 1e-3).cuda()
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    opts = RenderOpts(0.5, BG, 0.0)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    state = g.new_march_state(700, opts)
    g.render_train(ot, dt, opts, state)
    loss = torch.zeros(1, device="cuda")
    a = g.render_backward_train(ot, dt, gw, opts, state, lambda_sparsity=0.0, loss_sparsity=loss).cpu().numpy()
    b = g.render_backward_train(ot, dt, gw, opts, state).cpu().numpy()
    g.check()
    assert loss.item() == 0.0
    check_grads(a, b.astype(np.float64))


def test_sparsity_training_march_sparse512(cuda_lib):
    """Full size, in the training march's launch configuration: the 512^3 workload's 5000-ray batch,
    FP32 rows, photometric and prior gradients together, every gradient row and the prior's value."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    gt = synth.scene_config("sparse512")
    sc = synth.perturb(gt, 0.02, seed=1)
    R, n = sc.R, 5000
    cams = synth.cameras_config("hemi100_800")
    pix = synth.pixel_batch(100, 800, 800, n, seed=1003)
    o64, d64 = oracle.gen_rays(cams.astype(np.float64), pix)
    o, d = o64.astype(np.float32), d64.astype(np.float32)
    gw = (np.random.default_rng(78).normal(size=(n, 3)) * 1e-3).astype(np.float32)
    lam = 1e-5
    ref = oracle.render_backward(R, sc.idx, sc.rows, o.astype(float), d.astype(float), gw.astype(float), bg=BG)
    L_ref, ref = oracle.sparsity(R, sc.idx, sc.rows, o.astype(float), d.astype(float), lam, grad_rows=ref)
    g = Grid.from_host(R, sc.idx, sc.rows)
    grad, L = _gpu_adjoint(g, "train", o, d, gw, RenderOpts(0.5, BG, 0.0), lam)
    worst = check_grads(grad, ref)
    assert abs(L - L_ref) <= LOSS_RTOL * L_ref, (L, L_ref)
    print(f"512^3 sparsity: grad err/tol {worst:.3f}, loss {L:.6e} vs {L_ref:.6e}")
