"""The training march (plx_render_train / plx_render_backward_train, chunk work items and a march
state handed from the forward to the adjoint) against the FP64 oracle, through the C ABI."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from parity import FP32_SUM_U, bf16_grid_rows, check_colours, check_grads, delta_of, dense32_step_case, tie_flags

pytestmark = pytest.mark.gpu

BG = (0.9, 0.6, 0.3)


def _sparse_scene(R, frac_occ, seed, sigma=(0.0, 30.0), neg_frac=0.2):
    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=R ** 3) < frac_occ
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    M = int(occ.sum())
    rows = np.empty((M, 28), np.float32)
    rows[:, 0] = rng.uniform(*sigma, size=M)
    neg = rng.uniform(size=M) < neg_frac
    rows[neg, 0] = -rows[neg, 0]
    rows[:, 1:] = rng.normal(0, 0.4, size=(M, 27))
    return synth.Scene(R, idx, rows)


def _both(sc, o, d, gw, opts, form=0):
    """(rgb, T_end, grad) from the training march, and the oracle's (rgb, aux, grad), on the same rays."""
    from paper_2112_05131_gb300.grid import Grid

    g = Grid.from_host(sc.R, sc.idx, sc.rows, sh_form=form)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    state = g.new_march_state(o.shape[0], opts)
    T = torch.empty(o.shape[0], device="cuda")
    rgb = g.render_train(ot, dt, opts, state, T_end=T)
    grad = g.render_backward_train(ot, dt, torch.from_numpy(gw).cuda(), opts, state)
    g.check()
    rows = sc.rows if form == 0 else bf16_grid_rows(sc.rows)
    kw = dict(step_vox=opts.step_vox, bg=opts.bg, stop_thresh=opts.stop_thresh)
    ref, aux = oracle.render(sc.R, sc.idx, rows, o.astype(float), d.astype(float), **kw)
    gref = oracle.render_backward(sc.R, sc.idx, rows, o.astype(float), d.astype(float), gw.astype(float), **kw)
    return rgb.cpu().numpy(), T.cpu().numpy(), grad.cpu().numpy(), ref, aux, gref, rows


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("stop", [0.0, 1e-4])
def test_train_march_dense32(cuda_lib, form, stop):
    """The dense 32^3 workload's step (perturbed grid, MSE gradient against the ground truth's colours);
    random-sign dL/dC is exercised by the sparse cases below."""
    from paper_2112_05131_gb300.grid import RenderOpts

    sc, o, d, gw = dense32_step_case(2048, 41, stop_thresh=stop)
    opts = RenderOpts(0.5, (1.0, 1.0, 1.0), stop)
    rgb, T, grad, ref, aux, gref, rows = _both(sc, o, d, gw, opts, form)
    wc, nflag = check_colours(rgb, ref, aux, rows, delta_of(sc.R, 0.5), opts.bg, stop)
    assert np.allclose(T, aux[:, 0], rtol=1e-4, atol=1e-6 + stop)
    mag = oracle.render_backward_mag(sc.R, sc.idx, rows, o.astype(float), d.astype(float), gw.astype(float),
                                     step_vox=0.5, bg=opts.bg, stop_thresh=stop)
    wg = check_grads(grad, gref, extra_abs=FP32_SUM_U * mag)
    print(f"dense32 form={form} stop={stop}: colour err/tol {wc:.3f} (flagged {nflag}), grad err/tol {wg:.3f}")


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("R,n", [(48, 1237), (67, 3001),
                                 (96, 40011)])  # several CTAs, ragged tails; the last above the fused-combine limit
def test_train_march_sparse(cuda_lib, R, n, form):
    from paper_2112_05131_gb300.grid import RenderOpts

    sc = _sparse_scene(R, 0.15, 300 + R)
    o, d = synth.random_rays(n, seed=R + 1, spread=0.9)
    gw = (np.random.default_rng(R).normal(size=(n, 3)) * 1e-3).astype(np.float32)
    opts = RenderOpts(0.5, BG, 0.0)
    rgb, T, grad, ref, aux, gref, rows = _both(sc, o, d, gw, opts, form)
    wc, nflag = check_colours(rgb, ref, aux, rows, delta_of(R, 0.5), BG)
    wg = check_grads(grad, gref)
    assert np.all(grad[:, 28:] == 0.0)
    print(f"sparse R={R} form={form}: colour err/tol {wc:.3f} (flagged {nflag}), grad err/tol {wg:.3f}")


# Unit roundoffs granted to FP32 where the adjoint subtracts nearly equal numbers: the density term
# T_{s+1} c - R_s of a long ray whose colours resemble what lies behind it (and sums of gradient
# terms of both signs).  Each operand is formed by fewer than 64 rounded operations along any path
# of the warp scans, the per-ray chunk scan and the interpolation and SH sums.
FP32_CANCEL_U = 64 * 2.0 ** -24


def test_train_march_long_rays_many_chunks(cuda_lib):
    """A dense 64^3 grid marched at 0.05 voxel: rays of 1300-2200 samples, more than 32 chunks each,
    so the per-ray combine runs its multi-group prefix and suffix passes.  Thin density and colours
    close to the background make T_{s+1} c - R_s cancel by up to ~400x on some rows; the gradient
    tolerance there adds FP32_CANCEL_U times the oracle's magnitude adjoint (the size of the
    operands), the rounding bound of any FP32 evaluation of the same formula."""
    from paper_2112_05131_gb300.grid import RenderOpts

    R = 64
    rng = np.random.default_rng(5)
    idx = np.arange(R ** 3, dtype=np.int32)
    rows = np.empty((R ** 3, 28), np.float32)
    rows[:, 0] = rng.uniform(0.0, 0.6, size=R ** 3)  # thin enough that light crosses the whole box
    rows[:, 1:] = rng.normal(0, 0.3, size=(R ** 3, 27))
    rows[:, [1, 10, 19]] += 2.0
    sc = synth.Scene(R, idx, rows)
    o, d = synth.random_rays(300, seed=6, spread=0.3)
    gw = (rng.normal(size=(300, 3)) * 1e-3).astype(np.float32)
    opts = RenderOpts(0.05, BG, 0.0)
    rgb, T, grad, ref, aux, gref, rows_ = _both(sc, o, d, gw, opts)
    assert aux[:, 1].max() > 32 * 32, aux[:, 1].max()  # some ray has more than 32 chunks
    wc, _ = check_colours(rgb, ref, aux, rows_, delta_of(R, 0.05), BG)
    mag = oracle.render_backward_mag(R, sc.idx, rows_, o.astype(float), d.astype(float), gw.astype(float),
                                     step_vox=0.05, bg=BG)
    wg = check_grads(grad, gref, extra_abs=FP32_CANCEL_U * mag)
    print(f"long rays (max {int(aux[:, 1].max())} samples): colour err/tol {wc:.3f}, grad err/tol {wg:.3f}")


def test_train_march_large_batch_combine(cuda_lib):
    """A batch above the fused-combine limit (33001 rays) on a dense 128^3 grid, so that the separate
    combine kernel takes both of its paths: rays of at most 8 chunks (at most 256 samples) a thread each,
    longer rays (up to ~430 samples) a warp each.  Colours and gradients against the oracle; the long rays
    get the same cancellation allowance as in the long-ray test above.  Each row receives ~30 samples'
    contributions, so the FP32 atomic sums stay within that allowance (a 40^3 grid under the same rays
    gives rows thousands of additions, beyond what a per-path rounding bound covers).  The colours are
    kept away from the ReLU kink (a DC term of 3 per channel, the other coefficients N(0, 0.2)): among
    7.5 M samples with zero-mean colours a few pre-activations lie within FP32 rounding of 0, where the
    FP32 march (its stored pre-activations interpolate the corners in slot order) and the FP64 oracle
    may take different ReLU masks and so disagree by that sample's whole SH gradient."""
    from paper_2112_05131_gb300.grid import RenderOpts

    R = 128
    rng = np.random.default_rng(11)
    idx = np.arange(R ** 3, dtype=np.int32)
    rows = np.empty((R ** 3, 28), np.float32)
    rows[:, 0] = rng.uniform(0.0, 2.0, size=R ** 3)
    rows[:, 1:] = rng.normal(0, 0.2, size=(R ** 3, 27))
    rows[:, [1, 10, 19]] += 3.0
    sc = synth.Scene(R, idx, rows)
    n = 33001
    o, d = synth.random_rays(n, seed=12, spread=0.9)
    gw = (rng.normal(size=(n, 3)) * 1e-3).astype(np.float32)
    opts = RenderOpts(0.5, BG, 0.0)
    rgb, T, grad, ref, aux, gref, rows_ = _both(sc, o, d, gw, opts)
    ns = aux[:, 1]
    assert np.any(ns > 8 * 32) and np.any((ns > 32) & (ns <= 8 * 32)), (ns.max(), np.median(ns))
    wc, _ = check_colours(rgb, ref, aux, rows_, delta_of(R, 0.5), BG)
    mag = oracle.render_backward_mag(R, sc.idx, rows_, o.astype(float), d.astype(float), gw.astype(float),
                                     step_vox=0.5, bg=BG)
    wg = check_grads(grad, gref, extra_abs=FP32_CANCEL_U * mag)
    print(f"large batch (max {int(ns.max())} samples, {int(np.sum(ns > 256))} rays above 8 chunks): "
          f"colour err/tol {wc:.3f}, grad err/tol {wg:.3f}")


def test_train_march_matches_render_and_is_deterministic(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _sparse_scene(40, 0.2, 21)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    o, d = synth.random_rays(5000, seed=22)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    opts = RenderOpts(0.5, BG, 0.0)
    state = g.new_march_state(5000, opts)
    a = g.render_train(ot, dt, opts, state).cpu().numpy()
    b = g.render_train(ot, dt, opts, state).cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))  # item order varies, results do not
    ref = g.render(ot, dt, opts).cpu().numpy()
    assert np.allclose(a, ref, rtol=1e-5, atol=1e-7)


def test_train_march_edge_cases(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    opts = RenderOpts(0.5, BG, 0.0)
    sc = _sparse_scene(16, 0.3, 9)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    # zero rays
    empty = torch.empty((0, 3), device="cuda")
    st0 = g.new_march_state(0, opts)
    assert g.render_train(empty, empty, opts, st0).shape == (0, 3)
    grad0 = g.render_backward_train(empty, empty, torch.empty((0, 3), device="cuda"), opts, st0)
    assert torch.count_nonzero(grad0) == 0
    # misses, rays starting inside, rays along faces
    o = np.float32([[3, 3, 3], [0.1, -0.2, 0.3], [-3, 0.5, 0.25], [-3, 1.0, 0.0], [0.0, 0.0, 5.0], [-3, -1, -1]])
    d = np.float32([[1, 0, 0], [0.6, 0.0, 0.8], [1, 0, 0], [1, 0, 0], [0, 0, -1], [1, 0, 0]])
    gw = np.full((6, 3), 0.01, np.float32)
    # rays 2-5 run along a box axis from outside: (t_far - t_near) / delta is exactly 30, a tie
    # that FP32 and FP64 may resolve differently (one sample more or less).  Their colours are checked
    # with the one-sample bound; their gradients are left out (g = 0 on both sides).
    _, aux0 = oracle.render(sc.R, sc.idx, sc.rows, o.astype(float), d.astype(float), bg=BG)
    ties = tie_flags(aux0, delta_of(16, 0.5))
    assert ties.sum() >= 3
    gw[ties] = 0.0
    rgb, T, grad, ref, aux, gref, rows = _both(sc, o, d, gw, opts)
    check_colours(rgb, ref, aux, rows, delta_of(16, 0.5), BG)
    check_grads(grad, gref)
    assert np.any(gref != 0)
    assert np.all(rgb[0] == np.float32(BG))
    # an all-empty grid: background, no gradient
    ge = Grid.from_host(16, np.full(16 ** 3, -1, np.int32), np.zeros((0, 28), np.float32))
    o2, d2 = synth.random_rays(100, seed=3)
    ot, dt = torch.from_numpy(o2).cuda(), torch.from_numpy(d2).cuda()
    st = ge.new_march_state(100, opts)
    rgb2 = ge.render_train(ot, dt, opts, st).cpu().numpy()
    assert np.all(rgb2 == np.float32(BG)[None, :])


def test_train_march_rejects_a_foreign_state(cuda_lib):
    from paper_2112_05131_gb300._lib import PlxError
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    opts = RenderOpts(0.5, BG, 0.0)
    sc = _sparse_scene(24, 0.3, 10)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    o, d = synth.random_rays(500, seed=12)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    st = g.new_march_state(500, opts)
    g.render_train(ot, dt, opts, st)
    # other ray buffers than the forward's: the device check refuses, adds nothing, flags the grid
    ot2, dt2 = ot.clone(), dt.clone()
    grad = g.render_backward_train(ot2, dt2, torch.ones((500, 3), device="cuda"), opts, st)
    torch.cuda.synchronize()
    assert torch.count_nonzero(grad) == 0
    with pytest.raises(PlxError, match="PLX_EDEVICE"):
        g.check()
    g.check()  # the status word was cleared by the previous check
    # other options than the forward's: refused the same way
    grad = g.render_backward_train(ot, dt, torch.ones((500, 3), device="cuda"), RenderOpts(0.7, BG, 0.0), st)
    assert torch.count_nonzero(grad) == 0
    with pytest.raises(PlxError, match="PLX_EDEVICE"):
        g.check()
    # a state buffer that is too small is refused on the host, before any launch
    with pytest.raises(PlxError, match="PLX_EINVAL"):
        g.render_train(ot, dt, opts, st[: st.numel() // 2])
    # a matching state still works afterwards
    grad = g.render_backward_train(ot, dt, torch.ones((500, 3), device="cuda"), opts, st)
    g.check()
    assert torch.count_nonzero(grad) > 0


def test_plan_then_planned_equals_render_train(cuda_lib):
    from paper_2112_05131_gb300._lib import PlxError
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    opts = RenderOpts(0.5, BG, 0.0)
    sc = _sparse_scene(40, 0.2, 23)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    o, d = synth.random_rays(3000, seed=24)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    st = g.new_march_state(3000, opts)
    a = g.render_train(ot, dt, opts, st).cpu().numpy()
    g.march_plan(ot, dt, opts, st)
    b = g.render_planned(ot, dt, opts, st).cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    # a planned march of other rays than the plan's: nothing written, the grid flagged
    o2, d2 = ot.clone(), dt.clone()
    rgb = torch.full((3000, 3), -5.0, device="cuda")
    g.render_planned(o2, d2, opts, st, rgb)
    torch.cuda.synchronize()
    assert torch.all(rgb == -5.0)
    with pytest.raises(PlxError, match="PLX_EDEVICE"):
        g.check()


@pytest.mark.parametrize("form", [0, 1])
def test_overlapped_trainer_matches_serial(cuda_lib, form):
    """Three streams and a deferred update compute what the serial order computes: the first step's
    accumulated gradient (adjoint + TV) agrees with the serial calls' up to the order in which atomics
    add it; the deferred update is exactly RMSProp's first step on that gradient; and over further
    steps the losses of an overlapped and a serial run agree.  (Rows of the two runs are not compared
    entry by entry: where |g| is near eps / sqrt(1 - beta) the update depends on g's last bits.)"""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts, gen_rays, mse_grad
    from paper_2112_05131_gb300.train import StepConfig, Trainer, lr_sh, lr_sigma

    gt = synth.scene_config("dense32")
    sc = synth.perturb(gt, 0.05, seed=3)
    cams = torch.from_numpy(synth.cameras_config("sphere8_64")).cuda()
    opts = RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0)
    g_gt = Grid.from_host(gt.R, gt.idx, gt.rows)
    batches = []
    for s in range(4):
        pix = torch.from_numpy(synth.pixel_batch(8, 64, 64, 2048, seed=40 + s)).cuda()
        o, d = gen_rays(cams, pix, 64, 64)
        ss, sl = synth.tv_segments(gt.R, 0.3, 256, seed=50 + s)
        batches.append((pix, g_gt.render(o, d, opts), torch.from_numpy(ss).cuda(), torch.from_numpy(sl).cuda(),
                        int(sl.sum())))
    cfg = dict(batch=2048, opts=opts, lambda_tv_sigma=1e-3, lambda_tv_sh=1e-3)
    # the serial calls of step 0, by hand: the gradient before the update
    gs = Grid.from_host(sc.R, sc.idx, sc.rows, sh_form=form)
    b = batches[0]
    o, d = gen_rays(cams, b[0], 64, 64)
    st = gs.new_march_state(2048, opts)
    gs.march_plan(o, d, opts, st)
    rgb = gs.render_planned(o, d, opts, st)
    grad_ref = gs.render_backward_train(o, d, mse_grad(rgb, b[1]), opts, st)
    gs.tv_grad(b[2], b[3], b[4], 1e-3, 1e-3, grad_ref)
    grad_ref = grad_ref[:, :28].cpu().numpy()
    # overlapped trainer, step 0: its gradient is complete when the step returns (the update waits)
    ga = Grid.from_host(sc.R, sc.idx, sc.rows, sh_form=form)
    ta = Trainer(ga, cams, 64, 64, StepConfig(overlap=True, **cfg))
    ta.step(*b, lr_sigma(1000), lr_sh(1000))
    torch.cuda.synchronize()
    grad_a = ta.grad[:, :28].cpu().numpy()
    gmax = np.abs(grad_ref).max()
    assert np.allclose(grad_a, grad_ref, rtol=1e-5, atol=1e-7 * gmax)
    # the deferred update is RMSProp's first step on exactly that gradient
    ta.finish()
    torch.cuda.synchronize()
    xa = ga.rows[:, :28].cpu().numpy().astype(np.float64)
    g64 = grad_a.astype(np.float64)
    lr = np.array([lr_sigma(1000)] + [lr_sh(1000)] * 27)[None, :].astype(np.float32).astype(np.float64)
    step = np.where(g64 != 0, lr * g64 / (np.sqrt(0.05 * g64 * g64) + 1e-8), 0.0)
    x_expect = sc.rows.astype(np.float64) - step
    assert np.all(np.abs(xa - x_expect) <= 4 * np.finfo(np.float32).eps * (np.abs(x_expect) + np.abs(step)) + 1e-30)
    assert torch.count_nonzero(ta.grad) == 0
    # the serial trainer, for the losses of further steps
    gb = Grid.from_host(sc.R, sc.idx, sc.rows, sh_form=form)
    tb = Trainer(gb, cams, 64, 64, StepConfig(overlap=False, **cfg))
    tb.step(*b, lr_sigma(1000), lr_sh(1000))
    # further steps: the losses of the two runs agree
    # (the overlapped run plans each next batch during the step before it, except that the batch it is
    # told comes after the second step is not the one the third step gets: then it plans again)
    losses = {}
    nxt = [batches[2][0], batches[1][0], None]
    for t, key in ((ta, "a"), (tb, "b")):
        out = []
        for s, bb in enumerate(batches[1:]):
            t.loss.zero_()
            t.step(*bb, lr_sigma(1001 + s), lr_sh(1001 + s), next_pix=nxt[s] if t is ta else None)
            out.append(t.loss.item())
        t.finish()
        losses[key] = out
    torch.cuda.synchronize()
    ga.check()
    gb.check()
    assert np.allclose(losses["a"], losses["b"], rtol=1e-3), losses


def test_planned_mse_matches_oracle(cuda_lib):
    """plx_render_planned_mse: the colours, dL/dC = 2 (C - target) / n and L of the batch against the
    oracle's render and MSE."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    opts = RenderOpts(0.5, BG, 0.0)
    sc = _sparse_scene(40, 0.2, 25)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    n = 1500
    o, d = synth.random_rays(n, seed=26)
    tgt = np.random.default_rng(27).uniform(0, 1, size=(n, 3)).astype(np.float32)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    st = g.new_march_state(n, opts)
    rgb = torch.empty((n, 3), device="cuda")
    grad = torch.empty((n, 3), device="cuda")
    loss = torch.zeros(1, device="cuda")
    g.march_plan(ot, dt, opts, st)
    g.render_planned_mse(ot, dt, opts, st, torch.from_numpy(tgt).cuda(), rgb, grad, loss)
    g.check()
    ref, aux = oracle.render(sc.R, sc.idx, sc.rows, o.astype(float), d.astype(float), bg=BG)
    check_colours(rgb.cpu().numpy(), ref, aux, sc.rows, delta_of(40, 0.5), BG)
    L_ref, g_ref = oracle.mse(rgb.cpu().numpy().astype(np.float64), tgt.astype(np.float64))
    assert np.allclose(grad.cpu().numpy(), g_ref, rtol=1e-6, atol=1e-12)
    assert loss.item() == pytest.approx(L_ref, rel=1e-5)
    # the same state then drives the adjoint
    gr = g.render_backward_train(ot, dt, grad, opts, st)
    gref = oracle.render_backward(sc.R, sc.idx, sc.rows, o.astype(float), d.astype(float),
                                  grad.cpu().numpy().astype(np.float64), bg=BG)
    check_grads(gr.cpu().numpy(), gref)


@pytest.mark.parametrize("stop,lam_s", [(1e-3, 0.0), (0.0, 1e-4)])
def test_native_step_matches_serial_calls(cuda_lib, stop, lam_s):
    """plx_trainer_step with early termination (the recomputing march) and with the Cauchy prior: its
    first step's gradient and both losses equal the serial Trainer's (the same library calls in order),
    up to the order of atomic additions."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts, gen_rays
    from paper_2112_05131_gb300.train import StepConfig, Trainer

    gt = synth.scene_config("dense32")
    sc = synth.perturb(gt, 0.05, seed=3)
    cams = torch.from_numpy(synth.cameras_config("sphere8_64")).cuda()
    opts = RenderOpts(0.5, (1.0, 1.0, 1.0), stop)
    g_gt = Grid.from_host(gt.R, gt.idx, gt.rows)
    pix = torch.from_numpy(synth.pixel_batch(8, 64, 64, 1500, seed=61)).cuda()
    o, d = gen_rays(cams, pix, 64, 64)
    target = g_gt.render(o, d, opts)
    ss, sl = synth.tv_segments(gt.R, 0.2, 256, seed=62)
    ss_t, sl_t = torch.from_numpy(ss).cuda(), torch.from_numpy(sl).cuda()
    out = {}
    for overlap in (True, False):
        g = Grid.from_host(sc.R, sc.idx, sc.rows)
        tr = Trainer(g, cams, 64, 64, StepConfig(batch=1500, opts=opts, overlap=overlap, lambda_sparsity=lam_s,
                                                 lambda_tv_sigma=1e-3, lambda_tv_sh=1e-3))
        tr.step(pix, target, ss_t, sl_t, int(sl.sum()), 0.0, 0.0)  # zero rates: the update leaves rows as they are
        torch.cuda.synchronize()
        grad = tr.grad[:, :28].cpu().numpy().copy() if overlap else None
        if not overlap:  # the serial step has already applied (and cleared) it: recompute by the calls
            g2 = Grid.from_host(sc.R, sc.idx, sc.rows)
            st = g2.new_march_state(1500, opts)
            o2, d2 = gen_rays(cams, pix, 64, 64)
            g2.march_plan(o2, d2, opts, st)
            rgb = g2.render_planned(o2, d2, opts, st)
            from paper_2112_05131_gb300.grid import mse_grad
            gr = g2.render_backward_train(o2, d2, mse_grad(rgb, target), opts, st, lambda_sparsity=lam_s)
            g2.tv_grad(ss_t, sl_t, int(sl.sum()), 1e-3, 1e-3, gr)
            grad = gr[:, :28].cpu().numpy()
        tr.finish()
        torch.cuda.synchronize()
        g.check()
        out[overlap] = (grad, tr.loss.item(), tr.loss_sparsity.item())
    ga, gb = out[True][0], out[False][0]
    gmax = np.abs(gb).max()
    assert gmax > 0 and np.allclose(ga, gb, rtol=1e-5, atol=1e-6 * gmax)
    assert out[True][1] == pytest.approx(out[False][1], rel=1e-5)
    assert out[True][2] == pytest.approx(out[False][2], rel=1e-5, abs=1e-30)
    if lam_s > 0:
        assert out[True][2] > 0
