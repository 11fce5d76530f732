"""One full optimisation step on the dense 32^3 workload, GPU vs oracle, each side generating its own rays:
pixel batch -> rays -> render -> MSE gradient -> adjoint -> TV (all voxels) -> RMSProp."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import check_colours, check_grads, delta_of

pytestmark = pytest.mark.gpu

LR_SIGMA, LR_SH, BETA, EPS = 30.0, 1e-2, 0.95, 1e-8
LAM_TV = 1e-5


def test_full_step_dense32(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts, gen_rays, mse_grad

    gt = synth.scene_config("dense32")
    sc = synth.perturb(gt, 0.05, seed=1)
    cams = synth.cameras_config("sphere8_64")
    pix = synth.pixel_batch(8, 64, 64, 4096, seed=2)
    opts = RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0)
    R = gt.R

    # ---- oracle side (FP64): its own rays, held at the FP32 precision of the library's ray
    # buffers (the render inputs are float [n][3]); targets = oracle render of the ground truth
    o64, d64 = oracle.gen_rays(cams.astype(np.float64), pix)
    o64 = o64.astype(np.float32).astype(np.float64)
    d64 = d64.astype(np.float32).astype(np.float64)
    target, _ = oracle.render(R, gt.idx, gt.rows, o64, d64, step_vox=0.5, bg=opts.bg)
    target = target.astype(np.float32).astype(np.float64)  # the library receives FP32 targets
    rgb_ref, aux = oracle.render(R, sc.idx, sc.rows, o64, d64, step_vox=0.5, bg=opts.bg)
    L_ref, grgb_ref = oracle.mse(rgb_ref, target)
    g_ref = oracle.render_backward(R, sc.idx, sc.rows, o64, d64, grgb_ref, step_vox=0.5, bg=opts.bg)
    _, g_ref = oracle.tv(R, sc.idx, sc.rows, [0], [R ** 3], LAM_TV, LAM_TV, grad_rows=g_ref)
    x_ref, v_ref, _ = oracle.rmsprop(sc.rows, np.zeros_like(g_ref), g_ref, LR_SIGMA, LR_SH, BETA, EPS)

    # ---- GPU side (FP32), every step a library call
    g = Grid.from_host(R, sc.idx, sc.rows)
    cams_t = torch.from_numpy(cams).cuda()
    o, d = gen_rays(cams_t, torch.from_numpy(pix).cuda(), 64, 64)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    rgb = g.render(o, d, opts)
    loss = torch.zeros(1, device="cuda")
    grgb = mse_grad(rgb, tgt, loss=loss)
    grad = torch.zeros((g.M, 32), device="cuda")
    g.render_backward(o, d, grgb, opts, grad)
    g.tv_grad(torch.tensor([0], device="cuda"), torch.tensor([R ** 3], device="cuda"), R ** 3, LAM_TV, LAM_TV, grad)
    grad_np = grad.cpu().numpy()
    v = torch.zeros((g.M, 32), device="cuda")
    g.rmsprop_step(grad, v, LR_SIGMA, LR_SH, BETA, EPS, sparse=True)
    g.check()

    # the GPU's rays are the FP32 roundings of the exact rays, as are the oracle's here
    assert np.array_equal(d.cpu().numpy(), d64.astype(np.float32))
    worst_c, nflag = check_colours(rgb.cpu().numpy(), rgb_ref, aux, sc.rows, delta_of(R, 0.5), opts.bg)
    assert abs(loss.item() - L_ref) <= 1e-4 * L_ref
    # The MSE stage turns the colour tolerance (|dC| <= 1e-5 max(|C|, 1e-3), checked above) into an
    # uncertainty of dL/dC of 2 |dC| / n per ray and channel; the oracle's absolute-value adjoint
    # carries it into an entrywise bound on the gradient, added to the gradient tolerance.
    dC = 1e-5 * np.maximum(np.abs(rgb_ref), 1e-3)
    carried = oracle.render_backward_abs(R, sc.idx, sc.rows, o64, d64, 2.0 * dC / rgb_ref.shape[0],
                                         step_vox=0.5, bg=opts.bg)
    worst_g = check_grads(grad_np, g_ref, extra_abs=carried)
    # RMSProp's first step (v = 0) moves an entry by u(g) = lr g / (sqrt((1 - beta) g^2) + eps), which is
    # monotone in g: over the gradient's tolerance interval [g_ref - tol, g_ref + tol] the update can move
    # by at most max |u(g_ref +- tol) - u(g_ref)|; FP32 rounding of x adds a few ulp.
    x = g.rows[:, :28].cpu().numpy().astype(np.float64)
    lr = np.array([LR_SIGMA] + [LR_SH] * 27)[None, :]
    gmax = np.max(np.abs(g_ref))
    tol_g = 1e-4 * np.maximum(np.abs(g_ref), 1e-3 * gmax) + carried

    def u(gg):
        return lr * gg / (np.sqrt((1 - BETA) * gg * gg) + EPS)

    du = np.maximum(np.abs(u(g_ref + tol_g) - u(g_ref)), np.abs(u(g_ref - tol_g) - u(g_ref)))
    bound = du + 4 * np.finfo(np.float32).eps * (np.abs(x_ref) + np.abs(u(g_ref)))
    err = np.abs(x - x_ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    step_bound = lr / np.sqrt(1 - BETA) * 1.0001
    assert np.all(np.abs(x - sc.rows) <= step_bound + 1e-6)
    unresolved = int(np.sum(np.abs(g_ref) <= tol_g))
    print(f"step: colour err/tol {worst_c:.3f} (flagged {nflag}), grad err/tol {worst_g:.3f}, "
          f"entries whose sign the tolerance leaves open {unresolved}")
