"""plx_trainer_step_host: the overlapped step fed from page-locked host memory (inputs uploaded by the
trainer, the next batch staged and planned during the step, the loss downloaded beside the adjoint)
computes what the device-fed plx_trainer_step computes on the same batches."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _batches(gt_grid, cams_t, n, k, R):
    from paper_2112_05131_gb300.grid import RenderOpts, gen_rays

    out = []
    for b in range(k):
        pix = torch.from_numpy(synth.pixel_batch(8, 64, 64, n, seed=70 + b))
        o, d = gen_rays(cams_t, pix.cuda(), 64, 64)
        tgt = gt_grid.render(o, d, RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0)).cpu()
        ss, sl = synth.tv_segments(R, 0.05, 256, seed=80 + b)
        out.append((pix, tgt, torch.from_numpy(ss), torch.from_numpy(sl), int(sl.sum())))
    return out


def test_host_fed_steps_equal_device_fed_steps(cuda_lib):
    """Zero learning rates keep the rows fixed, so every step of both trainers sees the same grid: the loss
    of each step and its gradient (adjoint and TV) agree up to the order of FP32 additions (the colours
    are the same bits; the loss is an FP32 sum of the rays' squared errors whose grouping depends on which
    warp finishes which ray: 1e-5 relative bounds it for 2000 rays).  Steps are staged by the previous call except step 2,
    whose inputs are uploaded at its own start."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts
    from paper_2112_05131_gb300.train import StepConfig, Trainer

    sc = synth.scene_config("dense32")
    pert = synth.perturb(sc, 0.05, seed=3)
    cams_t = torch.from_numpy(synth.cameras_config("sphere8_64")).cuda()
    opts = RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0)
    n, K = 2000, 5
    batches = _batches(Grid.from_host(sc.R, sc.idx, sc.rows), cams_t, n, K, sc.R)
    max_seg = max(b[2].shape[0] for b in batches)
    cfg = StepConfig(batch=n, opts=opts, lambda_tv_sigma=1e-5, lambda_tv_sh=1e-3, max_segments=max_seg)

    ga = Grid.from_host(sc.R, pert.idx, pert.rows)
    ta = Trainer(ga, cams_t, 64, 64, cfg)
    dev = [tuple(x.cuda() if torch.is_tensor(x) else x for x in b) for b in batches]
    gb = Grid.from_host(sc.R, pert.idx, pert.rows)
    tb = Trainer(gb, cams_t, 64, 64, cfg)
    hb = [Trainer.host_batch(b[0].pin_memory(), b[1].pin_memory(), b[2].pin_memory(), b[3].pin_memory(), b[4])
          for b in batches]
    loss_out = torch.zeros(1).pin_memory()
    worst = 0.0
    for s in range(K):
        ta.loss.zero_()
        ta.step(*dev[s], 0.0, 0.0, next_pix=dev[s + 1][0] if s + 1 < K else None)
        nxt = hb[s + 1] if s + 1 < K and s != 1 else None
        tb.step_host(hb[s], 0.0, 0.0, next_batch=nxt, loss_out=loss_out)
        torch.cuda.synchronize()
        assert abs(loss_out.item() - ta.loss.item()) <= 1e-5 * abs(ta.loss.item()), (s, loss_out.item(), ta.loss.item())
        g_a, g_b = ta.grad[:, :28].cpu().numpy(), tb.grad[:, :28].cpu().numpy()
        tol = 1e-4 * np.maximum(np.abs(g_a), 1e-3 * np.abs(g_a).max())  # the gradient tolerance of the parity tests
        w = float(np.max(np.abs(g_b - g_a) / tol))
        assert w <= 1.0, (s, w, int(np.sum(np.abs(g_b - g_a) > tol)))
        worst = max(worst, w)
    ta.finish()
    tb.finish()
    torch.cuda.synchronize()
    ga.check()
    gb.check()
    print(f"host-fed vs device-fed, {K} steps: gradient err/tol {worst:.3f}")


def test_host_fed_step_rejects_bad_batches(cuda_lib):
    from paper_2112_05131_gb300._lib import PlxError
    from paper_2112_05131_gb300.grid import Grid, RenderOpts
    from paper_2112_05131_gb300.train import StepConfig, Trainer

    sc = synth.scene_config("dense32")
    cams_t = torch.from_numpy(synth.cameras_config("sphere8_64")).cuda()
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    tr = Trainer(g, cams_t, 64, 64, StepConfig(batch=100, opts=RenderOpts(), max_segments=2))
    pix = torch.zeros(100, dtype=torch.int64).pin_memory()
    tgt = torch.zeros((100, 3)).pin_memory()
    ss = torch.tensor([0, 256, 512], dtype=torch.int64).pin_memory()
    sl = torch.tensor([64, 64, 64], dtype=torch.int64).pin_memory()
    with pytest.raises(PlxError, match="max_segments"):  # three segments, two allowed
        tr.step_host(Trainer.host_batch(pix, tgt, ss, sl, 192), 0.0, 0.0)
    big = torch.zeros(101, dtype=torch.int64).pin_memory()
    with pytest.raises(PlxError, match="n out of range"):
        tr.step_host(Trainer.host_batch(big, torch.zeros((101, 3)).pin_memory()), 0.0, 0.0)
