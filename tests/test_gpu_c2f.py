"""The coarse-to-fine loop (Sec. 3.4, Supp. B.1) at a small scale: a dense 16^3 start, prune + upsample
to 32^3 and 64^3, training images from the ground-truth grid (spot-checked against the oracle)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import check_colours, delta_of

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prune_by", ["density", "weight"])
def test_coarse_to_fine_small(cuda_lib, prune_by):
    from paper_2112_05131_gb300.coarse_to_fine import C2FConfig, dense_grid, psnr, render_views, train
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    opts = RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0)
    gt = synth.scene_config("sparse64_0.08")
    g_gt = Grid.from_host(64, gt.idx, gt.rows)
    W = H = 64
    cams = synth.cameras(24, W, H, 40.0, 4.0, upper=True)
    test_cams = synth.cameras(4, W, H, 40.0, 4.0, upper=True, seed=9, jitter=0.2)
    cams_t, test_t = torch.from_numpy(cams).cuda(), torch.from_numpy(test_cams).cuda()
    images = render_views(g_gt, cams_t, W, H, opts)
    truth = render_views(g_gt, test_t, W, H, opts)

    # the training images are the forward of the ground truth: spot-check 64 pixels against the oracle
    pix = np.random.default_rng(3).integers(0, images.shape[0] * W * H, size=64)
    o, d = oracle.gen_rays(cams.astype(np.float64), pix)
    ref, aux = oracle.render(64, gt.idx, gt.rows, o.astype(np.float32).astype(float),
                             d.astype(np.float32).astype(float))
    check_colours(images.reshape(-1, 3)[pix], ref, aux, gt.rows, delta_of(64, 0.5), opts.bg)

    cfg = C2FConfig(steps=900, start_reso=16, upsample_at=(300, 600), batch=2048, tv_segment=256, chunk=100,
                    lambda_tv_sigma=1e-5, lambda_tv_sh=1e-4, prune_by=prune_by)
    log = []
    g = train(images, cams_t, W, H, cfg, log)
    assert g.reso == 64
    assert [r["to"][0] for r in log if "to" in r] == [32, 64]
    start = render_views(dense_grid(16, 0.1), test_t, W, H, opts)
    final = render_views(g, test_t, W, H, opts)
    p0, p1 = psnr(start, truth), psnr(final, truth)
    print(f"coarse-to-fine 16->32->64 ({prune_by} prune): held-out PSNR {p0:.2f} dB -> {p1:.2f} dB; stages {log}")
    assert p1 > p0 + 3.0


def test_tv_only_in_first_stage(cuda_lib):
    """tv_until (Supp. B.2: the synthetic scenes keep TV in the first stage only): from that step on the
    loop adds no TV gradient.  With the learning rates scaled to 0 the grid keeps its values, so each
    step's touched rows depend only on its rays and TV segments: the loop's count of rows with a gradient
    equals, exactly, that of the same batches stepped with TV before tv_until and the adjoint alone
    after it, and TV would have added rows at every step after it."""
    from paper_2112_05131_gb300.coarse_to_fine import C2FConfig, _Batches, train
    from paper_2112_05131_gb300.grid import Grid, RenderOpts
    from paper_2112_05131_gb300.train import StepConfig, Trainer

    R, W, H = 24, 32, 32
    rng = np.random.default_rng(5)
    idx = np.arange(R ** 3, dtype=np.int32)
    rows = rng.normal(0, 0.4, size=(R ** 3, 28)).astype(np.float32)
    rows[:, 0] = rng.uniform(0.5, 20.0, size=R ** 3).astype(np.float32)
    cams = synth.cameras(8, W, H, 40.0, 2.6, upper=False, seed=6)
    cams_t = torch.from_numpy(cams).cuda()
    images = rng.uniform(size=(8, H, W, 3)).astype(np.float32)
    cfg = C2FConfig(steps=10, start_reso=R, upsample_at=(), batch=64, tv_segment=256, tv_fraction=0.1, chunk=10,
                    tv_until=5, lambda_tv_sigma=1e-5, lambda_tv_sh=1e-3, track_touched=True, touched_every=1,
                    lr_scale=0.0)
    log = []
    g = train(images, cams_t, W, H, cfg, log, start=Grid.from_host(R, idx, rows))
    assert np.array_equal(g.rows[:, :28].cpu().numpy(), rows)  # zero learning rates: values unchanged
    frac = log[-1]["touched_frac"]
    got = np.array([round(frac[s] * g.M) for s in range(cfg.steps)])

    def counts(tv_steps):
        ref = Grid.from_host(R, idx, rows)
        tr = Trainer(ref, cams_t, W, H, StepConfig(batch=cfg.batch, opts=RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0),
                                                  lambda_tv_sigma=cfg.lambda_tv_sigma, lambda_tv_sh=cfg.lambda_tv_sh,
                                                  overlap=False, track_touched=True))
        b = _Batches(images, cfg, cams_t.device)
        for s in range(cfg.steps):
            pix, tgt, ss, sl, nsel = b.get(s, R)
            if s in tv_steps:
                tr.step(pix, tgt, ss, sl, nsel, 0.0, 0.0)
            else:
                tr.step(pix, tgt, None, None, 0, 0.0, 0.0)
        tr.finish()
        return tr.touched_counts()

    expect = counts(set(range(cfg.tv_until)))
    with_tv = counts(set(range(cfg.steps)))
    assert np.array_equal(got, expect), (got, expect)
    assert np.all(with_tv[cfg.tv_until:] > got[cfg.tv_until:])
    assert np.array_equal(with_tv[: cfg.tv_until], got[: cfg.tv_until])
    print(f"touched rows per step (of {g.M}), TV until step {cfg.tv_until}: {got.tolist()}; with TV throughout "
          f"{with_tv.tolist()}")
