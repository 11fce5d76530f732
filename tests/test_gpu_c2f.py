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
