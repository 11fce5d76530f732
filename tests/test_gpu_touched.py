"""Gradient sparsity (Sec. 3.8: few voxels receive a gradient once optimisation is under way):
plx_count_touched counts the rows the adjoint and TV have added to since the last RMSProp step.
Against the oracle it equals, exactly, the number of rows with a non-zero gradient (random values:
every contribution is non-zero); the Trainer's per-step log is the same in serial and overlapped
mode (with zero learning rates, so that both see the same rows), and RMSProp clears the mask
between steps."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import delta_of, tie_flags

pytestmark = pytest.mark.gpu

BG = (1.0, 1.0, 1.0)


def _scene(R, frac, seed):
    """Densities bounded away from 0, so that no interpolated density sits near the ReLU kink: there
    FP32 and FP64 could disagree on its sign, and with it on whether a row receives anything."""
    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=R ** 3) < frac
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    M = int(occ.sum())
    rows = rng.normal(0, 0.4, size=(M, 28)).astype(np.float32)
    rows[:, 0] = rng.uniform(0.5, 25.0, size=M).astype(np.float32)
    return synth.Scene(R, idx, rows)


@pytest.mark.parametrize("with_tv", [False, True])
def test_count_touched_equals_oracle_gradient_support(cuda_lib, with_tv):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _scene(40, 0.15, 31)
    # rays from inside the box: a ray entering through a face has its first sample exactly on the face,
    # where the oracle's corner weights on the far side are exactly 0 and the GPU's may be ~1e-9 (so the
    # GPU would touch rows the oracle leaves at zero)
    o, d = synth.random_rays(1200, seed=32, radius=0.7)
    _, aux = oracle.render(sc.R, sc.idx, sc.rows, o.astype(float), d.astype(float), bg=BG)
    keep = ~tie_flags(aux, delta_of(sc.R, 0.5))
    o, d = o[keep], d[keep]
    gw = (np.random.default_rng(33).normal(size=(o.shape[0], 3)) * 1e-3).astype(np.float32)
    ref = oracle.render_backward(sc.R, sc.idx, sc.rows, o.astype(float), d.astype(float), gw.astype(float), bg=BG)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    grad = g.render_backward(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(gw).cuda(),
                             RenderOpts(0.5, BG, 0.0))
    if with_tv:
        ss, sl = synth.tv_segments(sc.R, 0.02, 256, seed=34)
        _, ref = oracle.tv(sc.R, sc.idx, sc.rows, ss, sl, 1e-5, 1e-3, grad_rows=ref)
        g.tv_grad(torch.from_numpy(ss).cuda(), torch.from_numpy(sl).cuda(), int(sl.sum()), 1e-5, 1e-3, grad)
    count = int(g.count_touched().item())
    g.check()
    expect = int((ref != 0).any(1).sum())
    assert count == expect, (count, expect)
    assert count == int((grad.cpu().numpy()[:, :28] != 0).any(1).sum())
    # RMSProp clears the mask
    v = torch.zeros_like(grad)
    g.rmsprop_step(grad, v, 0.0, 0.0)
    assert int(g.count_touched().item()) == 0
    print(f"touched rows {count} of {sc.M} ({'adjoint + TV' if with_tv else 'adjoint'})")


def test_trainer_touched_log_serial_equals_overlap(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts
    from paper_2112_05131_gb300.grid import gen_rays
    from paper_2112_05131_gb300.train import StepConfig, Trainer

    sc = synth.scene_config("dense32")
    cams = synth.cameras_config("sphere8_64")
    cams_t = torch.from_numpy(cams).cuda()
    opts = RenderOpts(0.5, BG, 0.0)
    gt = Grid.from_host(sc.R, sc.idx, sc.rows)
    batches = []
    for b in range(6):
        pix = torch.from_numpy(synth.pixel_batch(8, 64, 64, 2000, seed=40 + b)).cuda()
        o, d = gen_rays(cams_t, pix, 64, 64)
        ss, sl = synth.tv_segments(sc.R, 0.01, 256, seed=50 + b)
        batches.append((pix, gt.render(o, d, opts), torch.from_numpy(ss).cuda(), torch.from_numpy(sl).cuda(),
                        int(sl.sum())))
    logs = []
    pert = synth.perturb(sc, 0.05, seed=3)
    for overlap in (False, True):
        g = Grid.from_host(sc.R, pert.idx, pert.rows)
        tr = Trainer(g, cams_t, 64, 64, StepConfig(batch=2000, opts=opts, overlap=overlap, track_touched=True))
        for s, b in enumerate(batches):  # zero learning rates: rows stay put, so both modes see the same rows
            tr.step(*b, 0.0, 0.0)
        tr.finish()
        logs.append(tr.touched_counts())
        g.check()
    assert logs[0].shape == (6,) and np.all(logs[0] > 0) and np.all(logs[0] <= g.M)
    assert np.array_equal(logs[0], logs[1]), logs
    print(f"touched rows per step (of {g.M}): {logs[0].tolist()}")
