"""Prune and upsample parity: index maps bit-exact, rows exact (prune) or within FP32 rounding (upsample)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _scene(R, frac, seed, dense=False):
    rng = np.random.default_rng(seed)
    occ = np.ones(R ** 3, bool) if dense else rng.uniform(size=R ** 3) < frac
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    M = int(occ.sum())
    rows = rng.normal(0, 1.0, size=(M, 28)).astype(np.float32)
    rows[:, 0] = rng.uniform(0, 10, size=M).astype(np.float32)
    return synth.Scene(R, idx, rows)


@pytest.mark.parametrize("R,frac,dense", [(17, 0.3, False), (37, 0.05, False), (32, 1.0, True), (2, 1.0, True)])
@pytest.mark.parametrize("dilate", [True, False])
def test_prune_bit_exact(cuda_lib, R, frac, dense, dilate):
    from paper_2112_05131_gb300.grid import Grid

    sc = _scene(R, frac, R, dense)
    tau = np.float32(7.5)
    sc.rows[: max(1, sc.M // 50), 0] = tau  # ties: sigma == tau is hot
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    gp = g.prune(float(tau), dilate)
    g.check()
    idx_ref, rows_ref = oracle.prune(sc.R, sc.idx, sc.rows, float(tau), dilate)
    assert np.array_equal(gp.idx.cpu().numpy(), idx_ref)
    got = gp.rows.cpu().numpy()
    assert got.shape[0] == rows_ref.shape[0]
    assert np.array_equal(got[:, :28], rows_ref.astype(np.float32))
    assert np.all(got[:, 28:] == 0)


def test_prune_everything_and_nothing(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid

    sc = _scene(12, 0.5, 3)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    none = g.prune(1e9)
    assert none.M == 0 and torch.all(none.idx == -1)
    allk = g.prune(-1e9)
    assert allk.M == sc.M
    assert np.array_equal(allk.idx.cpu().numpy(), sc.idx)


@pytest.mark.parametrize("R,R2,frac", [(9, 17, 1.0), (12, 24, 0.3), (16, 21, 0.1), (20, 13, 0.4)])
def test_upsample_parity(cuda_lib, R, R2, frac):
    from paper_2112_05131_gb300.grid import Grid

    sc = _scene(R, frac, 10 * R + R2, dense=frac >= 1.0)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    gu = g.upsample(R2)
    g.check()
    idx_ref, rows_ref = oracle.upsample(sc.R, sc.idx, sc.rows, R2)
    assert np.array_equal(gu.idx.cpu().numpy(), idx_ref)
    got = gu.rows.cpu().numpy()[:, :28].astype(np.float64)
    scale = np.max(np.abs(sc.rows), axis=0)[None, :]
    # FP32 weights and sums: error bounded by a few ulp of the largest input of the column
    assert np.all(np.abs(got - rows_ref) <= 4e-7 * (np.abs(rows_ref) + scale))


@pytest.mark.parametrize("R", [128, 256])
def test_prune_upsample_coarse_to_fine_sizes(cuda_lib, R):
    """The coarse-to-fine workload's grid operations at its own sizes (128^3 -> 256^3 -> 512^3): a sparse scene
    of the workload's generator, pruned at density 5 with dilation (bit-exact), then upsampled to 2R (map
    bit-exact, values within the FP32 bound above); the 512^3 output has about 10 M rows.  Values are
    compared in slices to bound host memory."""
    from paper_2112_05131_gb300.grid import Grid

    sc = synth.scene_config(f"sparse{R}_0.08", seed=3)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    gp = g.prune(5.0, True)
    idx_p, rows_p = oracle.prune(sc.R, sc.idx, sc.rows, 5.0, True)
    assert np.array_equal(gp.idx.cpu().numpy(), idx_p)
    assert np.array_equal(gp.rows.cpu().numpy()[:, :28], rows_p.astype(np.float32))
    del g
    R2 = 2 * R
    gu = gp.upsample(R2)
    gp.check()
    idx_ref, rows_ref = oracle.upsample(R, idx_p, rows_p, R2)
    assert np.array_equal(gu.idx.cpu().numpy(), idx_ref)
    assert gu.M == rows_ref.shape[0]
    scale = np.max(np.abs(rows_p), axis=0)[None, :]
    worst = 0.0
    for a in range(0, gu.M, 1 << 20):
        b = min(gu.M, a + (1 << 20))
        got = gu.rows[a:b, :28].cpu().numpy().astype(np.float64)
        ref = rows_ref[a:b]
        ratio = np.abs(got - ref) / (4e-7 * (np.abs(ref) + scale))
        worst = max(worst, float(ratio.max()))
    assert worst <= 1.0, worst
    print(f"prune + upsample {R}^3 -> {R2}^3: {gp.M} -> {gu.M} rows, value err/tol {worst:.3f}")
