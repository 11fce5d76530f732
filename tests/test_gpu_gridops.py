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
