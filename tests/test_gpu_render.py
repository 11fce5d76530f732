"""Forward-render and ray-generation parity: CUDA library (through the C ABI) vs the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import bf16_grid_rows, check_colours, delta_of, tie_flags

pytestmark = pytest.mark.gpu


def _grid(cuda_lib, scene, form=0):
    from paper_2112_05131_gb300.grid import Grid

    return Grid.from_host(scene.R, scene.idx, scene.rows, sh_form=form)


def _render_both(scene, o, d, opts, form=0):
    from paper_2112_05131_gb300.grid import Grid

    g = Grid.from_host(scene.R, scene.idx, scene.rows, sh_form=form)
    ot = torch.from_numpy(o).cuda()
    dt = torch.from_numpy(d).cuda()
    T = torch.empty(o.shape[0], device="cuda")
    rgb = g.render(ot, dt, opts, T_end=T).cpu().numpy()
    g.check()
    rows = scene.rows if form == 0 else bf16_grid_rows(scene.rows)
    ref, aux = oracle.render(scene.R, scene.idx, rows, o.astype(np.float64), d.astype(np.float64),
                             step_vox=opts.step_vox, bg=opts.bg, stop_thresh=opts.stop_thresh)
    return rgb, T.cpu().numpy(), ref, aux, rows


def _sparse_scene(R, frac_occ, seed, sigma=(0.0, 30.0), sh_std=0.4, neg_frac=0.0):
    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=R ** 3) < frac_occ
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    M = int(occ.sum())
    rows = np.empty((M, 28), np.float32)
    rows[:, 0] = rng.uniform(*sigma, size=M)
    if neg_frac > 0:
        neg = rng.uniform(size=M) < neg_frac
        rows[neg, 0] = -rows[neg, 0]
    rows[:, 1:] = rng.normal(0, sh_std, size=(M, 27))
    return synth.Scene(R, idx, rows)


@pytest.mark.parametrize("stop", [0.0, 1e-3])
def test_render_dense32_parity(cuda_lib, stop):
    from paper_2112_05131_gb300.grid import RenderOpts

    sc = synth.scene_config("dense32")
    o, d = synth.random_rays(4096, seed=7)
    opts = RenderOpts(0.5, (1.0, 1.0, 1.0), stop)
    rgb, T, ref, aux, rows = _render_both(sc, o, d, opts)
    worst, nflag = check_colours(rgb, ref, aux, rows, delta_of(sc.R, 0.5), opts.bg, stop)
    assert np.allclose(T, aux[:, 0], rtol=1e-4, atol=1e-6 + stop)
    print(f"dense32 stop={stop}: worst err/tol {worst:.3f}, flagged {nflag}")


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("R,n", [(48, 1237), (67, 3001)])  # several tiles and a ragged tail of rays
def test_render_sparse_parity(cuda_lib, R, n, form):
    from paper_2112_05131_gb300.grid import RenderOpts

    sc = _sparse_scene(R, 0.15, 100 + R, neg_frac=0.2)
    o, d = synth.random_rays(n, seed=R, spread=0.9)
    opts = RenderOpts(0.5, (0.9, 0.6, 0.3), 0.0)
    rgb, T, ref, aux, rows = _render_both(sc, o, d, opts, form)
    worst, nflag = check_colours(rgb, ref, aux, rows, delta_of(R, 0.5), opts.bg)
    print(f"sparse R={R} form={form}: worst err/tol {worst:.3f}, flagged {nflag}")


def test_render_step_sizes_and_anisotropic_box(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _sparse_scene(20, 0.4, 5, sigma=(0.0, 8.0))
    aabb = ((-1.0, -0.5, -1.5), (1.0, 1.0, 0.5))
    g = Grid.from_host(sc.R, sc.idx, sc.rows, aabb=aabb)
    o, d = synth.random_rays(700, seed=11, spread=0.5)
    o = o + np.float32([0.0, 0.25, -0.5])
    for step in (0.3, 1.0, 1.7):
        opts = RenderOpts(step, (1.0, 1.0, 1.0), 0.0)
        rgb = g.render(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), opts).cpu().numpy()
        ref, aux = oracle.render(sc.R, sc.idx, sc.rows, o.astype(float), d.astype(float), step_vox=step,
                                 bg=opts.bg, aabb=(*aabb[0], *aabb[1]))
        h = min((aabb[1][a] - aabb[0][a]) / (sc.R - 1) for a in range(3))
        check_colours(rgb, ref, aux, sc.rows, step * h, opts.bg)


def test_render_degenerate_cases(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _sparse_scene(16, 0.3, 9)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    opts = RenderOpts(0.5, (0.2, 0.4, 0.6), 0.0)
    # zero rays
    empty = torch.empty((0, 3), device="cuda")
    assert g.render(empty, empty, opts).shape == (0, 3)
    # rays that miss, start inside, run parallel to faces, graze an edge
    o = np.float32([[3, 3, 3], [0.1, -0.2, 0.3], [-3, 0.5, 0.25], [-3, 1.0, 0.0], [0.0, 0.0, 5.0], [-3, -1, -1],
                    [0.0, 0.0, 0.0]])
    d = np.float32([[1, 0, 0], [0.6, 0.0, 0.8], [1, 0, 0], [1, 0, 0], [0, 0, -1], [1, 0, 0], [0, 1, 0]])
    rgb = g.render(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), opts).cpu().numpy()
    ref, aux = oracle.render(sc.R, sc.idx, sc.rows, o.astype(float), d.astype(float), step_vox=0.5, bg=opts.bg)
    check_colours(rgb, ref, aux, sc.rows, delta_of(sc.R, 0.5), opts.bg)
    assert np.all(rgb[0] == np.float32(opts.bg))  # miss -> exactly the background
    # an all-empty grid renders the background exactly
    idx = np.full(16 ** 3, -1, np.int32)
    ge = Grid.from_host(16, idx, np.zeros((0, 28), np.float32))
    o2, d2 = synth.random_rays(100, seed=3)
    rgb2 = ge.render(torch.from_numpy(o2).cuda(), torch.from_numpy(d2).cuda(), opts).cpu().numpy()
    assert np.all(rgb2 == np.float32(opts.bg)[None, :])


def test_render_is_bitwise_deterministic(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _sparse_scene(40, 0.2, 21)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    o, d = synth.random_rays(5000, seed=22)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    a = g.render(ot, dt, RenderOpts()).cpu().numpy()
    b = g.render(ot, dt, RenderOpts()).cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_gen_rays_parity(cuda_lib):
    from paper_2112_05131_gb300.grid import gen_rays

    cams = synth.cameras_config("sphere8_64")
    pix = synth.pixel_batch(8, 64, 64, 4099, seed=5)
    o, d = gen_rays(torch.from_numpy(cams).cuda(), torch.from_numpy(pix).cuda(), 64, 64)
    o, d = o.cpu().numpy(), d.cpu().numpy()
    oref, dref = oracle.gen_rays(cams.astype(np.float64), pix)
    assert np.array_equal(o, oref.astype(np.float32))  # the camera centre, copied
    # the kernel returns the FP32 rounding of the exact direction: equal to the oracle's FP64
    # direction rounded to FP32, except within ~1e-14 of a rounding midpoint (then 1 ulp apart)
    d32 = dref.astype(np.float32)
    diff = d.view(np.int32).astype(np.int64) - d32.view(np.int32).astype(np.int64)
    assert np.all(np.abs(diff) <= 1)
    assert np.count_nonzero(diff) <= 2, np.count_nonzero(diff)
    # out-of-range ids give zero rays
    bad = torch.tensor([-1, 8 * 64 * 64], dtype=torch.int64, device="cuda")
    ob, db = gen_rays(torch.from_numpy(cams).cuda(), bad, 64, 64)
    assert torch.all(db == 0) and torch.all(ob == 0)


def test_count_nodes_on_a_dense_grid(cuda_lib):
    """On a grid with every node occupied every cell is non-empty: all samples are marched, and every
    counted node is occupied."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = synth.scene_config("dense32")
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    o, d = synth.random_rays(500, seed=71)
    counts = g.count_nodes(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), RenderOpts()).cpu().numpy()
    _, aux = oracle.render(sc.R, sc.idx, sc.rows, o.astype(float), d.astype(float))
    ok = ~tie_flags(aux, delta_of(sc.R, 0.5))
    assert np.array_equal(counts[ok, 2], aux[ok, 1].astype(np.int64))
    assert np.array_equal(counts[:, 0], counts[:, 1])
    assert np.all((counts[:, 0] > 0) == (aux[:, 1] > 0))


@pytest.mark.parametrize("R,node", [(16, (0, 0, 0)), (16, (9, 4, 13)), (16, (15, 15, 15)), (16, (0, 15, 7)),
                                    (16, (8, 8, 8)), (16, (7, 8, 15)), (41, (24, 8, 32)), (41, (40, 16, 0)),
                                    (41, (17, 23, 39))])
def test_render_single_occupied_node(cuda_lib, R, node):
    """Only one node occupied: the march bounds each ray's candidates by the box of non-empty cells (the
    cells around that node) and screens groups of samples against the 8^3-cell block mask, so rays must
    still see the node from every direction and position, including nodes on block faces (coordinates
    multiple of 8, whose cells straddle two blocks) and at the far faces of the grid."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    idx = np.full(R ** 3, -1, np.int32)
    i, j, k = node
    idx[(i * R + j) * R + k] = 0
    rows = np.zeros((1, 28), np.float32)
    rows[0, 0] = 40.0
    rows[0, [1, 10, 19]] = [2.0, 1.0, 0.5]
    g = Grid.from_host(R, idx, rows)
    # rays aimed at the node from all around, plus random ones, plus one starting next to it
    h = 2.0 / (R - 1)
    p = -1.0 + h * np.array(node, np.float64)
    rng = np.random.default_rng(sum(node))
    dirs = rng.normal(size=(600, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    o = (p[None, :] - 2.5 * dirs + rng.normal(0, 0.3 * h, size=(600, 3))).astype(np.float32)
    d = dirs.astype(np.float32)
    o2, d2 = synth.random_rays(400, seed=5)
    o = np.concatenate([o, o2, (p + 0.2 * h)[None, :].astype(np.float32)])
    d = np.concatenate([d, d2, np.float32([[0.6, 0.0, 0.8]])])
    opts = RenderOpts(0.5, (0.3, 0.3, 0.3), 0.0)
    rgb = g.render(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), opts).cpu().numpy()
    g.check()
    ref, aux = oracle.render(R, idx, rows, o.astype(float), d.astype(float), bg=opts.bg)
    check_colours(rgb, ref, aux, rows, delta_of(R, 0.5), opts.bg)
    assert np.sum(np.abs(ref - np.float64(opts.bg)).max(1) > 1e-3) > 100  # many rays do see the node


def test_render_sheets_on_block_faces(cuda_lib):
    """Occupied node planes at i = 8, j = 16 and k = 24 of a 33^3 grid (cells on either side of a face of
    the 8^3-cell blocks) and a thin diagonal line of nodes: every ray through them is checked against the
    oracle, so a group of samples wrongly screened out would show as a missing sheet."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    R = 33
    rng = np.random.default_rng(71)
    occ = np.zeros((R, R, R), bool)
    occ[8, :, :] = True
    occ[:, 16, :] = True
    occ[:, :, 24] = True
    t = np.arange(R)
    occ[t, (t * 7) % R, R - 1 - t] = True
    occ = occ.reshape(-1) & (rng.uniform(size=R ** 3) < 0.7)
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    rows = rng.normal(0, 0.4, size=(int(occ.sum()), 28)).astype(np.float32)
    rows[:, 0] = rng.uniform(0.0, 20.0, size=rows.shape[0]).astype(np.float32)
    sc = synth.Scene(R, idx, rows)
    o, d = synth.random_rays(3000, seed=72, spread=0.9)
    opts = RenderOpts(0.5, (1.0, 1.0, 1.0), 0.0)
    rgb, _, ref, aux, rows_used = _render_both(sc, o, d, opts)
    check_colours(rgb, ref, aux, rows_used, delta_of(R, 0.5), opts.bg)
    assert np.sum(np.abs(ref - 1.0).max(1) > 1e-2) > 2000  # most rays cross a sheet
