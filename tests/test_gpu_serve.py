"""Serving: plx_render_tiles (through the C ABI) against the FP64 oracle, and the continuous-batching
scheduler: every request's image is the same whether it is rendered alone or inside a mix of
requests of several scenes, and equal to plx_gen_rays + plx_render of its pixels."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from parity import bf16_grid_rows, check_colours, delta_of

pytestmark = pytest.mark.gpu

BG = (1.0, 1.0, 1.0)


def _scenes(form):
    from paper_2112_05131_gb300.grid import Grid

    out = []
    for R, occ, seed in ((40, 0.15, 1), (24, 0.3, 2), (33, 0.1, 3)):
        rng = np.random.default_rng(seed)
        o = rng.uniform(size=R ** 3) < occ
        idx = np.full(R ** 3, -1, np.int32)
        idx[o] = np.arange(int(o.sum()), dtype=np.int32)
        rows = np.empty((int(o.sum()), 28), np.float32)
        rows[:, 0] = rng.uniform(0, 30, size=rows.shape[0])
        rows[:, 1:] = rng.normal(0, 0.4, size=(rows.shape[0], 27))
        sc = synth.Scene(R, idx, rows)
        g = Grid.render_only_bf16(R, idx, rows) if form == 1 else Grid.from_host(R, idx, rows)
        out.append((sc, g))
    return out


def _requests():
    """Small requests with ragged sizes (tiles over the image edge) and both camera radii."""
    from paper_2112_05131_gb300.serve import Request

    cams = synth.cameras(6, 1, 1, 40.0, 2.6, upper=False, seed=4)
    reqs = []
    for i, (W, H) in enumerate([(37, 23), (64, 64), (16, 16), (50, 17), (1, 1), (29, 41)]):
        c = cams[i].copy()
        f = 0.5 * W / np.tan(np.radians(20.0))
        c[12:18] = [f, f, 0.5 * W, 0.5 * H, W, H]
        reqs.append(Request(i, i % 3, c, W, H, 0.0))
    return reqs


@pytest.mark.parametrize("form", [0, 1])
def test_tiles_parity_and_determinism(cuda_lib, form):
    from paper_2112_05131_gb300.grid import Grid, RenderOpts, gen_rays
    from paper_2112_05131_gb300.serve import TileServer

    scenes = _scenes(form)
    grids = [g for _, g in scenes]
    opts = RenderOpts(0.5, BG, 0.0)
    reqs = _requests()

    mixed = {d.rid: d.image for d in TileServer(grids, opts, max_rays_per_launch=4096, keep_images=True).run(reqs)}
    assert sorted(mixed) == [r.rid for r in reqs]
    for r in reqs:
        alone = TileServer(grids, opts, keep_images=True).run([r])[0].image
        assert np.array_equal(alone.view(np.uint32), mixed[r.rid].view(np.uint32)), f"request {r.rid}"
        sc, g = scenes[r.scene]
        pix = np.arange(r.W * r.H, dtype=np.int64)
        cams_t = torch.from_numpy(r.cam[None, :]).cuda()
        o, d = gen_rays(cams_t, torch.from_numpy(pix).cuda(), r.W, r.H)
        if form == 0:  # the same code on the same rays: the same bits as plx_render
            ref_gpu = g.render(o, d, opts).cpu().numpy().reshape(r.H, r.W, 3)
            assert np.array_equal(ref_gpu.view(np.uint32), mixed[r.rid].view(np.uint32))
        o64, d64 = oracle.gen_rays(r.cam[None, :].astype(np.float64), pix)
        rows = sc.rows if form == 0 else bf16_grid_rows(sc.rows)
        ref, aux = oracle.render(sc.R, sc.idx, rows, o64.astype(np.float32).astype(float),
                                 d64.astype(np.float32).astype(float), bg=BG)
        check_colours(mixed[r.rid].reshape(-1, 3), ref, aux, rows, delta_of(sc.R, 0.5), BG, what=f"req {r.rid}")


def test_tiles_bad_records_are_skipped_and_reported(cuda_lib):
    from paper_2112_05131_gb300._lib import PlxError
    from paper_2112_05131_gb300.grid import TILE_DTYPE, RenderOpts, render_tiles

    scenes = _scenes(0)
    grids = [g for _, g in scenes]
    img = torch.full((16, 16, 3), -1.0, device="cuda")
    rec = np.zeros(3, TILE_DTYPE)
    rec["W"], rec["H"], rec["d_rgb"] = 16, 16, img.data_ptr()
    rec["scene"] = [0, 7, 0]     # scene 7 does not exist
    rec["camera"] = [0, 0, 5]    # camera 5 does not exist
    cams = torch.from_numpy(synth.cameras(1, 16, 16, 40.0, 2.6, upper=False)).cuda()
    tiles = torch.from_numpy(rec.view(np.uint8)).cuda()
    render_tiles(grids, cams, tiles, 3, RenderOpts())
    torch.cuda.synchronize()
    assert torch.all(img != -1.0)  # the good tile rendered every pixel; the bad ones wrote nothing else
    with pytest.raises(PlxError, match="PLX_EDEVICE"):
        grids[0].check()
    # host-side validation: no grids, mixed forms
    with pytest.raises(PlxError, match="PLX_EINVAL"):
        render_tiles([], cams, tiles, 3, RenderOpts())


def test_server_poisson_trace(cuda_lib):
    from paper_2112_05131_gb300.grid import RenderOpts
    from paper_2112_05131_gb300.serve import TileServer, latency_stats, requests_from

    scenes = _scenes(1)
    grids = [g for _, g in scenes]
    reqs = requests_from(synth.serving_requests(40, 3, seed=9, rate=400.0))
    for r in reqs:  # keep the test small: shrink every request to at most 128x128
        r.W, r.H = min(r.W, 128), min(r.H, 128)
        r.cam = r.cam.copy()
        r.cam[14:18] = [0.5 * r.W, 0.5 * r.H, r.W, r.H]
    srv = TileServer(grids, RenderOpts(), max_rays_per_launch=1 << 14)
    done = srv.run(reqs)
    assert sorted(d.rid for d in done) == list(range(40))
    assert all(d.finished >= d.arrival for d in done)
    st = latency_stats(done, max(d.finished for d in done))
    assert st["p99_ms"] >= st["p50_ms"] > 0
    assert srv.launches >= 2


def test_server_admits_by_device_memory(cuda_lib):
    """A byte budget that holds only two of the requests' images: requests queue until memory frees up,
    the bytes held never exceed the budget, two requests do run at once, every request completes, and
    each image is the same as when it is rendered alone; a request larger than the whole budget is
    refused."""
    from paper_2112_05131_gb300.grid import RenderOpts
    from paper_2112_05131_gb300.serve import Request, TileServer, request_device_bytes

    scenes = _scenes(1)
    grids = [g for _, g in scenes]
    opts = RenderOpts(0.5, BG, 0.0)
    cams = synth.cameras(8, 1, 1, 40.0, 2.6, upper=False, seed=11)
    W = H = 192
    reqs = []
    for i in range(8):
        c = cams[i].copy()
        f = 0.5 * W / np.tan(np.radians(20.0))
        c[12:18] = [f, f, 0.5 * W, 0.5 * H, W, H]
        reqs.append(Request(i, i % 3, c, W, H, 0.0))
    one = request_device_bytes(W, H)
    budget = 2 * one + one // 2
    srv = TileServer(grids, opts, max_rays_per_launch=4096, keep_images=True, mem_budget=budget)
    done = srv.run(reqs)
    assert sorted(d.rid for d in done) == list(range(8))
    assert srv.mem_peak <= budget
    assert srv.mem_peak == 2 * one  # two requests were active together, never three
    assert srv.mem_in_use == 0
    waits = sorted(d.admission_wait for d in done)
    assert waits[-1] > 0.0  # later requests waited for memory
    for d in done:
        alone = TileServer(grids, opts, keep_images=True).run([reqs[d.rid]])[0].image
        assert np.array_equal(alone.view(np.uint32), d.image.view(np.uint32)), f"request {d.rid}"
    with pytest.raises(ValueError, match="budget"):
        TileServer(grids, opts, mem_budget=one - 1).submit(reqs[0])
