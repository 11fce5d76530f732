"""TV, RMSProp, BF16 packing and MSE parity vs the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import check_grads

pytestmark = pytest.mark.gpu


def _scene(R, frac, seed):
    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=R ** 3) < frac
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    M = int(occ.sum())
    rows = rng.normal(0, 1.0, size=(M, 28)).astype(np.float32)
    rows[:, 0] = rng.uniform(-5, 20, size=M)
    return synth.Scene(R, idx, rows)


@pytest.mark.parametrize("R,frac,seg_len", [(20, 0.3, 97), (33, 0.08, 512), (16, 1.0, 16 ** 3)])
def test_tv_parity(cuda_lib, R, frac, seg_len):
    from paper_2112_05131_gb300.grid import Grid

    sc = _scene(R, frac, R)
    starts, lens = synth.tv_segments(R, 0.4, seg_len, seed=R + 5)
    if R == 20:  # a ragged last segment that ends at the last node
        starts = np.append(starts[starts + seg_len < R ** 3 - 50], R ** 3 - 50)
        lens = np.append(lens[:starts.shape[0] - 1], 50)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    grad = torch.zeros((sc.M, 32), device="cuda")
    loss = torch.zeros(1, device="cuda")
    n_sel = int(lens.sum())
    g.tv_grad(torch.from_numpy(starts).cuda(), torch.from_numpy(lens).cuda(), n_sel, 1e-2, 3e-3, grad, loss)
    g.check()
    L_ref, g_ref = oracle.tv(sc.R, sc.idx, sc.rows, starts, lens, 1e-2, 3e-3)
    check_grads(grad.cpu().numpy(), g_ref)
    assert abs(loss.item() - L_ref) <= 1e-5 * abs(L_ref) + 1e-12


def _random_segments(R, n_seg, max_len, seed):
    """Non-overlapping runs at random (unaligned) starts with random lengths, sorted."""
    rng = np.random.default_rng(seed)
    N = R ** 3
    cuts = np.sort(rng.choice(np.arange(1, N), size=min(2 * n_seg, N - 1), replace=False))
    starts, lens = [], []
    for a, b in zip(cuts[0::2], cuts[1::2]):
        ln = int(min(b - a, rng.integers(1, max_len + 1)))
        starts.append(int(a))
        lens.append(ln)
    return np.array(starts, np.int64), np.array(lens, np.int64)


@pytest.mark.parametrize("R,frac,n_seg,max_len", [(2, 0.5, 2, 8), (3, 0.3, 3, 9), (9, 0.1, 6, 200),
                                                  (40, 0.02, 12, 1500), (40, 0.4, 12, 1500)])
def test_tv_parity_unaligned_segments(cuda_lib, R, frac, n_seg, max_len):
    """TV on runs that start and end anywhere (across regions, far faces and the last node), on
    sparse scenes whose empty cells the kernel skips by the occupancy mask and on dense ones."""
    from paper_2112_05131_gb300.grid import Grid

    sc = _scene(R, frac, 100 + R)
    starts, lens = _random_segments(R, n_seg, max_len, seed=R)
    starts = np.append(starts, R ** 3 - 1)  # the last node alone: every neighbour outside
    lens = np.append(lens, 1)
    keep = np.ones(starts.shape[0], bool)
    keep[:-1] = starts[:-1] + lens[:-1] <= R ** 3 - 1
    starts, lens = starts[keep], lens[keep]
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    grad = torch.zeros((sc.M, 32), device="cuda")
    loss = torch.zeros(1, device="cuda")
    g.tv_grad(torch.from_numpy(starts).cuda(), torch.from_numpy(lens).cuda(), int(lens.sum()), 1e-2, 3e-3, grad,
              loss)
    g.check()
    L_ref, g_ref = oracle.tv(sc.R, sc.idx, sc.rows, starts, lens, 1e-2, 3e-3)
    check_grads(grad.cpu().numpy(), g_ref)
    assert abs(loss.item() - L_ref) <= 1e-5 * abs(L_ref) + 1e-12
    assert np.array_equal((grad.cpu().numpy()[:, :28] != 0).any(1), (g_ref != 0).any(1))


def test_rmsprop_parity_dense(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid

    sc = _scene(24, 0.25, 40)
    M = sc.M
    rng = np.random.default_rng(41)
    g_np = rng.normal(0, 1e-2, size=(M, 28)).astype(np.float32)
    g_np[rng.uniform(size=(M, 28)) < 0.3] = 0.0        # zero entries are skipped
    g_np[rng.uniform(size=M) < 0.5] = 0.0              # whole rows without gradient
    v_np = rng.uniform(0, 1e-4, size=(M, 28)).astype(np.float32)
    lr_s, lr_h, beta, eps = 30.0, 1e-2, 0.95, 1e-8
    x_ref, v_ref, gz = oracle.rmsprop(sc.rows, v_np, g_np, lr_s, lr_h, beta, eps)
    assert np.all(gz == 0)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    grad = torch.zeros((M, 32), device="cuda")
    grad[:, :28] = torch.from_numpy(g_np).cuda()
    v = torch.zeros((M, 32), device="cuda")
    v[:, :28] = torch.from_numpy(v_np).cuda()
    g.rmsprop_step(grad, v, lr_s, lr_h, beta, eps, sparse=False)
    torch.cuda.synchronize()
    x = g.rows[:, :28].cpu().numpy()
    # FP32 update: a few ulp of x plus a few ulp of the step lr * g / sqrt(v)
    lr = np.array([lr_s] + [lr_h] * 27)[None, :]
    assert np.all(np.abs(x - x_ref) <= 4e-7 * np.abs(x_ref) + 4e-6 * lr)
    assert np.allclose(v[:, :28].cpu().numpy(), v_ref, rtol=2e-6, atol=0)
    assert torch.all(grad == 0)
    untouched = np.all(g_np == 0, axis=1)
    assert np.array_equal(x[untouched], sc.rows[untouched])
    assert np.array_equal(v[:, :28].cpu().numpy()[g_np == 0], v_np[g_np == 0])


def test_sparse_rmsprop_equals_dense_after_backward_and_tv(cuda_lib):
    """Rows marked by render_backward and tv_grad are exactly the rows with non-zero gradient:
    the sparse step on the marked rows equals the dense sweep on the same gradient."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _scene(32, 0.15, 50)
    o, d = synth.random_rays(600, seed=51)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    gw = torch.from_numpy(np.random.default_rng(52).normal(size=(600, 3)).astype(np.float32)).cuda()
    starts, lens = synth.tv_segments(32, 0.05, 128, seed=53)
    g = Grid.from_host(sc.R, sc.idx, sc.rows)
    grad = torch.zeros((sc.M, 32), device="cuda")
    v = torch.full((sc.M, 32), 1e-6, device="cuda")
    g.render_backward(ot, dt, gw, RenderOpts(), grad)
    g.tv_grad(torch.from_numpy(starts).cuda(), torch.from_numpy(lens).cuda(), int(lens.sum()), 1e-3, 1e-3, grad)
    rows0, grad0, v0 = g.rows.clone(), grad.clone(), v.clone()
    assert torch.count_nonzero(grad0.abs().sum(1)) > 0
    g.rmsprop_step(grad, v, 30.0, 1e-2, sparse=True)   # consumes and clears the marks
    sparse = (g.rows.clone(), v.clone(), grad.clone())
    g.rows.copy_(rows0)
    grad.copy_(grad0)
    v.copy_(v0)
    g.rmsprop_step(grad, v, 30.0, 1e-2, sparse=False)
    torch.cuda.synchronize()
    assert torch.equal(sparse[0], g.rows)
    assert torch.equal(sparse[1], v)
    assert torch.all(sparse[2] == 0) and torch.all(grad == 0)
    # the marks are cleared: a second sparse step with a fresh gradient on unmarked rows does nothing
    grad.copy_(grad0)
    rows1 = g.rows.clone()
    g.rmsprop_step(grad, v, 30.0, 1e-2, sparse=True)
    torch.cuda.synchronize()
    assert torch.equal(rows1, g.rows)


def test_pack_bf16_bit_exact(cuda_lib):
    from paper_2112_05131_gb300.grid import Grid

    sc = _scene(12, 0.5, 60)
    sc.rows[:, 1:] *= np.float32(10.0) ** np.random.default_rng(61).uniform(-6, 6, size=(sc.M, 27)).astype(np.float32)
    g = Grid.from_host(sc.R, sc.idx, sc.rows, sh_form=1)
    torch.cuda.synchronize()
    h = g.rows_h.cpu().numpy().view(np.uint16)
    sig = h[:, 0:2].copy().view(np.float32)[:, 0]
    assert np.array_equal(sig, sc.rows[:, 0])
    sh = (h[:, 2:29].astype(np.uint32) << 16).view(np.float32)
    assert np.array_equal(sh, oracle.round_bf16(sc.rows[:, 1:]))
    assert np.all(h[:, 29:] == 0)


def _check_bf16_shadow(g):
    """The grid's BF16-SH rows are the bit-exact packing of its FP32 rows (density bits, SH rounded to
    nearest even, padding zero)."""
    x = g.rows[:, :28].cpu().numpy()
    h = g.rows_h.cpu().numpy().view(np.uint16)
    assert np.array_equal(h[:, 0:2].copy().view(np.float32)[:, 0].view(np.uint32), x[:, 0].view(np.uint32))
    sh = (h[:, 2:29].astype(np.uint32) << 16).view(np.float32)
    assert np.array_equal(sh, oracle.round_bf16(x[:, 1:]))
    assert np.all(h[:, 29:] == 0)


@pytest.mark.parametrize("sparse", [False, True])
def test_rmsprop_refreshes_bf16_shadow(cuda_lib, sparse):
    """After an update of a BF16-SH grid, every row's BF16 shadow equals the packing of its updated
    FP32 row: rows with a gradient in one quarter only, in several, and rows without any."""
    from paper_2112_05131_gb300.grid import Grid, RenderOpts

    sc = _scene(24, 0.25, 80)
    g = Grid.from_host(sc.R, sc.idx, sc.rows, sh_form=1)
    M = sc.M
    grad = torch.zeros((M, 32), device="cuda")
    v = torch.full((M, 32), 1e-6, device="cuda")
    if sparse:  # marked by the adjoint
        o, d = synth.random_rays(500, seed=81)
        gw = torch.from_numpy(np.random.default_rng(82).normal(size=(500, 3)).astype(np.float32)).cuda()
        g.render_backward(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), gw, RenderOpts(), grad)
    else:
        rng = np.random.default_rng(83)
        g_np = rng.normal(0, 1e-2, size=(M, 28)).astype(np.float32)
        kind = rng.integers(0, 4, size=M)
        g_np[kind == 0] = 0.0                      # no gradient
        g_np[kind == 1, 4:] = 0.0                  # the first quarter only (density and 3 SH)
        g_np[kind == 2, :24] = 0.0                 # the last quarter only
        grad[:, :28] = torch.from_numpy(g_np).cuda()
    assert torch.count_nonzero(grad.abs().sum(1)) > 0
    rows0 = g.rows.clone()
    g.rmsprop_step(grad, v, 30.0, 1e-2, sparse=sparse)
    torch.cuda.synchronize()
    assert not torch.equal(rows0, g.rows)
    _check_bf16_shadow(g)


def test_mse_grad(cuda_lib):
    from paper_2112_05131_gb300.grid import mse_grad

    rng = np.random.default_rng(70)
    p, t = rng.uniform(size=(1003, 3)).astype(np.float32), rng.uniform(size=(1003, 3)).astype(np.float32)
    loss = torch.zeros(1, device="cuda")
    g = mse_grad(torch.from_numpy(p).cuda(), torch.from_numpy(t).cuda(), loss=loss).cpu().numpy()
    L, gref = oracle.mse(p.astype(float), t.astype(float))
    assert np.allclose(g, gref, rtol=1e-6, atol=1e-12)
    assert abs(loss.item() - L) <= 1e-5 * L
