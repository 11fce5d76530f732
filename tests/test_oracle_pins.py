"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against a closed form, an invariant, a
library routine, brute force on a tiny grid, or central finite differences,
chosen so that a plausible slip (a dropped term, a wrong sign, a swapped axis,
a missing half-pixel offset) fails at least one of them.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
Y00 = 1.0 / (2.0 * math.sqrt(math.pi))
NV = 28


def dense(R, rows):
    return np.arange(R ** 3, dtype=np.int32), np.asarray(rows, np.float64)


def node_pos(R, aabb=(-1, -1, -1, 1, 1, 1)):
    lo = np.array(aabb[:3], np.float64)
    hi = np.array(aabb[3:], np.float64)
    h = (hi - lo) / (R - 1)
    ijk = np.stack(np.meshgrid(np.arange(R), np.arange(R), np.arange(R), indexing="ij"), -1).reshape(-1, 3)
    return lo + ijk * h, ijk


def box_segment(o, d, lo=(-1, -1, -1), hi=(1, 1, 1)):
    """Entry/exit of a ray and a box by intersecting the six face planes and
    keeping the hits that lie on the closed box (independent of the slab test)."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    ts = []
    for a in range(3):
        if d[a] == 0:
            continue
        for plane in (lo[a], hi[a]):
            t = (plane - o[a]) / d[a]
            q = o + t * d
            if np.all(q >= lo - 1e-12) and np.all(q <= hi + 1e-12):
                ts.append(t)
    if len(ts) < 2 or max(ts) <= max(min(ts), 0.0):
        return None
    return max(min(ts), 0.0), max(ts)


# ----------------------------------------------------------------------------- SH

def test_sh_y00_matches_paper_constant():
    Y = oracle.sh_basis([[0.3, -0.2, math.sqrt(1 - 0.13)]])[0]
    assert Y[0] == pytest.approx(Y00, abs=1e-16)
    assert Y[0] == pytest.approx(GOLDEN["sh_y00"]["value"], abs=5e-9)
    assert 3 * 9 == GOLDEN["sh_coeffs_per_voxel"]["value"]


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform in phi integrates products of
    # degree <= 4 spherical polynomials exactly.
    xg, wg = np.polynomial.legendre.leggauss(32)
    nphi = 64
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_basis(dirs)
    G = (Y * w[:, None]).T @ Y
    assert np.max(np.abs(G - np.eye(9))) < 1e-12


def test_sh_addition_theorem():
    # sum_m Y_lm(d)^2 = (2l+1)/(4 pi) for every unit d, independent of sign conventions
    rng = np.random.default_rng(3)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(d)
    assert np.allclose((Y[:, 1:4] ** 2).sum(1), 3 / (4 * math.pi), atol=1e-14)
    assert np.allclose((Y[:, 4:9] ** 2).sum(1), 5 / (4 * math.pi), atol=1e-14)


def test_sh_matches_scipy_complex_harmonics():
    """Real basis built from scipy's complex SH (Condon-Shortley phase included):
    m<0: sqrt2 Im Y_l^|m|, m=0: Y_l^0, m>0: sqrt2 Re Y_l^m, ordered m=-l..l."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(4)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])

    def Ylm(l, m):
        if hasattr(sp, "sph_harm_y"):
            return sp.sph_harm_y(l, m, theta, phi)
        return sp.sph_harm(m, l, phi, theta)

    cols = []
    for l in range(3):
        for m in range(-l, l + 1):
            if m < 0:
                cols.append(math.sqrt(2) * Ylm(l, -m).imag)
            elif m == 0:
                cols.append(Ylm(l, 0).real)
            else:
                cols.append(math.sqrt(2) * Ylm(l, m).real)
    ref = np.stack(cols, 1)
    assert np.max(np.abs(oracle.sh_basis(d) - ref)) < 1e-12


# ----------------------------------------------------------------------------- interpolation

def test_interp_reproduces_affine_fields_exactly():
    R = 7
    aabb = (-1.0, -0.5, -2.0, 1.0, 1.5, 0.5)  # anisotropic cell sizes
    rng = np.random.default_rng(0)
    A = rng.normal(size=(NV, 3))
    b = rng.normal(size=NV)
    pos, _ = node_pos(R, aabb)
    rows = pos @ A.T + b
    idx, rows = dense(R, rows)
    lo, hi = np.array(aabb[:3]), np.array(aabb[3:])
    pts = lo + rng.uniform(size=(500, 3)) * (hi - lo)
    pts[:8] = [[lo[0] if (c >> 2) & 1 else hi[0], lo[1] if (c >> 1) & 1 else hi[1], lo[2] if c & 1 else hi[2]]
               for c in range(8)]  # the 8 box corners (clamp + base = R-2 path)
    out = oracle.interp(R, idx, rows, pts, aabb)
    assert np.max(np.abs(out - (pts @ A.T + b))) < 1e-12
    # points outside the box are clamped to it
    outside = lo - 0.5 + rng.uniform(size=(100, 3)) * (hi - lo + 1.0)
    out2 = oracle.interp(R, idx, rows, outside, aabb)
    assert np.max(np.abs(out2 - (np.clip(outside, lo, hi) @ A.T + b))) < 1e-12


def hat_interp(R, idx, rows, p, aabb=(-1, -1, -1, 1, 1, 1)):
    """Brute force: sum over all nodes of prod_a max(0, 1-|g_a - i_a|) * value."""
    lo, hi = np.array(aabb[:3], float), np.array(aabb[3:], float)
    g = np.clip((p - lo) / ((hi - lo) / (R - 1)), 0, R - 1)
    out = np.zeros(NV)
    for i, j, k in itertools.product(range(R), repeat=3):
        w = max(0.0, 1 - abs(g[0] - i)) * max(0.0, 1 - abs(g[1] - j)) * max(0.0, 1 - abs(g[2] - k))
        n = (i * R + j) * R + k
        if w > 0 and idx[n] >= 0:
            out += w * rows[idx[n]]
    return out


def random_sparse(R, frac_empty, seed, sigma_range=(0.0, 8.0), sh_std=0.5):
    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=R ** 3) >= frac_empty
    idx = np.full(R ** 3, -1, np.int32)
    idx[occ] = np.arange(int(occ.sum()), dtype=np.int32)
    rows = np.empty((int(occ.sum()), NV))
    rows[:, 0] = rng.uniform(*sigma_range, size=rows.shape[0])
    rows[:, 1:] = rng.normal(0, sh_std, size=(rows.shape[0], NV - 1))
    return idx, rows


def test_interp_matches_hat_function_brute_force_with_nulls():
    R = 4
    idx, rows = random_sparse(R, 0.4, 1, sigma_range=(-2, 5))
    rng = np.random.default_rng(2)
    pts = rng.uniform(-1.1, 1.1, size=(200, 3))
    out = oracle.interp(R, idx, rows, pts)
    ref = np.stack([hat_interp(R, idx, rows, p) for p in pts])
    assert np.max(np.abs(out - ref)) < 1e-12


# ----------------------------------------------------------------------------- rays

def test_gen_rays_pixel_centres_project_back():
    rng = np.random.default_rng(5)
    W, H = 37, 23
    cams = np.zeros((3, 18))
    for v in range(3):
        eye = rng.normal(size=3)
        eye = 3.0 * eye / np.linalg.norm(eye)
        cams[v, :12] = synth.look_at(eye, target=rng.uniform(-0.2, 0.2, 3)).reshape(-1)
        cams[v, 12:18] = [31.0 + 5 * v, 29.0, 17.2, 11.9, W, H]
    pix = rng.integers(0, 3 * W * H, size=300)
    o, d = oracle.gen_rays(cams, pix)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    for r in range(pix.shape[0]):
        view, rem = divmod(int(pix[r]), W * H)
        v, u = divmod(rem, W)
        c2w = cams[view, :12].reshape(3, 4)
        Rm, t = c2w[:, :3], c2w[:, 3]
        assert np.allclose(o[r], t, atol=0)
        X = o[r] + 2.7 * d[r]
        Xc = Rm.T @ (X - t)  # world -> camera
        assert Xc[2] < 0  # in front of a camera looking down -z
        fx, fy, cx, cy = cams[view, 12:16]
        up = cx + fx * Xc[0] / (-Xc[2])
        vp = cy - fy * Xc[1] / (-Xc[2])  # image rows grow downwards, camera y is up
        assert up == pytest.approx(u + 0.5, abs=1e-9)
        assert vp == pytest.approx(v + 0.5, abs=1e-9)


def test_clip_known_segments():
    o = np.array([[-3.0, 0.2, -0.4], [-2.0, -2.0, -2.0], [0.1, 0.2, 0.3], [-3.0, 1.5, 0.0],
                  [3.0, 0.0, 0.0], [0.5, -0.5, 4.0]])
    d = np.array([[1.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.0, 0.6, 0.8], [1.0, 0.0, 0.0],
                  [1.0, 0.0, 0.0], [0.0, 0.0, -1.0]])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out = oracle.clip(o, d)
    s3 = math.sqrt(3.0)
    assert out[0] == pytest.approx([2.0, 4.0, 1.0], abs=1e-14)
    assert out[1] == pytest.approx([s3, 3 * s3, 1.0], abs=1e-14)  # corner to corner
    assert out[2, 0] == 0.0 and out[2, 2] == 1.0  # starts inside: t_near = 0
    assert out[2, 1] == pytest.approx(min((1 - 0.2) / 0.6, (1 - 0.3) / 0.8), abs=1e-14)
    assert out[3, 2] == 0.0  # parallel to a face, outside the slab
    assert out[4, 2] == 0.0  # pointing away
    assert out[5] == pytest.approx([3.0, 5.0, 1.0], abs=1e-14)
    # against the face-plane construction on random rays
    o2, d2 = synth.random_rays(200, seed=9)
    o2, d2 = o2.astype(float), d2.astype(float)
    out2 = oracle.clip(o2, d2)
    for r in range(200):
        seg = box_segment(o2[r], d2[r])
        if seg is None:
            assert out2[r, 2] == 0.0
        else:
            assert out2[r, 2] == 1.0
            assert out2[r, :2] == pytest.approx(seg, abs=1e-12)


# ----------------------------------------------------------------------------- forward render

def constant_field(R, sigma0, k0_rgb):
    rows = np.zeros((R ** 3, NV))
    rows[:, 0] = sigma0
    for ch in range(3):
        rows[:, 1 + 9 * ch] = k0_rgb[ch]
    return dense(R, rows)


@pytest.mark.parametrize("stop", [0.0, 0.05])
def test_render_constant_field_closed_form(stop):
    """sigma = sigma0 and colour c everywhere: the sum telescopes (Supp. C form) to
    C = c (1 - exp(-sigma0 N delta)) + bg exp(-sigma0 N delta), N = number of samples."""
    R = 16
    sigma0 = 3.7
    k0 = (2.0, 1.0, -1.0)  # the blue channel is negative: ReLU clips it to 0
    idx, rows = constant_field(R, sigma0, k0)
    step_vox = 0.37
    delta = step_vox * 2.0 / (R - 1)
    bg = np.array([0.9, 0.5, 0.25])
    o = np.array([[-3.0, 0.2, -0.4], [-2.0, -2.0, -2.0], [0.3, -3.0, 0.1], [2.2, 2.9, -1.7]])
    d = np.array([[1.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.1, 1.0, -0.05], [-0.5, -0.8, 0.45]])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rgb, aux = oracle.render(R, idx, rows, o, d, step_vox=step_vox, bg=bg, stop_thresh=stop)
    c = np.maximum(0.0, Y00 * np.array(k0))
    for r in range(o.shape[0]):
        t0, t1 = box_segment(o[r], d[r])
        ratio = (t1 - t0) / delta
        assert abs(ratio - round(ratio)) > 1e-6
        N = math.ceil(ratio)
        if stop > 0:
            n_stop = math.ceil(math.log(1.0 / stop) / (sigma0 * delta))  # first s with T_s < stop
            N = min(N, n_stop)
        T = math.exp(-sigma0 * N * delta)
        assert aux[r, 1] == N
        assert aux[r, 0] == pytest.approx(T, rel=1e-13)
        assert rgb[r] == pytest.approx(c * (1 - T) + bg * T, rel=1e-13, abs=1e-15)


def test_render_weights_sum_with_T_end_to_one():
    R = 8
    idx, rows = random_sparse(R, 0.3, 11, sigma_range=(0.0, 20.0))
    rows[:, 1:] = 0.0
    rows[:, 1] = rows[:, 10] = rows[:, 19] = 1.0 / Y00  # colour 1 wherever occupied
    # the colour is then the occupancy-weighted interpolation, not 1, at mixed cells;
    # make every node occupied for an exact unit colour
    idx = np.arange(R ** 3, dtype=np.int32)
    rows = np.repeat(rows[:1], R ** 3, axis=0)
    rng = np.random.default_rng(12)
    rows[:, 0] = rng.uniform(0, 20, size=R ** 3)
    o, d = synth.random_rays(64, seed=13)
    rgb, aux = oracle.render(R, idx, rows, o, d, bg=(0.0, 0.0, 0.0))
    assert np.allclose(rgb[:, 0] + aux[:, 0], 1.0, atol=1e-13)


def test_render_matches_telescoped_form():
    """C = sum_i (T_i - T_{i+1}) c_i + T_N bg with T_i = exp(-sum_{j<i} sigma_j delta) (Supp. C)."""
    R = 6
    idx, rows = random_sparse(R, 0.3, 21, sigma_range=(-1.0, 9.0))
    o, d = synth.random_rays(32, seed=22)
    o, d = o.astype(float), d.astype(float)
    step_vox = 0.5
    delta = step_vox * 2 / (R - 1)
    bg = np.array([1.0, 1.0, 1.0])
    rgb, aux = oracle.render(R, idx, rows, o, d, step_vox=step_vox, bg=bg)
    Y = oracle.sh_basis(d)
    cl = oracle.clip(o, d)
    for r in range(o.shape[0]):
        if cl[r, 2] == 0:
            assert np.all(rgb[r] == bg)
            continue
        N = int(aux[r, 1])
        ts = cl[r, 0] + np.arange(N) * delta
        assert np.all(ts < cl[r, 1]) and not cl[r, 0] + N * delta < cl[r, 1]
        v = oracle.interp(R, idx, rows, o[r] + ts[:, None] * d[r])
        sig = np.maximum(v[:, 0], 0)
        col = np.maximum(0, np.stack([v[:, 1 + 9 * ch:10 + 9 * ch] @ Y[r] for ch in range(3)], 1))
        T = np.exp(-np.concatenate([[0.0], np.cumsum(sig * delta)]))
        ref = ((T[:-1] - T[1:])[:, None] * col).sum(0) + T[-1] * bg
        assert rgb[r] == pytest.approx(ref, rel=1e-12, abs=1e-14)


def brute_render(R, idx, rows, o, d, step_vox, bg, stop=0.0):
    seg = box_segment(o, d)
    if seg is None:
        return np.array(bg, float)
    t0, t1 = seg
    delta = step_vox * 2.0 / (R - 1)
    x, y, z = d
    Y = [Y00, -math.sqrt(3 / (4 * math.pi)) * y, math.sqrt(3 / (4 * math.pi)) * z,
         -math.sqrt(3 / (4 * math.pi)) * x, 0.5 * math.sqrt(15 / math.pi) * x * y,
         -0.5 * math.sqrt(15 / math.pi) * y * z, 0.25 * math.sqrt(5 / math.pi) * (3 * z * z - 1),
         -0.5 * math.sqrt(15 / math.pi) * x * z, 0.25 * math.sqrt(15 / math.pi) * (x * x - y * y)]
    C = np.zeros(3)
    T = 1.0
    s = 0
    while t0 + s * delta < t1 and T >= stop:
        v = hat_interp(R, idx, rows, o + (t0 + s * delta) * d)
        sig = max(0.0, v[0])
        c = np.array([max(0.0, float(np.dot(Y, v[1 + 9 * ch:10 + 9 * ch]))) for ch in range(3)])
        a = 1 - math.exp(-sig * delta)
        C += T * a * c
        T *= 1 - a
        s += 1
    return C + T * np.asarray(bg, float)


@pytest.mark.parametrize("stop", [0.0, 0.2])
def test_render_brute_force_4cubed(stop):
    R = 4
    idx, rows = random_sparse(R, 0.35, 31, sigma_range=(-1.0, 6.0))
    o, d = synth.random_rays(24, seed=32, spread=0.9)
    o, d = o.astype(float), d.astype(float)
    bg = (1.0, 0.8, 0.6)
    rgb, _ = oracle.render(R, idx, rows, o, d, step_vox=0.5, bg=bg, stop_thresh=stop)
    for r in range(o.shape[0]):
        assert rgb[r] == pytest.approx(brute_render(R, idx, rows, o[r], d[r], 0.5, bg, stop), rel=1e-12, abs=1e-14)


def test_render_empty_grid_gives_background_and_zero_gradient():
    R = 5
    rows = np.random.default_rng(0).normal(size=(10, NV))
    idx = np.full(R ** 3, -1, np.int32)
    o, d = synth.random_rays(20, seed=1)
    bg = (0.3, 0.6, 0.9)
    rgb, aux = oracle.render(R, idx, rows, o, d, bg=bg)
    assert np.all(rgb == np.array(bg))
    assert np.all(aux[:, 0] == 1.0)
    g = oracle.render_backward(R, idx, rows, o, d, np.ones((20, 3)), bg=bg)
    assert np.all(g == 0.0)


def test_render_gradient_support_is_near_the_ray():
    """Only nodes within one cell diagonal of a ray can be corners of a sampled cell."""
    R = 9
    idx, rows = random_sparse(R, 0.0, 41, sigma_range=(0.5, 3.0))
    rows[:, 1] += 1.0 / Y00
    o, d = synth.random_rays(1, seed=42)
    o, d = o.astype(float), d.astype(float)
    g = oracle.render_backward(R, idx, rows, o, d, np.ones((1, 3)))
    pos, _ = node_pos(R)
    rel = pos - o[0]
    dist = np.linalg.norm(rel - (rel @ d[0])[:, None] * d[0][None, :], axis=1)
    far = dist > math.sqrt(3) * 2.0 / (R - 1) + 1e-9
    assert np.any(far) and np.all(g[idx[far]] == 0.0)
    assert np.any(g[idx[~far]] != 0.0)


# ----------------------------------------------------------------------------- adjoint

def _loss_render(R, idx, rows, o, d, gw, stop, bg):
    rgb, _ = oracle.render(R, idx, rows, o, d, step_vox=0.5, bg=bg, stop_thresh=stop)
    return float((rgb * gw).sum())


@pytest.mark.parametrize("R,frac_empty,stop,sig_lo,dc", [
    (4, 0.0, 0.0, 0.2, 1.0), (4, 0.3, 0.0, 0.2, 1.0), (6, 0.3, 0.1, 0.2, 1.0),
    (5, 0.2, 0.0, -4.0, 0.0)])  # last: density and colour ReLUs both active and inactive
def test_render_backward_matches_central_differences(R, frac_empty, stop, sig_lo, dc):
    idx, rows = random_sparse(R, frac_empty, 50 + R, sigma_range=(sig_lo, 6.0), sh_std=0.1 if dc else 0.6)
    rows[:, 1] += dc / Y00  # dc = 1: colours sit well above the ReLU kink (Supp. B.1)
    rows[:, 10] += dc / Y00
    rows[:, 19] += dc / Y00
    o, d = synth.random_rays(16, seed=60 + R, spread=0.7)
    o, d = o.astype(float), d.astype(float)
    gw = np.random.default_rng(70).normal(size=(16, 3))
    bg = (1.0, 0.7, 0.2)
    an = oracle.render_backward(R, idx, rows, o, d, gw, step_vox=0.5, bg=bg, stop_thresh=stop)
    # h = 1e-5 balances the central-difference truncation error (~h^2) against
    # the FP64 rounding of the loss, which the tolerance bounds by 8 eps |L| / h.
    h = 1e-5
    fd = np.zeros_like(an)
    for m in range(rows.shape[0]):
        for v in range(NV):
            rp = rows.copy()
            rp[m, v] += h
            rm = rows.copy()
            rm[m, v] -= h
            fd[m, v] = (_loss_render(R, idx, rp, o, d, gw, stop, bg) - _loss_render(R, idx, rm, o, d, gw, stop, bg)) / (2 * h)
    scale = np.max(np.abs(an))
    assert scale > 0
    err = np.abs(fd - an)
    floor = 8 * np.finfo(float).eps * abs(_loss_render(R, idx, rows, o, d, gw, stop, bg)) / h
    assert np.all(err <= 1e-6 * np.maximum(np.abs(an), 1e-3 * scale) + floor)


# ----------------------------------------------------------------------------- Cauchy sparsity prior

@pytest.mark.parametrize("stop", [0.0, 0.05])
def test_sparsity_constant_field_closed_form(stop):
    """sigma = sigma0 on every node: each of a ray's N samples (the render's closed-form count) adds
    log(1 + 2 sigma0^2), and its gradient lambda 4 sigma0 / (1 + 2 sigma0^2) splits over corners whose
    trilinear weights sum to one, so the density column of the gradient sums to lambda N times that."""
    R, sigma0, lam, step_vox = 12, 2.3, 1e-3, 0.37
    idx, rows = constant_field(R, sigma0, (0.5, 0.5, 0.5))
    delta = step_vox * 2.0 / (R - 1)
    o = np.array([[-3.0, 0.2, -0.4], [0.3, -3.0, 0.1], [2.2, 2.9, -1.7]])
    d = np.array([[1.0, 0.0, 0.0], [0.1, 1.0, -0.05], [-0.5, -0.8, 0.45]])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    N = 0
    for r in range(o.shape[0]):
        t0, t1 = box_segment(o[r], d[r])
        n = math.ceil((t1 - t0) / delta)
        if stop > 0:
            n = min(n, math.ceil(math.log(1.0 / stop) / (sigma0 * delta)))
        N += n
    L, g = oracle.sparsity(R, idx, rows, o, d, lam, step_vox=step_vox, stop_thresh=stop)
    assert L == pytest.approx(lam * N * math.log(1 + 2 * sigma0 ** 2), rel=1e-13)
    assert g[:, 0].sum() == pytest.approx(lam * N * 4 * sigma0 / (1 + 2 * sigma0 ** 2), rel=1e-12)
    assert np.all(g[:, 1:] == 0.0)


def test_sparsity_matches_central_differences():
    R = 5
    idx, rows = random_sparse(R, 0.3, 81, sigma_range=(-3.0, 6.0))
    o, d = synth.random_rays(12, seed=82, spread=0.7)
    o, d = o.astype(float), d.astype(float)
    lam = 0.7
    L0, an = oracle.sparsity(R, idx, rows, o, d, lam)
    h = 1e-5
    fd = np.zeros(rows.shape[0])
    for m in range(rows.shape[0]):
        rp, rm = rows.copy(), rows.copy()
        rp[m, 0] += h
        rm[m, 0] -= h
        fd[m] = (oracle.sparsity(R, idx, rp, o, d, lam)[0] - oracle.sparsity(R, idx, rm, o, d, lam)[0]) / (2 * h)
    scale = np.max(np.abs(an[:, 0]))
    assert scale > 0 and L0 > 0
    floor = 8 * np.finfo(float).eps * abs(L0) / h
    assert np.all(np.abs(fd - an[:, 0]) <= 1e-6 * np.maximum(np.abs(an[:, 0]), 1e-3 * scale) + floor)


def test_sparsity_of_non_positive_density_is_zero():
    R = 6
    idx, rows = random_sparse(R, 0.2, 83, sigma_range=(-5.0, 0.0))
    o, d = synth.random_rays(30, seed=84)
    L, g = oracle.sparsity(R, idx, rows, o, d, 1.0)
    assert L == 0.0 and np.all(g == 0.0)


def test_backward_abs_bounds_the_adjoint():
    """|adjoint(g')| <= abs-adjoint(g) for every |g'| <= g (triangle inequality), with equality for a
    single ray and channel on the SH columns of its colour-channel (one sign per term there)."""
    R = 6
    idx, rows = random_sparse(R, 0.2, 140, sigma_range=(-1.0, 6.0))
    o, d = synth.random_rays(20, seed=141)
    o, d = o.astype(float), d.astype(float)
    rng = np.random.default_rng(142)
    gb = rng.uniform(0.1, 1.0, size=(20, 3))
    bound = oracle.render_backward_abs(R, idx, rows, o, d, gb)
    for trial in range(4):
        gp = gb * rng.uniform(-1, 1, size=gb.shape)
        a = oracle.render_backward(R, idx, rows, o, d, gp)
        assert np.all(np.abs(a) <= bound * (1 + 1e-12) + 1e-300)
    # a single ray, one channel: the SH gradient of channel 0 is g w [pre>0] Y_l per sample and corner
    # (all of one sign per (corner, l) only if Y_l keeps its sign, which it does for a fixed direction)
    g1 = np.zeros((1, 3))
    g1[0, 0] = 0.7
    a1 = oracle.render_backward(R, idx, rows, o[:1], d[:1], g1)
    b1 = oracle.render_backward_abs(R, idx, rows, o[:1], d[:1], g1)
    assert np.allclose(np.abs(a1[:, 1:10]), b1[:, 1:10], rtol=1e-13, atol=0)
    assert np.all(b1[:, 10:] == 0)


def test_backward_mag_dominates_abs_and_matches_it_without_cancellation():
    """The magnitude adjoint replaces |T_{s+1} c - R_s| by T_{s+1} c + R_s (both non-negative): it dominates
    the absolute-value adjoint, agrees with it on the SH columns, and equals it when every ray has one
    sample and the background is black (then R_s = 0 for that sample)."""
    R = 6
    idx, rows = random_sparse(R, 0.3, 150, sigma_range=(0.5, 6.0))
    o, d = synth.random_rays(30, seed=151)
    o, d = o.astype(float), d.astype(float)
    g = np.random.default_rng(152).uniform(0.1, 1.0, size=(30, 3))
    a = oracle.render_backward_abs(R, idx, rows, o, d, g, bg=(0.3, 0.5, 0.7))
    m = oracle.render_backward_mag(R, idx, rows, o, d, g, bg=(0.3, 0.5, 0.7))
    assert np.all(m >= a * (1 - 1e-13))
    assert np.allclose(m[:, 1:], a[:, 1:], rtol=1e-13, atol=0)
    assert np.any(m[:, 0] > a[:, 0] * (1 + 1e-6))  # the density column does see cancellation here
    # one sample per ray: the step is longer than the box diagonal; black background
    a1 = oracle.render_backward_abs(R, idx, rows, o, d, g, step_vox=20.0, bg=(0.0, 0.0, 0.0))
    m1 = oracle.render_backward_mag(R, idx, rows, o, d, g, step_vox=20.0, bg=(0.0, 0.0, 0.0))
    assert np.any(a1[:, 0] > 0)
    assert np.allclose(m1, a1, rtol=1e-13, atol=0)
    # signs of g do not matter to it
    assert np.allclose(oracle.render_backward_mag(R, idx, rows, o, d, -g, bg=(0.3, 0.5, 0.7)), m, rtol=1e-12, atol=0)


def test_mse_closed_form_constant_error():
    """Eq. 3's reconstruction term is the mean over the batch of the squared 2-norm over RGB.  With
    every channel of every ray off by the same c, each ray contributes ||(c, c, c)||^2 = 3 c^2, so the
    mean is 3 c^2 whatever the batch size, and the loss scales as c^2; a loss normalised by 3n (a
    per-channel mean) or not normalised at all gives c^2 or 3 n c^2 and fails here."""
    rng = np.random.default_rng(0)
    for n in (1, 7, 64):
        t = rng.uniform(size=(n, 3))
        for c in (0.25, -0.5, 1e-3):
            L, g = oracle.mse(t + c, t)
            assert L == pytest.approx(3.0 * c * c, rel=1e-12)
            # the gradient of 3 c^2 along the uniform direction, shared by the 3n inputs: 6 c / (3n) each
            assert np.allclose(g, 2.0 * c / n, rtol=1e-12, atol=0)
    L0, g0 = oracle.mse(t, t)
    assert L0 == 0.0 and not np.any(g0)


def test_mse_single_ray_error():
    """Only ray r differs, by the vector e: the loss is ||e||^2 / n (one term of the batch mean), and only
    ray r's three inputs get a gradient."""
    rng = np.random.default_rng(1)
    n, r = 9, 4
    t = rng.uniform(size=(n, 3))
    e = np.array([0.3, -0.1, 0.2])
    p = t.copy()
    p[r] += e
    L, g = oracle.mse(p, t)
    assert L == pytest.approx(float(e @ e) / n, rel=1e-12)
    assert np.all(g[np.arange(n) != r] == 0.0)
    assert np.any(g[r] != 0.0)


def test_mse_gradient_central_differences():
    """The returned gradient is the derivative of the returned loss: central differences of oracle.mse's
    own loss in every input (a dropped factor 2, or a gradient normalised differently from the loss,
    fails here).  The loss is quadratic, so the central difference is exact up to rounding."""
    rng = np.random.default_rng(2)
    n = 6
    p, t = rng.uniform(size=(n, 3)), rng.uniform(size=(n, 3))
    _, g = oracle.mse(p, t)
    h = 1e-5
    fd = np.zeros_like(p)
    for i in range(n):
        for ch in range(3):
            pp, pm = p.copy(), p.copy()
            pp[i, ch] += h
            pm[i, ch] -= h
            fd[i, ch] = (oracle.mse(pp, t)[0] - oracle.mse(pm, t)[0]) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-7, atol=1e-10)


# ----------------------------------------------------------------------------- TV

def _tv_scale(R):
    return R / GOLDEN["tv_resolution_reference"]["value"]


def test_tv_linear_ramp_closed_form():
    """V = a_d * i (+ b_d): every interior node has t = |a_d| R/256 and, with all
    interior nodes selected, interior gradients cancel; only i = 0 (and i = R-1
    through the neighbour term) receive gradient."""
    R = 6
    rng = np.random.default_rng(80)
    a = rng.uniform(0.5, 2.0, NV) * rng.choice([-1, 1], NV)
    b = rng.uniform(5, 6, NV)
    _, ijk = node_pos(R)
    rows = ijk[:, :1] * a[None, :] + b[None, :]
    idx, rows = dense(R, rows)
    starts, lens = [], []
    for i in range(R - 1):
        for j in range(R - 1):
            starts.append((i * R + j) * R)
            lens.append(R - 1)
    lam_s, lam_h = 0.7, 0.3
    L, g = oracle.tv(R, idx, rows, starts, lens, lam_s, lam_h)
    s = _tv_scale(R)
    assert L == pytest.approx(lam_s * abs(a[0]) * s + lam_h * np.abs(a[1:]).sum() * s, rel=1e-13)
    nsel = (R - 1) ** 3
    lam = np.array([lam_s] + [lam_h] * (NV - 1)) / nsel
    for n in range(R ** 3):
        i, j, k = ijk[n]
        if i == 0 and j < R - 1 and k < R - 1:
            exp = -s * np.sign(a) * lam
        elif i == R - 1 and j < R - 1 and k < R - 1:
            exp = s * np.sign(a) * lam
        else:
            exp = np.zeros(NV)
        assert np.allclose(g[n], exp, rtol=1e-12, atol=1e-18)


def test_tv_constant_field_edges():
    """Constant field c: only boundary nodes contribute, and only for density
    (missing density neighbour = 0; missing SH neighbour = own value, Supp. B.1)."""
    R = 5
    c = 2.5
    idx, rows = dense(R, np.full((R ** 3, NV), c))
    L, _ = oracle.tv(R, idx, rows, [0], [R ** 3], 1.0, 1.0)
    s = _tv_scale(R)
    expected = sum(math.comb(3, m) * (R - 1) ** (3 - m) * math.sqrt(m) for m in range(4)) * s * c / R ** 3
    assert L == pytest.approx(expected, rel=1e-13)


def test_tv_isolated_voxel_rules():
    """One occupied node in an empty grid.  Selecting it: density t = sqrt(3)|V| s,
    SH t = 0.  Selecting its empty -x neighbour: density and SH both see |V| s."""
    R = 5
    idx = np.full(R ** 3, -1, np.int32)
    n0 = (2 * R + 2) * R + 2
    idx[n0] = 0
    vals = np.linspace(-1.5, 2.0, NV)
    rows = vals[None, :].copy()
    s = _tv_scale(R)
    L, g = oracle.tv(R, idx, rows, [n0], [1], 1.0, 1.0)
    assert L == pytest.approx(math.sqrt(3) * abs(vals[0]) * s, rel=1e-14)
    assert g[0, 0] == pytest.approx(math.sqrt(3) * s * np.sign(vals[0]), rel=1e-14)
    assert np.all(g[0, 1:] == 0)
    nm = (1 * R + 2) * R + 2  # the -x neighbour, empty
    L2, g2 = oracle.tv(R, idx, rows, [nm], [1], 1.0, 1.0)
    assert L2 == pytest.approx(np.abs(vals).sum() * s, rel=1e-14)
    assert np.allclose(g2[0], s * np.sign(vals), rtol=1e-14)


def test_tv_gradient_matches_central_differences():
    R = 5
    idx, rows = random_sparse(R, 0.3, 90, sigma_range=(-3, 3), sh_std=1.0)
    starts, lens = synth.tv_segments(R, 0.5, 7, seed=91)
    lam_s, lam_h = 0.9, 0.4
    L0, an = oracle.tv(R, idx, rows, starts, lens, lam_s, lam_h)
    h = 1e-5  # as for the render adjoint: truncation ~h^2, rounding <= 8 eps |L| / h
    fd = np.zeros_like(an)
    for m in range(rows.shape[0]):
        for v in range(NV):
            rp = rows.copy()
            rp[m, v] += h
            rm = rows.copy()
            rm[m, v] -= h
            Lp, _ = oracle.tv(R, idx, rp, starts, lens, lam_s, lam_h)
            Lm, _ = oracle.tv(R, idx, rm, starts, lens, lam_s, lam_h)
            fd[m, v] = (Lp - Lm) / (2 * h)
    scale = np.max(np.abs(an))
    floor = 8 * np.finfo(float).eps * abs(L0) / h
    assert np.all(np.abs(fd - an) <= 1e-6 * np.maximum(np.abs(an), 1e-3 * scale) + floor)


# ----------------------------------------------------------------------------- RMSProp

def test_rmsprop_constant_gradient_closed_form():
    rng = np.random.default_rng(100)
    M = 7
    x0 = rng.normal(size=(M, NV))
    g = rng.normal(size=(M, NV))
    g[2, 5] = 0.0  # a zero-gradient entry is left alone
    beta, eps, lr_s, lr_h = 0.9, 1e-8, 3.0, 0.01
    x, v = x0.copy(), np.zeros((M, NV))
    v[2, 5] = 0.25
    steps = 6
    for _ in range(steps):
        x, v, gout = oracle.rmsprop(x, v, g, lr_s, lr_h, beta, eps)
        assert np.all(gout == 0)
    lr = np.array([lr_s] + [lr_h] * (NV - 1))[None, :]
    v_closed = [(1 - beta ** t) * g ** 2 for t in range(1, steps + 1)]
    x_closed = x0 - sum(lr * g / (np.sqrt(vt) + eps) for vt in v_closed)
    mask = g != 0
    assert np.allclose(v[mask], v_closed[-1][mask], rtol=1e-13)
    assert np.allclose(x[mask], x_closed[mask], rtol=1e-12, atol=1e-12)
    assert v[2, 5] == 0.25 and x[2, 5] == x0[2, 5]


# ----------------------------------------------------------------------------- prune / upsample

@pytest.mark.parametrize("mode", ["density", "key"])
def test_prune_matches_exhaustive_neighbourhoods(mode):
    R = 6
    idx, rows = random_sparse(R, 0.3, 110, sigma_range=(0, 10))
    tau = 7.0
    if mode == "density":
        rows[0, 0] = tau  # sigma == tau counts as hot
        key = rows[:, 0]
    else:  # an unrelated per-row key (the weight-threshold form)
        key = np.random.default_rng(111).uniform(0, 10, size=rows.shape[0])
        key[1] = tau
    for dilate in (True, False):
        if mode == "density":
            idx2, rows2 = oracle.prune(R, idx, rows, tau, dilate)
        else:
            idx2, rows2 = oracle.prune_key(R, idx, rows, key, tau, dilate)
        hot = lambda i, j, k: idx[(i * R + j) * R + k] >= 0 and key[idx[(i * R + j) * R + k]] >= tau
        expect_idx = np.full(R ** 3, -1, np.int32)
        kept = []
        for i, j, k in itertools.product(range(R), repeat=3):
            n = (i * R + j) * R + k
            if idx[n] < 0:
                continue
            if dilate:
                keep = any(hot(a, b, c) for a in range(max(0, i - 1), min(R, i + 2))
                           for b in range(max(0, j - 1), min(R, j + 2)) for c in range(max(0, k - 1), min(R, k + 2)))
            else:
                keep = hot(i, j, k)
            if keep:
                expect_idx[n] = len(kept)
                kept.append(rows[idx[n]])
        assert np.array_equal(idx2, expect_idx)
        assert np.array_equal(rows2, np.array(kept).reshape(-1, NV))


def test_prune_key_with_density_key_equals_density_prune():
    R = 7
    idx, rows = random_sparse(R, 0.5, 112, sigma_range=(0, 10))
    for dilate in (True, False):
        a = oracle.prune(R, idx, rows, 4.0, dilate)
        b = oracle.prune_key(R, idx, rows, rows[:, 0].copy(), 4.0, dilate)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ----------------------------------------------------------------------------- maximum weight (prune key)

@pytest.mark.parametrize("stop", [0.0, 0.5])
def test_max_weight_constant_field_closed_form(stop):
    """Density sigma0 on every node, a ray along +x at off-lattice grid coordinates (y, z) = (j0 + 0.3,
    k0 + 0.6), entering the box at grid x = 0, step 0.37 voxel.  Sample s sits at grid x = 0.37 s, has
    T_s = exp(-sigma0 s delta) and weight T_s (1 - exp(-sigma0 delta)), and is taken while T_s >= stop.
    It credits the 8 corners of cell floor(0.37 s): nodes (i, j, k) with i in {cell, cell + 1}, j in
    {j0, j0 + 1}, k in {k0, k0 + 1}.  Each of those nodes holds the largest weight crediting it (the
    earliest sample, weights falling along the ray); all other nodes hold 0."""
    R, step, sigma0 = 9, 0.37, 1.7
    h = 2.0 / (R - 1)
    delta = step * h
    j0, k0 = 3, 5
    idx, rows = constant_field(R, sigma0, (0.3, 0.2, 0.1))
    o = np.array([[-3.0, -1.0 + h * (j0 + 0.3), -1.0 + h * (k0 + 0.6)]])
    d = np.array([[1.0, 0.0, 0.0]])
    w = oracle.max_weight(R, idx, rows, o, d, step_vox=step, stop_thresh=stop)
    alpha = 1.0 - math.exp(-sigma0 * delta)
    expect = np.zeros(R ** 3)
    s = 0
    while 0.37 * s < R - 1:
        T = math.exp(-sigma0 * s * delta)
        if T < stop:
            break
        cell = min(math.floor(0.37 * s), R - 2)
        for i, j, k in itertools.product((cell, cell + 1), (j0, j0 + 1), (k0, k0 + 1)):
            n = (i * R + j) * R + k
            expect[n] = max(expect[n], T * alpha)
        s += 1
    assert np.count_nonzero(expect) == (4 * R if stop == 0 else np.count_nonzero(expect))
    assert np.max(np.abs(w - expect)) < 1e-14
    # the first sample (x = 0) credits the far corners of cell 0 although its trilinear weight there is 0
    assert w[(1 * R + j0) * R + k0] == pytest.approx(alpha, rel=1e-14)


def test_max_weight_union_of_ray_sets_is_the_elementwise_max():
    R = 10
    idx, rows = random_sparse(R, 0.6, 113, sigma_range=(0, 30))
    o, d = synth.random_rays(120, seed=114)
    wa = oracle.max_weight(R, idx, rows, o[:70], d[:70])
    wb = oracle.max_weight(R, idx, rows, o[70:], d[70:])
    wab = oracle.max_weight(R, idx, rows, o, d)
    assert np.array_equal(wab, np.maximum(wa, wb))
    again = oracle.max_weight(R, idx, rows, o[70:], d[70:], wmax=wa.copy())  # in-place continuation
    assert np.array_equal(again, wab)
    # every weight is at most the ray's total weight 1 - T_end (weights sum with T_end to one)
    _, aux = oracle.render(R, idx, rows, o, d, bg=0.0)
    assert 0.0 < wab.max() <= np.max(1.0 - aux[:, 0]) + 1e-15
    assert np.all(wab >= 0.0)


def test_max_weight_zero_density_is_zero():
    R = 6
    idx, rows = random_sparse(R, 0.2, 115, sigma_range=(0, 1))
    rows[:, 0] = 0.0
    o, d = synth.random_rays(40, seed=116)
    assert np.all(oracle.max_weight(R, idx, rows, o, d) == 0.0)


@pytest.mark.parametrize("R,R2", [(5, 9), (5, 10), (4, 7), (6, 11)])
def test_upsample_affine_field_exact(R, R2):
    rng = np.random.default_rng(120)
    A = rng.normal(size=(NV, 3))
    b = rng.normal(size=NV)
    pos, _ = node_pos(R)
    idx, rows = dense(R, pos @ A.T + b)
    idx2, rows2 = oracle.upsample(R, idx, rows, R2)
    pos2, _ = node_pos(R2)
    assert np.array_equal(idx2, np.arange(R2 ** 3))
    assert np.max(np.abs(rows2 - (pos2 @ A.T + b))) < 1e-12


def test_upsample_matches_exact_rational_support():
    R, R2 = 5, 8
    idx, rows = random_sparse(R, 0.6, 130)
    idx2, rows2 = oracle.upsample(R, idx, rows, R2)
    expect = []
    expect_idx = np.full(R2 ** 3, -1, np.int32)
    for i2, j2, k2 in itertools.product(range(R2), repeat=3):
        g = [Fraction(p * (R - 1), R2 - 1) for p in (i2, j2, k2)]
        occ = False
        val = np.zeros(NV)
        for i, j, k in itertools.product(range(R), repeat=3):
            w = Fraction(1)
            for ga, na in zip(g, (i, j, k)):
                w *= max(Fraction(0), 1 - abs(ga - na))
            if w == 0:
                continue
            n = (i * R + j) * R + k
            if idx[n] >= 0:
                occ = True
                val += float(w) * rows[idx[n]]
        if occ:
            expect_idx[(i2 * R2 + j2) * R2 + k2] = len(expect)
            expect.append(val)
    assert np.array_equal(idx2, expect_idx)
    assert np.max(np.abs(rows2 - np.array(expect))) < 1e-12


# ----------------------------------------------------------------------------- BF16 storage rounding

def test_round_bf16_ties_and_carries():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -(1 + 3 * 2 ** -8),
                  2 ** 0 - 2 ** -9, 3.0e-39, 65504.0], np.float32)
    y = oracle.round_bf16(x)
    assert y[0] == 1.0
    assert y[1] == 1.0  # tie, even mantissa
    assert y[2] == 1 + 2 ** -6  # tie, odd -> up
    assert y[3] == 1 + 2 ** -7  # above the tie
    assert y[4] == -(1 + 2 ** -6)
    assert y[5] == 1.0  # carry into the exponent
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    z = (rng.normal(size=10000) * 10 ** rng.uniform(-6, 6, 10000)).astype(np.float32)
    ref = torch.from_numpy(z).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.round_bf16(z), ref)
    assert np.array_equal(y, torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy())
