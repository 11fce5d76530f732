"""Comparison rules shared by the GPU parity tests (CUDA library vs the FP64 oracle).

Tolerances (colours and gradients are FP32 on the GPU, FP64 in the oracle):
  colours    |dC| <= 1e-5 * max(|C_ref|, 1e-3)
  gradients  |dg| <= 1e-4 * max(|g_ref|, 1e-3 * max|g_ref|)       (per row entry)
  maps       bit-exact (index volumes after prune/upsample)
Two discrete decisions may legitimately differ between FP32 and FP64 and are
flagged per ray, then checked against the size of one sample's contribution:
  * the sample count, when (t_far - t_near)/delta sits within 1e-9 of an
    integer (the kernels hold t as a double-float);
  * the early-termination sample, when stop_thresh > 0: |dC| <= stop_thresh *
    (c_max + |bg|) is added, as one sample at T < stop_thresh contributes at most that.
"""
from __future__ import annotations

import math

import numpy as np

COLOUR_RTOL = 1e-5
COLOUR_FLOOR = 1e-3
GRAD_RTOL = 1e-4
GRAD_FLOOR = 1e-3


def ulp32(x):
    x = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.maximum(x, 1e-30)))
    return np.exp2(e - 23)


def delta_of(R, step_vox, aabb=((-1, -1, -1), (1, 1, 1))):
    h = min((aabb[1][a] - aabb[0][a]) / (R - 1) for a in range(3))
    return step_vox * h


def colour_bound(rows28, bg):
    """Largest colour any sample can have (each channel sum_l |Y_l| |k_l| <= 1.1 sum_l |k_l|)."""
    if rows28.shape[0] == 0:
        return float(np.max(np.abs(bg)))
    k = np.abs(rows28[:, 1:]).reshape(-1, 3, 9).sum(2).max()
    return float(1.1 * k + np.max(np.abs(bg)))


def tie_flags(aux, delta):
    """Rays whose sample count the GPU cannot resolve: aux = oracle [n,4] (T_end, n, ratio, hit).
    The kernels carry t as a double-float (about 2^-44 relative), so only rays whose
    (t_far - t_near)/delta lies within 1e-9 of an integer are flagged."""
    ratio = aux[:, 2]
    frac = np.abs(ratio - np.round(ratio))
    return (aux[:, 3] > 0) & (frac < 1e-9)


def check_colours(gpu, ref, aux, rows28, delta, bg, stop_thresh=0.0, sigma_max=None, what="rgb", extra_tol=None):
    """Assert colour parity; returns (worst error/tolerance ratio over unflagged rays, n flagged).
    `extra_tol` ([n,3], optional) widens the bound where the two sides' inputs differ by a known amount."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape
    assert np.all(np.isfinite(gpu)), f"{what}: non-finite GPU output"
    tol = COLOUR_RTOL * np.maximum(np.abs(ref), COLOUR_FLOOR)
    if extra_tol is not None:
        tol = tol + extra_tol
    cmax = colour_bound(rows28, bg)
    if stop_thresh > 0:
        tol = tol + stop_thresh * cmax
    flags = tie_flags(aux, delta)
    err = np.abs(gpu - ref)
    ok = err <= tol
    if sigma_max is None:
        sigma_max = float(np.max(rows28[:, 0])) if rows28.shape[0] else 0.0
    one_sample = delta * max(sigma_max, 0.0) * cmax
    ok_flag = err <= tol + one_sample
    bad = ~np.where(flags[:, None], ok_flag, ok)
    worst = float(np.max(np.where(flags[:, None], 0.0, err / tol))) if err.size else 0.0
    if np.any(bad):
        r, c = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {int(bad.any(1).sum())} rays out of tolerance; first ray {r} ch {c}: "
                             f"gpu {gpu[r, c]!r} ref {ref[r, c]!r} err {err[r, c]:.3e} tol {tol[r, c]:.3e} "
                             f"(worst unflagged err/tol {worst:.3f}, flagged {int(flags.sum())})")
    return worst, int(flags.sum())


def check_grads(gpu, ref, what="grad", rows=None, extra_abs=None):
    """Assert per-entry gradient parity on [M, 28] arrays (optionally only `rows`).
    `extra_abs` ([M, 28], optional) adds a derived bound where the two sides' inputs differ."""
    gpu = np.asarray(gpu, np.float64)[:, :28]
    ref = np.asarray(ref, np.float64)[:, :28]
    gmax = float(np.max(np.abs(ref))) if ref.size else 0.0
    extra = np.zeros_like(ref) if extra_abs is None else np.asarray(extra_abs, np.float64)[:, :28]
    if rows is not None:
        gpu = gpu[rows]
        ref = ref[rows]
        extra = extra[rows]
    assert np.all(np.isfinite(gpu)), f"{what}: non-finite GPU gradient"
    tol = GRAD_RTOL * np.maximum(np.abs(ref), GRAD_FLOOR * gmax) + extra
    err = np.abs(gpu - ref)
    bad = err > tol
    worst = float(np.max(err / np.maximum(tol, 1e-300))) if err.size else 0.0
    if np.any(bad):
        m, d = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {int(bad.sum())} entries out of tolerance; first row {m} col {d}: "
                             f"gpu {gpu[m, d]!r} ref {ref[m, d]!r} err {err[m, d]:.3e} tol {tol[m, d]:.3e} "
                             f"(worst err/tol {worst:.3f}, max|g| {gmax:.3e})")
    return worst


def bf16_grid_rows(rows28):
    """The values a BF16-SH grid holds: SH rounded to bfloat16 (nearest even), density exact."""
    import oracle

    out = np.array(rows28, np.float32, copy=True)
    out[:, 1:] = oracle.round_bf16(out[:, 1:])
    return out


def rmsprop_first_step_bound(g_ref, tol_g, x_ref, lr_sigma, lr_sh, beta, eps):
    """Entrywise bound on |x_gpu - x_ref| after RMSProp's first step (v = 0) when the GPU gradient is
    only known to lie in [g_ref - tol_g, g_ref + tol_g].  The update u(g) = lr g / (sqrt((1 - beta) g^2)
    + eps) is monotone in g, so over that interval it moves by at most max |u(g_ref +- tol) - u(g_ref)|;
    FP32 rounding of x adds a few ulp."""
    lr = np.array([lr_sigma] + [lr_sh] * 27)[None, :]

    def u(gg):
        return lr * gg / (np.sqrt((1 - beta) * gg * gg) + eps)

    du = np.maximum(np.abs(u(g_ref + tol_g) - u(g_ref)), np.abs(u(g_ref - tol_g) - u(g_ref)))
    return du + 4 * np.finfo(np.float32).eps * (np.abs(x_ref) + np.abs(u(g_ref)))


def grad_tolerance(g_ref, extra_abs=None):
    """The per-entry gradient tolerance check_grads applies (without row selection)."""
    g_ref = np.asarray(g_ref, np.float64)[:, :28]
    gmax = float(np.max(np.abs(g_ref))) if g_ref.size else 0.0
    tol = GRAD_RTOL * np.maximum(np.abs(g_ref), GRAD_FLOOR * gmax)
    if extra_abs is not None:
        tol = tol + np.asarray(extra_abs, np.float64)[:, :28]
    return tol


def psnr(x, y):
    """Peak signal-to-noise ratio in dB for colours on a unit peak."""
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(y, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else -10.0 * math.log10(mse)


# FP32 summation allowance for gradient entries whose terms cancel.  Each term of an adjoint entry is a
# product of several rounded FP32 quantities (transmittance, alpha, colour gradient, trilinear and basis
# factors), so it carries a relative error of a few units of roundoff, and the atomic accumulation adds
# one rounding per addition in an order that changes from run to run.  Where the terms cancel, the
# entry's error is a few roundoffs of the summed magnitudes, not of the entry, and can exceed the floor
# 1e-4 * 1e-3 max|g| (about 1.7 roundoffs of max|g|).  On the dense 32^3 step the largest error measured
# on a GB300 was 3.7 roundoffs of the oracle's magnitude adjoint; the allowance is 8.
FP32_SUM_U = 8 * 2.0 ** -24


def dense32_step_case(n, seed, opts_bg=(1.0, 1.0, 1.0), stop_thresh=0.0):
    """The dense 32^3 workload's own adjoint input: the perturbed grid (the ground truth plus N(0, 0.05)
    on every value) rendered along n seeded rays, and dL/dC of the MSE against the ground truth's render
    (Eq. 3), both from the oracle.  Returns (scene, o, d, dL/dC float32)."""
    import oracle
    import synth

    gt = synth.scene_config("dense32")
    sc = synth.perturb(gt, 0.05, seed=1)
    o, d = synth.random_rays(n, seed=seed)
    kw = dict(bg=opts_bg, stop_thresh=stop_thresh)
    target, _ = oracle.render(gt.R, gt.idx, gt.rows, o.astype(float), d.astype(float), **kw)
    pred, _ = oracle.render(gt.R, sc.idx, sc.rows, o.astype(float), d.astype(float), **kw)
    gw = oracle.mse(pred, target.astype(np.float32).astype(np.float64))[1].astype(np.float32)
    return sc, o, d, gw
