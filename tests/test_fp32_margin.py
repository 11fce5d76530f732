"""The march's cheap occupancy test works on FP32 grid coordinates and falls back to double-float
arithmetic within a per-ray margin of every cell face.  The margin is a bound on the FP32 coordinate
error, u (inv_h (3 |o - lo| + 5 t) + |x|) with u = 2^-24, plus a quarter.  This test runs the same
FP32 operations (ray setup, sample parameter, coordinate) in numpy and checks the bound against
float64 coordinates over many rays, samples, grid sizes and camera distances."""
import numpy as np
import pytest

U = 2.0 ** -24


def fma32(a, b, c):
    """float32 fused multiply-add: the exact product plus c, rounded once (float64 holds the product
    of two float32 exactly; the final sum rounds in float64 first, a second rounding that is at most
    one float32 ulp in rare ties and far inside the bound's slack)."""
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(np.float32)


@pytest.mark.parametrize("R", [32, 512, 2048])
@pytest.mark.parametrize("radius", [2.5, 4.0, 12.0])
def test_fp32_coordinate_error_within_margin(R, radius):
    rng = np.random.default_rng(R + int(radius * 10))
    n = 4000
    lo = np.float32(-1.0)
    h = 2.0 / (R - 1)
    inv_h32 = np.float32(1.0 / h)
    # rays from a sphere of `radius` towards random points of the box
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    o = (radius * dirs).astype(np.float32)
    tgt = rng.uniform(-0.9, 0.9, size=(n, 3))
    d = (tgt - o).astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = d.astype(np.float32)
    # box clip in float64 (the kernels' double-float clip is exact to ~2^-44)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (-1.0 - o.astype(np.float64)) / d
        tb = (1.0 - o.astype(np.float64)) / d
    tn = np.clip(np.max(np.minimum(ta, tb), axis=1), 0.0, None)
    tf = np.min(np.maximum(ta, tb), axis=1)
    hit = tf > tn
    o, d, tn, tf = o[hit], d[hit], tn[hit], tf[hit]
    delta = 0.5 * h
    delta32 = np.float32(delta)
    tn_hi = tn.astype(np.float32)
    og = ((o - lo).astype(np.float32) * inv_h32).astype(np.float32)
    dg = (d * inv_h32).astype(np.float32)
    om = np.max(np.abs(o - lo), axis=1).astype(np.float64)
    bound = U * (float(inv_h32) * (3.0 * om + 5.0 * np.abs(tf)) + R)
    worst = 0.0
    for s in range(0, int(np.ceil((tf - tn).max() / delta)) + 1, 7):
        live = tn + s * delta < tf
        if not live.any():
            break
        t32 = fma32(np.float32(s), delta32, tn_hi)
        t = tn + s * delta
        for a in range(3):
            x32 = fma32(t32, dg[:, a], og[:, a]).astype(np.float64)
            x = (o[:, a].astype(np.float64) - lo + t * d[:, a].astype(np.float64)) / h
            err = np.abs(x32 - x)[live]
            ratio = err / bound[live]
            worst = max(worst, float(ratio.max()))
    assert worst <= 1.0, worst
    print(f"R={R} radius={radius}: worst error / bound {worst:.3f}")
