"""The march's cheap occupancy test works on FP32 grid coordinates and falls back to double-float
arithmetic within a per-ray margin of every cell face.  Sample s of a ray sits at grid coordinates
g0 + s st (g0: the point at t_near, st: the step between samples, both kept as double-floats); the
cheap coordinate is fma(s, st_hi, g0_hi) and the margin is a bound on its error,
u (2 max|g0| + 2 (s_end + 8) max|st|) with u = 2^-24, plus a quarter.  This test runs the same FP32
operations in numpy and checks the bound against float64 coordinates over many rays, samples (up to
8 past the last one, as the group screen evaluates), grid sizes and camera distances."""
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
    # the double-float anchor and step, rounded to their FP32 high parts
    g0 = (o.astype(np.float64) - lo + tn[:, None] * d.astype(np.float64)) / h
    st = delta * d.astype(np.float64) / h
    g0_hi = g0.astype(np.float32)
    st_hi = st.astype(np.float32)
    s_end = np.ceil((tf - tn) / delta)
    bound = U * (2.0 * np.abs(g0_hi).max(axis=1) + 2.0 * (s_end + 8) * np.abs(st_hi).max(axis=1))
    worst = 0.0
    for s in range(0, int(s_end.max()) + 8, 7):
        live = s < s_end + 8
        if not live.any():
            break
        for a in range(3):
            x32 = fma32(np.float32(s), st_hi[:, a], g0_hi[:, a]).astype(np.float64)
            x = (o[:, a].astype(np.float64) - lo + (tn + s * delta) * d[:, a].astype(np.float64)) / h
            err = np.abs(x32 - x)[live]
            ratio = err / bound[live]
            worst = max(worst, float(ratio.max()))
    assert worst <= 1.0, worst
    print(f"R={R} radius={radius}: worst error / bound {worst:.3f}")
