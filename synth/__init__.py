"""Seeded synthetic inputs for the Plenoxels renderer: scenes, cameras, ray batches, TV segments.

This module is the only code shared by the CUDA path's tests/benchmark and the
FP64 oracle, and it holds none of the method's arithmetic: it draws grids,
camera poses, pixel ids and voxel segments; rendering, interpolation, SH,
compositing, TV, RMSProp, pruning and upsampling live on each side separately.

The paper's workloads (NeRF-synthetic: 100 views of 800x800 on the upper
hemisphere, white background, Sec. 4.1; 256^3 -> 512^3 grids, Supp. B.2) are
datasets that are not available; the generators below stand in for them with
the same shapes.  Scene recipes:

* ``scene_dense_blobs`` -- dense R^3 grid, density = sum of isotropic Gaussian
  blobs (peak 50, std ``blob_std_vox`` voxels, centres ~ U[-0.5,0.5]^3) evaluated
  on every node (strictly positive), SH ~ N(0, sh_std).
* ``scene_sparse`` -- R^3 grid whose density is 20 Gaussian blobs (peak 50,
  std ~ U(0.04, 0.12) world units) plus a thin spherical shell (radius 0.6,
  Gaussian profile of width 1.5 voxels, peak 50).  The top ``occupancy``
  fraction of nodes by density is occupied; occupied nodes keep their density
  and get SH ~ N(0, sh_std); the rest are NULL.

Node (i,j,k) has linear id (i*R + j)*R + k and world position
-1 + 2*(i,j,k)/(R-1) (the [-1,1]^3 box).  Rows are float32 [M, 28] laid out as
[sigma, R0..R8, G0..G8, B0..B8].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

NV = 28


@dataclass
class Scene:
    R: int
    idx: np.ndarray   # int32 [R^3], -1 = empty
    rows: np.ndarray  # float32 [M, 28]

    @property
    def M(self) -> int:
        return int(self.rows.shape[0])


def _node_coords_1d(R: int) -> np.ndarray:
    return (-1.0 + 2.0 * np.arange(R, dtype=np.float64) / (R - 1)).astype(np.float32)


def _add_blob(sigma: np.ndarray, R: int, centre, std: float, peak: float, truncate: bool = True) -> None:
    """Add peak*exp(-|x-c|^2/(2 std^2)), either on the whole grid or inside a +-4 std box
    (values beyond it are below 4e-6 * peak, far under the occupancy thresholds of sparse scenes)."""
    h = 2.0 / (R - 1)
    if truncate:
        lo = [max(0, int(math.floor((c - 4 * std + 1.0) / h))) for c in centre]
        hi = [min(R - 1, int(math.ceil((c + 4 * std + 1.0) / h))) for c in centre]
    else:
        lo, hi = [0, 0, 0], [R - 1, R - 1, R - 1]
    xs = [(-1.0 + h * np.arange(lo[a], hi[a] + 1)).astype(np.float32) - np.float32(centre[a]) for a in range(3)]
    inv = np.float32(1.0 / (2.0 * std * std))
    ex = np.exp(-(xs[0] ** 2) * inv)
    ey = np.exp(-(xs[1] ** 2) * inv)
    ez = np.exp(-(xs[2] ** 2) * inv)
    block = np.float32(peak) * ex[:, None, None] * ey[None, :, None] * ez[None, None, :]
    sigma[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] += block


def scene_dense_blobs(R: int = 32, n_blobs: int = 3, peak: float = 50.0, blob_std_vox: float = 4.0,
                      sh_std: float = 0.3, seed: int = 0) -> Scene:
    """Dense grid (every node occupied, idx = arange)."""
    rng = np.random.default_rng(seed)
    h = 2.0 / (R - 1)
    centres = rng.uniform(-0.5, 0.5, size=(n_blobs, 3))
    sigma = np.zeros((R, R, R), np.float32)
    for b in range(n_blobs):
        _add_blob(sigma, R, centres[b], blob_std_vox * h, peak, truncate=False)
    M = R ** 3
    rows = np.empty((M, NV), np.float32)
    rows[:, 0] = sigma.reshape(-1)
    rows[:, 1:] = rng.normal(0.0, sh_std, size=(M, NV - 1)).astype(np.float32)
    idx = np.arange(M, dtype=np.int32)
    return Scene(R, idx, rows)


def scene_sparse(R: int, occupancy: float, n_blobs: int = 20, peak: float = 50.0,
                 shell_radius: float = 0.6, shell_width_vox: float = 1.5,
                 sh_std: float = 0.2, seed: int = 0) -> Scene:
    """Sparse blobs + shell scene; occupancy = fraction of nodes kept (top by density)."""
    rng = np.random.default_rng(seed)
    h = 2.0 / (R - 1)
    centres = rng.uniform(-0.6, 0.6, size=(n_blobs, 3))
    stds = rng.uniform(0.04, 0.12, size=n_blobs)
    sigma = np.zeros((R, R, R), np.float32)
    for b in range(n_blobs):
        _add_blob(sigma, R, centres[b], float(stds[b]), peak)
    # thin shell: peak * exp(-(r - r0)^2 / (2 w^2)), evaluated slab by slab
    x = _node_coords_1d(R)
    w = shell_width_vox * h
    inv = np.float32(1.0 / (2.0 * w * w))
    yz2 = x[:, None] ** 2 + x[None, :] ** 2
    for i in range(R):
        r = np.sqrt(x[i] ** 2 + yz2)
        sigma[i] += np.float32(peak) * np.exp(-((r - np.float32(shell_radius)) ** 2) * inv)
    flat = sigma.reshape(-1)
    N = flat.shape[0]
    keep = int(round(occupancy * N))
    if keep >= N:
        occ = np.ones(N, bool)
    else:
        thresh = np.partition(flat, N - keep)[N - keep]
        occ = flat >= thresh
    idx = np.full(N, -1, np.int32)
    nz = np.flatnonzero(occ)
    idx[nz] = np.arange(nz.shape[0], dtype=np.int32)
    M = nz.shape[0]
    rows = np.empty((M, NV), np.float32)
    rows[:, 0] = flat[nz]
    rows[:, 1:] = rng.normal(0.0, sh_std, size=(M, NV - 1)).astype(np.float32)
    return Scene(R, idx, rows)


def perturb(scene: Scene, std: float, seed: int = 1) -> Scene:
    """The same occupancy with N(0, std) noise added to all 28 values of every row."""
    rng = np.random.default_rng(seed)
    rows = scene.rows + rng.normal(0.0, std, size=scene.rows.shape).astype(np.float32)
    return Scene(scene.R, scene.idx.copy(), rows.astype(np.float32))


def scene_config(name: str, seed: int = 0) -> Scene:
    """The named synthetic workloads: 'dense32', 'sparse256' (8%), 'sparse512' (3%), or 'sparseR_f'."""
    if name == "dense32":
        return scene_dense_blobs(32, 3, 50.0, 4.0, 0.3, seed)
    if name == "sparse256":
        return scene_sparse(256, 0.08, seed=seed)
    if name == "sparse512":
        return scene_sparse(512, 0.03, seed=seed)
    if name.startswith("sparse"):
        r, f = name[6:].split("_")
        return scene_sparse(int(r), float(f), seed=seed)
    raise ValueError(name)


# --------------------------------------------------------------------------- cameras

def fibonacci_directions(n: int, upper: bool) -> np.ndarray:
    """n near-uniform unit vectors on the sphere (or on the z>0 hemisphere)."""
    k = np.arange(n, dtype=np.float64) + 0.5
    z = (1.0 - k / n) if upper else (1.0 - 2.0 * k / n)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def look_at(eye: np.ndarray, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """3x4 camera-to-world matrix of a camera at ``eye`` looking at ``target``.

    Camera axes follow the OpenGL convention the renderer assumes: x right,
    y up, looking down -z.
    """
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    upv = np.asarray(up, np.float64)
    if abs(float(np.dot(fwd, upv))) > 0.999:
        upv = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, upv)
    right /= np.linalg.norm(right)
    cam_up = np.cross(right, fwd)
    c2w = np.zeros((3, 4), np.float64)
    c2w[:, 0] = right
    c2w[:, 1] = cam_up
    c2w[:, 2] = -fwd
    c2w[:, 3] = eye
    return c2w


def cameras(n_views: int, W: int, H: int, fov_deg: float, radius: float, upper: bool,
            seed: int = 0, jitter: float = 0.0) -> np.ndarray:
    """float32 [n_views, 18] = c2w (3x4 row-major), fx, fy, cx, cy, W, H."""
    rng = np.random.default_rng(seed)
    dirs = fibonacci_directions(n_views, upper)
    if jitter > 0:
        dirs = dirs + rng.normal(0.0, jitter, size=dirs.shape)
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        if upper:
            dirs[:, 2] = np.abs(dirs[:, 2])
    f = 0.5 * W / math.tan(math.radians(fov_deg) / 2.0)
    cams = np.zeros((n_views, 18), np.float64)
    for v in range(n_views):
        cams[v, :12] = look_at(radius * dirs[v]).reshape(-1)
        cams[v, 12:16] = [f, f, 0.5 * W, 0.5 * H]
        cams[v, 16:18] = [W, H]
    return cams.astype(np.float32)


def cameras_config(name: str, seed: int = 0) -> np.ndarray:
    """'sphere8_64': 8 views 64x64 on a sphere r=2.5, fov 40 deg;
    'hemi100_800': 100 views 800x800 on the upper hemisphere r=4, fov 40 deg;
    'hemi25_800_test': 25 held-out 800x800 views (different seed/jitter)."""
    if name == "sphere8_64":
        return cameras(8, 64, 64, 40.0, 2.5, upper=False, seed=seed)
    if name == "hemi100_800":
        return cameras(100, 800, 800, 40.0, 4.0, upper=True, seed=seed)
    if name == "hemi25_800_test":
        return cameras(25, 800, 800, 40.0, 4.0, upper=True, seed=seed + 1000, jitter=0.15)
    raise ValueError(name)


def pixel_batch(n_views: int, W: int, H: int, n: int, seed: int) -> np.ndarray:
    """n pixel ids (view*H*W + v*W + u) uniform over all pixels of all views, with replacement."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_views * W * H, size=n, dtype=np.int64)


def tv_segments(R: int, fraction: float, seg_len: int, seed: int):
    """Random contiguous runs of ``seg_len`` linear node ids covering ~``fraction`` of R^3
    (Supp. B.1: TV on random contiguous segments in pointer-grid order).  Non-overlapping,
    sorted; returns (start int64 [S], length int64 [S])."""
    rng = np.random.default_rng(seed)
    N = R ** 3
    n_slots = max(1, N // seg_len)
    n_seg = max(1, min(n_slots, int(round(fraction * N / seg_len))))
    slots = np.sort(rng.choice(n_slots, size=n_seg, replace=False)).astype(np.int64)
    start = slots * seg_len
    length = np.minimum(seg_len, N - start).astype(np.int64)
    return start, length


def random_rays(n: int, seed: int, radius: float = 2.5, spread: float = 0.6):
    """float32 rays from points on a sphere of ``radius`` aimed near the origin: (o [n,3], d [n,3]).

    Directions are normalised in float64 and then rounded to float32; both
    sides take these exact float32 values as input."""
    rng = np.random.default_rng(seed)
    eye = rng.normal(size=(n, 3))
    eye = radius * eye / np.linalg.norm(eye, axis=1, keepdims=True)
    target = rng.uniform(-spread, spread, size=(n, 3))
    d = target - eye
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return eye.astype(np.float32), d.astype(np.float32)


SERVING_RESOLUTIONS = ((256, 256), (800, 800), (1280, 720), (1920, 1080))


def serving_requests(n: int, n_scenes: int, seed: int, rate=None, fov_deg: float = 40.0, radius: float = 4.0):
    """n image requests as (scene, cam float32 [18], W, H, arrival s): scene uniform over n_scenes,
    resolution uniform over SERVING_RESOLUTIONS, a camera at a uniform point of the upper hemisphere
    of radius `radius` looking at the origin, Poisson arrivals at `rate` per second (all 0 if None)."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for _ in range(n):
        W, H = SERVING_RESOLUTIONS[int(rng.integers(len(SERVING_RESOLUTIONS)))]
        z = rng.uniform(0.05, 1.0)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        r = math.sqrt(1.0 - z * z)
        c2w = look_at(radius * np.array([r * math.cos(phi), r * math.sin(phi), z]))
        f = 0.5 * W / math.tan(0.5 * math.radians(fov_deg))
        cam = np.concatenate([c2w.reshape(-1), [f, f, 0.5 * W, 0.5 * H, W, H]]).astype(np.float32)
        if rate is not None:
            t += rng.exponential(1.0 / rate)
        out.append((int(rng.integers(n_scenes)), cam, W, H, t))
    return out
