// plx_render.cu -- ray generation, the forward march (Eq. 1) and its adjoint.
//
// Parallelisation (sm_103a design): one warp per ray, and the 32 lanes take
// 32 samples of that ray at a time ("chunks"): the samples that lie in cells
// with an occupied corner, compacted in order (see "sample compaction").  Each
// lane does the full trilinear gather of its own sample (8 index reads, 8 x
// 112-byte row reads as float4 vectors), the warp turns per-sample alphas into
// transmittances with a prefix product, and early termination ends the loop at
// chunk granularity.  Compared with one warp per ray and one lane per SH
// coefficient (the design Supp. B.1 describes for a Titan RTX), this cuts the
// serial chain of dependent loads per ray by 32x, which is what bounds a
// 5000-ray batch on a 152-SM part.  Cells with no occupied corner (a bit in
// the grid's occupancy mask) cost one mask read, issued kCand at a time.
//
// Transmittance is the running product T_{s+1} = T_s exp(-sigma_s delta),
// formed per chunk by a warp prefix product (relative error grows like the
// square root of the sample count, independent of the optical depth).  The
// ray parameter and sample coordinates are double-floats (see DF).
#include <cstring>

#include "plx_march.cuh"

namespace plx {

// --------------------------------------------------------------------------- rays
// The pixel-centre ray of pixel (u, v) of camera c (float [18]: c2w 3x4, fx, fy, cx, cy, W, H),
// camera looking down -z with y up: d = normalize(R ((u + 1/2 - cx)/fx, -(v + 1/2 - cy)/fy, -1)),
// o = the camera centre.  Double-float throughout, then one rounding: d is the FP32 rounding of
// the exact direction (up to inputs within ~1e-14 of a rounding midpoint).
__device__ __forceinline__ void pixel_ray(const float *__restrict__ c, int u, int v, float o[3], float d[3]) {
    const DF dc0 = df_div(df_two_sum((float)u + 0.5f, -c[14]), c[12]);
    DF dc1 = df_div(df_two_sum((float)v + 0.5f, -c[15]), c[13]);
    dc1.hi = -dc1.hi;
    dc1.lo = -dc1.lo;
    DF dw[3];
    DF len2 = {0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dw[i] = df_add(df_add(df_mul_f(dc0, c[4 * i + 0]), df_mul_f(dc1, c[4 * i + 1])), DF{-c[4 * i + 2], 0.0f});
        len2 = df_add(len2, df_mul(dw[i], dw[i]));
    }
    const DF len = df_sqrt(len2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const DF q = df_div_df(dw[i], len);
        d[i] = q.hi + q.lo;
        o[i] = c[4 * i + 3];
    }
}

__global__ void gen_rays_kernel(const float *__restrict__ cams, int n_cams, int W, int H,
                                const int64_t *__restrict__ pix, int64_t n, float *__restrict__ o,
                                float *__restrict__ d) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t p = pix[r];
    int64_t hw = (int64_t)W * H;
    float oo[3] = {0.0f, 0.0f, 0.0f}, dd[3] = {0.0f, 0.0f, 0.0f};
    if (p >= 0 && p < hw * n_cams) {
        const int64_t view = p / hw;
        const int64_t rem = p - view * hw;
        const int v = (int)(rem / W);
        const int u = (int)(rem - (int64_t)v * W);
        pixel_ray(cams + 18 * view, u, v, oo, dd);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o[3 * r + i] = oo[i];
        d[3 * r + i] = dd[i];
    }
}

cudaError_t launch_gen_rays(const float *cams, int n_cams, int W, int H, const int64_t *pix, int64_t n,
                            float *o, float *d, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    gen_rays_kernel<<<(unsigned)blocks, threads, 0, s>>>(cams, n_cams, W, H, pix, n, o, d);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- MSE
__global__ void mse_grad_kernel(const float *__restrict__ rgb, const float *__restrict__ target, int64_t n3,
                                float inv_n, float *__restrict__ grad, float *__restrict__ loss) {
    float acc = 0.0f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
        const float diff = rgb[e] - target[e];
        grad[e] = 2.0f * diff * inv_n;
        acc = fmaf(diff, diff, acc);
    }
    if (loss) {
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0 && acc != 0.0f) atomicAdd(loss, acc * inv_n);
    }
}

cudaError_t launch_mse_grad(const float *rgb, const float *target, int64_t n, float *grad, float *loss,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t n3 = 3 * n;
    int64_t blocks = (n3 + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    mse_grad_kernel<<<(unsigned)blocks, 256, 0, s>>>(rgb, target, n3, (float)(1.0 / (double)n), grad, loss);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- forward
constexpr int kFwdWarps = 4;
// Resident warps per SM the one-warp-per-ray render kernels are compiled for, per row form: the
// register cap it implies trades a few spilled bytes for more warps to hide the gathers' latency.
constexpr int kFwdWarpsSMF32 = 24;
constexpr int kFwdWarpsSMBF16 = 24;
constexpr int fwd_blocks(int form) { return (form == PLX_SH_BF16 ? kFwdWarpsSMBF16 : kFwdWarpsSMF32) / kFwdWarps; }
// Rays per warp in the render kernels: the rays are set up in parallel, a lane each (double-float clip
// and anchor, SH basis, candidate range; in plx_render by the CTA's first warp for all its rays, in the
// tiles kernel by lanes 0 .. kRayBatch-1 of each warp) into shared memory, and each warp then marches its
// kRayBatch rays one after another, so the setup's cost is shared instead of repeated in every lane of
// every ray's warp.
constexpr int kRayBatch = 4;
// The CTA's kFwdWarps * kRayBatch consecutive rays are dealt to its warps in turn (ray r of warp w is the
// CTA's ray r kFwdWarps + w), so that neighbouring rays, which cost about the same, are spread over the
// warps and the CTA's warps finish together.
constexpr bool kDealRays = true;
static_assert(kDealRays && kFwdWarps * kRayBatch <= 32, "render_fwd_kernel's first warp sets up the CTA's rays");
__device__ __forceinline__ int64_t batch_ray(int64_t cta_ray0, int wid, int r) {
    return cta_ray0 + (kDealRays ? (int64_t)r * kFwdWarps + wid : (int64_t)wid * kRayBatch + r);
}

// The forward march of one ray by one warp (Eq. 1 over the compacted samples, chunk by chunk):
// returns, in every lane, the composited colour without the background and the final
// transmittance.  ring: this warp's kRing ints of shared memory.
template <int FORM>
__device__ __forceinline__ void march_forward(const GridView &g, const RenderParams &p, const RaySetup &rs, int *ring,
                                              int lane, float C[3], float &Tc) {
    C[0] = C[1] = C[2] = 0.0f;
    Tc = 1.0f;  // transmittance before the current chunk
    if (rs.hit > 0) {
        Stream st = {rs.s_lo, rs.s_lo, rs.s_lo, false};
        for (;;) {
            refill(g, rs, ring, st, lane);
            int s;
            const int cnt = take_chunk(ring, st, lane, s);
            if (cnt == 0) break;
            const bool valid = lane < cnt;
            float sig = 0.0f, col[3] = {0.0f, 0.0f, 0.0f};
            if (valid) {
                DF gc[3];
                coords_at(rs, s, gc);
                float acc[kNV];
                int32_t rr[8];
                float ff[3];
                if (gather_sample<true>(g, FORM, gc, acc, rr, ff)) {
                    sig = fmaxf(acc[0], 0.0f);
                    float pre[3];
                    colour_of(acc, rs.Y, pre, col);
                }
            }
            const Composite cp = composite(sig, valid, Tc, p, lane);
            if (cp.take) {
                const float w = cp.T * cp.alpha;
                C[0] = fmaf(w, col[0], C[0]);
                C[1] = fmaf(w, col[1], C[1]);
                C[2] = fmaf(w, col[2], C[2]);
            }
            Tc *= cp.chunk_prod;
            if (cp.tmask != __ballot_sync(kFull, valid)) break;  // T fell below stop_thresh
        }
    }
    C[0] = warp_sum(C[0]);
    C[1] = warp_sum(C[1]);
    C[2] = warp_sum(C[2]);
}

template <int FORM>
__global__ void __launch_bounds__(kFwdWarps * 32, fwd_blocks(FORM)) render_fwd_kernel(GridView g, const float *__restrict__ ro,
                                                                    const float *__restrict__ rd, int64_t n,
                                                                    RenderParams p, float *__restrict__ rgb,
                                                                    float *__restrict__ T_out) {
    __shared__ int s_ring[kFwdWarps][kRing];
    __shared__ RaySetup s_rs[kFwdWarps][kRayBatch];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t cta_ray0 = (int64_t)blockIdx.x * kFwdWarps * kRayBatch;
    // the first warp sets up all of the CTA's rays, a lane each (one pass of the setup's instructions for
    // kFwdWarps * kRayBatch rays instead of one per warp)
    if (wid == 0 && lane < kFwdWarps * kRayBatch) {
        const int64_t ray = cta_ray0 + lane;  // = batch_ray(cta_ray0, lane % kFwdWarps, lane / kFwdWarps)
        if (ray < n) s_rs[lane % kFwdWarps][lane / kFwdWarps] = ray_setup(g, p, ro, rd, ray);
    }
    __syncthreads();
    for (int r = 0; r < kRayBatch; ++r) {
        const int64_t ray = batch_ray(cta_ray0, wid, r);
        if (ray >= n) break;  // uniform per warp
        float C[3], Tc;
        march_forward<FORM>(g, p, s_rs[wid][r], s_ring[wid], lane, C, Tc);
        if (lane == 0) {
            rgb[3 * ray + 0] = fmaf(Tc, p.bg[0], C[0]);
            rgb[3 * ray + 1] = fmaf(Tc, p.bg[1], C[1]);
            rgb[3 * ray + 2] = fmaf(Tc, p.bg[2], C[2]);
            if (T_out) T_out[ray] = Tc;
        }
    }
}

cudaError_t launch_render(const GridView &g, const float *o, const float *d, int64_t n,
                          const RenderParams &p, float *rgb, float *T_end, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t per_block = (int64_t)kFwdWarps * kRayBatch;
    const int64_t blocks = (n + per_block - 1) / per_block;
    if (g.form == PLX_SH_F32)
        render_fwd_kernel<PLX_SH_F32><<<(unsigned)blocks, kFwdWarps * 32, 0, s>>>(g, o, d, n, p, rgb, T_end);
    else
        render_fwd_kernel<PLX_SH_BF16><<<(unsigned)blocks, kFwdWarps * 32, 0, s>>>(g, o, d, n, p, rgb, T_end);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- serving
// plx_render_tiles: image requests of several resident scenes in one launch.
// Each tile is 16x16 pixels of one request; ray w of the launch is pixel (w mod 256)
// of tile w / 256.  Each warp takes kRayBatch consecutive rays: its lanes generate
// them in-kernel with the same code as plx_gen_rays and set them up, and the warp
// marches them with the same code as plx_render, so a pixel's value does not
// depend on what else is in the launch.
struct SceneTable {
    GridView g[PLX_TILES_MAX_SCENES];
    RenderParams p[PLX_TILES_MAX_SCENES];
};

template <int FORM>
__global__ void __launch_bounds__(kFwdWarps * 32, fwd_blocks(FORM)) render_tiles_kernel(
    const __grid_constant__ SceneTable tab, int n_scenes, const float *__restrict__ cams, int n_cams,
    const plx_tile *__restrict__ tiles, int64_t n_rays) {
    __shared__ int s_ring[kFwdWarps][kRing];
    __shared__ RaySetup s_rs[kFwdWarps][kRayBatch];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t cta_ray0 = (int64_t)blockIdx.x * kFwdWarps * kRayBatch;
    const int64_t my_ray = batch_ray(cta_ray0, wid, lane);
    if (lane < kRayBatch && my_ray < n_rays) {
        const int64_t ray = my_ray;
        const plx_tile tile = tiles[ray / (PLX_TILE_W * PLX_TILE_H)];
        const int px = (int)(ray % (PLX_TILE_W * PLX_TILE_H));
        const int x = tile.x0 + px % PLX_TILE_W;
        const int y = tile.y0 + px / PLX_TILE_W;
        RaySetup &rs = s_rs[wid][lane];
        if (x < 0 || y < 0 || x >= tile.W || y >= tile.H) {  // a tile over the image's edge
            rs.hit = -1;
        } else if (tile.scene < 0 || tile.scene >= n_scenes || tile.camera < 0 || tile.camera >= n_cams ||
                   !tile.d_rgb) {
            report(tab.g[0].status, kDevBadTile);
            rs.hit = -1;
        } else {
            float o[3], d[3];
            pixel_ray(cams + 18 * (int64_t)tile.camera, x, y, o, d);
            rs = ray_setup_od(tab.g[tile.scene], tab.p[tile.scene], o, d);
        }
    }
    __syncwarp();
    for (int r = 0; r < kRayBatch; ++r) {
        const int64_t ray = batch_ray(cta_ray0, wid, r);
        if (ray >= n_rays) break;            // uniform per warp
        if (s_rs[wid][r].hit < 0) continue;  // uniform
        const plx_tile tile = tiles[ray / (PLX_TILE_W * PLX_TILE_H)];
        const int px = (int)(ray % (PLX_TILE_W * PLX_TILE_H));
        const int x = tile.x0 + px % PLX_TILE_W;
        const int y = tile.y0 + px / PLX_TILE_W;
        const GridView &g = tab.g[tile.scene];
        const RenderParams &p = tab.p[tile.scene];
        float C[3], Tc;
        march_forward<FORM>(g, p, s_rs[wid][r], s_ring[wid], lane, C, Tc);
        if (lane == 0) {
            float *out = tile.d_rgb + ((int64_t)y * tile.W + x) * 3;
            out[0] = fmaf(Tc, p.bg[0], C[0]);
            out[1] = fmaf(Tc, p.bg[1], C[1]);
            out[2] = fmaf(Tc, p.bg[2], C[2]);
        }
    }
}

cudaError_t launch_render_tiles(const GridView *g, const RenderParams *p, int n_scenes, const float *cams,
                                int n_cams, const plx_tile *tiles, int64_t n_tiles, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    SceneTable tab;
    memset(&tab, 0, sizeof(tab));
    for (int i = 0; i < n_scenes; ++i) {
        tab.g[i] = g[i];
        tab.p[i] = p[i];
    }
    const int64_t n_rays = n_tiles * PLX_TILE_W * PLX_TILE_H;
    const int64_t per_block = (int64_t)kFwdWarps * kRayBatch;
    const int64_t blocks = (n_rays + per_block - 1) / per_block;
    if (g[0].form == PLX_SH_F32)
        render_tiles_kernel<PLX_SH_F32><<<(unsigned)blocks, kFwdWarps * 32, 0, s>>>(tab, n_scenes, cams, n_cams, tiles,
                                                                                     n_rays);
    else
        render_tiles_kernel<PLX_SH_BF16><<<(unsigned)blocks, kFwdWarps * 32, 0, s>>>(tab, n_scenes, cams, n_cams, tiles,
                                                                                      n_rays);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- backward
// Pass 1 marches forward on density alone over the compacted samples,
// recording for every chunk its transmittance at the start, its first sample
// index and whether it holds any positive density.  Pass 2 walks the chunks in
// reverse, re-deriving each chunk's samples from its index range, so the
// remaining colour R_s = sum_{j>s} w_j c_j + T_end bg is an explicit suffix sum
// (no cancellation against the forward colour); it recomputes each sample's
// full gather and scatters its 28 gradients to the 8 corners with float4
// atomics.  Samples with sigma_pre <= 0 have alpha = 0 and a masked density
// gradient, so they contribute nothing and are skipped.
constexpr int kBwdWarps = 4;
constexpr int kMaxChunks = 256;  // 8192 samples per ray

template <int FORM>
__global__ void __launch_bounds__(kBwdWarps * 32, kGatherBlocks) render_bwd_kernel(GridView g, const float *__restrict__ ro,
                                                                    const float *__restrict__ rd, int64_t n,
                                                                    RenderParams p,
                                                                    const float *__restrict__ grad_rgb,
                                                                    float *__restrict__ grad_rows) {
    __shared__ float s_T[kBwdWarps][kMaxChunks];
    __shared__ int s_first[kBwdWarps][kMaxChunks + 1];
    __shared__ uint32_t s_live[kBwdWarps][kMaxChunks / 32];
    __shared__ int s_ring[kBwdWarps][kRing];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t ray = (int64_t)blockIdx.x * kBwdWarps + wid;
    if (ray >= n) return;
    const RaySetup rs = ray_setup(g, p, ro, rd, ray);
    if (rs.hit <= 0) return;
    for (int q = lane; q < kMaxChunks / 32; q += 32) s_live[wid][q] = 0u;
    __syncwarp();
    int *ring = s_ring[wid];

    // ---- pass 1: density-only forward march over the compacted samples
    float Tc = 1.0f;
    int n_chunks = 0;
    {
        Stream st = {rs.s_lo, rs.s_lo, rs.s_lo, false};
        for (;;) {
            refill(g, rs, ring, st, lane);
            int s;
            const int cnt = take_chunk(ring, st, lane, s);
            if (cnt == 0) break;
            if (n_chunks >= p.max_chunks || n_chunks >= kMaxChunks) {  // cannot happen for a clipped ray
                if (lane == 0) report(g.status, kDevTooManySamples);
                return;
            }
            const bool valid = lane < cnt;
            float sig = 0.0f;
            if (valid) {
                DF gc[3];
                coords_at(rs, s, gc);
                sig = fmaxf(gather_sigma(g, FORM, gc), 0.0f);
            }
            const Composite cp = composite(sig, valid, Tc, p, lane);
            const unsigned lmask = __ballot_sync(kFull, cp.take && sig > 0.0f);
            const int last = __shfl_sync(kFull, s, cnt - 1);
            if (lane == 0) {
                s_T[wid][n_chunks] = Tc;
                s_first[wid][n_chunks] = s;
                s_first[wid][n_chunks + 1] = last + 1;
                if (lmask) s_live[wid][n_chunks >> 5] |= 1u << (n_chunks & 31);
            }
            ++n_chunks;
            Tc *= cp.chunk_prod;
            if (cp.tmask != __ballot_sync(kFull, valid)) break;
        }
    }
    __syncwarp();
    const float gr[3] = {__ldg(grad_rgb + 3 * ray), __ldg(grad_rgb + 3 * ray + 1), __ldg(grad_rgb + 3 * ray + 2)};
    float Rsuf[3] = {Tc * p.bg[0], Tc * p.bg[1], Tc * p.bg[2]};

    // ---- pass 2: reverse over chunks
    for (int chunk = n_chunks - 1; chunk >= 0; --chunk) {
        if (!((s_live[wid][chunk >> 5] >> (chunk & 31)) & 1u)) continue;  // uniform: no density, no gradient
        const int cnt = scan_range(g, rs, s_first[wid][chunk], s_first[wid][chunk + 1], ring, lane);
        const bool valid = lane < min(cnt, 32);
        const int s = valid ? ring[lane] : 0;
        __syncwarp();
        float acc[kNV];
        int32_t rr[8];
        float ff[3];
        int64_t cell = -1;
        float sig = 0.0f, pre[3] = {0.0f, 0.0f, 0.0f}, col[3] = {0.0f, 0.0f, 0.0f};
        bool occupied = false;
        if (valid) {
            DF gc[3];
            coords_at(rs, s, gc);
            occupied = gather_sample(g, FORM, gc, acc, rr, ff, &cell);
            if (occupied) {
                sig = fmaxf(acc[0], 0.0f);
                colour_of(acc, rs.Y, pre, col);
            }
        }
        const Composite cp = composite(sig, valid, s_T[wid][chunk], p, lane);
        const bool take = cp.take;
        const float w = take ? cp.T * cp.alpha : 0.0f;
        float Rs[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float wc = w * col[ch];
            const float suf = warp_incl_suffix(wc, lane);
            float suf_ex = __shfl_down_sync(kFull, suf, 1);
            if (lane == 31) suf_ex = 0.0f;
            Rs[ch] = Rsuf[ch] + suf_ex;
            Rsuf[ch] += __shfl_sync(kFull, suf, 0);
        }
        const float gprior = sparsity_prior(p, take && occupied, sig);
        scatter_chunk(g, take && occupied && sig > 0.0f, cell, rr, ff, rs.Y, gr, pre, col, w, cp.Tn, Rs, p.delta,
                      gprior, grad_rows, lane);
    }
}

cudaError_t launch_render_backward(const GridView &g, const float *o, const float *d, int64_t n,
                                   const RenderParams &p, const float *grad_rgb, float *grad_rows,
                                   cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (p.max_chunks > kMaxChunks) return cudaErrorInvalidValue;
    const int64_t blocks = (n + kBwdWarps - 1) / kBwdWarps;
    if (g.form == PLX_SH_F32)
        render_bwd_kernel<PLX_SH_F32><<<(unsigned)blocks, kBwdWarps * 32, 0, s>>>(g, o, d, n, p, grad_rgb, grad_rows);
    else
        render_bwd_kernel<PLX_SH_BF16><<<(unsigned)blocks, kBwdWarps * 32, 0, s>>>(g, o, d, n, p, grad_rgb, grad_rows);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- node counting
// Algorithmic-traffic accounting for the forward march: per ray, the number of
// distinct lattice nodes that are corners of sampled cells with at least one
// occupied corner (each costs an index read), how many of them are occupied
// (each costs a row read), and how many samples are marched.  The cells sharing a node form a
// contiguous run along the ray, so a node is counted at the first such cell,
// i.e. unless it is also a corner of the previous non-empty sampled cell.
// Exact for occupied nodes (every cell around one is non-empty); an empty node
// whose run is interrupted by an all-empty cell may be counted twice (4 bytes).
__device__ __forceinline__ bool is_corner_of(int64_t node, int64_t base, int64_t R) {
    if (base < 0) return false;
    const int64_t ni = node / (R * R), nj = (node / R) % R, nk = node % R;
    const int64_t bi = base / (R * R), bj = (base / R) % R, bk = base % R;
    return ni - bi >= 0 && ni - bi <= 1 && nj - bj >= 0 && nj - bj <= 1 && nk - bk >= 0 && nk - bk <= 1;
}

__global__ void __launch_bounds__(kFwdWarps * 32) count_nodes_kernel(GridView g, const float *__restrict__ ro,
                                                                     const float *__restrict__ rd, int64_t n,
                                                                     RenderParams p, int64_t *__restrict__ out) {
    __shared__ int s_ring[kFwdWarps][kRing];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t ray = (int64_t)blockIdx.x * kFwdWarps + wid;
    if (ray >= n) return;
    const RaySetup rs = ray_setup(g, p, ro, rd, ray);
    int64_t nodes = 0, occ_nodes = 0, samples = 0;  // samples: uniform over the warp
    if (rs.hit > 0) {
        int *ring = s_ring[wid];
        Stream st = {rs.s_lo, rs.s_lo, rs.s_lo, false};
        float Tc = 1.0f;
        int64_t carry = -1;  // cell of the last sample of the previous chunk
        for (;;) {
            refill(g, rs, ring, st, lane);
            int s;
            const int cnt = take_chunk(ring, st, lane, s);
            if (cnt == 0) break;
            const bool valid = lane < cnt;
            float sig = 0.0f;
            int64_t cell = -1;
            if (valid) {
                DF gc[3];
                coords_at(rs, s, gc);
                cell = locate(g, gc).base;
                sig = fmaxf(gather_sigma(g, g.form, gc), 0.0f);
            }
            const Composite cp = composite(sig, valid, Tc, p, lane);
            int64_t prev = __shfl_up_sync(kFull, cell, 1);
            if (lane == 0) prev = carry;
            if (cp.take && cell != prev) {
                for (int c = 0; c < 8; ++c) {
                    const int64_t node = corner_node(g, cell, c);
                    if (is_corner_of(node, prev, g.R)) continue;
                    ++nodes;
                    if (__ldg(g.idx + node) >= 0) ++occ_nodes;
                }
            }
            const int k = __popc(cp.tmask);
            if (k > 0) carry = __shfl_sync(kFull, cell, k - 1);
            samples += k;
            Tc *= cp.chunk_prod;
            if (cp.tmask != __ballot_sync(kFull, valid)) break;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        nodes += __shfl_xor_sync(kFull, nodes, off);
        occ_nodes += __shfl_xor_sync(kFull, occ_nodes, off);
    }
    if (lane == 0) {
        out[3 * ray] = nodes;
        out[3 * ray + 1] = occ_nodes;
        out[3 * ray + 2] = samples;
    }
}

cudaError_t launch_count_nodes(const GridView &g, const float *o, const float *d, int64_t n, const RenderParams &p,
                               int64_t *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    count_nodes_kernel<<<(unsigned)((n + kFwdWarps - 1) / kFwdWarps), kFwdWarps * 32, 0, s>>>(g, o, d, n, p, out);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- weight-threshold prune key
// plx_max_weight: over the given rays, the largest weight T_s alpha_s of the samples
// crediting each row (Sec. 3.4, weight-threshold pruning).  A sample credits the 8
// corner nodes of its cell, the nodes its values come from, whatever their
// trilinear weights; NULL corners have no row.  The march, its samples and its
// weights are those of plx_render (samples in all-empty cells have weight 0 and
// credit no row, so compaction changes nothing).  Weights are positive floats,
// whose order is their bit patterns' order as unsigned integers: the maximum is
// an unsigned atomicMax, issued only when the weight beats the value in L2.
__global__ void __launch_bounds__(kFwdWarps * 32) max_weight_kernel(GridView g, const float *__restrict__ ro,
                                                                    const float *__restrict__ rd, int64_t n,
                                                                    RenderParams p, float *__restrict__ wmax) {
    __shared__ int s_ring[kFwdWarps][kRing];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t ray = (int64_t)blockIdx.x * kFwdWarps + wid;
    if (ray >= n) return;  // uniform per warp
    const RaySetup rs = ray_setup(g, p, ro, rd, ray);
    if (rs.hit <= 0) return;   // uniform per warp
    int *ring = s_ring[wid];
    Stream st = {rs.s_lo, rs.s_lo, rs.s_lo, false};
    float Tc = 1.0f;
    for (;;) {
        refill(g, rs, ring, st, lane);
        int s;
        const int cnt = take_chunk(ring, st, lane, s);
        if (cnt == 0) break;
        const bool valid = lane < cnt;
        float sig = 0.0f;
        int32_t r[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = -1;
        if (valid) {
            DF gc[3];
            coords_at(rs, s, gc);
            const Cell c = locate(g, gc);
#pragma unroll
            for (int k = 0; k < 8; ++k) r[k] = row_of(g, corner_node(g, c.base, k));
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (r[k] >= 0) acc = fmaf(corner_weight(c.f, k), row_sigma(g, g.form, r[k]), acc);
            sig = fmaxf(acc, 0.0f);
        }
        const Composite cp = composite(sig, valid, Tc, p, lane);
        const float w = cp.T * cp.alpha;
        if (cp.take && w > 0.0f) {
            const unsigned wb = __float_as_uint(w);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (r[k] < 0) continue;
                unsigned *a = reinterpret_cast<unsigned *>(wmax + r[k]);
                if (wb > __ldcg(a)) atomicMax(a, wb);
            }
        }
        Tc *= cp.chunk_prod;
        if (cp.tmask != __ballot_sync(kFull, valid)) break;  // T fell below stop_thresh
    }
}

cudaError_t launch_max_weight(const GridView &g, const float *o, const float *d, int64_t n, const RenderParams &p,
                              float *wmax, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    max_weight_kernel<<<(unsigned)((n + kFwdWarps - 1) / kFwdWarps), kFwdWarps * 32, 0, s>>>(g, o, d, n, p, wmax);
    return cudaGetLastError();
}

}  // namespace plx
