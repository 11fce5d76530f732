// plx_render.cu -- ray generation, the forward march (Eq. 1) and its adjoint.
//
// Parallelisation (sm_103a design): one warp per ray, and the 32 lanes take
// 32 samples of that ray at a time ("chunks"): the samples that lie in cells
// with an occupied corner, compacted in order (see "sample compaction").  Each
// lane does the full trilinear gather of its own sample (8 index reads, 8 x
// 112-byte row reads as float4 vectors), the warp turns per-sample alphas into
// transmittances with a prefix product, and early termination ends the loop at
// chunk granularity.  Compared with one warp per ray and one lane per SH
// coefficient (the design Supp. A.1 describes for a Titan RTX), this cuts the
// serial chain of dependent loads per ray by 32x, which is what bounds a
// 5000-ray batch on a 152-SM part.  Cells with no occupied corner (a bit in
// the grid's occupancy mask) cost one mask read, issued kCand at a time.
//
// Transmittance is the running product T_{s+1} = T_s exp(-sigma_s delta),
// formed per chunk by a warp prefix product (relative error grows like the
// square root of the sample count, independent of the optical depth).  The
// ray parameter and sample coordinates are double-floats (see DF).
#include "plx_internal.cuh"

namespace plx {

// --------------------------------------------------------------------------- rays
__global__ void gen_rays_kernel(const float *__restrict__ cams, int n_cams, int W, int H,
                                const int64_t *__restrict__ pix, int64_t n, float *__restrict__ o,
                                float *__restrict__ d) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t p = pix[r];
    int64_t hw = (int64_t)W * H;
    if (p < 0 || p >= hw * n_cams) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            o[3 * r + i] = 0.0f;
            d[3 * r + i] = 0.0f;
        }
        return;
    }
    int64_t view = p / hw;
    int64_t rem = p - view * hw;
    int v = (int)(rem / W);
    int u = (int)(rem - (int64_t)v * W);
    const float *c = cams + 18 * view;
    // double-float throughout, then one rounding: the result is the FP32 rounding of the
    // exact ray (up to inputs within ~1e-14 of a rounding midpoint)
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
        d[3 * r + i] = q.hi + q.lo;
        o[3 * r + i] = c[4 * i + 3];
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

// --------------------------------------------------------------------------- per-ray setup
struct RaySetup {
    DF A[3];       // origin minus box corner, exact as a double-float
    float d[3];    // unit direction as given
    DF tn, tf;     // clipped parameter range
    float og[3];   // FP32 grid-coordinate origin and direction, for the cheap candidate test
    float dg[3];
    float Y[9];    // SH basis at the direction
    bool hit;
};

__device__ __forceinline__ RaySetup ray_setup(const GridView &g, const float *__restrict__ ro,
                                              const float *__restrict__ rd, int64_t ray) {
    RaySetup rs;
    float o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = __ldg(ro + 3 * ray + a);
        rs.d[a] = __ldg(rd + 3 * ray + a);
    }
    rs.hit = clip_box(g, o, rs.d, rs.tn, rs.tf);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        rs.A[a] = df_two_sum(o[a], -g.lo[a]);
        rs.og[a] = (o[a] - g.lo[a]) * g.inv_h[a];
        rs.dg[a] = rs.d[a] * g.inv_h[a];
    }
    sh_basis(rs.d, rs.Y);
    return rs;
}

// t_s = t_near + s * delta as a double-float (s * delta_hi is exact for s < 2^24).
__device__ __forceinline__ DF sample_t(const RaySetup &rs, const RenderParams &p, int s) {
    DF sd = df_two_prod((float)s, p.delta);
    sd.lo = fmaf((float)s, p.delta_lo, sd.lo);
    return df_add(rs.tn, sd);
}

// Grid coordinates of the point at parameter t: ((o - lo) + t d) / h per axis.
__device__ __forceinline__ void sample_coords(const GridView &g, const RaySetup &rs, DF t, DF gc[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        DF td = df_two_prod(t.hi, rs.d[a]);
        td.lo = fmaf(t.lo, rs.d[a], td.lo);
        gc[a] = df_mul(df_add(rs.A[a], td), DF{g.inv_h[a], g.inv_h_lo[a]});
    }
}

// Read-only vector loads issued as volatile asm: the compiler keeps them in
// program order ahead of their uses instead of sinking each next to its FMAs.
__device__ __forceinline__ float4 ldg4_pinned(const float4 *p) {
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ldg4_pinned(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

// Full sample: interpolated values at grid point gc, whose cell the caller has
// already found occupied (compaction).  rows_out/f_out receive the corners.
__device__ __forceinline__ bool gather_sample(const GridView &g, int form, const DF gc[3], float acc[kNV],
                                              int32_t rows_out[8], float f_out[3]) {
#pragma unroll
    for (int q = 0; q < kNV; ++q) acc[q] = 0.0f;
    Cell c = locate(g, gc);
    f_out[0] = c.f[0];
    f_out[1] = c.f[1];
    f_out[2] = c.f[2];
    int32_t r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = row_of(g, corner_node(g, c.base, k));
    // every corner's row is requested before any is used: one memory round trip per
    // chunk instead of eight (a NULL corner contributes w * 0, i.e. nothing)
    if (form == PLX_SH_F32) {
        float4 v[8][7];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 *p = reinterpret_cast<const float4 *>(g.rows + (int64_t)max(r[k], 0) * kRowF);
#pragma unroll
            for (int q = 0; q < 7; ++q) v[k][q] = r[k] >= 0 ? ldg4_pinned(p + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        // an empty volatile use of every loaded value, after all the loads: no FMA can be
        // scheduled between two loads, so all 56 requests are in flight together
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int q = 0; q < 7; ++q)
                asm volatile("" : "+f"(v[k][q].x), "+f"(v[k][q].y), "+f"(v[k][q].z), "+f"(v[k][q].w));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float w = corner_weight(c.f, k);
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                acc[4 * q + 0] = fmaf(w, v[k][q].x, acc[4 * q + 0]);
                acc[4 * q + 1] = fmaf(w, v[k][q].y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(w, v[k][q].z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(w, v[k][q].w, acc[4 * q + 3]);
            }
        }
    } else {
        uint4 v[8][4];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint4 *p = reinterpret_cast<const uint4 *>(g.rows_h + (int64_t)max(r[k], 0) * kRowH);
#pragma unroll
            for (int q = 0; q < 4; ++q) v[k][q] = r[k] >= 0 ? ldg4_pinned(p + q) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q) asm volatile("" : "+r"(v[k][q].x), "+r"(v[k][q].y), "+r"(v[k][q].z), "+r"(v[k][q].w));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float w = corner_weight(c.f, k);
            const uint32_t wd[16] = {v[k][0].x, v[k][0].y, v[k][0].z, v[k][0].w, v[k][1].x, v[k][1].y,
                                     v[k][1].z, v[k][1].w, v[k][2].x, v[k][2].y, v[k][2].z, v[k][2].w,
                                     v[k][3].x, v[k][3].y, v[k][3].z, v[k][3].w};
            acc[0] = fmaf(w, __uint_as_float(wd[0]), acc[0]);
#pragma unroll
            for (int sh = 0; sh < 27; ++sh) {
                const uint32_t word = wd[1 + (sh >> 1)];
                const uint32_t bits = (sh & 1) ? (word & 0xffff0000u) : (word << 16);
                acc[1 + sh] = fmaf(w, __uint_as_float(bits), acc[1 + sh]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) rows_out[k] = r[k];
    return true;
}

// Density only (backward pass 1 and node counting).  The caller has already
// found the sample's cell occupied (compaction), so the mask is not re-read.
__device__ __forceinline__ float gather_sigma(const GridView &g, int form, const DF gc[3]) {
    Cell c = locate(g, gc);
    int32_t r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = row_of(g, corner_node(g, c.base, k));
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (r[k] >= 0) s = fmaf(corner_weight(c.f, k), row_sigma(g, form, r[k]), s);
    return s;
}

__device__ __forceinline__ void colour_of(const float acc[kNV], const float Y[9], float pre[3], float c[3]) {
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float p = 0.0f;
#pragma unroll
        for (int l = 0; l < 9; ++l) p = fmaf(Y[l], acc[1 + 9 * ch + l], p);
        pre[ch] = p;
        c[ch] = fmaxf(p, 0.0f);
    }
}

// Warp inclusive prefix product (lane order).
__device__ __forceinline__ float warp_incl_prod(float x, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float v = __shfl_up_sync(kFull, x, off);
        if (lane >= off) x *= v;
    }
    return x;
}

// Per-chunk compositing state shared by the kernels: given this lane's
// density, returns alpha, T_s (before the sample), T_{s+1} and whether the
// sample is taken (valid and T_s >= stop); Tc is the transmittance before
// the chunk.  Transmittance is the running product of exp(-sigma delta).
struct Composite {
    float alpha, T, Tn;
    bool take;
    unsigned tmask;
    float chunk_prod;  // product over the taken lanes, to advance Tc
};

__device__ __forceinline__ Composite composite(float sig, bool valid, float Tc, const RenderParams &p, int lane) {
    Composite r;
    r.alpha = -expm1f(-sig * p.delta);
    const float e = 1.0f - r.alpha;
    const float incl = warp_incl_prod(e, lane);
    float excl = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) excl = 1.0f;
    r.T = Tc * excl;
    r.Tn = Tc * incl;
    r.take = valid && r.T >= p.stop;
    r.tmask = __ballot_sync(kFull, r.take);
    const int k = __popc(r.tmask);
    r.chunk_prod = k > 0 ? __shfl_sync(kFull, incl, k - 1) : 1.0f;
    return r;
}

// --------------------------------------------------------------------------- sample compaction
// The candidates (all samples of the ray, in order) are tested against the
// cell occupancy mask, kCand per lane at a time so that many mask loads are in
// flight; samples whose cell has an occupied corner are appended, in order, to
// a per-warp ring buffer in shared memory and processed 32 at a time.  A
// skipped sample lies in a cell whose 8 corners are NULL (all values zero):
// its alpha is exactly 0, it multiplies T by exactly 1 and adds nothing, so
// the compacted march evaluates the same sum.
constexpr int kCand = 8;    // candidates per lane per refill
constexpr int kRing = 512;  // ring capacity >= 31 + 32 kCand, a power of two

struct Cand {
    bool valid, occ;
};

// Is sample s inside the clipped ray (valid), and is its cell non-empty (occ)?
// The answer must equal the double-float one exactly (it decides which samples
// are marched).  Plain FP32 coordinates are within ~3e-4 of a cell of the
// double-float ones (rounding of t_near, delta, the direction and the grid
// scale, for R <= 2048); a candidate whose FP32 coordinate lies within kFaceEps
// of a cell face on any axis, or whose t lies within kTEps of t_far, is
// re-evaluated in double-float, so the cheap path is taken only where both agree.
constexpr float kFaceEps = 2e-3f;

__device__ __forceinline__ Cand test_candidate(const GridView &g, const RaySetup &rs, const RenderParams &p, int s) {
    Cand c;
    c.occ = false;
    c.valid = false;
    if (s >= p.max_chunks * 32) return c;
    const float t32 = fmaf((float)s, p.delta, rs.tn.hi);
    const float kTEps = 1e-5f * (fabsf(rs.tf.hi) + 1.0f);
    bool exact = fabsf(t32 - rs.tf.hi) <= kTEps;
    if (!exact && t32 > rs.tf.hi) return c;  // clearly past t_far
    int b[3];
    const float rm1 = (float)(g.R - 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = fmaf(t32, rs.dg[a], rs.og[a]);
        const float fl = floorf(x);
        exact = exact || (x - fl) < kFaceEps || (fl + 1.0f - x) < kFaceEps || x < kFaceEps || x > rm1 - kFaceEps;
        b[a] = (int)fl;
    }
    if (exact) {
        const DF t = sample_t(rs, p, s);
        c.valid = df_lt(t, rs.tf);
        if (c.valid) {
            DF gc[3];
            sample_coords(g, rs, t, gc);
            c.occ = cell_occupied(g, locate(g, gc).base);
        }
        return c;
    }
    c.valid = true;
    c.occ = cell_occupied(g, ((int64_t)b[0] * g.R + b[1]) * g.R + b[2]);
    return c;
}

struct Stream {
    int next;   // next candidate sample index to test
    int head;   // ring read position (absolute)
    int tail;   // ring write position (absolute)
    bool exhausted;
};

// Append occupied candidates until 32 are queued or the ray has no candidates left.
__device__ __forceinline__ void refill(const GridView &g, const RaySetup &rs, const RenderParams &p, int *ring,
                                       Stream &st, int lane) {
    const unsigned lt = (1u << lane) - 1u;
    while (st.tail - st.head < 32 && !st.exhausted) {
        Cand c[kCand];
#pragma unroll
        for (int j = 0; j < kCand; ++j) c[j] = test_candidate(g, rs, p, st.next + 32 * j + lane);
#pragma unroll
        for (int j = 0; j < kCand; ++j) {
            const unsigned m = __ballot_sync(kFull, c[j].occ);
            if (c[j].occ) ring[(st.tail + __popc(m & lt)) & (kRing - 1)] = st.next + 32 * j + lane;
            st.tail += __popc(m);
        }
        // valid candidates form a prefix of the sample indices
        st.exhausted = __ballot_sync(kFull, c[kCand - 1].valid) != kFull;
        st.next += 32 * kCand;
    }
    __syncwarp();
}

// Take the next (up to) 32 queued samples: returns the count; lane i gets sample s (if i < count).
__device__ __forceinline__ int take_chunk(const int *ring, Stream &st, int lane, int &s) {
    const int cnt = min(st.tail - st.head, 32);
    s = lane < cnt ? ring[(st.head + lane) & (kRing - 1)] : 0;
    st.head += cnt;
    __syncwarp();
    return cnt;
}

// The occupied samples with index in [first, end), in order, into buf (at most 32 are kept).
__device__ __forceinline__ int scan_range(const GridView &g, const RaySetup &rs, const RenderParams &p, int first,
                                          int end, int *buf, int lane) {
    const unsigned lt = (1u << lane) - 1u;
    int cnt = 0;
    for (int base = first; base < end; base += 32 * kCand) {
        Cand c[kCand];
#pragma unroll
        for (int j = 0; j < kCand; ++j) {
            const int s = base + 32 * j + lane;
            if (s < end) {
                c[j] = test_candidate(g, rs, p, s);
            } else {
                c[j].valid = c[j].occ = false;
            }
        }
#pragma unroll
        for (int j = 0; j < kCand; ++j) {
            const unsigned m = __ballot_sync(kFull, c[j].occ);
            const int pos = cnt + __popc(m & lt);
            if (c[j].occ && pos < 32) buf[pos] = base + 32 * j + lane;
            cnt += __popc(m);
        }
    }
    __syncwarp();
    return cnt;
}

// --------------------------------------------------------------------------- forward
// Four resident 4-warp CTAs per SM: up to 128 registers a thread, enough for the
// gather to keep most of a chunk's row loads in flight (measured on the 512^3
// training batch against 2 and 3 CTAs, which buy more registers but fewer warps).
constexpr int kGatherBlocks = 4;
constexpr int kFwdWarps = 4;

template <int FORM>
__global__ void __launch_bounds__(kFwdWarps * 32, kGatherBlocks) render_fwd_kernel(GridView g, const float *__restrict__ ro,
                                                                    const float *__restrict__ rd, int64_t n,
                                                                    RenderParams p, float *__restrict__ rgb,
                                                                    float *__restrict__ T_out) {
    __shared__ int s_ring[kFwdWarps][kRing];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t ray = (int64_t)blockIdx.x * kFwdWarps + wid;
    if (ray >= n) return;  // uniform per warp
    const RaySetup rs = ray_setup(g, ro, rd, ray);
    float C[3] = {0.0f, 0.0f, 0.0f};
    float Tc = 1.0f;  // transmittance before the current chunk
    if (rs.hit) {
        int *ring = s_ring[wid];
        Stream st = {0, 0, 0, false};
        for (;;) {
            refill(g, rs, p, ring, st, lane);
            int s;
            const int cnt = take_chunk(ring, st, lane, s);
            if (cnt == 0) break;
            const bool valid = lane < cnt;
            float sig = 0.0f, col[3] = {0.0f, 0.0f, 0.0f};
            if (valid) {
                DF gc[3];
                sample_coords(g, rs, sample_t(rs, p, s), gc);
                float acc[kNV];
                int32_t rr[8];
                float ff[3];
                if (gather_sample(g, FORM, gc, acc, rr, ff)) {
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
    if (lane == 0) {
        rgb[3 * ray + 0] = fmaf(Tc, p.bg[0], C[0]);
        rgb[3 * ray + 1] = fmaf(Tc, p.bg[1], C[1]);
        rgb[3 * ray + 2] = fmaf(Tc, p.bg[2], C[2]);
        if (T_out) T_out[ray] = Tc;
    }
}

cudaError_t launch_render(const GridView &g, const float *o, const float *d, int64_t n,
                          const RenderParams &p, float *rgb, float *T_end, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n + kFwdWarps - 1) / kFwdWarps;
    if (g.form == PLX_SH_F32)
        render_fwd_kernel<PLX_SH_F32><<<(unsigned)blocks, kFwdWarps * 32, 0, s>>>(g, o, d, n, p, rgb, T_end);
    else
        render_fwd_kernel<PLX_SH_BF16><<<(unsigned)blocks, kFwdWarps * 32, 0, s>>>(g, o, d, n, p, rgb, T_end);
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
    const RaySetup rs = ray_setup(g, ro, rd, ray);
    if (!rs.hit) return;
    for (int q = lane; q < kMaxChunks / 32; q += 32) s_live[wid][q] = 0u;
    __syncwarp();
    int *ring = s_ring[wid];

    // ---- pass 1: density-only forward march over the compacted samples
    float Tc = 1.0f;
    int n_chunks = 0;
    {
        Stream st = {0, 0, 0, false};
        for (;;) {
            refill(g, rs, p, ring, st, lane);
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
                sample_coords(g, rs, sample_t(rs, p, s), gc);
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
        const int cnt = scan_range(g, rs, p, s_first[wid][chunk], s_first[wid][chunk + 1], ring, lane);
        const bool valid = lane < min(cnt, 32);
        const int s = valid ? ring[lane] : 0;
        __syncwarp();
        float acc[kNV];
        int32_t rr[8];
        float ff[3];
        float sig = 0.0f, pre[3] = {0.0f, 0.0f, 0.0f}, col[3] = {0.0f, 0.0f, 0.0f};
        bool occupied = false;
        if (valid) {
            DF gc[3];
            sample_coords(g, rs, sample_t(rs, p, s), gc);
            occupied = gather_sample(g, FORM, gc, acc, rr, ff);
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
        if (take && occupied && sig > 0.0f) {
            // per-sample gradients w.r.t. the interpolated values
            float gsig = 0.0f;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) gsig = fmaf(gr[ch], cp.Tn * col[ch] - Rs[ch], gsig);
            gsig *= p.delta;
            float gpre[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) gpre[ch] = pre[ch] > 0.0f ? gr[ch] * w : 0.0f;
            // scatter to corners
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (rr[k] < 0) continue;
                const float wk = corner_weight(ff, k);
                if (wk == 0.0f) continue;
                float v[kNV];
                v[0] = wk * gsig;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float gw = wk * gpre[ch];
#pragma unroll
                    for (int l = 0; l < 9; ++l) v[1 + 9 * ch + l] = gw * rs.Y[l];
                }
                float4 *dst = reinterpret_cast<float4 *>(grad_rows + (int64_t)rr[k] * kRowF);
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    atomicAdd(dst + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
                mark_touched(g, rr[k]);
            }
        }
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
// occupied corner (each costs an index read) and how many of them are
// occupied (each costs a row read).  The cells sharing a node form a
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
    const RaySetup rs = ray_setup(g, ro, rd, ray);
    int64_t nodes = 0, occ_nodes = 0;
    if (rs.hit) {
        int *ring = s_ring[wid];
        Stream st = {0, 0, 0, false};
        float Tc = 1.0f;
        int64_t carry = -1;  // cell of the last sample of the previous chunk
        for (;;) {
            refill(g, rs, p, ring, st, lane);
            int s;
            const int cnt = take_chunk(ring, st, lane, s);
            if (cnt == 0) break;
            const bool valid = lane < cnt;
            float sig = 0.0f;
            int64_t cell = -1;
            if (valid) {
                DF gc[3];
                sample_coords(g, rs, sample_t(rs, p, s), gc);
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
        out[2 * ray] = nodes;
        out[2 * ray + 1] = occ_nodes;
    }
}

cudaError_t launch_count_nodes(const GridView &g, const float *o, const float *d, int64_t n, const RenderParams &p,
                               int64_t *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    count_nodes_kernel<<<(unsigned)((n + kFwdWarps - 1) / kFwdWarps), kFwdWarps * 32, 0, s>>>(g, o, d, n, p, out);
    return cudaGetLastError();
}

}  // namespace plx
