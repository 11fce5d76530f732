// plx_optim.cu -- the kernels around the renderer: the cell-occupancy mask
// used for empty-space skipping, BF16-SH packing, the total-variation gradient
// (Sec. 3.4, Supp. A.1) and the RMSProp update (Sec. 3.4).
#include "plx_internal.cuh"

namespace plx {

// --------------------------------------------------------------------------- occupancy
// Bit n of `occ` is 1 iff node n is the (0,0,0) corner of a cell (i,j,k < R-1)
// with at least one occupied corner.  One warp writes one 32-bit word.
__global__ void build_occupancy_kernel(GridView g, uint32_t *__restrict__ occ, int64_t n_words) {
    const int lane = threadIdx.x & 31;
    const int64_t R = g.R;
    const int64_t N = R * R * R;
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n_words;
         w += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int64_t n = w * 32 + lane;
        bool any = false;
        if (n < N) {
            const int64_t i = n / (R * R), j = (n / R) % R, k = n % R;
            if (i < R - 1 && j < R - 1 && k < R - 1) {
#pragma unroll
                for (int c = 0; c < 8; ++c) any = any || (__ldg(g.idx + corner_node(g, n, c)) >= 0);
            }
        }
        const unsigned word = __ballot_sync(kFull, any);
        if (lane == 0) occ[w] = word;
    }
}

cudaError_t launch_build_occupancy(const GridView &g, uint32_t *occ, cudaStream_t s) {
    const int64_t R = g.R;
    const int64_t n_words = (R * R * R + 31) / 32;
    const int threads = 256;
    int64_t blocks = (n_words + 7) / 8;
    if (blocks > 152 * 64) blocks = 152 * 64;
    build_occupancy_kernel<<<(unsigned)blocks, threads, 0, s>>>(g, occ, n_words);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- BF16 packing
__device__ __forceinline__ uint16_t bf16_bits_rn(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// One warp per row: lane l writes slot l of the 32-slot BF16 row.
__global__ void pack_bf16_kernel(const float *__restrict__ rows, uint16_t *__restrict__ rows_h, int64_t M) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < M;
         r += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const float *src = rows + r * kRowF;
        uint16_t out = 0;
        if (lane < 2) {
            const uint32_t sb = __float_as_uint(__ldg(src));
            out = lane == 0 ? (uint16_t)(sb & 0xffffu) : (uint16_t)(sb >> 16);
        } else if (lane < 29) {
            out = bf16_bits_rn(__ldg(src + (lane - 1)));
        }
        rows_h[r * kRowH + lane] = out;
    }
}

cudaError_t launch_pack_bf16(const GridView &g, uint16_t *rows_h, cudaStream_t s) {
    if (g.M == 0) return cudaSuccess;
    int64_t blocks = (g.M + 7) / 8;
    if (blocks > 152 * 64) blocks = 152 * 64;
    pack_bf16_kernel<<<(unsigned)blocks, 256, 0, s>>>(g.rows, rows_h, g.M);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- TV
// Thread per selected node.  A node whose own row and +x/+y/+z neighbours are
// all empty has t = 0 for every value and is skipped; the others load the
// (up to) four rows as float4 groups and scatter float4 gradients:
//   D_a = (V_d(v+e_a) - V_d(v)) * R/256; t = |D|; L += lam_d t;
//   missing neighbour (NULL or outside): density 0, SH = V_d(v).
// Each segment is split over kTvParts CTAs so short and long runs both fill the GPU.
constexpr int kTvThreads = 256;
constexpr int kTvParts = 8;

__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

__device__ __forceinline__ float comp(const float4 &v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }

__device__ __forceinline__ void tv_node(const GridView &g, int32_t rs, const int32_t rn[3], float scale, float lam_sigma,
                                        float lam_sh, float *__restrict__ grad, float &loss_acc) {
#pragma unroll 1
    for (int q = 0; q < 7; ++q) {
        const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float4 self4 = rs >= 0 ? ld4(g.rows + (int64_t)rs * kRowF + 4 * q) : z4;
        float4 nb4[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) nb4[a] = rn[a] >= 0 ? ld4(g.rows + (int64_t)rn[a] * kRowF + 4 * q) : z4;
        float gs[4], gn[3][4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int d = 4 * q + c;
            const float lam = d == 0 ? lam_sigma : lam_sh;
            const float self = comp(self4, c);
            float D[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float nv = rn[a] >= 0 ? comp(nb4[a], c) : (d == 0 ? 0.0f : self);
                D[a] = (nv - self) * scale;
            }
            const float t = sqrtf(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
            loss_acc = fmaf(lam, t, loss_acc);
            const float k = t > 0.0f ? lam * scale / t : 0.0f;
            float acc = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                gn[a][c] = D[a] * k;
                if (rn[a] >= 0 || d == 0) acc -= D[a];
            }
            gs[c] = acc * k;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (rn[a] >= 0)
                atomicAdd(reinterpret_cast<float4 *>(grad + (int64_t)rn[a] * kRowF + 4 * q),
                          make_float4(gn[a][0], gn[a][1], gn[a][2], gn[a][3]));
        if (rs >= 0)
            atomicAdd(reinterpret_cast<float4 *>(grad + (int64_t)rs * kRowF + 4 * q), make_float4(gs[0], gs[1], gs[2], gs[3]));
    }
    if (rs >= 0) mark_touched(g, rs);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (rn[a] >= 0) mark_touched(g, rn[a]);
}

__global__ void __launch_bounds__(kTvThreads) tv_kernel(GridView g, const int64_t *__restrict__ seg_start,
                                                        const int64_t *__restrict__ seg_len, int64_t n_seg,
                                                        float lam_sigma, float lam_sh, float *__restrict__ grad,
                                                        float *__restrict__ loss) {
    const int64_t R = g.R;
    const int64_t N = R * R * R;
    const float scale = (float)R / 256.0f;
    float loss_acc = 0.0f;
    for (int64_t item = blockIdx.x; item < n_seg * kTvParts; item += gridDim.x) {
        const int64_t sg = item / kTvParts;
        const int part = (int)(item % kTvParts);
        const int64_t start = seg_start[sg];
        const int64_t len = seg_len[sg];
        for (int64_t off = (int64_t)part * kTvThreads + threadIdx.x; off < len; off += (int64_t)kTvParts * kTvThreads) {
            const int64_t n = start + off;
            if (n < 0 || n >= N) continue;
            const int64_t i = n / (R * R), j = (n / R) % R, k = n % R;
            const int32_t rs = row_of(g, n);
            int32_t rn[3];
            rn[0] = i + 1 < R ? row_of(g, n + R * R) : -1;
            rn[1] = j + 1 < R ? row_of(g, n + R) : -1;
            rn[2] = k + 1 < R ? row_of(g, n + 1) : -1;
            if (rs < 0 && rn[0] < 0 && rn[1] < 0 && rn[2] < 0) continue;
            tv_node(g, rs, rn, scale, lam_sigma, lam_sh, grad, loss_acc);
        }
    }
    if (loss) {
        loss_acc = warp_sum(loss_acc);
        if ((threadIdx.x & 31) == 0 && loss_acc != 0.0f) atomicAdd(loss, loss_acc);
    }
}

cudaError_t launch_tv(const GridView &g, const int64_t *seg_start, const int64_t *seg_len, int64_t n_seg,
                      float lam_sigma, float lam_sh, float *grad_rows, float *loss, cudaStream_t s) {
    if (n_seg == 0) return cudaSuccess;
    int64_t blocks = n_seg * kTvParts;
    if (blocks > 152 * 32) blocks = 152 * 32;
    tv_kernel<<<(unsigned)blocks, kTvThreads, 0, s>>>(g, seg_start, seg_len, n_seg, lam_sigma, lam_sh, grad_rows, loss);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- RMSProp
// One warp per word of the touched mask (32 rows): the word's marked rows (all
// rows in dense mode) are updated four at a time with 8 lanes per row (lane q
// owns values 4q..4q+3), so each warp instruction covers 4 whole rows.  The
// grid has enough warps to keep every touched row's loads in flight at once,
// which the scattered rows need to reach DRAM efficiently.  Entries with a zero
// gradient keep x and v; a row with any update is re-packed into its BF16-SH
// form when the grid has one.
__device__ __forceinline__ void rms_quarter(int64_t r, int q, float *__restrict__ rows, uint16_t *__restrict__ rows_h,
                                            float *__restrict__ grad, float *__restrict__ v, float lr_sigma, float lr_sh,
                                            float beta, float eps, bool active) {
    float4 g4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (active && q < 7) g4 = reinterpret_cast<const float4 *>(grad + r * kRowF)[q];
    const bool nz = g4.x != 0.0f || g4.y != 0.0f || g4.z != 0.0f || g4.w != 0.0f;
    const unsigned grp = __ballot_sync(kFull, nz);
    const int lane = threadIdx.x & 31;
    const bool row_any = (grp >> (lane & ~7)) & 0xffu;
    if (!active || !row_any || q == 7) return;
    float4 *xp = reinterpret_cast<float4 *>(rows + r * kRowF) + q;
    float4 *vp = reinterpret_cast<float4 *>(v + r * kRowF) + q;
    float4 x4 = *xp, v4 = *vp;
    float *xe = &x4.x, *ve = &v4.x;
    const float *ge = &g4.x;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float gg = ge[c];
        if (gg != 0.0f) {
            const float lr = (q == 0 && c == 0) ? lr_sigma : lr_sh;
            const float vv = fmaf(beta, ve[c], (1.0f - beta) * gg * gg);
            ve[c] = vv;
            xe[c] = xe[c] - lr * gg / (sqrtf(vv) + eps);
        }
    }
    *xp = x4;
    *vp = v4;
    if (nz) reinterpret_cast<float4 *>(grad + r * kRowF)[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (rows_h) {
        // column col sits in BF16 slot col + 1 (SH), density bits in slots 0-1
        uint16_t *hp = rows_h + r * kRowH;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int col = 4 * q + c;
            if (col == 0)
                *reinterpret_cast<uint32_t *>(hp) = __float_as_uint(xe[0]);
            else
                hp[col + 1] = bf16_bits_rn(xe[c]);
        }
    }
}

__global__ void __launch_bounds__(256) rmsprop_kernel(GridView g, float *__restrict__ rows, uint16_t *__restrict__ rows_h,
                                                      float *__restrict__ grad, float *__restrict__ v, float lr_sigma,
                                                      float lr_sh, float beta, float eps, int sparse, int64_t n_words) {
    const int lane = threadIdx.x & 31;
    const int q = lane & 7;
    const int grp = lane >> 3;
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n_words;
         w += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const uint32_t word = g.touched[w];
        uint32_t mask = sparse ? word : 0xffffffffu;
        const int64_t left = g.M - w * 32;  // rows beyond M in the last word
        if (left < 32) mask &= (1u << left) - 1u;
        __syncwarp();
        if (lane == 0 && word) g.touched[w] = 0u;  // both modes leave the mask clear
        while (mask) {  // uniform
            const int n = __popc(mask);
            const bool active = grp < n;
            const int bit = active ? __fns(mask, 0, grp + 1) : 0;
            rms_quarter(w * 32 + bit, q, rows, rows_h, grad, v, lr_sigma, lr_sh, beta, eps, active);
            // drop the (up to) four rows just handled
            for (int k = 0; k < 4 && mask; ++k) mask &= mask - 1;
        }
    }
}

cudaError_t launch_rmsprop(const GridView &g, float *rows, uint16_t *rows_h, float *grad, float *v, float lr_sigma,
                           float lr_sh, float beta, float eps, int sparse, cudaStream_t s) {
    const int64_t n_words = (g.M + 31) / 32;
    if (n_words == 0) return cudaSuccess;
    int64_t blocks = (n_words + 7) / 8;
    if (blocks > 152 * 64) blocks = 152 * 64;
    rmsprop_kernel<<<(unsigned)blocks, 256, 0, s>>>(g, rows, rows_h, grad, v, lr_sigma, lr_sh, beta, eps, sparse,
                                                    n_words);
    return cudaGetLastError();
}

}  // namespace plx
