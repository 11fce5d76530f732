// plx_gridops.cu -- coarse-to-fine grid operations (Sec. 3.4 "Coarse to
// Fine"): density-threshold pruning with 3x3x3 dilation and trilinear
// resampling to a new resolution.  Both are two-phase: a count pass builds a
// bit map of surviving nodes and per-block counts in a caller workspace, a
// single-CTA exclusive scan turns counts into block offsets (the total is the
// new row count), and an apply pass writes the new index volume and rows in
// ascending node order, so the result is unique and bit-exact.
#include "plx_internal.cuh"

namespace plx {

constexpr int kBlockNodes = 1024;  // nodes per CTA block = 32 warps x 32 lanes

struct MapLayout {
    size_t bits_off, keep_off, counts_off, offsets_off, total;
    int64_t n_words, n_blocks;
    static size_t r256(size_t b) { return (b + 255) & ~size_t(255); }
    static MapLayout make(int64_t n_nodes, bool two_maps) {
        MapLayout L;
        L.n_words = (n_nodes + 31) / 32;
        L.n_blocks = (n_nodes + kBlockNodes - 1) / kBlockNodes;
        L.bits_off = 256;
        L.keep_off = L.bits_off + (two_maps ? r256(size_t(L.n_words) * 4) : 0);
        L.counts_off = L.keep_off + r256(size_t(L.n_words) * 4);
        L.offsets_off = L.counts_off + r256(size_t(L.n_blocks) * 4);
        L.total = L.offsets_off + r256(size_t(L.n_blocks) * 4);
        return L;
    }
};

size_t prune_ws_bytes(int64_t R) { return MapLayout::make(R * R * R, true).total; }
size_t upsample_ws_bytes(int64_t R2) { return MapLayout::make(R2 * R2 * R2, false).total; }

__device__ __forceinline__ bool test_bit(const uint32_t *bits, int64_t n) {
    return (__ldg(bits + (n >> 5)) >> (n & 31)) & 1u;
}

// Block-level sum of 32 per-warp popcounts into counts[blockIdx.x].
__device__ __forceinline__ void block_count(unsigned word, uint32_t *counts, int64_t b) {
    __shared__ uint32_t s_cnt[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_cnt[wid] = __popc(word);
    __syncthreads();
    if (wid == 0) {
        uint32_t c = s_cnt[lane];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(kFull, c, off);
        if (lane == 0) counts[b] = c;
    }
}

// Position of this lane's set bit among all set bits of the block (32 words).
__device__ __forceinline__ uint32_t block_rank(unsigned word) {
    __shared__ uint32_t s_pre[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_pre[wid] = __popc(word);
    __syncthreads();
    if (wid == 0) {
        uint32_t c = s_pre[lane];
        uint32_t x = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t v = __shfl_up_sync(kFull, x, off);
            if (lane >= off) x += v;
        }
        s_pre[lane] = x - c;  // exclusive
    }
    __syncthreads();
    return s_pre[wid] + __popc(word & ((1u << lane) - 1u));
}

// Single-CTA exclusive scan of counts[nb] -> offsets[nb]; total -> *total.
__global__ void __launch_bounds__(1024) scan_kernel(const uint32_t *__restrict__ counts, uint32_t *__restrict__ offsets,
                                                    int64_t nb, int64_t *__restrict__ total) {
    __shared__ uint64_t s_part[1024];
    const int tid = threadIdx.x;
    const int64_t per = (nb + 1023) / 1024;
    const int64_t b0 = tid * per, b1 = min(nb, b0 + per);
    uint64_t sum = 0;
    for (int64_t b = b0; b < b1; ++b) sum += counts[b];
    s_part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint64_t v = tid >= off ? s_part[tid - off] : 0;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    uint64_t run = s_part[tid] - sum;
    for (int64_t b = b0; b < b1; ++b) {
        offsets[b] = (uint32_t)run;
        run += counts[b];
    }
    if (tid == 1023) *total = (int64_t)s_part[1023];
}

// --------------------------------------------------------------------------- prune
// hot(n): node n occupied and its key >= tau; the key is the row's density, or key[row] when given.
__global__ void prune_hot_kernel(GridView g, const float *__restrict__ key, float tau, uint32_t *__restrict__ hot,
                                 int64_t n_words) {
    const int lane = threadIdx.x & 31;
    const int64_t N = (int64_t)g.R * g.R * g.R;
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n_words;
         w += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int64_t n = w * 32 + lane;
        bool h = false;
        if (n < N) {
            const int32_t r = row_of(g, n);
            h = r >= 0 && (key ? __ldg(key + r) : __ldg(g.rows + (int64_t)r * kRowF)) >= tau;
        }
        const unsigned word = __ballot_sync(kFull, h);
        if (lane == 0) hot[w] = word;
    }
}

__global__ void __launch_bounds__(1024) prune_keep_kernel(GridView g, int dilate, const uint32_t *__restrict__ hot,
                                                          uint32_t *__restrict__ keep, uint32_t *__restrict__ counts) {
    const int64_t R = g.R, N = R * R * R;
    const int64_t n = (int64_t)blockIdx.x * kBlockNodes + threadIdx.x;
    bool k = false;
    if (n < N && row_of(g, n) >= 0) {
        if (!dilate) {
            k = test_bit(hot, n);
        } else {
            const int64_t i = n / (R * R), j = (n / R) % R, kk = n % R;
            for (int di = -1; di <= 1 && !k; ++di) {
                const int64_t a = i + di;
                if (a < 0 || a >= R) continue;
                for (int dj = -1; dj <= 1 && !k; ++dj) {
                    const int64_t b = j + dj;
                    if (b < 0 || b >= R) continue;
                    for (int dk = -1; dk <= 1 && !k; ++dk) {
                        const int64_t c = kk + dk;
                        if (c < 0 || c >= R) continue;
                        k = test_bit(hot, (a * R + b) * R + c);
                    }
                }
            }
        }
    }
    const unsigned word = __ballot_sync(kFull, k);
    const int64_t w = n >> 5;
    if ((threadIdx.x & 31) == 0 && w * 32 < N) keep[w] = word;
    block_count(word, counts, blockIdx.x);
}

__global__ void __launch_bounds__(1024) prune_apply_kernel(GridView g, const uint32_t *__restrict__ keep,
                                                           const uint32_t *__restrict__ offsets, int64_t n_keep,
                                                           int32_t *__restrict__ idx_new, float *__restrict__ rows_new) {
    const int64_t N = (int64_t)g.R * g.R * g.R;
    const int64_t n = (int64_t)blockIdx.x * kBlockNodes + threadIdx.x;
    const unsigned word = (n >> 5) * 32 < N ? __ldg(keep + (n >> 5)) : 0u;
    const uint32_t rank = block_rank(word);
    if (n >= N) return;
    const bool k = (word >> (threadIdx.x & 31)) & 1u;
    if (!k) {
        idx_new[n] = -1;
        return;
    }
    const uint32_t id = offsets[blockIdx.x] + rank;
    if ((int64_t)id >= n_keep) {  // workspace and count disagree: write nothing out of range
        report(g.status, kDevCountMismatch);
        idx_new[n] = -1;
        return;
    }
    idx_new[n] = (int32_t)id;
    const int32_t r = __ldg(g.idx + n);
    const float4 *src = reinterpret_cast<const float4 *>(g.rows + (int64_t)r * kRowF);
    float4 *dst = reinterpret_cast<float4 *>(rows_new + (int64_t)id * kRowF);
#pragma unroll
    for (int q = 0; q < 7; ++q) dst[q] = __ldg(src + q);
    dst[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

cudaError_t launch_prune_count(const GridView &g, const float *key, float tau, int dilate, void *ws, cudaStream_t s) {
    const int64_t N = (int64_t)g.R * g.R * g.R;
    MapLayout L = MapLayout::make(N, true);
    char *base = static_cast<char *>(ws);
    uint32_t *hot = reinterpret_cast<uint32_t *>(base + L.bits_off);
    uint32_t *keep = reinterpret_cast<uint32_t *>(base + L.keep_off);
    uint32_t *counts = reinterpret_cast<uint32_t *>(base + L.counts_off);
    uint32_t *offsets = reinterpret_cast<uint32_t *>(base + L.offsets_off);
    int64_t blocks = (L.n_words + 7) / 8;
    if (blocks > 152 * 64) blocks = 152 * 64;
    prune_hot_kernel<<<(unsigned)blocks, 256, 0, s>>>(g, key, tau, hot, L.n_words);
    prune_keep_kernel<<<(unsigned)L.n_blocks, 1024, 0, s>>>(g, dilate, hot, keep, counts);
    scan_kernel<<<1, 1024, 0, s>>>(counts, offsets, L.n_blocks, reinterpret_cast<int64_t *>(base + kWsCountOff));
    return cudaGetLastError();
}

cudaError_t launch_prune_apply(const GridView &g, const void *ws, int64_t n_keep, int32_t *idx_new, float *rows_new,
                               cudaStream_t s) {
    const int64_t N = (int64_t)g.R * g.R * g.R;
    MapLayout L = MapLayout::make(N, true);
    const char *base = static_cast<const char *>(ws);
    prune_apply_kernel<<<(unsigned)L.n_blocks, 1024, 0, s>>>(
        g, reinterpret_cast<const uint32_t *>(base + L.keep_off), reinterpret_cast<const uint32_t *>(base + L.offsets_off),
        n_keep, idx_new, rows_new);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- upsample
// New node p' along one axis: num = p'(R-1); base = num / (R'-1); rem = num mod (R'-1).
struct AxisMap {
    int base;
    int rem;
};

__device__ __forceinline__ AxisMap axis_map(int64_t p2, int64_t R, int64_t R2) {
    const int64_t num = p2 * (R - 1);
    AxisMap m;
    m.base = (int)(num / (R2 - 1));
    m.rem = (int)(num - (int64_t)m.base * (R2 - 1));
    return m;
}

__global__ void __launch_bounds__(1024) upsample_count_kernel(GridView g, int R2, uint32_t *__restrict__ occ2,
                                                              uint32_t *__restrict__ counts) {
    const int64_t R = g.R, N2 = (int64_t)R2 * R2 * R2;
    const int64_t n2 = (int64_t)blockIdx.x * kBlockNodes + threadIdx.x;
    bool occ = false;
    if (n2 < N2) {
        const int64_t p[3] = {n2 / ((int64_t)R2 * R2), (n2 / R2) % R2, n2 % R2};
        AxisMap m[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) m[a] = axis_map(p[a], R, R2);
        for (int c = 0; c < 8 && !occ; ++c) {
            const int cb[3] = {(c >> 2) & 1, (c >> 1) & 1, c & 1};
            if ((cb[0] && m[0].rem == 0) || (cb[1] && m[1].rem == 0) || (cb[2] && m[2].rem == 0)) continue;
            const int64_t n = ((int64_t)(m[0].base + cb[0]) * R + (m[1].base + cb[1])) * R + (m[2].base + cb[2]);
            occ = __ldg(g.idx + n) >= 0;
        }
    }
    const unsigned word = __ballot_sync(kFull, occ);
    const int64_t w = n2 >> 5;
    if ((threadIdx.x & 31) == 0 && w * 32 < N2) occ2[w] = word;
    block_count(word, counts, blockIdx.x);
}

__global__ void __launch_bounds__(1024) upsample_apply_kernel(GridView g, int R2, const uint32_t *__restrict__ occ2,
                                                              const uint32_t *__restrict__ offsets, int64_t n_new,
                                                              int32_t *__restrict__ idx_new, float *__restrict__ rows_new) {
    const int64_t R = g.R, N2 = (int64_t)R2 * R2 * R2;
    const int64_t n2 = (int64_t)blockIdx.x * kBlockNodes + threadIdx.x;
    const unsigned word = (n2 >> 5) * 32 < N2 ? __ldg(occ2 + (n2 >> 5)) : 0u;
    const uint32_t rank = block_rank(word);
    if (n2 >= N2) return;
    if (!((word >> (threadIdx.x & 31)) & 1u)) {
        idx_new[n2] = -1;
        return;
    }
    const uint32_t id = offsets[blockIdx.x] + rank;
    if ((int64_t)id >= n_new) {
        report(g.status, kDevCountMismatch);
        idx_new[n2] = -1;
        return;
    }
    idx_new[n2] = (int32_t)id;
    const int64_t p[3] = {n2 / ((int64_t)R2 * R2), (n2 / R2) % R2, n2 % R2};
    AxisMap m[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m[a] = axis_map(p[a], R, R2);
        f[a] = (float)m[a].rem / (float)(R2 - 1);
    }
    float acc[kNV];
#pragma unroll
    for (int q = 0; q < kNV; ++q) acc[q] = 0.0f;
    for (int c = 0; c < 8; ++c) {
        const int cb[3] = {(c >> 2) & 1, (c >> 1) & 1, c & 1};
        if ((cb[0] && m[0].rem == 0) || (cb[1] && m[1].rem == 0) || (cb[2] && m[2].rem == 0)) continue;
        const int64_t n = ((int64_t)(m[0].base + cb[0]) * R + (m[1].base + cb[1])) * R + (m[2].base + cb[2]);
        const int32_t r = row_of(g, n);
        if (r < 0) continue;
        accum_row(g, PLX_SH_F32, r, corner_weight(f, c), acc);
    }
    float4 *dst = reinterpret_cast<float4 *>(rows_new + (int64_t)id * kRowF);
#pragma unroll
    for (int q = 0; q < 7; ++q) dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    dst[7] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

cudaError_t launch_upsample_count(const GridView &g, int R2, void *ws, cudaStream_t s) {
    const int64_t N2 = (int64_t)R2 * R2 * R2;
    MapLayout L = MapLayout::make(N2, false);
    char *base = static_cast<char *>(ws);
    uint32_t *occ2 = reinterpret_cast<uint32_t *>(base + L.keep_off);
    uint32_t *counts = reinterpret_cast<uint32_t *>(base + L.counts_off);
    uint32_t *offsets = reinterpret_cast<uint32_t *>(base + L.offsets_off);
    upsample_count_kernel<<<(unsigned)L.n_blocks, 1024, 0, s>>>(g, R2, occ2, counts);
    scan_kernel<<<1, 1024, 0, s>>>(counts, offsets, L.n_blocks, reinterpret_cast<int64_t *>(base + kWsCountOff));
    return cudaGetLastError();
}

cudaError_t launch_upsample_apply(const GridView &g, int R2, const void *ws, int64_t n_new, int32_t *idx_new,
                                  float *rows_new, cudaStream_t s) {
    const int64_t N2 = (int64_t)R2 * R2 * R2;
    MapLayout L = MapLayout::make(N2, false);
    const char *base = static_cast<const char *>(ws);
    upsample_apply_kernel<<<(unsigned)L.n_blocks, 1024, 0, s>>>(
        g, R2, reinterpret_cast<const uint32_t *>(base + L.keep_off),
        reinterpret_cast<const uint32_t *>(base + L.offsets_off), n_new, idx_new, rows_new);
    return cudaGetLastError();
}

}  // namespace plx
