// plx_optim.cu -- the kernels around the renderer: the cell-occupancy mask
// used for empty-space skipping, BF16-SH packing, the total-variation gradient
// (Sec. 3.5, Supp. B.1) and the RMSProp update (Sec. 3.5).
#include <algorithm>

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

// The box of cells with an occupied corner (for the march's ray clip): a grid-stride pass over the
// occupancy words, reduced per CTA in shared memory, then one atomicMax per CTA and bound.  Stored as
// R-1-lo and hi, so that the zeroed status block starts as the empty box.
__global__ void __launch_bounds__(256) occ_box_kernel(GridView g, const uint32_t *__restrict__ occ, int64_t n_words,
                                                      int *__restrict__ box) {
    __shared__ int s_box[6];
    if (threadIdx.x < 6) s_box[threadIdx.x] = 0;
    __syncthreads();
    const int64_t R = g.R;
    int b[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_words; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = __ldg(occ + w);
        while (word) {
            const int bit = __ffs(word) - 1;
            word &= word - 1u;
            const int64_t c = w * 32 + bit;
            const int64_t ijk[3] = {c / (R * R), (c / R) % R, c % R};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                b[a] = max(b[a], (int)(R - 1 - ijk[a]));
                b[3 + a] = max(b[3 + a], (int)ijk[a]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        int v = b[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
        if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(&s_box[i], v);
    }
    __syncthreads();
    if (threadIdx.x < 6 && s_box[threadIdx.x] > 0) atomicMax(&box[threadIdx.x], s_box[threadIdx.x]);
}

// The coarse mask: one thread per block of 8^3 cells ORs the cell bits of its 64 rows of up to 8 cells
// (cells (i, j, k) with 0 <= i, j, k <= R - 2; the bit of cell (i, j, k) sits at node id (i R + j) R + k).
__global__ void __launch_bounds__(256) coarse_occupancy_kernel(GridView g, const uint32_t *__restrict__ occ,
                                                               uint32_t *__restrict__ coarse) {
    const int64_t R = g.R, nb = g.nb;
    const int64_t n_blocks = nb * nb * nb;
    const int64_t n_words = (n_blocks + 31) / 32;
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n_words;
         w += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int64_t b = w * 32 + (threadIdx.x & 31);
        bool any = false;
        if (b < n_blocks) {
            const int64_t bi = b / (nb * nb), bj = (b / nb) % nb, bk = b % nb;
            const int64_t k0 = bk << kBlockLog, k1 = min(k0 + (1 << kBlockLog), R - 1);  // cells [k0, k1)
            const uint64_t want = (k1 > k0) ? ((1ull << (k1 - k0)) - 1ull) : 0ull;
            for (int64_t i = bi << kBlockLog; i < min((bi + 1) << kBlockLog, R - 1) && !any; ++i)
                for (int64_t j = bj << kBlockLog; j < min((bj + 1) << kBlockLog, R - 1) && !any; ++j) {
                    const int64_t n0 = (i * R + j) * R + k0;  // first cell bit of the row's run
                    const int64_t w0 = n0 >> 5;
                    const int sh = (int)(n0 & 31);
                    uint64_t bits = __ldg(occ + w0);
                    if (sh + (k1 - k0) > 32) bits |= (uint64_t)__ldg(occ + w0 + 1) << 32;
                    any = ((bits >> sh) & want) != 0ull;
                }
        }
        const unsigned word = __ballot_sync(kFull, any);
        if ((threadIdx.x & 31) == 0) coarse[w] = word;
    }
}

cudaError_t launch_build_occupancy(const GridView &g, uint32_t *occ, uint32_t *occ_coarse, cudaStream_t s) {
    const int64_t R = g.R;
    const int64_t n_words = (R * R * R + 31) / 32;
    const int threads = 256;
    int64_t blocks = (n_words + 7) / 8;
    if (blocks > 152 * 64) blocks = 152 * 64;
    build_occupancy_kernel<<<(unsigned)blocks, threads, 0, s>>>(g, occ, n_words);
    const int64_t bblocks = std::min<int64_t>((n_words + 255) / 256, 152 * 8);
    occ_box_kernel<<<(unsigned)bblocks, 256, 0, s>>>(g, occ, n_words, const_cast<int *>(g.occ_box));
    const int64_t nb = g.nb;
    const int64_t c_words = (nb * nb * nb + 31) / 32;
    const int64_t cblocks = std::max<int64_t>(1, std::min<int64_t>((c_words + 7) / 8, 152 * 64));
    coarse_occupancy_kernel<<<(unsigned)cblocks, 256, 0, s>>>(g, occ, occ_coarse);
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
// A node whose own row and +x/+y/+z neighbours are all empty has t = 0 for every
// value and is skipped; the others are handled four at a time, 8 lanes per node,
// each lane loading one float4 quarter of the (up to) four rows and scattering
// float4 gradients:
//   D_a = (V_d(v+e_a) - V_d(v)) * R/256; t = |D|; L += lam_d t;
//   missing neighbour (NULL or outside): density 0, SH = V_d(v).
// A CTA takes a region of kTvRegion consecutive nodes of a segment at a time; each
// segment is split over as many CTAs ("parts", sized on the host from the average
// segment length) as it has regions, so short and long runs both fill the GPU.
constexpr int kTvThreads = 128;
constexpr int kTvLaneNodes = 16;                 // nodes each lane of the first warp screens (4, 8, 32 measured slower)
constexpr int kTvRegion = 32 * kTvLaneNodes;    // nodes a CTA takes at once
constexpr int kTvGridPerSm = 16;  // at most this many CTAs per SM in the grid

__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

__device__ __forceinline__ float comp(const float4 &v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }

// TV (Sec. 3.5; Supp. B.1) of one float4 quarter q (< 7) of one node: per value d of the quarter,
// D_a = (V_d(n + e_a) - V_d(n)) R/256, t = sqrt(sum_a D_a^2), loss += lam_d t, and the gradient
// lam_d (R/256) D_a / t to the +a neighbour and minus its sum to the node (0 when t = 0).  A missing
// neighbour (NULL or outside) has density 0 and SH equal to the node's own (no gradient for it).
__device__ __forceinline__ void tv_quarter(const GridView &g, int32_t rs, const int32_t rn[3], int q, float scale,
                                           float lam_sigma, float lam_sh, float *__restrict__ grad,
                                           float &loss_acc) {
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

// The row entries TV needs for one node: its own and those of its +x, +y, +z neighbours (-1: NULL or
// outside the grid).
struct TvNode {
    int32_t rs, rn[3];
};

// Candidates among the (up to) 32 nodes n_a .. n_a + cnt - 1 of one lane: bit t set when node n_a + t may
// have an occupied row among self and +x/+y/+z.  An interior node and those neighbours are four corners
// of the cell based at the node, so the cell's occupancy bit decides; a node on a far face (i, j or k =
// R - 1) is the base of no cell and stays a candidate, to be decided by its index entries.
__device__ __forceinline__ uint32_t tv_candidates(const GridView &g, int64_t n_a, int cnt) {
    const int64_t R = g.R;
    const int64_t n_words = (R * R * R + 31) >> 5;
    const int64_t w = n_a >> 5;
    const int sh = (int)(n_a & 31);
    uint32_t bits = __ldg(g.occ + w) >> sh;
    if (sh && w + 1 < n_words) bits |= __ldg(g.occ + w + 1) << (32 - sh);
    int64_t i = n_a / (R * R);
    const int64_t rem = n_a - i * R * R;
    int64_t j = rem / R;
    int64_t k = rem - j * R;
    uint32_t face = 0u;
    for (int t = 0; t < cnt;) {  // one pass per grid row the nodes touch
        const int run = (int)min((int64_t)(cnt - t), R - k);
        if (i == R - 1 || j == R - 1)
            face |= (run == 32 ? kFull : ((1u << run) - 1u)) << t;
        else if (k + run == R)
            face |= 1u << (t + run - 1);
        t += run;
        k = 0;
        if (++j == R) {
            j = 0;
            ++i;
        }
    }
    const uint32_t valid = cnt == 32 ? kFull : ((1u << cnt) - 1u);
    return (bits | face) & valid;
}

// Per region of a segment, three phases separated by CTA barriers: (1) the first warp screens the
// region's nodes against the occupancy bit map (one bit per node instead of four index entries) and
// lists the candidates in shared memory; (2) every thread reads the index entries of one candidate at a
// time and keeps, in a second list, the nodes with an occupied row among self and +x/+y/+z; (3) each
// warp takes the kept nodes four at a time with 8 lanes per node (one float4 quarter each), so a node's
// rows take one memory round trip.  Only occupied nodes' neighbourhoods cost index reads, and all kept
// nodes of a region are in flight at once.
__global__ void __launch_bounds__(kTvThreads) tv_kernel(GridView g, const int64_t *__restrict__ seg_start,
                                                        const int64_t *__restrict__ seg_len, int64_t n_seg,
                                                        int64_t parts, float lam_sigma, float lam_sh,
                                                        float *__restrict__ grad, float *__restrict__ loss) {
    __shared__ uint16_t s_cand[kTvRegion];
    __shared__ TvNode s_node[kTvRegion];
    __shared__ int s_ncand, s_nnode;
    const float scale = (float)g.R / 256.0f;
    const int lane = threadIdx.x & 31;
    const int q = lane & 7;
    const int grp = lane >> 3;
    const int wid = threadIdx.x >> 5;
    constexpr int kWarps = kTvThreads / 32;
    const int64_t R = g.R;
    const int64_t N = R * R * R;
    float loss_acc = 0.0f;
    for (int64_t item = blockIdx.x; item < n_seg * parts; item += gridDim.x) {
        const int64_t sg = item / parts;
        const int64_t part = item % parts;
        const int64_t start = seg_start[sg];
        const int64_t len = seg_len[sg];
        for (int64_t r0 = part * kTvRegion; r0 < len; r0 += parts * kTvRegion) {  // uniform over the CTA
            if (wid == 0) {
                const int64_t off = r0 + lane * kTvLaneNodes;
                const int64_t n_a = start + off;
                uint32_t cand = 0u;
                if (off < len && n_a >= 0 && n_a < N)
                    cand = tv_candidates(g, n_a, (int)min((int64_t)kTvLaneNodes, min(len - off, N - n_a)));
                const int c = __popc(cand);
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += t;
                }
                int pos = incl - c;
                while (cand) {
                    const int bit = __ffs(cand) - 1;
                    cand &= cand - 1u;
                    s_cand[pos++] = (uint16_t)(lane * kTvLaneNodes + bit);
                }
                if (lane == 31) s_ncand = incl;
                if (lane == 0) s_nnode = 0;
            }
            __syncthreads();
            const int ncand = s_ncand;
            for (int c = threadIdx.x; c < ncand; c += kTvThreads) {
                const int64_t n = start + r0 + s_cand[c];
                int64_t i, j, k;
                if (N <= (int64_t)UINT32_MAX) {  // 32-bit divisions where the ids fit
                    const uint32_t n32 = (uint32_t)n, R32 = (uint32_t)R;
                    const uint32_t ij = n32 / R32;
                    k = n32 - ij * R32;
                    i = ij / R32;
                    j = ij - (uint32_t)i * R32;
                } else {
                    i = n / (R * R);
                    const int64_t rem = n - i * R * R;
                    j = rem / R;
                    k = rem - j * R;
                }
                TvNode t;
                t.rs = row_of(g, n);
                t.rn[0] = i + 1 < R ? row_of(g, n + R * R) : -1;
                t.rn[1] = j + 1 < R ? row_of(g, n + R) : -1;
                t.rn[2] = k + 1 < R ? row_of(g, n + 1) : -1;
                if (t.rs >= 0 || t.rn[0] >= 0 || t.rn[1] >= 0 || t.rn[2] >= 0) s_node[atomicAdd(&s_nnode, 1)] = t;
            }
            __syncthreads();
            const int nn = s_nnode;
            for (int b = wid * 4; b < nn; b += kWarps * 4) {  // uniform over the warp
                const int m = b + grp;
                if (m < nn && q < 7) {
                    const TvNode t = s_node[m];
                    tv_quarter(g, t.rs, t.rn, q, scale, lam_sigma, lam_sh, grad, loss_acc);
                    if (q == 0) {
                        if (t.rs >= 0) mark_touched(g, t.rs);
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            if (t.rn[a] >= 0) mark_touched(g, t.rn[a]);
                    }
                }
            }
            __syncthreads();  // the lists are rewritten by the next region
        }
    }
    if (loss) {
        loss_acc = warp_sum(loss_acc);
        if (lane == 0 && loss_acc != 0.0f) atomicAdd(loss, loss_acc);
    }
}

cudaError_t launch_tv(const GridView &g, const int64_t *seg_start, const int64_t *seg_len, int64_t n_seg,
                      int64_t n_selected, float lam_sigma, float lam_sh, float *grad_rows, float *loss,
                      cudaStream_t s) {
    if (n_seg == 0) return cudaSuccess;
    // parts per segment: the regions of the average segment; one CTA per item (the block scheduler
    // balances the short-lived CTAs), at most 2^20 items
    const int64_t avg = (n_selected + n_seg - 1) / n_seg;
    const int64_t parts = std::max<int64_t>(1, std::min<int64_t>((avg + kTvRegion - 1) / kTvRegion, 1 << 20));
    int sms = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int64_t blocks = std::min<int64_t>(n_seg * parts, (int64_t)sms * kTvGridPerSm);
    tv_kernel<<<(unsigned)blocks, kTvThreads, 0, s>>>(g, seg_start, seg_len, n_seg, parts, lam_sigma, lam_sh,
                                                      grad_rows, loss);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- RMSProp
// Sparse mode lists the rows marked in the touched bitmask (rms_compact_kernel),
// then a warp takes 32 listed rows (32 consecutive rows in dense mode) and updates
// them four at a time with 8 lanes per row (lane q owns values 4q..4q+3), so each
// warp instruction covers 4 whole rows.  The grid has enough warps to keep every
// touched row's loads in flight at once, which the scattered rows need to reach
// DRAM efficiently.  Entries with a zero gradient keep x and v; a row with any
// update is re-packed into its BF16-SH form when the grid has one.
// RMSProp (Sec. 3.5) on one float4 quarter q (< 7) of a row: for every entry with g != 0,
// v <- beta v + (1 - beta) g^2, x <- x - lr g / (sqrt(v) + eps), then g <- 0.  g4, x4, v4 were
// loaded by the caller; x4 returns updated, and the result says whether any entry changed (the caller
// then refreshes the row's BF16-SH shadow).
__device__ __forceinline__ bool rms_update(int64_t r, int q, float4 g4, float4 &x4, float4 v4, float *__restrict__ rows,
                                           float *__restrict__ grad, float *__restrict__ v, float lr_sigma,
                                           float lr_sh, float beta, float eps) {
    const bool nz = g4.x != 0.0f || g4.y != 0.0f || g4.z != 0.0f || g4.w != 0.0f;
    if (!nz) return false;
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
    reinterpret_cast<float4 *>(rows + r * kRowF)[q] = x4;
    reinterpret_cast<float4 *>(v + r * kRowF)[q] = v4;
    reinterpret_cast<float4 *>(grad + r * kRowF)[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    return true;
}

// plx_count_touched: the number of rows marked in the touched bitmask, i.e. the rows that received a
// gradient (adjoint or TV) since the last RMSProp step (Sec. 3.8: the gradient is sparse).  One CTA
// sums the popcounts of the mask words and writes the total.
__global__ void __launch_bounds__(1024) count_touched_kernel(GridView g, int64_t n_words, int64_t *__restrict__ out) {
    __shared__ unsigned long long s_part[32];
    unsigned long long c = 0;
    for (int64_t w = threadIdx.x; w < n_words; w += blockDim.x) {
        uint32_t word = __ldcg(g.touched + w);
        const int64_t left = g.M - w * 32;  // >= 1
        if (left < 32) word &= (1u << left) - 1u;
        c += (unsigned long long)__popc(word);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(kFull, c, off);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        c = threadIdx.x < (blockDim.x >> 5) ? s_part[threadIdx.x] : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(kFull, c, off);
        if (threadIdx.x == 0) *out = (int64_t)c;
    }
}

// Sparse mode, pass 1: the rows marked in the touched bitmask, as a list, and the mask cleared.  A CTA
// takes 256 consecutive mask words at a time (a word per thread), adds its count to the list's length
// with one atomic and writes its rows in ascending order: warp by warp, then word by word, the lanes of
// a word's set bits storing consecutive entries (one coalesced store per non-empty word).  The list is
// ascending within each CTA's range, which keeps the update's row accesses in long ascending runs.
// The count this call's update reads starts at zero; the call also zeroes the other count, which the
// next call uses (the two alternate, so no separate reset sits between the adjoint and the update).
constexpr int kCompactThreads = 256;
__global__ void __launch_bounds__(kCompactThreads) rms_compact_kernel(GridView g, int64_t n_words,
                                                                      int *__restrict__ next_count) {
    chain_release();  // the update (chained) may be scheduled as this pass drains
    __shared__ int s_warp[kCompactThreads / 32];
    __shared__ int s_base;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    if (blockIdx.x == 0 && threadIdx.x == 0) *next_count = 0;
    for (int64_t c0 = (int64_t)blockIdx.x * kCompactThreads; c0 < n_words; c0 += (int64_t)gridDim.x * kCompactThreads) {
        const int64_t w = c0 + threadIdx.x;
        uint32_t word = 0u;
        if (w < n_words) {
            word = g.touched[w];
            if (word) g.touched[w] = 0u;
            const int64_t left = g.M - w * 32;  // >= 1
            if (left < 32) word &= (1u << left) - 1u;
        }
        const int c = __popc(word);
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
#pragma unroll
            for (int q = 0; q < kCompactThreads / 32; ++q) {
                const int t = s_warp[q];
                s_warp[q] = tot;
                tot += t;
            }
            s_base = tot ? atomicAdd(g.tcount, tot) : 0;
        }
        __syncthreads();
        const int excl = s_base + s_warp[wid] + incl - c;  // list position of this word's first row
        unsigned nz = __ballot_sync(kFull, word != 0u);
        while (nz) {
            const int src = __ffs(nz) - 1;
            nz &= nz - 1u;
            const uint32_t wj = __shfl_sync(kFull, word, src);
            const int pj = __shfl_sync(kFull, excl, src);
            if ((wj >> lane) & 1u) g.tlist[pj + __popc(wj & lt)] = (int32_t)((c0 + 32 * wid + src) * 32 + lane);
        }
        __syncthreads();  // s_warp and s_base are rewritten by the next round
    }
}

// Pass 2: rows from the list (sparse) or all rows (dense).  A warp takes 32 rows at a time, 8 lanes per
// row (quarters 0..6; lane 7 only stores the last 8 bytes of a BF16 shadow), kRmsGroups groups of 4 rows
// per round so that 3 kRmsGroups float4 loads of each lane are in flight together.
constexpr int kRmsGroups = 2;
constexpr int kRmsGridPerSm = 8;  // CTAs per SM in the grid (warps loop over 32-row slices)
template <bool SPARSE>
__global__ void __launch_bounds__(256) rms_apply_kernel(GridView g, float *__restrict__ rows,
                                                        uint16_t *__restrict__ rows_h, float *__restrict__ grad,
                                                        float *__restrict__ v, float lr_sigma, float lr_sh, float beta,
                                                        float eps) {
    chain_wait();
    chain_release();
    const int lane = threadIdx.x & 31;
    const int q = lane & 7;
    const int grp = lane >> 3;
    const int64_t total = SPARSE ? (int64_t)*g.tcount : g.M;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32; base < total; base += n_warps * 32) {
        const int64_t li = base + lane;
        const int32_t mine = li < total ? (SPARSE ? g.tlist[li] : (int32_t)li) : -1;
#pragma unroll 1
        for (int sub = 0; sub < 8; sub += kRmsGroups) {
            int32_t r[kRmsGroups];
#pragma unroll
            for (int j = 0; j < kRmsGroups; ++j) r[j] = __shfl_sync(kFull, mine, 4 * (sub + j) + grp);
            const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float4 gg[kRmsGroups], xx[kRmsGroups], vv[kRmsGroups];
#pragma unroll
            for (int j = 0; j < kRmsGroups; ++j) {
                gg[j] = xx[j] = vv[j] = z;
                if (r[j] >= 0 && q < 7) {
                    gg[j] = reinterpret_cast<const float4 *>(grad + (int64_t)r[j] * kRowF)[q];
                    xx[j] = reinterpret_cast<const float4 *>(rows + (int64_t)r[j] * kRowF)[q];
                    vv[j] = reinterpret_cast<const float4 *>(v + (int64_t)r[j] * kRowF)[q];
                }
            }
#pragma unroll
            for (int j = 0; j < kRmsGroups; ++j) {
                bool nz = false;
                if (r[j] >= 0 && q < 7) nz = rms_update(r[j], q, gg[j], xx[j], vv[j], rows, grad, v, lr_sigma, lr_sh, beta, eps);
                if (rows_h) {  // uniform over the warp
                    // The row's BF16 shadow, rewritten whole when any quarter changed, 8 aligned bytes per
                    // lane: slots 4q..4q+3 hold column 4q - 1 (lane q - 1's fourth value) and columns
                    // 4q..4q+2 (density bits in slots 0-1, column c in slot c + 1, slots 29-31 zero).
                    const float prev = __shfl_up_sync(kFull, xx[j].w, 1, 8);
                    const unsigned row_nz = (__ballot_sync(kFull, nz) >> (8 * grp)) & 0xffu;
                    if (r[j] >= 0 && row_nz) {
                        const uint32_t lo = q == 0 ? __float_as_uint(xx[j].x)
                                                   : (uint32_t)bf16_bits_rn(prev) | ((uint32_t)bf16_bits_rn(xx[j].x) << 16);
                        const uint32_t hi = (uint32_t)bf16_bits_rn(xx[j].y) | ((uint32_t)bf16_bits_rn(xx[j].z) << 16);
                        reinterpret_cast<uint2 *>(rows_h + (int64_t)r[j] * kRowH)[q] = make_uint2(lo, hi);
                    }
                }
            }
        }
    }
}

cudaError_t launch_rmsprop(const GridView &g, float *rows, uint16_t *rows_h, float *grad, float *v, float lr_sigma,
                           float lr_sh, float beta, float eps, int sparse, int *next_count, cudaStream_t s) {
    const int64_t n_words = (g.M + 31) / 32;
    if (n_words == 0) return cudaSuccess;
    int sms = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int64_t apply_blocks = std::min<int64_t>((g.M + 255) / 256, (int64_t)sms * kRmsGridPerSm);
    if (sparse) {
        if (!next_count) return cudaErrorInvalidValue;
        const int64_t blocks = std::min<int64_t>((n_words + kCompactThreads - 1) / kCompactThreads, (int64_t)sms * 8);
        rms_compact_kernel<<<(unsigned)blocks, kCompactThreads, 0, s>>>(g, n_words, next_count);
        return launch_chained(rms_apply_kernel<true>, (unsigned)apply_blocks, 256, s, g, rows, rows_h, grad, v,
                              lr_sigma, lr_sh, beta, eps);
    }
    cudaError_t e = launch_chained(rms_apply_kernel<false>, (unsigned)apply_blocks, 256, s, g, rows, rows_h, grad, v,
                                   lr_sigma, lr_sh, beta, eps);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(g.touched, 0, (size_t)n_words * 4, s);
}

cudaError_t launch_count_touched(const GridView &g, int64_t *out, cudaStream_t s) {
    count_touched_kernel<<<1, 1024, 0, s>>>(g, (g.M + 31) / 32, out);
    return cudaGetLastError();
}

}  // namespace plx
