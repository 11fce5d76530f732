// plx_internal.cuh -- device-side view of a Plenoxel grid and the helpers the
// kernels share (SH basis, box clip, warp scans, status reporting).
//
// Layout facts used throughout (Sec. 3.2; Supp. B.1):
//   node (i,j,k) -> n = (i*R + j)*R + k; idx[n] = -1 for a NULL node;
//   F32 row  = 32 floats   [sigma, 27 SH (R0..R8, G0..G8, B0..B8), 4 pad];
//   BF16 row = 32 uint16   [sigma FP32 (2 slots), 27 SH bf16, 3 pad].
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>

#include "plenoxel.h"

namespace plx {

constexpr int kNV = 28;          // values per node: density + 27 SH
constexpr int kRowF = 32;        // floats per F32 row (128 bytes)
constexpr int kRowH = 32;        // uint16 per BF16 row (64 bytes)
constexpr unsigned kFull = 0xffffffffu;

// Chained launches (programmatic dependent launch).  A kernel started by launch_chained may be
// scheduled while the kernel before it in the stream is still finishing; its first statement is
// chain_wait(), which returns once every earlier kernel of the stream has completed and its memory
// is visible, so no thread touches global memory before the stream order allows (launched plainly,
// chain_wait() returns at once).  chain_release() lets the next chained kernel be scheduled once
// every CTA of this grid has issued it.  Only the launch latency and CTA ramp are overlapped.
// Used for the RMSProp update after its compaction and for the large-batch combine after the chunk
// kernel; chaining the 5000-ray march kernels as well made each faster alone but took from the TV
// kernel beside them the SM slots it fills between launches, and the overlapped step measured slower.
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void chain_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s,
                                  Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// device status codes (stored in the grid workspace's first word)
enum : int { kDevOk = 0, kDevBadRow = 1, kDevTooManySamples = 2, kDevCountMismatch = 3, kDevStateMismatch = 4, kDevBadTile = 5 };

// Workspace layout of a grid: [status block 256 B][occupancy bits][touched bits][touched-row list].
// The status block holds the device status word at byte 0, the touched-list length at byte 64 and the
// box of non-empty cells at byte 128 (six ints: R-1-lo per axis, then hi per axis).
// Coarse blocks of 8^3 cells: one bit per block, set when a cell of the block has an occupied corner.
constexpr int kBlockLog = 3;
__host__ __device__ inline int64_t coarse_blocks_per_axis(int64_t R) { return ((R - 2) >> kBlockLog) + 1; }

struct WorkspaceLayout {
    size_t status_off, occ_off, coarse_off, touched_off, list_off, total;
    static constexpr size_t kListCountOff = 64;   // two list lengths, used by alternate sparse RMSProp calls
    static constexpr size_t kListCount2Off = 96;
    static constexpr size_t kOccBoxOff = 128;
    static size_t round256(size_t b) { return (b + 255) & ~size_t(255); }
    static WorkspaceLayout make(int64_t R, int64_t M) {
        WorkspaceLayout L;
        int64_t nodes = R * R * R;
        const int64_t nb = coarse_blocks_per_axis(R);
        L.status_off = 0;
        L.occ_off = 256;
        L.coarse_off = L.occ_off + round256(size_t((nodes + 31) / 32) * 4);
        L.touched_off = L.coarse_off + round256(size_t((nb * nb * nb + 31) / 32) * 4);
        L.list_off = L.touched_off + round256(size_t((M + 31) / 32 + 1) * 4);
        L.total = L.list_off + round256(size_t(M) * 4);
        return L;
    }
};

struct GridView {
    const int32_t *idx;
    const float *rows;          // F32 rows (may be null for a render-only BF16 grid)
    const uint16_t *rows_h;     // BF16-SH rows (null for the F32 form)
    const uint32_t *occ;        // bit per base node: 1 if any of the cell's 8 nodes is occupied
    const uint32_t *occ_coarse; // bit per block of 8^3 cells: 1 if any of its cells is non-empty
    int nb;                     // blocks per axis, coarse_blocks_per_axis(R)
    const int *occ_box;         // cells with an occupied corner lie in [R-1-box[a], box[3+a]] on axis a
    uint32_t *touched;          // bit per row: set when a gradient lands on the row
    int32_t *tlist;             // the touched rows as a list (built by the sparse RMSProp step)
    int *tcount;                // its length
    int *status;
    int R;
    int form;
    int64_t M;
    float lo[3], hi[3], inv_h[3];
    float inv_h_lo[3];          // inv_h + inv_h_lo = 1/h to ~2^-48 relative (double-float)
    float hmin;
};

// ------------------------------------------------------------------ double-float arithmetic
// A value hi + lo held as two floats (Dekker / Knuth error-free transformations).
// The march keeps the ray parameter t and the grid coordinates of each sample
// in this form: a plain FP32 coordinate near g ~ 500 is quantised to ~3e-5 of
// a cell, which on steep density fields moves colours by more than 1e-5; the
// pair form keeps the cell fraction exact to FP32 rounding of [0, 1).
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ DF df_two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

// (x.hi + x.lo) * (m.hi + m.lo)
__device__ __forceinline__ DF df_mul(DF x, DF m) {
    DF p = df_two_prod(x.hi, m.hi);
    return df_fast_two_sum(p.hi, p.lo + fmaf(x.hi, m.lo, x.lo * m.hi));
}

// (n.hi + n.lo) / d for a float d != 0
__device__ __forceinline__ DF df_div(DF n, float d) {
    const float q = n.hi / d;
    const float r = fmaf(-q, d, n.hi);  // exact remainder
    return df_fast_two_sum(q, (r + n.lo) / d);
}

__device__ __forceinline__ bool df_lt(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// (x.hi + x.lo) * m for a float m
__device__ __forceinline__ DF df_mul_f(DF x, float m) {
    DF p = df_two_prod(x.hi, m);
    return df_fast_two_sum(p.hi, fmaf(x.lo, m, p.lo));
}

// (n.hi + n.lo) / (d.hi + d.lo)
__device__ __forceinline__ DF df_div_df(DF n, DF d) {
    const float q1 = n.hi / d.hi;
    const DF r = df_add(n, df_mul_f(d, -q1));  // n - q1 d
    const float q2 = r.hi / d.hi;
    return df_fast_two_sum(q1, q2);
}

// sqrt(x.hi + x.lo), x > 0 (one Newton correction of the FP32 root)
__device__ __forceinline__ DF df_sqrt(DF x) {
    const float s = sqrtf(x.hi);
    const DF s2 = df_two_prod(s, s);
    const float corr = ((x.hi - s2.hi) - s2.lo + x.lo) / (2.0f * s);
    return df_fast_two_sum(s, corr);
}

__device__ __forceinline__ void report(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Real spherical harmonics of degree <= 2 at unit direction d (Sec. 3.2),
// order m = -l..l per degree: Y0 | -c1 y, c1 z, -c1 x | c2 xy, -c2 yz,
// c3 (3z^2-1), -c2 xz, c4 (x^2-y^2); c1 = sqrt(3/(4pi)), c2 = sqrt(15/pi)/2,
// c3 = sqrt(5/pi)/4, c4 = sqrt(15/pi)/4.
__device__ __forceinline__ void sh_basis(const float d[3], float Y[9]) {
    const float c0 = 0.28209479177387814f;
    const float c1 = 0.48860251190291992f;
    const float c2 = 1.09254843059207907f;
    const float c3 = 0.31539156525252005f;
    const float c4 = 0.54627421529603959f;
    const float x = d[0], y = d[1], z = d[2];
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c2 * x * y;
    Y[5] = -c2 * y * z;
    Y[6] = c3 * (3.0f * z * z - 1.0f);
    Y[7] = -c2 * x * z;
    Y[8] = c4 * (x * x - y * y);
}

// Slab clip against the grid box in double-float; t_near = max(t_in, 0).
// Returns hit (false for a miss, a zero direction or non-finite input).
__device__ __forceinline__ bool clip_box(const GridView &g, const float o[3], const float d[3], DF &tn, DF &tf) {
    DF t0 = {0.0f, 0.0f}, t1 = {INFINITY, 0.0f};
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            ok = ok && !(o[a] < g.lo[a] || o[a] > g.hi[a]);
        } else {
            const DF ta = df_div(df_two_sum(g.lo[a], -o[a]), d[a]);
            const DF tb = df_div(df_two_sum(g.hi[a], -o[a]), d[a]);
            const bool sw = df_lt(tb, ta);
            const DF tmin = sw ? tb : ta, tmax = sw ? ta : tb;
            if (df_lt(t0, tmin)) t0 = tmin;
            if (df_lt(tmax, t1)) t1 = tmax;
        }
    }
    tn = t0;
    tf = t1;
    // t1 stays +inf only for a zero (or NaN) direction: no march
    return ok && df_lt(t0, t1) && t1.hi < INFINITY && t0.hi == t0.hi;
}

// Warp inclusive prefix sum (lane order).
__device__ __forceinline__ float warp_incl_scan(float x, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        float v = __shfl_up_sync(kFull, x, off);
        if (lane >= off) x += v;
    }
    return x;
}

// Warp inclusive suffix sum (sum over lanes >= this lane).
__device__ __forceinline__ float warp_incl_suffix(float x, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        float v = __shfl_down_sync(kFull, x, off);
        if (lane + off < 32) x += v;
    }
    return x;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(kFull, x, off);
    return x;
}

// Cell of a sample: grid coordinates clamped to [0, R-1], base = min(floor, R-2),
// f = g - base, from double-float coordinates.
struct Cell {
    int64_t base;   // linear id of the cell's (0,0,0) node
    float f[3];     // fractions
    int par;        // parities of the cell's integer coordinates: bit 2 x, bit 1 y, bit 0 z
};

__device__ __forceinline__ Cell locate(const GridView &g, const DF gc[3]) {
    Cell c;
    int b[3];
    const float rm1 = (float)(g.R - 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        DF x = gc[a];
        if (!(x.hi > 0.0f) || (x.hi == 0.0f)) x = {0.0f, 0.0f};  // also maps NaN to 0
        if (x.hi >= rm1) x = {rm1, 0.0f};
        float fl = floorf(x.hi);
        if (fl == x.hi && x.lo < 0.0f) fl -= 1.0f;
        int bi = (int)fl;
        bi = max(0, min(bi, g.R - 2));
        b[a] = bi;
        const float fr = (x.hi - (float)bi) + x.lo;
        c.f[a] = fminf(fmaxf(fr, 0.0f), 1.0f);
    }
    c.base = ((int64_t)b[0] * g.R + b[1]) * g.R + b[2];
    c.par = ((b[0] & 1) << 2) | ((b[1] & 1) << 1) | (b[2] & 1);
    return c;
}

// The 8 corners of a cell in slot order.  Slot i takes, along each axis a, the node whose coordinate has
// the parity of i's bit for a (bit 2 x, bit 1 y, bit 0 z): slot i of every cell is its one corner with
// parity pattern i.  Two cells sharing a node then hold it in the same slot, so when a warp's lanes load
// their cells' slot i in one instruction, every node shared by neighbouring samples is one address and
// is fetched once.  Canonical order (par = 0) is slot i = corner i.
struct Corners {
    int64_t base;
    int off[3][2];   // node offset along each axis for slot bit 0 / 1
    float w[3][2];   // trilinear weight factor along each axis for slot bit 0 / 1
};

__device__ __forceinline__ Corners corners_of(const GridView &g, const Cell &c, int par) {
    Corners k;
    k.base = c.base;
    const int stride[3] = {g.R * g.R, g.R, 1};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int p = (par >> (2 - a)) & 1;  // slot bit b selects the node at offset b ^ p
        k.off[a][0] = p ? stride[a] : 0;
        k.off[a][1] = p ? 0 : stride[a];
        k.w[a][0] = p ? c.f[a] : 1.0f - c.f[a];
        k.w[a][1] = p ? 1.0f - c.f[a] : c.f[a];
    }
    return k;
}

__device__ __forceinline__ int64_t slot_node(const Corners &k, int i) {
    return k.base + (k.off[0][(i >> 2) & 1] + k.off[1][(i >> 1) & 1] + k.off[2][i & 1]);
}

__device__ __forceinline__ float slot_weight(const Corners &k, int i) {
    return k.w[0][(i >> 2) & 1] * k.w[1][(i >> 1) & 1] * k.w[2][i & 1];
}

__device__ __forceinline__ bool cell_occupied(const GridView &g, int64_t base) {
    return (__ldg(g.occ + (base >> 5)) >> (base & 31)) & 1u;
}

__device__ __forceinline__ int64_t corner_node(const GridView &g, int64_t base, int c) {
    const int64_t R = g.R;
    return base + ((c >> 2) & 1) * R * R + ((c >> 1) & 1) * R + (c & 1);
}

__device__ __forceinline__ float corner_weight(const float f[3], int c) {
    float wx = ((c >> 2) & 1) ? f[0] : 1.0f - f[0];
    float wy = ((c >> 1) & 1) ? f[1] : 1.0f - f[1];
    float wz = (c & 1) ? f[2] : 1.0f - f[2];
    return wx * wy * wz;
}

// Row index of node n, or -1 (NULL, or out-of-range row recorded as corrupt).
__device__ __forceinline__ int32_t row_of(const GridView &g, int64_t n) {
    int32_t r = __ldg(g.idx + n);
    if (r >= 0 && (int64_t)r >= g.M) {
        report(g.status, kDevBadRow);
        r = -1;
    }
    return r;
}

// Accumulate w * row r (all 28 values) into acc.
__device__ __forceinline__ void accum_row(const GridView &g, int form, int32_t r, float w, float acc[kNV]) {
    if (form == PLX_SH_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(g.rows + (int64_t)r * kRowF);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            float4 v = __ldg(p + q);
            acc[4 * q + 0] = fmaf(w, v.x, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(w, v.y, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(w, v.z, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(w, v.w, acc[4 * q + 3]);
        }
    } else {
        const uint4 *p = reinterpret_cast<const uint4 *>(g.rows_h + (int64_t)r * kRowH);
        uint32_t wd[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4 v = __ldg(p + q);
            wd[4 * q + 0] = v.x;
            wd[4 * q + 1] = v.y;
            wd[4 * q + 2] = v.z;
            wd[4 * q + 3] = v.w;
        }
        acc[0] = fmaf(w, __uint_as_float(wd[0]), acc[0]);
        // SH value s (0..26) is the bf16 in slot 2 + s: word 1 + s/2, low half if s even.
#pragma unroll
        for (int s = 0; s < 27; ++s) {
            uint32_t word = wd[1 + (s >> 1)];
            uint32_t bits = (s & 1) ? (word & 0xffff0000u) : (word << 16);
            acc[1 + s] = fmaf(w, __uint_as_float(bits), acc[1 + s]);
        }
    }
}

__device__ __forceinline__ float row_sigma(const GridView &g, int form, int32_t r) {
    if (form == PLX_SH_F32) return __ldg(g.rows + (int64_t)r * kRowF);
    return __uint_as_float(__ldg(reinterpret_cast<const uint32_t *>(g.rows_h + (int64_t)r * kRowH)));
}

// Set row r's bit in the touched mask (fire-and-forget reduction; the result is unused).
__device__ __forceinline__ void mark_touched(const GridView &g, int32_t r) {
    atomicOr(g.touched + (r >> 5), 1u << (r & 31));
}

// ------------------------------------------------------------------ launchers (host)
struct RenderParams {
    float delta;      // sample spacing (world units), hi part
    float delta_lo;   // lo part: delta + delta_lo = step_vox * min h to double-float accuracy
    float bg[3];
    float stop;
    int max_chunks;
    // Cauchy sparsity prior (adjoints only): lam_s sum log(1 + 2 sigma^2) over the taken samples;
    // lam_s = 0 leaves it out, loss_s (nullable) accumulates its value
    float lam_s;
    float *loss_s;
};

// March state written by plx_render_train and read by plx_render_backward_train.
// Per ray: the number of compacted (occupied-cell) samples and, per chunk of 32
// of them, the sample-index range [first, last + 1) that holds them; per
// chunk a float4 that first holds the chunk's local colour and transmittance
// product (C_loc, P) and, after the per-ray combine, the remaining colour after
// the chunk and the transmittance before it (R_after, T_before); a flag for
// chunks with positive density; the flat list of (ray, chunk) work items; and,
// when sample indices fit in 16 bits, each chunk's 32 sample indices and the
// forward's interpolated density and colour pre-activations of each sample
// (so the adjoint needs the corner indices and weights only, not the rows).
struct MarchHeader {
    uint32_t magic;
    int32_t max_chunks;
    int64_t n;
    int32_t total_items;  // appended to by the plan kernel
    int32_t R;
    int64_t M;
    float delta, delta_lo, stop;
    int32_t mode;         // kMarchChunked, or kMarchRecompute when the adjoint re-marches
    const void *ro, *rd;  // the rays the state belongs to
    const void *rows;     // the grid's row storage
};
constexpr uint32_t kMarchMagic = 0x53584c50u;
enum : int32_t { kMarchChunked = 1, kMarchRecompute = 2 };

constexpr size_t kRaySetupBytes = 128;  // the march's per-ray setup (RaySetup, plx_march.cuh)

struct MarchLayout {
    size_t hdr_off, nocc_off, done_off, first_off, items_off, part_off, live_off, samp_off, vals_off, setup_off, total;
    // the plan stores each chunk's sample indices (uint16) when every index fits
    static bool store_samples(int max_chunks) { return (int64_t)max_chunks * 32 <= 65536; }
    static size_t round256(size_t b) { return (b + 255) & ~size_t(255); }
    static MarchLayout make(int64_t n, int max_chunks) {
        MarchLayout L;
        const size_t slots = size_t(n) * size_t(max_chunks);
        L.hdr_off = 0;
        L.nocc_off = 256;
        L.done_off = L.nocc_off + round256(size_t(n) * 4);
        L.first_off = L.done_off + round256(size_t(n) * 4);
        L.items_off = L.first_off + round256(slots * 8);
        L.part_off = L.items_off + round256(slots * 8);
        L.live_off = L.part_off + round256(slots * 16);
        L.samp_off = L.live_off + round256(slots);
        L.vals_off = L.samp_off + (store_samples(max_chunks) ? round256(slots * 64) : 0);
        L.setup_off = L.vals_off + (store_samples(max_chunks) ? round256(slots * 32 * 16) : 0);
        L.total = L.setup_off + round256(size_t(n) * kRaySetupBytes);
        return L;
    }
};

struct MarchPtrs {
    MarchHeader *hdr;
    int32_t *n_occ;   // [n] compacted samples per ray
    int32_t *done;    // [n] the ray's chunks the forward has finished (set to 0 by the plan)
    int2 *range;      // [n][max_chunks] the sample-index range [first, last + 1) of each chunk
    int2 *items;      // [total_items] (ray, chunk)
    float4 *part;     // [n][max_chunks] (C_loc, P), then (R_after, T_before)
    uint8_t *live;    // [n][max_chunks] 1 if any sample of the chunk has positive density
    uint16_t *samp;   // [n][max_chunks][32] the chunk's sample indices, or null (then chunks rescan)
    float4 *vals;     // [n][max_chunks][32] each sample's (sigma, pre_R, pre_G, pre_B) from the forward, or null
    void *setup;      // [n] the rays' march setup (RaySetup: clip, grid-space origin and direction, SH basis)
    int max_chunks;
};

cudaError_t launch_gen_rays(const float *cams, int n_cams, int W, int H, const int64_t *pix, int64_t n,
                            float *o, float *d, cudaStream_t s);
cudaError_t launch_render(const GridView &g, const float *o, const float *d, int64_t n,
                          const RenderParams &p, float *rgb, float *T_end, cudaStream_t s);
cudaError_t launch_render_backward(const GridView &g, const float *o, const float *d, int64_t n,
                                   const RenderParams &p, const float *grad_rgb, float *grad_rows,
                                   cudaStream_t s);
cudaError_t launch_march_plan(const GridView &g, const float *o, const float *d, int64_t n, const RenderParams &p,
                              const MarchPtrs &st, const MarchHeader &hdr, cudaStream_t s);
cudaError_t launch_render_planned(const GridView &g, const float *o, const float *d, int64_t n,
                                  const RenderParams &p, const MarchPtrs &st, const MarchHeader &hdr, float *rgb,
                                  float *T_end, const float *target, float *grad_rgb, float *loss, cudaStream_t s);
cudaError_t launch_render_train(const GridView &g, const float *o, const float *d, int64_t n, const RenderParams &p,
                                const MarchPtrs &st, const MarchHeader &hdr, float *rgb, float *T_end, cudaStream_t s);
cudaError_t launch_render_backward_train(const GridView &g, const float *o, const float *d, int64_t n,
                                         const RenderParams &p, const MarchPtrs &st, const MarchHeader &hdr,
                                         const float *grad_rgb, float *grad_rows, cudaStream_t s);
cudaError_t launch_render_tiles(const GridView *g, const RenderParams *p, int n_scenes, const float *cams,
                                int n_cams, const plx_tile *tiles, int64_t n_tiles, cudaStream_t s);
cudaError_t launch_count_nodes(const GridView &g, const float *o, const float *d, int64_t n, const RenderParams &p,
                               int64_t *out, cudaStream_t s);
cudaError_t launch_max_weight(const GridView &g, const float *o, const float *d, int64_t n, const RenderParams &p,
                              float *wmax, cudaStream_t s);
cudaError_t launch_count_touched(const GridView &g, int64_t *out, cudaStream_t s);
cudaError_t launch_mse_grad(const float *rgb, const float *target, int64_t n, float *grad, float *loss,
                            cudaStream_t s);
cudaError_t launch_build_occupancy(const GridView &g, uint32_t *occ, uint32_t *occ_coarse, cudaStream_t s);
cudaError_t launch_pack_bf16(const GridView &g, uint16_t *rows_h, cudaStream_t s);
cudaError_t launch_tv(const GridView &g, const int64_t *seg_start, const int64_t *seg_len, int64_t n_seg,
                      int64_t n_selected, float scale_sigma, float scale_sh, float *grad_rows, float *loss,
                      cudaStream_t s);
// sparse: g.tcount is this call's list length (zero on entry), next_count the next call's (zeroed here)
cudaError_t launch_rmsprop(const GridView &g, float *rows, uint16_t *rows_h, float *grad, float *v,
                           float lr_sigma, float lr_sh, float beta, float eps, int sparse, int *next_count,
                           cudaStream_t s);

// prune / upsample (plx_gridops.cu)
size_t prune_ws_bytes(int64_t R);
size_t upsample_ws_bytes(int64_t R2);
// key: a per-row value compared with tau (the weight-threshold form), or nullptr for the density
cudaError_t launch_prune_count(const GridView &g, const float *key, float tau, int dilate, void *ws, cudaStream_t s);
cudaError_t launch_prune_apply(const GridView &g, const void *ws, int64_t n_keep, int32_t *idx_new,
                               float *rows_new, cudaStream_t s);
cudaError_t launch_upsample_count(const GridView &g, int R2, void *ws, cudaStream_t s);
cudaError_t launch_upsample_apply(const GridView &g, int R2, const void *ws, int64_t n_new, int32_t *idx_new,
                                  float *rows_new, cudaStream_t s);
// total kept/occupied count written by the count kernels, at this byte offset of ws
constexpr size_t kWsCountOff = 0;

// host helpers defined in plx_api.cu for entry points in other translation units
const GridView *grid_view(const plx_grid *grid);  // NULL for a NULL grid
plx_status set_error(plx_status s, const char *message);

}  // namespace plx
