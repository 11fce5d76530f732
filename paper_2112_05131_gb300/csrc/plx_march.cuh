// plx_march.cuh -- the pieces of the ray march (Eq. 1) that the forward, the
// adjoint and the chunk-parallel training kernels share: per-ray setup, sample
// positions, the trilinear gather, SH colour, chunk compositing and sample
// compaction against the occupancy mask.
#pragma once

#include "plx_internal.cuh"

namespace plx {

// Four resident 4-warp CTAs per SM: up to 128 registers a thread, enough for the
// gather to keep most of a chunk's row loads in flight (measured on the 512^3
// training batch against 2 and 3 CTAs, which buy more registers but fewer warps).
constexpr int kGatherBlocks = 4;

// --------------------------------------------------------------------------- per-ray setup
struct __align__(16) RaySetup {  // 128 bytes: the training march keeps one per ray in its state
    DF A[3];       // origin minus box corner, exact as a double-float
    float d[3];    // unit direction as given
    DF tn, tf;     // clipped parameter range
    float og[3];   // FP32 grid-coordinate origin and direction, for the cheap candidate test
    float dg[3];
    float Y[9];    // SH basis at the direction
    float feps;    // bound on |FP32 - exact| grid coordinate of any sample of the ray (see test_candidate)
    int hit;       // the ray meets the box
    int s_lo, s_hi;  // samples outside [s_lo, s_hi) lie in empty cells (outside the box of non-empty cells)
};
static_assert(sizeof(RaySetup) == 128, "RaySetup layout");

__device__ __forceinline__ RaySetup ray_setup_od(const GridView &g, const RenderParams &p, const float o[3],
                                                 const float d[3]) {
    RaySetup rs;
#pragma unroll
    for (int a = 0; a < 3; ++a) rs.d[a] = d[a];
    rs.hit = clip_box(g, o, rs.d, rs.tn, rs.tf);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        rs.A[a] = df_two_sum(o[a], -g.lo[a]);
        rs.og[a] = (o[a] - g.lo[a]) * g.inv_h[a];
        rs.dg[a] = rs.d[a] * g.inv_h[a];
    }
    sh_basis(rs.d, rs.Y);
    // The cheap test's coordinate x32 = fma(t32, dg, og) with t32 = fma(s, delta, t_near.hi) differs from
    // the exact (o - lo + t d) / h by at most u (inv_h (3 |o - lo| + 5 t) + |x|), u = 2^-24: og carries
    // 3 roundings, dg 2, t32 3 (t_near.lo, delta_lo, the fma), and the final fma 1.  Over the ray
    // t <= t_far and |x| <= R; the margin is that bound plus a quarter.
    float om = 0.0f, ih = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        om = fmaxf(om, fabsf(o[a] - g.lo[a]));
        ih = fmaxf(ih, g.inv_h[a]);
    }
    const float tmax = rs.hit ? fabsf(rs.tf.hi) : 0.0f;
    rs.feps = 1.25f * 5.9604645e-8f * (ih * (3.0f * om + 5.0f * tmax) + (float)g.R);
    // The candidate range: every cell with an occupied corner lies in the box of cells [lo, hi] (grid
    // coordinates [lo, hi + 1]); a sample whose coordinate is outside that box widened by one cell on
    // every side (far more than the FP32 error) is in an empty cell.  Slab test in FP32, then sample
    // indices widened by two on each side; samples beyond max_chunks * 32 do not exist.
    rs.s_lo = 0;
    rs.s_hi = 0;
    if (rs.hit) {
        float t0 = rs.tn.hi, t1 = rs.tf.hi;
        bool any = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float blo = (float)(g.R - 1 - __ldg(g.occ_box + a)) - 1.0f;
            const float bhi = (float)__ldg(g.occ_box + 3 + a) + 2.0f;
            any = any && blo <= bhi;
            if (rs.dg[a] == 0.0f) {
                any = any && rs.og[a] >= blo && rs.og[a] <= bhi;
            } else {
                const float ta = (blo - rs.og[a]) / rs.dg[a], tb = (bhi - rs.og[a]) / rs.dg[a];
                t0 = fmaxf(t0, fminf(ta, tb));
                t1 = fminf(t1, fmaxf(ta, tb));
            }
        }
        if (any && t0 <= t1) {
            const float sa = floorf((t0 - rs.tn.hi) / p.delta) - 2.0f;
            const float sb = ceilf((t1 - rs.tn.hi) / p.delta) + 3.0f;
            const float smax = (float)(p.max_chunks * 32);
            rs.s_lo = (int)fminf(fmaxf(sa, 0.0f), smax);
            rs.s_hi = (int)fminf(fmaxf(sb, 0.0f), smax);
        }
    }
    return rs;
}

__device__ __forceinline__ RaySetup ray_setup(const GridView &g, const RenderParams &p, const float *__restrict__ ro,
                                              const float *__restrict__ rd, int64_t ray) {
    float o[3], d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = __ldg(ro + 3 * ray + a);
        d[a] = __ldg(rd + 3 * ray + a);
    }
    return ray_setup_od(g, p, o, d);
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

// Packed FP32 arithmetic (fma.rn.f32x2): one instruction computes two independent fmaf, each
// rounded once as fmaf is, so results equal the scalar code's bit for bit.
__device__ __forceinline__ uint64_t f32x2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
// (a0, a1) += (w, w) * (x0, x1), with ww = f32x2(w, w)
__device__ __forceinline__ void fma2(float &a0, float &a1, uint64_t ww, float x0, float x1) {
    asm("{\n\t.reg .b64 acc, xx;\n\t"
        "mov.b64 acc, {%0, %1};\n\t"
        "mov.b64 xx, {%3, %4};\n\t"
        "fma.rn.f32x2 acc, %2, xx, acc;\n\t"
        "mov.b64 {%0, %1}, acc;\n\t}"
        : "+f"(a0), "+f"(a1)
        : "l"(ww), "f"(x0), "f"(x1));
}

// Full sample: interpolated values at grid point gc, whose cell the caller has
// already found occupied (compaction).  rows_out/f_out (and base_out, if given)
// receive the corners.
__device__ __forceinline__ bool gather_sample(const GridView &g, int form, const DF gc[3], float acc[kNV],
                                              int32_t rows_out[8], float f_out[3], int64_t *base_out = nullptr) {
#pragma unroll
    for (int q = 0; q < kNV; ++q) acc[q] = 0.0f;
    Cell c = locate(g, gc);
    if (base_out) *base_out = c.base;
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
            // scalar FMAs here: the packed form needs register pairs, and at the FP32 render kernels'
            // register cap it spilled more and measured slower
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
            const uint64_t ww = f32x2(w, w);
            acc[0] = fmaf(w, __uint_as_float(wd[0]), acc[0]);
            // SH pairs (2i, 2i+1) share word 1 + i: low half, then high half
#pragma unroll
            for (int i = 0; i < 13; ++i)
                fma2(acc[1 + 2 * i], acc[2 + 2 * i], ww, __uint_as_float(wd[1 + i] << 16),
                     __uint_as_float(wd[1 + i] & 0xffff0000u));
            acc[27] = fmaf(w, __uint_as_float(wd[14] << 16), acc[27]);
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
// are marched).  Plain FP32 coordinates are within rs.feps of the exact ones
// (the bound derived in ray_setup_od); a candidate whose FP32 coordinate lies
// within rs.feps of a cell face or of the box on any axis, or whose t lies
// within kTEps of t_far, is re-evaluated in double-float, so the cheap path is
// taken only where both agree.

__device__ __forceinline__ Cand test_candidate(const GridView &g, const RaySetup &rs, const RenderParams &p, int s) {
    Cand c;
    c.occ = false;
    c.valid = false;
    if (s >= rs.s_hi) return c;  // beyond the non-empty box (or past max_chunks * 32): no more samples
    if (s < rs.s_lo) {            // before the non-empty box: valid and empty
        c.valid = true;
        return c;
    }
    const float t32 = fmaf((float)s, p.delta, rs.tn.hi);
    const float kTEps = 1e-5f * (fabsf(rs.tf.hi) + 1.0f);
    bool exact = fabsf(t32 - rs.tf.hi) <= kTEps;
    if (!exact && t32 > rs.tf.hi) return c;  // clearly past t_far
    int b[3];
    // near a cell face: the fraction within feps of 0 or 1; near the box: x within feps of 0 or R-1
    const float half = 0.5f * (float)(g.R - 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = fmaf(t32, rs.dg[a], rs.og[a]);
        const float fl = floorf(x);
        exact = exact || fabsf((x - fl) - 0.5f) > 0.5f - rs.feps || fabsf(x - half) > half - rs.feps;
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
    // here 0 <= b < R - 1 on every axis; the linear id fits 32 bits below R = 1291
    const int64_t base = g.R <= 1290 ? (int64_t)((b[0] * g.R + b[1]) * g.R + b[2])
                                     : ((int64_t)b[0] * g.R + b[1]) * g.R + b[2];
    c.occ = cell_occupied(g, base);
    return c;
}

// --------------------------------------------------------------------------- coarse skipping
// Before the per-sample test, candidates are screened in groups of kGroup consecutive samples
// against the coarse mask (one bit per 8^3-cell block): a group none of whose samples can lie in a
// non-empty cell is skipped whole.  A round of 32 kCand = 256 candidates is 32 groups, one per lane;
// candidate 32 j + l of the round belongs to group 4 j + l / 8.
constexpr int kGroup = 8;
static_assert(32 * kCand == 32 * kGroup, "a round is one group per lane");

// Can a sample with index in [s0, s0 + kGroup) lie in a cell with an occupied corner?  Never false
// when one does.  The samples lie on the segment between the first and the last, whose FP32 grid
// coordinates are within rs.feps of the exact ones (the bound holds a fortiori a few samples past
// t_far, where the extra error is ~1e-6 of a cell against the bound's 25% slack), so their cells
// lie in the box of cells of the two endpoints widened by feps, clamped as locate() clamps; the
// coarse bits of that box's blocks (at most 2 per axis; a wider box answers yes) decide.
__device__ __forceinline__ bool group_live(const GridView &g, const RaySetup &rs, const RenderParams &p, int s0) {
    if (s0 >= rs.s_hi) return false;
    const float ta = fmaf((float)s0, p.delta, rs.tn.hi);
    const float tb = fmaf((float)(s0 + kGroup - 1), p.delta, rs.tn.hi);
    const float cmax = (float)(g.R - 2);
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xa = fmaf(ta, rs.dg[a], rs.og[a]);
        const float xb = fmaf(tb, rs.dg[a], rs.og[a]);
        const float c0 = fminf(fmaxf(floorf(fminf(xa, xb) - rs.feps), 0.0f), cmax);
        const float c1 = fminf(fmaxf(floorf(fmaxf(xa, xb) + rs.feps), 0.0f), cmax);
        lo[a] = (int)c0 >> kBlockLog;
        hi[a] = (int)c1 >> kBlockLog;
    }
    if (hi[0] - lo[0] > 1 || hi[1] - lo[1] > 1 || hi[2] - lo[2] > 1) return true;
    for (int i = lo[0]; i <= hi[0]; ++i)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int k = lo[2]; k <= hi[2]; ++k) {
                const int b = (i * g.nb + j) * g.nb + k;
                if ((__ldg(g.occ_coarse + (b >> 5)) >> (b & 31)) & 1u) return true;
            }
    return false;
}

// Tests the candidates of one round starting at sample `first` (candidate 32 j + lane in c[j]), the
// ones in skipped groups answering (invalid, empty), and returns the ballot of live groups.
__device__ __forceinline__ unsigned test_round(const GridView &g, const RaySetup &rs, const RenderParams &p, int first,
                                               int end, int lane, Cand c[kCand]) {
    const unsigned live = __ballot_sync(kFull, group_live(g, rs, p, first + kGroup * lane));
#pragma unroll
    for (int j = 0; j < kCand; ++j) {
        const int s = first + 32 * j + lane;
        c[j].valid = c[j].occ = false;
        if (((live >> (4 * j + (lane >> 3))) & 1u) && s < end) c[j] = test_candidate(g, rs, p, s);
    }
    return live;
}

struct Stream {
    int next;   // next candidate sample index to test
    int head;   // ring read position (absolute)
    int tail;   // ring write position (absolute)
    bool exhausted;
};

// Append occupied candidates until 32 are queued or the ray has no candidates left (none at or
// beyond s_hi).
__device__ __forceinline__ void refill(const GridView &g, const RaySetup &rs, const RenderParams &p, int *ring,
                                       Stream &st, int lane) {
    const unsigned lt = (1u << lane) - 1u;
    while (st.tail - st.head < 32 && !st.exhausted) {
        Cand c[kCand];
        if (test_round(g, rs, p, st.next, rs.s_hi, lane, c)) {  // uniform
#pragma unroll
            for (int j = 0; j < kCand; ++j) {
                const unsigned m = __ballot_sync(kFull, c[j].occ);
                if (c[j].occ) ring[(st.tail + __popc(m & lt)) & (kRing - 1)] = st.next + 32 * j + lane;
                st.tail += __popc(m);
            }
        }
        st.next += 32 * kCand;
        st.exhausted = st.next >= rs.s_hi;
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
        if (!test_round(g, rs, p, base, end, lane, c)) continue;  // uniform
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


// The Cauchy sparsity prior (Sec. 3.7, Eq. 4) at one sample of density sigma >= 0 (taken: every
// taken sample counts; sigma = 0 adds nothing): returns its density gradient
// lam_s 4 sigma / (1 + 2 sigma^2) and adds lam_s sum log(1 + 2 sigma^2) over the warp's samples to
// *p.loss_s (one atomic per warp).  Call from all 32 lanes.
__device__ __forceinline__ float sparsity_prior(const RenderParams &p, bool taken, float sigma) {
    if (p.lam_s == 0.0f) return 0.0f;  // uniform
    const float s2 = taken ? 2.0f * sigma * sigma : 0.0f;
    if (p.loss_s) {
        const float l = warp_sum(log1pf(s2));
        if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(p.loss_s, p.lam_s * l);
    }
    return taken ? p.lam_s * 4.0f * sigma / (1.0f + s2) : 0.0f;
}

// --------------------------------------------------------------------------- adjoint of one sample
// Gradients of one taken sample with positive density with respect to its
// interpolated values (the adjoint of Eq. 1 with SH colour and ReLUs), scattered
// to the cell's 8 corners with their trilinear weights (NULL corners skip):
//   dL/dsigma = delta sum_ch g_ch (T_{s+1} c_ch - R_ch) + gsig_prior,   R = colour after the sample,
//   dL/dk_{ch,l} = g_ch w [pre_ch > 0] Y_l,
// gsig_prior being the density gradient of a per-sample prior (sparsity_prior).
// Rows are accumulated with float4 atomics and marked in the touched mask.
//
// scatter_chunk does this for the 32 samples of a chunk, called by all 32 lanes (`scat`: this lane's sample is taken
// and has positive density).  Consecutive samples of a ray often share a cell (two per cell at half a
// voxel's step), and then their gradients go to the same 8 rows: since Y is the ray's, a corner k
// receives wk (gsig, gpre_0 Y, gpre_1 Y, gpre_2 Y), so four numbers per corner and sample carry all of it.
// Lanes are paired within each run of equal cells (positions 0-1, 2-3, ... of the run); the even lane
// adds its partner's 32 numbers (8 corners x 4, by shuffles) and scatters both, the odd lane nothing,
// which halves the atomics of such runs; then pairs of the remaining lanes whose cells are one step
// apart merge their 4 shared corners the same way.  `cell`: the sample's cell base node (any value when
// !scat).
__device__ __forceinline__ void scatter_chunk(const GridView &g, bool scat, int64_t cell, const int32_t rr[8],
                                              const float ff[3], const float Y[9], const float gr[3],
                                              const float pre[3], const float col[3], float w, float Tn,
                                              const float Rs[3], float delta, float gsig_prior,
                                              float *__restrict__ grad_rows, int lane) {
    float gsig = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) gsig = fmaf(gr[ch], Tn * col[ch] - Rs[ch], gsig);
    gsig = fmaf(gsig, delta, gsig_prior);
    float gpre[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) gpre[ch] = pre[ch] > 0.0f ? gr[ch] * w : 0.0f;
    float a[8], b[8][3];
    unsigned wmask = 0u;  // corners with a non-zero trilinear weight and a row
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float wk = scat && rr[k] >= 0 ? corner_weight(ff, k) : 0.0f;
        if (wk != 0.0f) wmask |= 1u << k;
        a[k] = wk * gsig;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) b[k][ch] = wk * gpre[ch];
    }
    // runs of equal cells among the scattering lanes; a lane continues a run when the previous one has
    // its cell (the key of a lane that does not scatter is unique)
    const int64_t key = scat ? cell : -1 - (int64_t)lane;
    const int64_t prev_key = __shfl_up_sync(kFull, key, 1);
    const unsigned cont = __ballot_sync(kFull, lane > 0 && prev_key == key);
    const unsigned upto = lane == 31 ? kFull : ((2u << lane) - 1u);
    const int start = 31 - __clz(~cont & upto);   // bit 0 of ~cont is always set
    const bool odd = ((lane - start) & 1) != 0;
    const bool absorb = !odd && lane < 31 && ((cont >> (lane + 1)) & 1u);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float an = __shfl_down_sync(kFull, a[k], 1);
        if (absorb) a[k] += an;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float bn = __shfl_down_sync(kFull, b[k][ch], 1);
            if (absorb) b[k][ch] += bn;
        }
    }
    const unsigned wn = __shfl_down_sync(kFull, wmask, 1);
    if (absorb) wmask |= wn;
    // Second level: the lanes left to scatter ("heads"), in lane order, are usually in cells one step
    // apart along an axis, which share 4 corners.  Heads are paired by rank (0-1, 2-3, ...); when a pair's
    // cells are one step apart, the even one adds the odd one's values for the 4 shared corners and the
    // odd one leaves them out.  Corner k = 4 cx + 2 cy + cz; along axis a the shared corners differ in
    // bit 4 >> a.
    const bool head = scat && !odd;
    const unsigned heads = __ballot_sync(kFull, head);
    const unsigned above = lane == 31 ? 0u : heads & ~((2u << lane) - 1u);
    const unsigned below = heads & ((1u << lane) - 1u);
    const int next_head = above ? __ffs(above) - 1 : lane;
    const int prev_head = below ? 31 - __clz(below) : lane;
    const bool even_rank = (__popc(below) & 1) == 0;
    // this head's partner: the next head (even rank) or the previous one (odd rank)
    const int partner = even_rank ? next_head : prev_head;
    const int64_t pcell = __shfl_sync(kFull, cell, partner);
    int bit = 0;       // the axis bit of the shared corners, 0: the cells are not one step apart
    bool up = false;   // the odd head's cell is the even head's plus one step
    if (head && partner != lane) {
        const int64_t R = g.R;
        const int64_t dlt = even_rank ? pcell - cell : cell - pcell;  // odd head's cell minus even head's
        const int64_t st = dlt < 0 ? -dlt : dlt;
        bit = st == 1 ? 1 : st == R ? 2 : st == R * R ? 4 : 0;
        up = dlt > 0;
    }
    float pa[8], pb[8][3];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        pa[k] = __shfl_sync(kFull, a[k], next_head);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) pb[k][ch] = __shfl_sync(kFull, b[k][ch], next_head);
    }
    const unsigned pw = __shfl_sync(kFull, wmask, next_head);
    if (bit != 0 && even_rank) {
        // corner k (with bit set iff up) is the odd head's corner k ^ bit
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool shared = up ? (k & bit) != 0 : (k & bit) == 0;
            if (!shared) continue;
            const int src = bit == 4 ? (k ^ 4) : bit == 2 ? (k ^ 2) : (k ^ 1);
            float sa = 0.0f, sb[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j == src) {
                    sa = pa[j];
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) sb[ch] = pb[j][ch];
                }
            a[k] += sa;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) b[k][ch] += sb[ch];
            wmask |= ((pw >> src) & 1u) << k;
        }
    } else if (bit != 0) {
        // the odd head leaves out its shared corners: those with bit clear iff up
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool shared = up ? (k & bit) == 0 : (k & bit) != 0;
            if (shared) wmask &= ~(1u << k);
        }
    }
    if (!scat || odd) return;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (!((wmask >> k) & 1u)) continue;
        float v[kNV];
        v[0] = a[k];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
#pragma unroll
            for (int l = 0; l < 9; ++l) v[1 + 9 * ch + l] = b[k][ch] * Y[l];
        float4 *dst = reinterpret_cast<float4 *>(grad_rows + (int64_t)rr[k] * kRowF);
#pragma unroll
        for (int q = 0; q < 7; ++q) atomicAdd(dst + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
        mark_touched(g, rr[k]);
    }
}

}  // namespace plx
