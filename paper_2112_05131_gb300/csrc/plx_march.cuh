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
// Sample s of a ray lies at t_s = t_near + s delta (Eq. 1's fixed step), i.e. at grid coordinates
// g0 + s st per axis, with g0 = (o - lo + t_near d) / h the point where the ray enters the box and
// st = delta d / h the step between samples.  Both are double-floats formed once per ray, so a
// sample's coordinates cost one exact product and one double-float addition.
struct __align__(16) RaySetup {  // 128 bytes: the training march keeps one per ray in its state
    DF g0[3];      // grid coordinates at t_near
    DF st[3];      // grid-coordinate step between consecutive samples
    float Y[9];    // SH basis at the direction
    float feps;    // bound on |FP32 - exact| grid coordinate of any candidate of the ray (see test_candidate)
    int hit;       // the ray meets the box (1), misses it (0); < 0: no ray (a pixel outside its image)
    int s_lo, s_hi;  // samples outside [s_lo, s_hi) are past t_far or lie in empty cells
    float pad_[7];
};
static_assert(sizeof(RaySetup) == 128, "RaySetup layout");

// t_s = t_near + s * delta as a double-float (s * delta_hi is exact for s < 2^24).
__device__ __forceinline__ DF sample_t(DF tn, const RenderParams &p, int s) {
    DF sd = df_two_prod((float)s, p.delta);
    sd.lo = fmaf((float)s, p.delta_lo, sd.lo);
    return df_add(tn, sd);
}

__device__ __forceinline__ RaySetup ray_setup_od(const GridView &g, const RenderParams &p, const float o[3],
                                                 const float d[3]) {
    RaySetup rs;
    DF tn, tf;
    rs.hit = clip_box(g, o, d, tn, tf);
    sh_basis(d, rs.Y);
    rs.s_lo = rs.s_hi = 0;
    rs.feps = 0.0f;
#pragma unroll
    for (int q = 0; q < 7; ++q) rs.pad_[q] = 0.0f;
    if (!rs.hit) {
#pragma unroll
        for (int a = 0; a < 3; ++a) rs.g0[a] = rs.st[a] = DF{0.0f, 0.0f};
        return rs;
    }
    const DF del = {p.delta, p.delta_lo};
    float gmax = 0.0f, smax = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const DF ih = {g.inv_h[a], g.inv_h_lo[a]};
        rs.g0[a] = df_mul(df_add(df_two_sum(o[a], -g.lo[a]), df_mul_f(tn, d[a])), ih);
        rs.st[a] = df_mul(df_mul_f(del, d[a]), ih);
        gmax = fmaxf(gmax, fabsf(rs.g0[a].hi));
        smax = fmaxf(smax, fabsf(rs.st[a].hi));
    }
    // s_end: the number of samples with t_s < t_far, decided in double-float (the FP32 estimate is
    // within one sample of it); samples beyond max_chunks * 32 do not exist.
    const int cap = p.max_chunks * 32;
    int k = (int)fminf(fmaxf(ceilf((tf.hi - tn.hi) / p.delta), 0.0f), (float)cap);
    for (int it = 0; it < 8 && k > 0 && !df_lt(sample_t(tn, p, k - 1), tf); ++it) --k;
    for (int it = 0; it < 8 && k < cap && df_lt(sample_t(tn, p, k), tf); ++it) ++k;
    const int s_end = k;
    // The cheap test's coordinate x32 = fma(s, st.hi, g0.hi) differs from the exact g0 + s st by at most
    // u |x32| + |g0.lo| + s |st.lo| <= u (2 |g0| + 2 s |st|) with u = 2^-24 (one rounding; the lo parts
    // are at most u of their hi parts).  Candidates, and the last sample of a candidate group, have
    // s < s_end + 8; the margin is that bound plus a quarter.
    rs.feps = 1.25f * 5.9604645e-8f * (2.0f * gmax + 2.0f * (float)(s_end + 8) * smax);
    // The candidate range: every cell with an occupied corner lies in the box of cells [lo, hi] (grid
    // coordinates [lo, hi + 1]); a sample whose coordinate is outside that box widened by one cell on
    // every side (far more than the FP32 error) is in an empty cell.  Slab test in FP32 on the sample
    // index, widened by two samples on each side, within [0, s_end).
    float s0 = 0.0f, s1 = (float)s_end;
    bool any = s_end > 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float blo = (float)(g.R - 1 - __ldg(g.occ_box + a)) - 1.0f;
        const float bhi = (float)__ldg(g.occ_box + 3 + a) + 2.0f;
        any = any && blo <= bhi;
        if (rs.st[a].hi == 0.0f) {
            any = any && rs.g0[a].hi >= blo && rs.g0[a].hi <= bhi;
        } else {
            const float inv = 1.0f / rs.st[a].hi;
            const float ta = (blo - rs.g0[a].hi) * inv, tb = (bhi - rs.g0[a].hi) * inv;
            s0 = fmaxf(s0, fminf(ta, tb));
            s1 = fminf(s1, fmaxf(ta, tb));
        }
    }
    if (any && s0 <= s1) {
        rs.s_lo = (int)fminf(fmaxf(floorf(s0) - 2.0f, 0.0f), (float)s_end);
        rs.s_hi = (int)fminf(fmaxf(ceilf(s1) + 3.0f, 0.0f), (float)s_end);
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

// Grid coordinates of sample s: g0 + s st per axis, as double-floats (s st.hi is exact).
__device__ __forceinline__ void coords_at(const RaySetup &rs, int s, DF gc[3]) {
    const float sf = (float)s;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        DF q = df_two_prod(sf, rs.st[a].hi);
        q.lo = fmaf(sf, rs.st[a].lo, q.lo);
        gc[a] = df_add(rs.g0[a], q);
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

// 256-bit read-only loads (sm_100 and later): eight 32-bit values from a 32-byte aligned address in one
// instruction, so a 128-byte F32 row takes four loads and a 64-byte BF16-SH row two.
struct F8 {
    float v[8];
};
struct U8 {
    uint32_t v[8];
};
__device__ __forceinline__ F8 ldg8_pinned(const float *p) {
    F8 r;
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]),
                   "=f"(r.v[7])
                 : "l"(p));
    return r;
}
__device__ __forceinline__ U8 ldg8_pinned(const uint32_t *p) {
    U8 r;
    asm volatile("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]), "=r"(r.v[6]),
                   "=r"(r.v[7])
                 : "l"(p));
    return r;
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
// receive the corners: rows_out[k] is corner k's row (canonical order), unless
// SLOTS, when the corners are loaded and returned in slot order (corners_of), which
// lets lanes share the loads of common nodes; forward-only callers use that.
template <bool SLOTS = false>
__device__ __forceinline__ bool gather_sample(const GridView &g, int form, const DF gc[3], float acc[kNV],
                                              int32_t rows_out[8], float f_out[3], int64_t *base_out = nullptr) {
#pragma unroll
    for (int q = 0; q < kNV; ++q) acc[q] = 0.0f;
    const Cell c = locate(g, gc);
    const Corners cn = corners_of(g, c, SLOTS ? c.par : 0);
    if (base_out) *base_out = c.base;
    f_out[0] = c.f[0];
    f_out[1] = c.f[1];
    f_out[2] = c.f[2];
    int32_t r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = row_of(g, slot_node(cn, k));
    // every corner's row is requested before any is used: one memory round trip per
    // chunk instead of eight (a NULL corner contributes w * 0, i.e. nothing)
    if (form == PLX_SH_F32) {
        // four 256-bit loads per row (the last holds SH 23..26 and the row's 4 pad floats)
        F8 v[8][4];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float *p = g.rows + (int64_t)max(r[k], 0) * kRowF;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (r[k] >= 0) {
                    v[k][q] = ldg8_pinned(p + 8 * q);
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[k][q].v[e] = 0.0f;
                }
            }
        }
        // an empty volatile use of every loaded value, after all the loads: no FMA can be
        // scheduled between two loads, so all 32 requests are in flight together
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int e = 0; e < 8; e += 4)
                    asm volatile("" : "+f"(v[k][q].v[e]), "+f"(v[k][q].v[e + 1]), "+f"(v[k][q].v[e + 2]),
                                 "+f"(v[k][q].v[e + 3]));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float w = slot_weight(cn, k);
            // scalar FMAs: packed pairs (fma.rn.f32x2) measured no faster here (the F32 gather is bound by
            // its loads, not by FMA issue)
#pragma unroll
            for (int q = 0; q < kNV; ++q) acc[q] = fmaf(w, v[k][q >> 3].v[q & 7], acc[q]);
        }
    } else {
        U8 v[8][2];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t *p = reinterpret_cast<const uint32_t *>(g.rows_h + (int64_t)max(r[k], 0) * kRowH);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (r[k] >= 0) {
                    v[k][q] = ldg8_pinned(p + 8 * q);
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[k][q].v[e] = 0u;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int e = 0; e < 8; e += 4)
                    asm volatile("" : "+r"(v[k][q].v[e]), "+r"(v[k][q].v[e + 1]), "+r"(v[k][q].v[e + 2]),
                                 "+r"(v[k][q].v[e + 3]));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float w = slot_weight(cn, k);
            uint32_t wd[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) wd[e] = v[k][e >> 3].v[e & 7];
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
constexpr int kGroupLog = 3;
constexpr int kCand = 1 << kGroupLog;  // candidates per lane per refill
constexpr int kRing = kCand <= 8 ? 512 : 1024;  // ring capacity >= 31 + 32 kCand, a power of two
static_assert(kRing >= 31 + 32 * kCand, "ring capacity");

// Is the cell of sample s (s_lo <= s < s_hi: every such sample is before t_far) non-empty?  The answer
// must equal the double-float one exactly (it decides which samples are marched).  Plain FP32
// coordinates are within rs.feps of the exact ones (the bound derived in ray_setup_od); a candidate whose
// FP32 coordinate lies within rs.feps of a cell face or of the box on any axis is re-evaluated in
// double-float, so the cheap path is taken only where both agree.
// The double-float decision for sample s (rare: near a cell face or the box), kept out of line so
// that the unrolled candidate loops stay small.
// Everything is passed by value, so that no caller's setup has to live in addressable memory.
static __device__ __noinline__ bool exact_occupied(const uint32_t *__restrict__ occ, int R, float g0x, float g0x_lo,
                                            float g0y, float g0y_lo, float g0z, float g0z_lo, float stx,
                                            float stx_lo, float sty, float sty_lo, float stz, float stz_lo, int s) {
    RaySetup rs;
    rs.g0[0] = DF{g0x, g0x_lo};
    rs.g0[1] = DF{g0y, g0y_lo};
    rs.g0[2] = DF{g0z, g0z_lo};
    rs.st[0] = DF{stx, stx_lo};
    rs.st[1] = DF{sty, sty_lo};
    rs.st[2] = DF{stz, stz_lo};
    DF gc[3];
    coords_at(rs, s, gc);
    GridView g;
    g.R = R;
    g.occ = occ;
    return cell_occupied(g, locate(g, gc).base);
}

__device__ __forceinline__ bool test_candidate(const GridView &g, const RaySetup &rs, int s) {
    const float sf = (float)s;
    bool exact = false;
    int b[3];
    const float half = 0.5f * (float)(g.R - 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = fmaf(sf, rs.st[a].hi, rs.g0[a].hi);
        const float fl = floorf(x);
        exact = exact || fabsf((x - fl) - 0.5f) > 0.5f - rs.feps;
        exact = exact || fabsf(x - half) > half - rs.feps;
        b[a] = (int)fl;
    }
    if (exact)
        return exact_occupied(g.occ, g.R, rs.g0[0].hi, rs.g0[0].lo, rs.g0[1].hi, rs.g0[1].lo, rs.g0[2].hi, rs.g0[2].lo,
                              rs.st[0].hi, rs.st[0].lo, rs.st[1].hi, rs.st[1].lo, rs.st[2].hi, rs.st[2].lo, s);
    // here 0 <= b < R - 1 on every axis; the linear id fits 32 bits below R = 1291
    const int64_t base = g.R <= 1290 ? (int64_t)((b[0] * g.R + b[1]) * g.R + b[2])
                                     : ((int64_t)b[0] * g.R + b[1]) * g.R + b[2];
    return cell_occupied(g, base);
}

// --------------------------------------------------------------------------- coarse skipping
// Before the per-sample test, candidates are screened in groups of kGroup consecutive samples
// against the coarse mask (one bit per 8^3-cell block): a group none of whose samples can lie in a
// non-empty cell is skipped whole.  A round of 32 kCand candidates is 32 groups, one per lane;
// candidate 32 j + l of the round belongs to group (32 j + l) / kGroup.
constexpr int kGroup = 1 << kGroupLog;
static_assert(32 * kCand == 32 * kGroup, "a round is one group per lane");

// Can a sample with index in [s0, s0 + kGroup) lie in a cell with an occupied corner?  Never false
// when one does.  The samples lie on the segment between the first and the last, whose FP32 grid
// coordinates are within rs.feps of the exact ones (the bound covers s < s_end + 8), so their cells
// lie in the box of cells of the two endpoints widened by feps, clamped as locate() clamps; the
// coarse bits of that box's blocks (at most 2 per axis; a wider box answers yes) decide.
__device__ __forceinline__ bool group_live(const GridView &g, const RaySetup &rs, int s0) {
    if (s0 >= rs.s_hi) return false;
    const float sa = (float)s0, sb = (float)(s0 + kGroup - 1);
    const float cmax = (float)(g.R - 2);
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xa = fmaf(sa, rs.st[a].hi, rs.g0[a].hi);
        const float xb = fmaf(sb, rs.st[a].hi, rs.g0[a].hi);
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

// Tests the candidates of one round starting at sample `first` (candidate 32 j + lane in occ[j]; those
// at or beyond `end` <= s_hi, or in skipped groups, answer empty) and returns the ballot of live groups.
__device__ __forceinline__ unsigned test_round(const GridView &g, const RaySetup &rs, int first, int end, int lane,
                                               bool occ[kCand]) {
    const unsigned live = __ballot_sync(kFull, group_live(g, rs, first + kGroup * lane));
#pragma unroll
    for (int j = 0; j < kCand; ++j) {
        const int s = first + 32 * j + lane;
        occ[j] = ((live >> ((32 * j + lane) >> kGroupLog)) & 1u) && s < end && test_candidate(g, rs, s);
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
__device__ __forceinline__ void refill(const GridView &g, const RaySetup &rs, int *ring, Stream &st, int lane) {
    const unsigned lt = (1u << lane) - 1u;
    while (st.tail - st.head < 32 && !st.exhausted) {
        bool occ[kCand];
        const unsigned live = test_round(g, rs, st.next, rs.s_hi, lane, occ);
        if (live) {  // uniform
#pragma unroll
            for (int j = 0; j < kCand; ++j) {
                // candidates 32 j .. 32 j + 31 form the round's groups 32 j / kGroup onwards: none of them
                // live, none occupied
                constexpr int kPerIter = 32 / kGroup;
                constexpr unsigned kIterMask = kPerIter >= 32 ? kFull : (1u << kPerIter) - 1u;
                if (((live >> (kPerIter * j)) & kIterMask) == 0u) continue;  // uniform
                const unsigned m = __ballot_sync(kFull, occ[j]);
                if (occ[j]) ring[(st.tail + __popc(m & lt)) & (kRing - 1)] = st.next + 32 * j + lane;
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

// The occupied samples with index in [first, end) (end <= s_hi), in order, into buf (at most 32 are kept).
__device__ __forceinline__ int scan_range(const GridView &g, const RaySetup &rs, int first, int end, int *buf,
                                          int lane) {
    const unsigned lt = (1u << lane) - 1u;
    int cnt = 0;
    for (int base = first; base < end; base += 32 * kCand) {
        bool occ[kCand];
        if (!test_round(g, rs, base, end, lane, occ)) continue;  // uniform
#pragma unroll
        for (int j = 0; j < kCand; ++j) {
            const unsigned m = __ballot_sync(kFull, occ[j]);
            const int pos = cnt + __popc(m & lt);
            if (occ[j] && pos < 32) buf[pos] = base + 32 * j + lane;
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
