// plx_train.cu -- the chunk-parallel march of the optimisation step (Eq. 1 and
// its adjoint for a batch of training rays, Sec. 3.5 / Supp. B.1).
//
// Why a second march: a 5000-ray batch is about two waves of one-warp-per-ray
// work on a 152-SM part, and a ray through the dense shell and blobs carries
// 10-20x the average number of non-empty samples.  With a warp per ray those
// rays set the kernel time while most SMs idle.  Here every chunk of 32
// compacted samples of every ray is one work item of equal cost:
//
//   plan     (CTA per ray)     compacts the ray's samples against the
//                              occupancy mask, records the sample range of each
//                              chunk of 32, and appends its (ray, chunk) items;
//   chunks   (one resident wave, warps stride over the items)
//                              gathers a chunk and composites it from T = 1:
//                              local colour C_loc and transmittance product P;
//   combine  (in the chunks kernel, by the warp that finishes a ray's last chunk)
//                              T_before(k) = prod_{j<k} P_j, C = sum_k
//                              T_before(k) C_loc(k) + T_end bg, and, for the
//                              adjoint, R_after(k) = sum_{j>k} T_before(j)
//                              C_loc(j) + T_end bg (a suffix sum of
//                              non-negative terms: no cancellation);
//   adjoint  (one resident wave over the same items)
//                              takes each sample's density and colour
//                              pre-activations from the forward, recomputes
//                              T_s = T_before(k) x (in-chunk prefix) and R_s =
//                              R_after(k) + (in-chunk suffix), looks up the
//                              corner rows and scatters.
//
// The state between the calls lives in a caller buffer (MarchLayout).  The
// results equal plx_render / plx_render_backward up to FP32 summation order.
// Early termination (stop_thresh > 0) needs the global transmittance inside a
// chunk, so with stop_thresh > 0 the pair falls back to the one-warp-per-ray
// kernels, recorded in the state's mode.
#include <algorithm>
#include <mutex>

#include "plx_march.cuh"

namespace plx {

namespace {

constexpr int kPlanWarps = 4;
// Batches up to this many rays combine each ray inside the chunk kernel (one launch fewer on the
// step's critical path); larger ones launch the combine as a kernel of its own.
constexpr int64_t kFuseCombineMaxRays = 32768;
constexpr int kChunkWarps = 4;
// Resident CTAs per SM of the forward chunk kernel: 80 registers (at 4, 5 and 8 CTAs, 128, 96 and 64
// registers, the 5000-ray step measured 109.1, 109.0 and 111.2 us against 106.8 us at 6).
constexpr int kChunkFwdBlocks = 6;

int sm_count() {
    static std::mutex mu;
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

__global__ void march_header_kernel(MarchHeader *dst, MarchHeader v) { *dst = v; }

// ---------------------------------------------------------------------------- ray setup
// The per-ray setup (double-float clip, grid-space origin and direction, SH basis, FP32 margin),
// computed once per ray and read by the plan and by every chunk of the ray.
__device__ __forceinline__ const RaySetup &setup_of(const MarchPtrs &st, int64_t ray) {
    return reinterpret_cast<const RaySetup *>(st.setup)[ray];
}

__global__ void __launch_bounds__(128) march_setup_kernel(GridView g, RenderParams p, const float *__restrict__ ro,
                                                          const float *__restrict__ rd, int64_t n, MarchPtrs st) {
    const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n) return;
    reinterpret_cast<RaySetup *>(st.setup)[ray] = ray_setup(g, p, ro, rd, ray);
}

// ---------------------------------------------------------------------------- plan
// One CTA per ray: its kPlanWarps warps test interleaved spans of 256 candidates (span q by warp
// q mod kPlanWarps, candidate q 256 + 32 j + lane as in the other marches), keeping each span's
// ballot masks in shared memory; a prefix over the spans' counts then gives every occupied sample its
// rank, so a long ray is planned by four warps at once.  Spans are handled kPlanMaxSpans at a time.
constexpr int kPlanMaxSpans = 64;
constexpr int kSpan = 32 * kCand;  // candidates tested by one warp at a time

__global__ void __launch_bounds__(kPlanWarps * 32) march_plan_kernel(GridView g, const float *__restrict__ ro,
                                                                     const float *__restrict__ rd, int64_t n,
                                                                     RenderParams p, MarchPtrs st) {
    __shared__ uint32_t s_mask[kPlanMaxSpans * kCand];
    __shared__ int s_cnt[kPlanMaxSpans + 1];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t ray = blockIdx.x; ray < n; ray += gridDim.x) {  // uniform over the CTA
        const RaySetup rs = setup_of(st, ray);  // every thread: a broadcast load, no barrier
        if (threadIdx.x == 0) s_last = -1;  // read after phase 1's barrier
        const int mc = st.max_chunks;
        int2 *range = st.range + ray * mc;
        uint16_t *samp = st.samp ? st.samp + ray * mc * 32 : nullptr;  // chunk k's samples at [32 k, 32 k + 32)
        // s_hi <= max_chunks * 32, so every rank / 32 < max_chunks
        const int L = rs.hit > 0 ? rs.s_hi : 0;  // candidates outside [s_lo, s_hi) are empty or past t_far
        const int s_first = rs.s_lo;
        const int n_spans = L > s_first ? (L - s_first + kSpan - 1) / kSpan : 0;
        int n_occ = 0;
        for (int w0 = 0; w0 < n_spans; w0 += kPlanMaxSpans) {
            const int nw = min(kPlanMaxSpans, n_spans - w0);
            // phase 1: masks and counts of this window's spans
            for (int q = wid; q < nw; q += kPlanWarps) {
                const int base = s_first + (w0 + q) * kSpan;
                bool occ[kCand];
                test_round(g, rs, base, L, lane, occ);
                int cnt = 0;
#pragma unroll
                for (int j = 0; j < kCand; ++j) {
                    const unsigned m = __ballot_sync(kFull, occ[j]);
                    if (lane == 0) s_mask[q * kCand + j] = m;
                    cnt += __popc(m);
                }
                if (lane == 0) s_cnt[q] = cnt;
            }
            __syncthreads();
            // phase 2: exclusive prefix of the counts (from the ranks already given), and the last sample
            if (wid == 0) {
                int carry = n_occ;
                for (int q0 = 0; q0 < nw; q0 += 32) {
                    const int q = q0 + lane;
                    const int c = q < nw ? s_cnt[q] : 0;
                    int incl = c;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int v = __shfl_up_sync(kFull, incl, off);
                        if (lane >= off) incl += v;
                    }
                    if (q < nw) s_cnt[q] = carry + incl - c;
                    const unsigned nz = __ballot_sync(kFull, c > 0);
                    if (nz && lane == 0) {
                        const int ql = q0 + 31 - __clz((int)nz);  // last span with an occupied sample so far
                        for (int j = kCand - 1; j >= 0; --j) {
                            const unsigned m = s_mask[ql * kCand + j];
                            if (m) {
                                s_last = s_first + (w0 + ql) * kSpan + 32 * j + 31 - __clz((int)m);
                                break;
                            }
                        }
                    }
                    carry += __shfl_sync(kFull, incl, 31);
                }
                if (lane == 0) s_cnt[nw] = carry;
            }
            __syncthreads();
            // phase 3: every occupied sample of the window writes its chunk boundary and list entry
            for (int q = wid; q < nw; q += kPlanWarps) {
                const int base = s_first + (w0 + q) * kSpan;
                int rank0 = s_cnt[q];
#pragma unroll
                for (int j = 0; j < kCand; ++j) {
                    const unsigned m = s_mask[q * kCand + j];
                    if ((m >> lane) & 1u) {
                        const int rank = rank0 + __popc(m & lt);
                        const int sidx = base + 32 * j + lane;
                        if ((rank & 31) == 0) range[rank >> 5].x = sidx;
                        if ((rank & 31) == 31) range[rank >> 5].y = sidx + 1;
                        if (samp) samp[rank] = (uint16_t)sidx;
                    }
                    rank0 += __popc(m);
                }
            }
            n_occ = s_cnt[nw];
            __syncthreads();  // the next window reuses the shared arrays
        }
        if (threadIdx.x == 0) {
            const int nch = (n_occ + 31) >> 5;
            if (nch > 0) {
                range[nch - 1].y = s_last + 1;
                const int base = atomicAdd(&st.hdr->total_items, nch);
                for (int k = 0; k < nch; ++k) st.items[base + k] = make_int2((int)ray, k);
            }
            st.n_occ[ray] = n_occ;
            st.done[ray] = 0;
        }
        __syncthreads();  // the next ray reuses the shared setup
    }
}

// Does the state's header describe a plan of these rays, this grid and these options?
__device__ __forceinline__ bool header_matches(const MarchHeader &h, const MarchHeader &e) {
    return h.magic == kMarchMagic && h.mode == kMarchChunked && h.n == e.n && h.max_chunks == e.max_chunks &&
           h.R == e.R && h.M == e.M && __float_as_uint(h.delta) == __float_as_uint(e.delta) &&
           __float_as_uint(h.delta_lo) == __float_as_uint(e.delta_lo) &&
           __float_as_uint(h.stop) == __float_as_uint(e.stop) && h.ro == e.ro && h.rd == e.rd &&
           h.rows == e.rows && h.total_items >= 0 && (int64_t)h.total_items <= e.n * (int64_t)e.max_chunks;
}

// The inputs of one work item, loaded one item ahead so that their round trips overlap the
// previous item's gather: the ray, its compacted-sample count, and this lane's sample index when
// the plan stored the chunk's list.  The ray's setup follows through shared memory (SetupPipe).
struct ItemIn {
    int ray, k;  // ray -1: past the end of the list
    int n_occ;
    int s;
};

__device__ __forceinline__ int2 item_at(const MarchPtrs &st, int it, int total) {
    return it < total ? st.items[it] : make_int2(-1, 0);
}

__device__ __forceinline__ ItemIn load_item(const MarchPtrs &st, const float *__restrict__ ro,
                                            const float *__restrict__ rd, int2 id, int lane) {
    ItemIn r;
    r.ray = id.x;
    r.k = id.y;
    r.n_occ = 0;
    r.s = 0;
    if (id.x >= 0) {
        const int64_t ray = id.x;
        r.n_occ = st.n_occ[ray];
        // lanes past the chunk's count read unused slots of the list; their value is never used
        if (st.samp) r.s = st.samp[(ray * st.max_chunks + id.y) * 32 + lane];
    }
    return r;
}

// A warp's two shared-memory slots for ray setups: the next item's setup is copied in with cp.async
// (lanes 0-7, 16 bytes each) while the current item is processed, and read in place from there.
struct SetupPipe {
    RaySetup slot[2];
};

__device__ __forceinline__ void setup_fetch(SetupPipe &p, int buf, const MarchPtrs &st, int ray, int lane) {
    if (ray >= 0 && lane < 8) {
        const char *src = reinterpret_cast<const char *>(st.setup) + (int64_t)ray * kRaySetupBytes + 16 * lane;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char *>(&p.slot[buf]) + 16 * lane);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Waits until every fetch but the most recent one has landed, and makes it visible to the warp.
__device__ __forceinline__ void setup_wait_prev() {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncwarp();
}

// The samples of the item: returns the count (lane i gets sample s if i < count), from the plan's list
// when it stored one, else rescanned from the chunk's range; -1 when the rescan disagrees with the plan
// (reported; cannot happen for a deterministic occupancy test).
__device__ __forceinline__ int item_samples(const GridView &g, const RaySetup &rs, const RenderParams &p,
                                            const MarchPtrs &st, const ItemIn &in, int *buf, int lane, int &s) {
    const int expect = min(32, in.n_occ - 32 * in.k);
    if (st.samp) {
        s = lane < expect ? in.s : 0;
        return expect;
    }
    const int2 r = st.range[(int64_t)in.ray * st.max_chunks + in.k];
    const int cnt = scan_range(g, rs, r.x, r.y, buf, lane);
    s = lane < cnt ? buf[lane] : 0;
    __syncwarp();
    if (cnt != expect) {
        if (lane == 0) report(g.status, kDevCountMismatch);
        return -1;
    }
    return cnt;
}

// ---------------------------------------------------------------------------- combine
// One ray's combine: T before each chunk, the colour (and, with `target`, the MSE gradient 2 (C - target)
// / n of Sec. 3.5), and the colour arriving after each chunk for the adjoint.  Returns, in lane 0, the
// ray's squared error |C - target|^2 (0 without a target).
__device__ __forceinline__ float combine_ray(const RenderParams &p, const MarchPtrs &st, int64_t ray, int lane,
                                             float *__restrict__ rgb, float *__restrict__ T_out,
                                             const float *__restrict__ target, float *__restrict__ grad_rgb,
                                             float inv_n) {
    const int mc = st.max_chunks;
    const int nch = (st.n_occ[ray] + 31) >> 5;
    float4 *part = st.part + ray * mc;
    // forward over chunks: T_before and the colour
    float Tc = 1.0f;
    float C[3] = {0.0f, 0.0f, 0.0f};
    for (int b = 0; b < nch; b += 32) {
        const int k = b + lane;
        const bool valid = k < nch;
        const float4 q = valid ? part[k] : make_float4(0.0f, 0.0f, 0.0f, 1.0f);
        const float incl = warp_incl_prod(q.w, lane);
        float excl = __shfl_up_sync(kFull, incl, 1);
        if (lane == 0) excl = 1.0f;
        const float Tb = Tc * excl;
        C[0] = fmaf(Tb, q.x, C[0]);
        C[1] = fmaf(Tb, q.y, C[1]);
        C[2] = fmaf(Tb, q.z, C[2]);
        if (valid) part[k].w = Tb;
        Tc *= __shfl_sync(kFull, incl, 31);
    }
    C[0] = warp_sum(C[0]);
    C[1] = warp_sum(C[1]);
    C[2] = warp_sum(C[2]);
    float sq = 0.0f;
    if (lane == 0) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float c = fmaf(Tc, p.bg[ch], C[ch]);
            rgb[3 * ray + ch] = c;
            if (target) {
                const float diff = c - __ldg(target + 3 * ray + ch);
                grad_rgb[3 * ray + ch] = 2.0f * diff * inv_n;
                sq = fmaf(diff, diff, sq);
            }
        }
        if (T_out) T_out[ray] = Tc;
    }
    // reverse over chunks: the colour that arrives after each chunk
    float Rs[3] = {Tc * p.bg[0], Tc * p.bg[1], Tc * p.bg[2]};
    for (int b = nch > 0 ? ((nch - 1) >> 5) << 5 : -32; b >= 0; b -= 32) {
        const int k = b + lane;
        const bool valid = k < nch;
        const float4 q = valid ? part[k] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // (C_loc, T_before)
        const float cl[3] = {q.x, q.y, q.z};
        float Ra[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float suf = warp_incl_suffix(q.w * cl[ch], lane);
            float suf_ex = __shfl_down_sync(kFull, suf, 1);
            if (lane == 31) suf_ex = 0.0f;
            Ra[ch] = Rs[ch] + suf_ex;
            Rs[ch] += __shfl_sync(kFull, suf, 0);
        }
        if (valid) part[k] = make_float4(Ra[0], Ra[1], Ra[2], q.w);
    }
    return sq;
}

// ---------------------------------------------------------------------------- chunks (forward)
// With `fuse`, the warp that finishes a ray's last chunk (a counter per ray, after a fence that publishes
// the chunk) combines the ray (combine_ray), and after the items the warps combine the rays without
// chunks; with `target`, L = sum |C - target|^2 / n is added to *loss (one atomic per CTA).  For large
// batches (kFuseCombineMaxRays) the combine is a kernel of its own instead: the resident wave would
// otherwise combine tens of rays per warp, one dependent round trip after another.
template <int FORM>
__global__ void __launch_bounds__(kChunkWarps * 32, kChunkFwdBlocks) march_chunks_fwd_kernel(
    GridView g, const float *__restrict__ ro, const float *__restrict__ rd, RenderParams p, MarchPtrs st,
    MarchHeader expect, int fuse, int64_t n, float *__restrict__ rgb, float *__restrict__ T_out,
    const float *__restrict__ target, float *__restrict__ grad_rgb, float *__restrict__ loss, float inv_n) {
    __shared__ int s_buf[kChunkWarps][32];
    __shared__ SetupPipe s_pipe[kChunkWarps];
    __shared__ float s_loss[kChunkWarps];
    chain_release();  // a chained combine (large batches) may be scheduled; it waits for this grid to finish
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const MarchHeader h = *st.hdr;
    if (!header_matches(h, expect)) {  // uniform over the grid: no plan of these rays
        if (fuse && blockIdx.x == 0 && threadIdx.x == 0) report(g.status, kDevStateMismatch);
        return;
    }
    float sq_warp = 0.0f;  // lane 0: the squared errors of the rays this warp combined
    const int total = h.total_items;
    const int stride = gridDim.x * kChunkWarps;
    const int mc = st.max_chunks;
    int it = blockIdx.x * kChunkWarps + wid;
    ItemIn cur = load_item(st, ro, rd, item_at(st, it, total), lane);
    setup_fetch(s_pipe[wid], 0, st, cur.ray, lane);
    int2 id_next = item_at(st, it + stride, total);
    int buf = 0;
    for (; it < total; it += stride, buf ^= 1) {
        const ItemIn nxt = load_item(st, ro, rd, id_next, lane);
        setup_fetch(s_pipe[wid], buf ^ 1, st, nxt.ray, lane);
        id_next = item_at(st, it + 2 * stride, total);
        const int64_t ray = cur.ray;
        const int k = cur.k;
        const int nch = (cur.n_occ + 31) >> 5;
        setup_wait_prev();
        const RaySetup &rs = s_pipe[wid].slot[buf];
        int s;
        int cnt = item_samples(g, rs, p, st, cur, s_buf[wid], lane, s);
        cur = nxt;
        if (cnt < 0) cnt = 0;  // a rescan that disagrees with the plan (reported): the chunk adds nothing
        const bool valid = lane < cnt;
        float sig = 0.0f, col[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
            DF gc[3];
            coords_at(rs, s, gc);
            float acc[kNV];
            int32_t rr[8];
            float ff[3];
            gather_sample<true>(g, FORM, gc, acc, rr, ff);
            sig = fmaxf(acc[0], 0.0f);
            float pre[3];
            colour_of(acc, rs.Y, pre, col);
            if (st.vals) st.vals[(ray * mc + k) * 32 + lane] = make_float4(sig, pre[0], pre[1], pre[2]);
        }
        const Composite cp = composite(sig, valid, 1.0f, p, lane);  // stop_thresh is 0 on this path
        const float w = cp.take ? cp.T * cp.alpha : 0.0f;
        const float c0 = warp_sum(w * col[0]);
        const float c1 = warp_sum(w * col[1]);
        const float c2 = warp_sum(w * col[2]);
        const unsigned live = __ballot_sync(kFull, valid && sig > 0.0f);
        int finished = 0;
        if (lane == 0) {
            st.part[ray * mc + k] = make_float4(c0, c1, c2, cp.chunk_prod);
            st.live[ray * mc + k] = live ? 1 : 0;
            if (fuse) {
                __threadfence();  // the chunk is visible before the count says so
                finished = atomicAdd(st.done + ray, 1) + 1;
            }
        }
        finished = __shfl_sync(kFull, finished, 0);
        if (fuse && finished == nch) {  // uniform: every chunk of the ray is in; combine it
            __threadfence();
            sq_warp += combine_ray(p, st, ray, lane, rgb, T_out, target, grad_rgb, inv_n);
        }
        __syncwarp();  // every lane is done with this slot before the next fetch overwrites it
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (!fuse) return;
    // the rays without a chunk (no sample in a non-empty cell): colour = background
    for (int64_t ray = (int64_t)blockIdx.x * kChunkWarps + wid; ray < n; ray += (int64_t)gridDim.x * kChunkWarps)
        if (st.n_occ[ray] == 0) sq_warp += combine_ray(p, st, ray, lane, rgb, T_out, target, grad_rgb, inv_n);
    if (target && loss) {
        if (lane == 0) s_loss[wid] = sq_warp;
        __syncthreads();
        if (threadIdx.x == 0) {
            float acc = 0.0f;
            for (int w = 0; w < kChunkWarps; ++w) acc += s_loss[w];
            if (acc != 0.0f) atomicAdd(loss, acc * inv_n);
        }
    }
}

// The combine of a ray of at most kCombineShort chunks by one thread: the same quantities as combine_ray,
// accumulated chunk by chunk (for one or two chunks the same roundings as combine_ray's warp sums).
// Returns the ray's squared error |C - target|^2 (0 without a target).
constexpr int kCombineShort = 8;
__device__ __forceinline__ float combine_short(const RenderParams &p, const MarchPtrs &st, int64_t ray, int nch,
                                               float *__restrict__ rgb, float *__restrict__ T_out,
                                               const float *__restrict__ target, float *__restrict__ grad_rgb,
                                               float inv_n) {
    float4 *part = st.part + ray * st.max_chunks;
    float4 q[kCombineShort];
#pragma unroll
    for (int k = 0; k < kCombineShort; ++k) q[k] = k < nch ? part[k] : make_float4(0.0f, 0.0f, 0.0f, 1.0f);
    float Tc = 1.0f, Tb[kCombineShort];
    float C[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < kCombineShort; ++k) {
        Tb[k] = Tc;
        if (k < nch) {
            C[0] = __fadd_rn(C[0], __fmul_rn(Tc, q[k].x));
            C[1] = __fadd_rn(C[1], __fmul_rn(Tc, q[k].y));
            C[2] = __fadd_rn(C[2], __fmul_rn(Tc, q[k].z));
            Tc *= q[k].w;
        }
    }
    float sq = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float c = fmaf(Tc, p.bg[ch], C[ch]);
        rgb[3 * ray + ch] = c;
        if (target) {
            const float diff = c - __ldg(target + 3 * ray + ch);
            grad_rgb[3 * ray + ch] = 2.0f * diff * inv_n;
            sq = fmaf(diff, diff, sq);
        }
    }
    if (T_out) T_out[ray] = Tc;
    // back to front: the colour arriving after each chunk
    float R[3] = {Tc * p.bg[0], Tc * p.bg[1], Tc * p.bg[2]};
#pragma unroll
    for (int k = kCombineShort - 1; k >= 0; --k) {
        if (k < nch) {
            part[k] = make_float4(R[0], R[1], R[2], Tb[k]);
            R[0] = __fadd_rn(R[0], __fmul_rn(Tb[k], q[k].x));
            R[1] = __fadd_rn(R[1], __fmul_rn(Tb[k], q[k].y));
            R[2] = __fadd_rn(R[2], __fmul_rn(Tb[k], q[k].z));
        }
    }
    return sq;
}

// The combine as a kernel of its own (large batches): a thread per ray for the rays of at most
// kCombineShort chunks (most rays), the longer rays listed in shared memory and then combined a warp per
// ray (combine_ray); with `target`, L is added to *loss (one atomic per CTA).
constexpr int kCombineThreads = 256;
__global__ void __launch_bounds__(kCombineThreads) march_combine_kernel(GridView g, int64_t n, RenderParams p,
                                                                        MarchPtrs st, MarchHeader expect,
                                                                        float *__restrict__ rgb,
                                                                        float *__restrict__ T_out,
                                                                        const float *__restrict__ target,
                                                                        float *__restrict__ grad_rgb,
                                                                        float *__restrict__ loss, float inv_n) {
    constexpr int kWarps = kCombineThreads / 32;
    __shared__ int s_long[kCombineThreads];
    __shared__ int s_nlong;
    __shared__ float s_loss[kWarps];
    chain_wait();  // launched chained to the chunk kernel: nothing is read before it has finished
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    if (!header_matches(*st.hdr, expect)) {  // uniform over the grid: no plan of these rays
        if (blockIdx.x == 0 && threadIdx.x == 0) report(g.status, kDevStateMismatch);
        return;
    }
    if (threadIdx.x == 0) s_nlong = 0;
    __syncthreads();
    const int64_t ray0 = (int64_t)blockIdx.x * kCombineThreads;
    const int64_t ray = ray0 + threadIdx.x;
    float sq = 0.0f;
    if (ray < n) {
        const int nch = (st.n_occ[ray] + 31) >> 5;
        if (nch > kCombineShort)
            s_long[atomicAdd(&s_nlong, 1)] = threadIdx.x;
        else
            sq = combine_short(p, st, ray, nch, rgb, T_out, target, grad_rgb, inv_n);
    }
    __syncthreads();
    const int nl = s_nlong;
    for (int i = wid; i < nl; i += kWarps)  // uniform over the warp
        sq += combine_ray(p, st, ray0 + s_long[i], lane, rgb, T_out, target, grad_rgb, inv_n);
    if (target && loss) {
        sq = warp_sum(sq);
        if (lane == 0) s_loss[wid] = sq;
        __syncthreads();
        if (threadIdx.x == 0) {
            float acc = 0.0f;
            for (int w = 0; w < kWarps; ++w) acc += s_loss[w];
            if (acc != 0.0f) atomicAdd(loss, acc * inv_n);
        }
    }
}

// ---------------------------------------------------------------------------- adjoint

// With the forward's stored values (VALS) the adjoint gathers no rows: half the registers, twice the
// resident warps to hide the index loads and atomics.
constexpr int kBwdValsBlocks = 5;

template <int FORM, bool VALS>
__global__ void __launch_bounds__(kChunkWarps * 32, VALS ? kBwdValsBlocks : kGatherBlocks) march_chunks_bwd_kernel(
    GridView g, const float *__restrict__ ro, const float *__restrict__ rd, RenderParams p, MarchPtrs st,
    MarchHeader expect, const float *__restrict__ grad_rgb, float *__restrict__ grad_rows) {
    __shared__ int s_buf[kChunkWarps][32];
    __shared__ SetupPipe s_pipe[kChunkWarps];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const MarchHeader h = *st.hdr;
    if (!header_matches(h, expect)) {  // uniform over the grid
        if (threadIdx.x == 0 && blockIdx.x == 0) report(g.status, kDevStateMismatch);
        return;
    }
    const int total = h.total_items;
    const int stride = gridDim.x * kChunkWarps;
    const int mc = st.max_chunks;
    int it = blockIdx.x * kChunkWarps + wid;
    // the items whose chunk has no positive density add nothing: skip them when fetching
    auto next_live = [&](int from) {
        int2 id = item_at(st, from, total);
        while (id.x >= 0 && !st.live[(int64_t)id.x * mc + id.y]) {
            from += stride;
            id = item_at(st, from, total);
        }
        it = from;
        return id;
    };
    int2 id = next_live(it);
    int it_cur = it;
    ItemIn cur = load_item(st, ro, rd, id, lane);
    setup_fetch(s_pipe[wid], 0, st, cur.ray, lane);
    int2 id_next = next_live(it_cur + stride);
    int buf = 0;
    for (; cur.ray >= 0; buf ^= 1) {
        const ItemIn nxt = load_item(st, ro, rd, id_next, lane);
        setup_fetch(s_pipe[wid], buf ^ 1, st, nxt.ray, lane);
        id_next = next_live(it + stride);
        const int64_t ray = cur.ray;
        const int k = cur.k;
        const float4 q = st.part[ray * mc + k];  // (R_after, T_before)
        const float gr[3] = {__ldg(grad_rgb + 3 * ray), __ldg(grad_rgb + 3 * ray + 1), __ldg(grad_rgb + 3 * ray + 2)};
        setup_wait_prev();
        const RaySetup &rs = s_pipe[wid].slot[buf];
        int s;
        const int cnt = item_samples(g, rs, p, st, cur, s_buf[wid], lane, s);
        cur = nxt;
        if (cnt < 0) {
            __syncwarp();
            continue;
        }
        const bool valid = lane < cnt;
        int32_t rr[8];
        float ff[3];
        int64_t cell = -1;
        float sig = 0.0f, pre[3] = {0.0f, 0.0f, 0.0f}, col[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
            DF gc[3];
            coords_at(rs, s, gc);
            if (VALS) {  // the forward's values; only the corners are looked up again
                const float4 v = st.vals[(ray * mc + k) * 32 + lane];
                const Cell c = locate(g, gc);
                cell = c.base;
#pragma unroll
                for (int a = 0; a < 3; ++a) ff[a] = c.f[a];
#pragma unroll
                for (int kc = 0; kc < 8; ++kc) rr[kc] = row_of(g, corner_node(g, c.base, kc));
                sig = v.x;
                pre[0] = v.y;
                pre[1] = v.z;
                pre[2] = v.w;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) col[ch] = fmaxf(pre[ch], 0.0f);
            } else {
                float acc[kNV];
                gather_sample(g, FORM, gc, acc, rr, ff, &cell);
                sig = fmaxf(acc[0], 0.0f);
                colour_of(acc, rs.Y, pre, col);
            }
        }
        const Composite cp = composite(sig, valid, q.w, p, lane);
        const float w = cp.take ? cp.T * cp.alpha : 0.0f;
        const float Ra[3] = {q.x, q.y, q.z};
        float Rs[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float suf = warp_incl_suffix(w * col[ch], lane);
            float suf_ex = __shfl_down_sync(kFull, suf, 1);
            if (lane == 31) suf_ex = 0.0f;
            Rs[ch] = Ra[ch] + suf_ex;
        }
        const float gprior = sparsity_prior(p, cp.take, sig);
        scatter_chunk(g, cp.take && sig > 0.0f, cell, rr, ff, rs.Y, gr, pre, col, w, cp.Tn, Rs, p.delta, gprior,
                      grad_rows, lane);
        __syncwarp();  // every lane is done with this slot before the next fetch overwrites it
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// One resident wave: blocks_per_sm CTAs per SM, but no more warps than items can exist.
unsigned chunk_grid(int64_t n, int max_chunks, int blocks_per_sm = kGatherBlocks) {
    const int64_t slots = n * (int64_t)max_chunks;
    const int64_t need = (slots + kChunkWarps - 1) / kChunkWarps;
    const int64_t wave = (int64_t)sm_count() * blocks_per_sm;
    return (unsigned)std::max<int64_t>(1, std::min(need, wave));
}

}  // namespace

cudaError_t launch_march_plan(const GridView &g, const float *o, const float *d, int64_t n, const RenderParams &p,
                              const MarchPtrs &st, const MarchHeader &hdr, cudaStream_t s) {
    march_header_kernel<<<1, 1, 0, s>>>(st.hdr, hdr);
    if (hdr.mode == kMarchChunked && n > 0) {
        march_setup_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, p, o, d, n, st);
        march_plan_kernel<<<(unsigned)n, kPlanWarps * 32, 0, s>>>(g, o, d, n, p, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_render_planned(const GridView &g, const float *o, const float *d, int64_t n,
                                  const RenderParams &p, const MarchPtrs &st, const MarchHeader &hdr, float *rgb,
                                  float *T_end, const float *target, float *grad_rgb, float *loss, cudaStream_t s) {
    if (hdr.mode == kMarchRecompute) {
        cudaError_t e = launch_render(g, o, d, n, p, rgb, T_end, s);
        if (e == cudaSuccess && target) e = launch_mse_grad(rgb, target, n, grad_rgb, loss, s);
        return e;
    }
    if (n == 0) return cudaSuccess;
    const unsigned grid = chunk_grid(n, st.max_chunks, kChunkFwdBlocks);
    const float inv_n = (float)(1.0 / (double)n);
    const int fuse = n <= kFuseCombineMaxRays ? 1 : 0;
    if (g.form == PLX_SH_F32)
        march_chunks_fwd_kernel<PLX_SH_F32><<<grid, kChunkWarps * 32, 0, s>>>(g, o, d, p, st, hdr, fuse, n, rgb,
                                                                                T_end, target, grad_rgb, loss, inv_n);
    else
        march_chunks_fwd_kernel<PLX_SH_BF16><<<grid, kChunkWarps * 32, 0, s>>>(g, o, d, p, st, hdr, fuse, n, rgb,
                                                                                 T_end, target, grad_rgb, loss, inv_n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || fuse) return e;
    return launch_chained(march_combine_kernel, (unsigned)((n + kCombineThreads - 1) / kCombineThreads),
                          kCombineThreads, s, g, n, p, st, hdr, rgb, T_end, target, grad_rgb, loss, inv_n);
}

cudaError_t launch_render_train(const GridView &g, const float *o, const float *d, int64_t n, const RenderParams &p,
                                const MarchPtrs &st, const MarchHeader &hdr, float *rgb, float *T_end,
                                cudaStream_t s) {
    cudaError_t e = launch_march_plan(g, o, d, n, p, st, hdr, s);
    if (e != cudaSuccess) return e;
    return launch_render_planned(g, o, d, n, p, st, hdr, rgb, T_end, nullptr, nullptr, nullptr, s);
}

cudaError_t launch_render_backward_train(const GridView &g, const float *o, const float *d, int64_t n,
                                         const RenderParams &p, const MarchPtrs &st, const MarchHeader &hdr,
                                         const float *grad_rgb, float *grad_rows, cudaStream_t s) {
    if (hdr.mode == kMarchRecompute) return launch_render_backward(g, o, d, n, p, grad_rgb, grad_rows, s);
    if (n == 0) return cudaSuccess;
    if (st.vals) {
        const unsigned grid = chunk_grid(n, st.max_chunks, kBwdValsBlocks);
        if (g.form == PLX_SH_F32)
            march_chunks_bwd_kernel<PLX_SH_F32, true><<<grid, kChunkWarps * 32, 0, s>>>(g, o, d, p, st, hdr, grad_rgb,
                                                                                      grad_rows);
        else
            march_chunks_bwd_kernel<PLX_SH_BF16, true><<<grid, kChunkWarps * 32, 0, s>>>(g, o, d, p, st, hdr,
                                                                                       grad_rgb, grad_rows);
    } else {
        const unsigned grid = chunk_grid(n, st.max_chunks);
        if (g.form == PLX_SH_F32)
            march_chunks_bwd_kernel<PLX_SH_F32, false><<<grid, kChunkWarps * 32, 0, s>>>(g, o, d, p, st, hdr,
                                                                                       grad_rgb, grad_rows);
        else
            march_chunks_bwd_kernel<PLX_SH_BF16, false><<<grid, kChunkWarps * 32, 0, s>>>(g, o, d, p, st, hdr,
                                                                                        grad_rgb, grad_rows);
    }
    return cudaGetLastError();
}

}  // namespace plx
