// plx_trainer.cu -- the optimisation step (Sec. 3.5; Supp. B.1: batches of rays, RMSProp, TV on
// contiguous segments) as one native call: ray generation, plan, forward with the MSE gradient,
// adjoint (with the Cauchy prior when configured), TV and RMSProp, scheduled on three streams.
//
// Dependencies within and across steps: the RMSProp update of step k-1 must precede the forward of
// step k (it changes the rows the forward reads) and TV of step k (same); TV adds into the gradient
// with atomics and only reads rows, so it runs beside the forward and adjoint; ray generation and the
// plan read no rows.  The update of a step is deferred to the start of the next call (or to
// plx_trainer_finish), so it runs beside the next batch's plan.  Rays and march state are kept in two
// sets, so that the next batch (d_next_pix) is generated and planned during this step's march.
//
// The trainer only orders library calls (the same entry points a caller would use) on its streams;
// every computation is in the library's kernels.
#include <cstdint>
#include <new>
#include <string>

#include "plenoxel.h"
#include "plx_internal.cuh"

namespace {

constexpr size_t kAlign = 256;
size_t up(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
    size_t ray[2][2];  // [set][o, d]
    size_t rgb, grad_rgb;
    size_t state[2];
    size_t state_bytes;
    size_t in_pix[2], in_tgt[2], in_ss[2], in_sl[2];  // host-fed steps: each set's inputs
    size_t loss[2];                                     // host-fed steps: each set's loss
    size_t total;
};

bool make_layout(const plx_grid *grid, const plx_trainer_desc *desc, Layout *L) {
    const size_t n = (size_t)desc->batch;
    const size_t rays = up(n * 3 * sizeof(float));
    L->state_bytes = plx_march_state_bytes(grid, desc->batch, &desc->opts);
    if (L->state_bytes == 0) return false;
    size_t off = 0;
    for (int k = 0; k < 2; ++k)
        for (int a = 0; a < 2; ++a) {
            L->ray[k][a] = off;
            off += rays;
        }
    L->rgb = off;
    off += rays;
    L->grad_rgb = off;
    off += rays;
    for (int k = 0; k < 2; ++k) {
        L->state[k] = off;
        off += up(L->state_bytes);
    }
    const size_t segs = up((size_t)(desc->max_segments > 0 ? desc->max_segments : 0) * sizeof(int64_t));
    for (int k = 0; k < 2; ++k) {
        L->in_pix[k] = off;
        off += up(n * sizeof(int64_t));
        L->in_tgt[k] = off;
        off += rays;
        L->in_ss[k] = off;
        off += segs;
        L->in_sl[k] = off;
        off += segs;
        L->loss[k] = off;
        off += kAlign;
    }
    L->total = off;
    return true;
}

}  // namespace

struct plx_trainer {
    plx_grid *grid;
    plx_trainer_desc desc;
    const float *cams;
    int32_t n_cams, W, H;
    float *grad, *v;
    char *ws;
    Layout L;
    cudaStream_t march = nullptr, plan = nullptr, tv = nullptr, io = nullptr;
    cudaEvent_t ev_start = nullptr, ev_rms = nullptr, ev_tv = nullptr, ev_end = nullptr;
    cudaEvent_t ev_in = nullptr, ev_fwd = nullptr, ev_io = nullptr;  // host-fed steps
    const int64_t *staged_host_pix = nullptr;  // the host batch whose inputs the last call staged, and its n
    int64_t staged_n = 0;
    cudaEvent_t ev_plan[2] = {nullptr, nullptr}, ev_bwd[2] = {nullptr, nullptr};
    bool bwd_recorded[2] = {false, false};
    int set = 0;
    const int64_t *ahead_pix = nullptr;  // the batch planned ahead, its size and set
    int64_t ahead_n = 0;
    int ahead_set = -1;
    bool pending = false;  // an update not yet applied, and its learning rates
    float pend_lrs = 0.0f, pend_lrh = 0.0f;

    int64_t *in_pix(int k) { return reinterpret_cast<int64_t *>(ws + L.in_pix[k]); }
    float *in_tgt(int k) { return reinterpret_cast<float *>(ws + L.in_tgt[k]); }
    int64_t *in_ss(int k) { return reinterpret_cast<int64_t *>(ws + L.in_ss[k]); }
    int64_t *in_sl(int k) { return reinterpret_cast<int64_t *>(ws + L.in_sl[k]); }
    float *loss(int k) { return reinterpret_cast<float *>(ws + L.loss[k]); }
    float *o(int k) { return reinterpret_cast<float *>(ws + L.ray[k][0]); }
    float *d(int k) { return reinterpret_cast<float *>(ws + L.ray[k][1]); }
    void *state(int k) { return ws + L.state[k]; }
};

namespace {

plx_status cuda_fail(cudaError_t e, const char *where) {
    return plx::set_error(PLX_ECUDA, (std::string(where) + ": " + cudaGetErrorString(e)).c_str());
}

void destroy_handles(plx_trainer *t) {
    for (cudaEvent_t e : {t->ev_start, t->ev_rms, t->ev_tv, t->ev_end, t->ev_plan[0], t->ev_plan[1], t->ev_bwd[0],
                          t->ev_bwd[1], t->ev_in, t->ev_fwd, t->ev_io})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : {t->march, t->plan, t->tv, t->io})
        if (s) cudaStreamDestroy(s);
}

// Host-to-device copies of a host batch into input set k, on stream s.
cudaError_t upload_batch(plx_trainer *t, const plx_host_batch *b, int k, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(t->in_pix(k), b->pix, (size_t)b->n * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t->in_tgt(k), b->target, (size_t)b->n * 3 * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && b->n_seg > 0)
        e = cudaMemcpyAsync(t->in_ss(k), b->seg_start, (size_t)b->n_seg * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && b->n_seg > 0)
        e = cudaMemcpyAsync(t->in_sl(k), b->seg_len, (size_t)b->n_seg * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    return e;
}

// What a host-fed step adds to the device step: the uploads of its own batch (when not staged) and of
// the next one, and the download of the loss.
struct HostIO {
    const plx_host_batch *cur;   // upload into the step's set first (nullptr: staged by the previous call)
    const plx_host_batch *next;  // upload into the other set before its plan (nullptr: none)
    float *h_loss;               // download of the step's loss (nullptr: none)
};

// Rays and plan of the n pixels d_pix into set k on the plan stream, after set k's last adjoint.
plx_status plan_batch(plx_trainer *t, const int64_t *d_pix, int64_t n, int k) {
    cudaError_t e = cudaSuccess;
    if (t->bwd_recorded[k]) e = cudaStreamWaitEvent(t->plan, t->ev_bwd[k], 0);
    if (e != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    plx_status st = plx_gen_rays(t->cams, t->n_cams, t->W, t->H, d_pix, n, t->o(k), t->d(k), t->plan);
    if (st == PLX_OK)
        st = plx_march_plan(t->grid, t->o(k), t->d(k), n, &t->desc.opts, t->state(k), t->L.state_bytes, t->plan);
    if (st != PLX_OK) return st;
    e = cudaEventRecord(t->ev_plan[k], t->plan);
    return e == cudaSuccess ? PLX_OK : cuda_fail(e, "plx_trainer_step");
}

plx_status apply_update(plx_trainer *t, cudaStream_t s) {
    if (!t->pending) return PLX_OK;
    t->pending = false;
    return plx_rmsprop_step(t->grid, t->grad, t->v, t->pend_lrs, t->pend_lrh, t->desc.beta, t->desc.eps,
                            t->desc.sparse_rmsprop, s);
}

}  // namespace

extern "C" {

size_t plx_trainer_workspace_bytes(const plx_grid *grid, const plx_trainer_desc *desc) {
    if (!grid || !desc || desc->batch <= 0) return 0;
    Layout L;
    return make_layout(grid, desc, &L) ? L.total : 0;
}

plx_status plx_trainer_create(plx_grid *grid, const plx_trainer_desc *desc, const float *d_cams, int32_t n_cams,
                              int32_t W, int32_t H, float *d_grad_rows, float *d_v, void *d_workspace,
                              size_t workspace_bytes, plx_trainer **out) {
    if (!out) return plx::set_error(PLX_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !desc) return plx::set_error(PLX_EINVAL, "NULL grid or descriptor");
    if (desc->batch <= 0) return plx::set_error(PLX_EINVAL, "batch must be positive");
    if (!d_cams || n_cams <= 0 || W <= 0 || H <= 0) return plx::set_error(PLX_EINVAL, "bad cameras or image size");
    if (!d_grad_rows || !d_v) return plx::set_error(PLX_EINVAL, "NULL gradient or RMSProp state");
    if (!(desc->beta >= 0.0f && desc->beta < 1.0f) || !(desc->eps >= 0.0f))
        return plx::set_error(PLX_EINVAL, "bad RMSProp hyper-parameters");
    if (!(desc->lambda_sparsity >= 0.0f)) return plx::set_error(PLX_EINVAL, "lambda_sparsity must be >= 0");
    if (desc->sparse_rmsprop != 0 && desc->sparse_rmsprop != 1) return plx::set_error(PLX_EINVAL, "sparse_rmsprop");
    if (desc->max_segments < 0) return plx::set_error(PLX_EINVAL, "max_segments must be >= 0");
    Layout L;
    if (!make_layout(grid, desc, &L)) return plx::set_error(PLX_EINVAL, "no march state for this grid and batch");
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & (kAlign - 1)) != 0)
        return plx::set_error(PLX_EINVAL, "d_workspace must be non-NULL and 256-byte aligned");
    if (workspace_bytes < L.total) return plx::set_error(PLX_EINVAL, "workspace too small");
    plx_trainer *t = new (std::nothrow) plx_trainer();
    if (!t) return plx::set_error(PLX_ENOMEM, "host allocation of the trainer failed");
    t->grid = grid;
    t->desc = *desc;
    t->cams = d_cams;
    t->n_cams = n_cams;
    t->W = W;
    t->H = H;
    t->grad = d_grad_rows;
    t->v = d_v;
    t->ws = static_cast<char *>(d_workspace);
    t->L = L;
    // the march and the plan one level above TV, which has the lowest priority: when both have blocks
    // waiting, the block scheduler starts the march's first and TV fills the SMs it leaves (one level, not
    // the device's highest for the plan or the march, measured fastest)
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    const int above = lo - 1 >= hi ? lo - 1 : hi;  // numerically lower is higher priority
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&t->march, cudaStreamNonBlocking, above);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&t->plan, cudaStreamNonBlocking, above);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&t->tv, cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&t->io, cudaStreamNonBlocking, above);
    for (cudaEvent_t *ev : {&t->ev_start, &t->ev_rms, &t->ev_tv, &t->ev_end, &t->ev_plan[0], &t->ev_plan[1],
                            &t->ev_bwd[0], &t->ev_bwd[1], &t->ev_in, &t->ev_fwd, &t->ev_io})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        destroy_handles(t);
        delete t;
        return cuda_fail(e, "plx_trainer_create");
    }
    *out = t;
    return PLX_OK;
}

plx_status plx_trainer_destroy(plx_trainer *t) {
    if (!t) return PLX_OK;
    destroy_handles(t);
    delete t;
    return PLX_OK;
}

}  // extern "C"

namespace {

// The step on device inputs; with io, a host-fed step (the inputs of set k are then the trainer's own,
// d_pix etc. pointing at them).
plx_status step_impl(plx_trainer *t, const int64_t *d_pix, int64_t n, const float *d_target,
                     const int64_t *d_seg_start, const int64_t *d_seg_len, int64_t n_seg, int64_t n_selected,
                     float lr_sigma, float lr_sh, const int64_t *d_next_pix, int32_t pix_is_ahead, float *d_loss,
                     float *d_loss_sparsity, int64_t *d_touched, void *const *events, int32_t *set_out,
                     cudaStream_t caller, const HostIO *io, int io_set) {
    cudaStream_t ms = t->march, ps = t->plan;
    auto mark = [&](int i) -> cudaError_t {
        return events ? cudaEventRecord(static_cast<cudaEvent_t>(events[i]), ms) : cudaSuccess;
    };
    // this step's set: the one planned ahead for these pixels, else the other one
    const bool planned = pix_is_ahead && t->ahead_set >= 0 && t->ahead_pix == d_pix && t->ahead_n == n;
    const int k = io ? io_set : planned ? t->ahead_set : 1 - t->set;
    t->ahead_set = -1;
    t->set = k;
    if (set_out) *set_out = k;
    const bool do_tv = d_seg_start && d_seg_len && n_seg > 0 && n_selected > 0;

    // the march and plan streams start after everything the caller enqueued (inputs, loss resets)
    cudaError_t e = cudaEventRecord(t->ev_start, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ms, t->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ps, t->ev_start, 0);
    if (e != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    if (io && io->cur) {  // this batch's inputs, before its plan (plan stream) and its TV (waits for ev_in)
        e = upload_batch(t, io->cur, k, ps);
        if (e == cudaSuccess) e = cudaEventRecord(t->ev_in, ps);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t->tv, t->ev_in, 0);
        if (e != cudaSuccess) return cuda_fail(e, "plx_trainer_step_host");
    }
    plx_status st = PLX_OK;
    if (!planned) st = plan_batch(t, d_pix, n, k);
    if (st != PLX_OK) return st;
    // the previous step's update, beside the plan
    if ((e = mark(0)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    if ((st = apply_update(t, ms)) != PLX_OK) return st;
    if ((e = mark(1)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    // TV of this step after that update, beside the march
    if (do_tv) {
        e = cudaEventRecord(t->ev_rms, ms);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t->tv, t->ev_rms, 0);
        if (e != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
        st = plx_tv_grad(t->grid, d_seg_start, d_seg_len, n_seg, n_selected, t->desc.lambda_tv_sigma,
                         t->desc.lambda_tv_sh, t->grad, nullptr, t->tv);
        if (st != PLX_OK) return st;
        if ((e = cudaEventRecord(t->ev_tv, t->tv)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    }
    // forward with the MSE gradient, then the adjoint, on the march stream once the plan is there
    if ((e = cudaStreamWaitEvent(ms, t->ev_plan[k], 0)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    if ((e = mark(2)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    float *rgb = reinterpret_cast<float *>(t->ws + t->L.rgb);
    float *grgb = reinterpret_cast<float *>(t->ws + t->L.grad_rgb);
    if (io && (e = cudaMemsetAsync(d_loss, 0, sizeof(float), ms)) != cudaSuccess)
        return cuda_fail(e, "plx_trainer_step_host");
    st = plx_render_planned_mse(t->grid, t->o(k), t->d(k), n, &t->desc.opts, d_target, rgb, grgb, d_loss, t->state(k),
                                t->L.state_bytes, ms);
    if (st != PLX_OK) return st;
    if (io && io->h_loss) {  // the loss is complete after the forward: download it beside the adjoint
        e = cudaEventRecord(t->ev_fwd, ms);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t->io, t->ev_fwd, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(io->h_loss, d_loss, sizeof(float), cudaMemcpyDeviceToHost, t->io);
        if (e == cudaSuccess) e = cudaEventRecord(t->ev_io, t->io);
        if (e != cudaSuccess) return cuda_fail(e, "plx_trainer_step_host");
    }
    if ((e = mark(3)) != cudaSuccess || (e = mark(4)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    st = plx_render_backward_train(t->grid, t->o(k), t->d(k), n, &t->desc.opts, grgb, t->state(k), t->L.state_bytes,
                                   t->grad, t->desc.lambda_sparsity, d_loss_sparsity, ms);
    if (st != PLX_OK) return st;
    if ((e = cudaEventRecord(t->ev_bwd[k], ms)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    t->bwd_recorded[k] = true;
    if ((e = mark(5)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    if (do_tv && (e = cudaStreamWaitEvent(ms, t->ev_tv, 0)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    if (d_touched && (st = plx_count_touched(t->grid, d_touched, ms)) != PLX_OK) return st;
    t->pending = true;
    t->pend_lrs = lr_sigma;
    t->pend_lrh = lr_sh;
    if ((e = mark(6)) != cudaSuccess || (e = mark(7)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step");
    // the next batch's rays and plan, beside this step's march (a host-fed next batch is uploaded first;
    // the inputs of set 1 - k were last read by the previous step, which ended before this one started)
    if (d_next_pix) {
        if (io && io->next) {
            if ((e = upload_batch(t, io->next, 1 - k, ps)) != cudaSuccess) return cuda_fail(e, "plx_trainer_step_host");
        }
        if ((st = plan_batch(t, d_next_pix, io && io->next ? io->next->n : n, 1 - k)) != PLX_OK) return st;
        t->ahead_pix = d_next_pix;
        t->ahead_n = io && io->next ? io->next->n : n;
        t->ahead_set = 1 - k;
    }
    // the caller's stream resumes after the step, after the next batch's plan has read its pixels, and after
    // the loss download
    e = cudaEventRecord(t->ev_end, ms);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, t->ev_end, 0);
    if (e == cudaSuccess && d_next_pix) e = cudaStreamWaitEvent(caller, t->ev_plan[1 - k], 0);
    if (e == cudaSuccess && io && io->h_loss) e = cudaStreamWaitEvent(caller, t->ev_io, 0);
    return e == cudaSuccess ? PLX_OK : cuda_fail(e, "plx_trainer_step");
}

}  // namespace

extern "C" {

plx_status plx_trainer_step(plx_trainer *t, const int64_t *d_pix, int64_t n, const float *d_target,
                            const int64_t *d_seg_start, const int64_t *d_seg_len, int64_t n_seg, int64_t n_selected,
                            float lr_sigma, float lr_sh, const int64_t *d_next_pix, int32_t pix_is_ahead,
                            float *d_loss, float *d_loss_sparsity, int64_t *d_touched, void *const *events,
                            int32_t *set_out, void *stream) {
    if (!t) return plx::set_error(PLX_EINVAL, "trainer is NULL");
    if (n <= 0 || n > t->desc.batch) return plx::set_error(PLX_EINVAL, "n out of range (1..batch)");
    if (!d_pix || !d_target) return plx::set_error(PLX_EINVAL, "NULL pixels or targets");
    t->staged_host_pix = nullptr;  // a device-fed step ends any host staging
    return step_impl(t, d_pix, n, d_target, d_seg_start, d_seg_len, n_seg, n_selected, lr_sigma, lr_sh, d_next_pix,
                     pix_is_ahead, d_loss, d_loss_sparsity, d_touched, events, set_out,
                     static_cast<cudaStream_t>(stream), nullptr, 0);
}

static plx_status check_host_batch(const plx_trainer *t, const plx_host_batch *b, const char *what) {
    if (!b->pix || !b->target) return plx::set_error(PLX_EINVAL, (std::string(what) + ": NULL pixels or targets").c_str());
    if (b->n <= 0 || b->n > t->desc.batch)
        return plx::set_error(PLX_EINVAL, (std::string(what) + ": n out of range (1..batch)").c_str());
    if (b->n_seg < 0 || b->n_seg > t->desc.max_segments || (b->n_seg > 0 && (!b->seg_start || !b->seg_len)))
        return plx::set_error(PLX_EINVAL, (std::string(what) + ": TV segments beyond max_segments or NULL").c_str());
    if (b->n_selected < 0) return plx::set_error(PLX_EINVAL, (std::string(what) + ": n_selected < 0").c_str());
    return PLX_OK;
}

plx_status plx_trainer_step_host(plx_trainer *t, const plx_host_batch *batch, const plx_host_batch *next,
                                 float lr_sigma, float lr_sh, float *h_loss, void *stream) {
    if (!t || !batch) return plx::set_error(PLX_EINVAL, "trainer or batch is NULL");
    plx_status st = check_host_batch(t, batch, "batch");
    if (st == PLX_OK && next) st = check_host_batch(t, next, "next");
    if (st != PLX_OK) return st;
    // staged: the previous call uploaded and planned this batch into the set it left ahead
    const bool staged = t->staged_host_pix == batch->pix && t->staged_n == batch->n && t->ahead_set >= 0;
    const int k = staged ? t->ahead_set : 1 - t->set;
    HostIO io = {staged ? nullptr : batch, next, h_loss};
    const bool do_tv = batch->n_seg > 0 && batch->n_selected > 0;
    t->staged_host_pix = nullptr;
    st = step_impl(t, t->in_pix(k), batch->n, t->in_tgt(k), do_tv ? t->in_ss(k) : nullptr,
                   do_tv ? t->in_sl(k) : nullptr, batch->n_seg, batch->n_selected, lr_sigma, lr_sh,
                   next ? t->in_pix(1 - k) : nullptr, staged ? 1 : 0, t->loss(k), nullptr, nullptr, nullptr, nullptr,
                   static_cast<cudaStream_t>(stream), &io, k);
    if (st == PLX_OK && next) {
        t->staged_host_pix = next->pix;
        t->staged_n = next->n;
    }
    return st;
}

plx_status plx_trainer_finish(plx_trainer *t, void *stream) {
    if (!t) return plx::set_error(PLX_EINVAL, "trainer is NULL");
    return apply_update(t, static_cast<cudaStream_t>(stream));
}

plx_status plx_trainer_buffers(const plx_trainer *t, int32_t set, float **d_origins, float **d_dirs, float **d_rgb,
                               void **d_state, size_t *state_bytes) {
    if (!t || set < 0 || set > 1) return plx::set_error(PLX_EINVAL, "bad trainer or set");
    plx_trainer *m = const_cast<plx_trainer *>(t);
    if (d_origins) *d_origins = m->o(set);
    if (d_dirs) *d_dirs = m->d(set);
    if (d_rgb) *d_rgb = reinterpret_cast<float *>(m->ws + m->L.rgb);
    if (d_state) *d_state = m->state(set);
    if (state_bytes) *state_bytes = m->L.state_bytes;
    return PLX_OK;
}

}  // extern "C"
