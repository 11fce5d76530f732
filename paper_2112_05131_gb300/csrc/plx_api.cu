// plx_api.cu -- the extern "C" entry points declared in include/plenoxel.h:
// argument validation on the host, the opaque grid handle, workspace
// layout, error reporting, and the launches into the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "plx_internal.cuh"

struct plx_grid {
    plx_grid_desc desc;
    const int32_t *idx;
    float *rows;
    uint16_t *rows_h;
    char *ws;
    plx::WorkspaceLayout layout;
    plx::GridView view;
    int rms_parity;  // which of the two list lengths the next sparse RMSProp call uses
};

namespace {

thread_local std::string g_last_error;

plx_status fail(plx_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
plx_status fail(plx_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

plx_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return PLX_OK;
    return fail(PLX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

plx_status check_desc(const plx_grid_desc *d) {
    if (!d) return fail(PLX_EINVAL, "descriptor is NULL");
    if (d->reso < 2 || d->reso > 2048) return fail(PLX_EINVAL, "reso %d outside [2, 2048]", d->reso);
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(d->aabb_min[a]) || !std::isfinite(d->aabb_max[a]) || !(d->aabb_max[a] > d->aabb_min[a]))
            return fail(PLX_EINVAL, "aabb axis %d is empty or not finite", a);
    }
    if (d->n_rows < 0 || d->n_rows >= (int64_t(1) << 31)) return fail(PLX_EINVAL, "n_rows %lld out of range", (long long)d->n_rows);
    if (d->sh_form != PLX_SH_F32 && d->sh_form != PLX_SH_BF16) return fail(PLX_EINVAL, "unknown sh_form %d", d->sh_form);
    return PLX_OK;
}

plx_status check_grid(const plx_grid *g) {
    if (!g) return fail(PLX_EINVAL, "grid is NULL");
    return PLX_OK;
}

plx_status check_opts(const plx_render_opts *o) {
    if (!o) return fail(PLX_EINVAL, "render options are NULL");
    if (!(o->step_vox > 0.0f) || !std::isfinite(o->step_vox)) return fail(PLX_EINVAL, "step_vox must be positive and finite");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(o->bg[c])) return fail(PLX_EINVAL, "background colour is not finite");
    if (!(o->stop_thresh >= 0.0f) || !(o->stop_thresh <= 1.0f)) return fail(PLX_EINVAL, "stop_thresh must be in [0, 1]");
    return PLX_OK;
}

plx::RenderParams make_params(const plx_grid *g, const plx_render_opts *o) {
    plx::RenderParams p;
    double hmin = 1e300, diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double ext = (double)g->desc.aabb_max[a] - (double)g->desc.aabb_min[a];
        hmin = std::fmin(hmin, ext / (double)(g->desc.reso - 1));
        diag2 += ext * ext;
    }
    double delta = (double)o->step_vox * hmin;
    p.delta = (float)delta;
    p.delta_lo = (float)(delta - (double)p.delta);
    for (int c = 0; c < 3; ++c) p.bg[c] = o->bg[c];
    p.stop = o->stop_thresh;
    double max_samples = std::sqrt(diag2) / delta + 2.0;
    p.max_chunks = (int)std::fmin(1e9, std::ceil(max_samples / 32.0) + 1.0);
    p.lam_s = 0.0f;
    p.loss_s = nullptr;
    return p;
}

}  // namespace

namespace plx {
const GridView *grid_view(const plx_grid *grid) { return grid ? &grid->view : nullptr; }
plx_status set_error(plx_status s, const char *message) { return fail(s, "%s", message); }
}  // namespace plx

extern "C" {

const char *plx_status_str(plx_status s) {
    switch (s) {
    case PLX_OK: return "ok";
    case PLX_EINVAL: return "invalid argument";
    case PLX_ENOMEM: return "buffer too small";
    case PLX_ECUDA: return "CUDA error";
    case PLX_ETIMEOUT: return "timed out";
    case PLX_EBUSY: return "busy";
    case PLX_EUNSUPPORTED: return "unsupported";
    case PLX_EDEVICE: return "device reported corrupt data";
    }
    return "unknown status";
}

const char *plx_last_error(void) { return g_last_error.c_str(); }

const char *plx_version(void) { return "plenoxel-gb300 0.1 (sm_103a)"; }

size_t plx_grid_workspace_bytes(const plx_grid_desc *desc) {
    if (check_desc(desc) != PLX_OK) return 0;
    return plx::WorkspaceLayout::make(desc->reso, desc->n_rows).total;
}

plx_status plx_grid_create(const plx_grid_desc *desc, const int32_t *d_idx, float *d_rows_f32, uint16_t *d_rows_bf16,
                           void *d_workspace, void *stream, plx_grid **out) {
    plx_status st = check_desc(desc);
    if (st != PLX_OK) return st;
    if (!out) return fail(PLX_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d_idx) return fail(PLX_EINVAL, "d_idx is NULL");
    if (!d_workspace || !aligned(d_workspace, 256)) return fail(PLX_EINVAL, "d_workspace must be non-NULL and 256-byte aligned");
    const bool have_rows = desc->n_rows > 0;
    if (desc->sh_form == PLX_SH_F32) {
        if (have_rows && !d_rows_f32) return fail(PLX_EINVAL, "F32 form needs d_rows_f32");
        if (d_rows_bf16) return fail(PLX_EINVAL, "F32 form takes no d_rows_bf16");
    } else {
        if (have_rows && !d_rows_bf16) return fail(PLX_EINVAL, "BF16 form needs d_rows_bf16");
    }
    if (d_rows_f32 && !aligned(d_rows_f32, 16)) return fail(PLX_EINVAL, "d_rows_f32 must be 16-byte aligned");
    if (d_rows_bf16 && !aligned(d_rows_bf16, 16)) return fail(PLX_EINVAL, "d_rows_bf16 must be 16-byte aligned");
    if (!aligned(d_idx, 4)) return fail(PLX_EINVAL, "d_idx must be 4-byte aligned");

    plx_grid *g = new (std::nothrow) plx_grid();
    if (!g) return fail(PLX_ENOMEM, "host allocation of the grid handle failed");
    g->desc = *desc;
    g->idx = d_idx;
    g->rows = d_rows_f32;
    g->rows_h = d_rows_bf16;
    g->ws = static_cast<char *>(d_workspace);
    g->layout = plx::WorkspaceLayout::make(desc->reso, desc->n_rows);
    plx::GridView &v = g->view;
    v.idx = d_idx;
    v.rows = d_rows_f32;
    v.rows_h = d_rows_bf16;
    v.occ = reinterpret_cast<const uint32_t *>(g->ws + g->layout.occ_off);
    v.occ_coarse = reinterpret_cast<const uint32_t *>(g->ws + g->layout.coarse_off);
    v.nb = (int)plx::coarse_blocks_per_axis(desc->reso);
    v.occ_box = reinterpret_cast<const int *>(g->ws + g->layout.status_off + plx::WorkspaceLayout::kOccBoxOff);
    v.touched = reinterpret_cast<uint32_t *>(g->ws + g->layout.touched_off);
    v.tlist = reinterpret_cast<int32_t *>(g->ws + g->layout.list_off);
    v.tcount = reinterpret_cast<int *>(g->ws + g->layout.status_off + plx::WorkspaceLayout::kListCountOff);
    v.status = reinterpret_cast<int *>(g->ws + g->layout.status_off);
    v.R = desc->reso;
    v.form = desc->sh_form;
    v.M = desc->n_rows;
    v.hmin = 1e30f;
    for (int a = 0; a < 3; ++a) {
        v.lo[a] = desc->aabb_min[a];
        v.hi[a] = desc->aabb_max[a];
        double h = ((double)desc->aabb_max[a] - (double)desc->aabb_min[a]) / (double)(desc->reso - 1);
        v.inv_h[a] = (float)(1.0 / h);
        v.inv_h_lo[a] = (float)(1.0 / h - (double)v.inv_h[a]);
        v.hmin = std::fmin(v.hmin, (float)h);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // status block and touched bits start at zero; occupancy is rebuilt from the index volume
    cudaError_t e = cudaMemsetAsync(g->ws + g->layout.status_off, 0, 256, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(g->ws + g->layout.touched_off, 0, g->layout.list_off - g->layout.touched_off, s);
    if (e == cudaSuccess)
        e = plx::launch_build_occupancy(v, reinterpret_cast<uint32_t *>(g->ws + g->layout.occ_off),
                                        reinterpret_cast<uint32_t *>(g->ws + g->layout.coarse_off), s);
    if (e != cudaSuccess) {
        delete g;
        return cuda_status(e, "plx_grid_create");
    }
    *out = g;
    return PLX_OK;
}

plx_status plx_grid_destroy(plx_grid *grid) {
    delete grid;
    return PLX_OK;
}

plx_status plx_grid_get_desc(const plx_grid *grid, plx_grid_desc *out) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    if (!out) return fail(PLX_EINVAL, "out is NULL");
    *out = grid->desc;
    return PLX_OK;
}

plx_status plx_pack_bf16(plx_grid *grid, void *stream) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    if (!grid->rows || !grid->rows_h) return fail(PLX_EINVAL, "plx_pack_bf16 needs both F32 and BF16 rows");
    return cuda_status(plx::launch_pack_bf16(grid->view, grid->rows_h, static_cast<cudaStream_t>(stream)), "plx_pack_bf16");
}

plx_status plx_check(const plx_grid *grid, void *stream) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int code = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&code, grid->view.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && code != 0) e = cudaMemset(grid->view.status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_status(e, "plx_check");
    if (code == plx::kDevBadRow) return fail(PLX_EDEVICE, "an index volume entry is >= n_rows");
    if (code == plx::kDevTooManySamples) return fail(PLX_EDEVICE, "a ray needed more samples than the backward supports");
    if (code == plx::kDevCountMismatch)
        return fail(PLX_EDEVICE, "a count disagreed with its plan (apply given a row count its workspace does not "
                                 "hold, or a training chunk rescan found a different sample count)");
    if (code == plx::kDevBadTile)
        return fail(PLX_EDEVICE, "plx_render_tiles skipped a tile with an out-of-range scene or camera or a NULL image");
    if (code == plx::kDevStateMismatch)
        return fail(PLX_EDEVICE, "a training march was given a state that holds no plan of these rays, this grid and "
                                 "these options; it wrote and added nothing");
    if (code != 0) return fail(PLX_EDEVICE, "device status %d", code);
    return PLX_OK;
}

plx_status plx_gen_rays(const float *d_cams, int32_t n_cams, int32_t W, int32_t H, const int64_t *d_pix, int64_t n,
                        float *d_origins, float *d_dirs, void *stream) {
    if (n < 0) return fail(PLX_EINVAL, "n < 0");
    if (n_cams < 1 || W < 1 || H < 1) return fail(PLX_EINVAL, "need n_cams, W, H >= 1");
    if (n > 0 && (!d_cams || !d_pix || !d_origins || !d_dirs)) return fail(PLX_EINVAL, "NULL buffer");
    if (n >= (int64_t(1) << 40)) return fail(PLX_EINVAL, "n too large");
    return cuda_status(plx::launch_gen_rays(d_cams, n_cams, W, H, d_pix, n, d_origins, d_dirs,
                                            static_cast<cudaStream_t>(stream)), "plx_gen_rays");
}

plx_status plx_render(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                      const plx_render_opts *opts, float *d_rgb, float *d_T_end, void *stream) {
    plx_status st = check_grid(grid);
    if (st == PLX_OK) st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (n < 0 || n >= (int64_t(1) << 36)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_origins || !d_dirs || !d_rgb)) return fail(PLX_EINVAL, "NULL ray or output buffer");
    if (grid->desc.sh_form == PLX_SH_F32 && grid->desc.n_rows > 0 && !grid->rows) return fail(PLX_EINVAL, "grid has no F32 rows");
    plx::RenderParams p = make_params(grid, opts);
    return cuda_status(plx::launch_render(grid->view, d_origins, d_dirs, n, p, d_rgb, d_T_end,
                                          static_cast<cudaStream_t>(stream)), "plx_render");
}

plx_status plx_render_backward(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                               const plx_render_opts *opts, const float *d_grad_rgb, float *d_grad_rows,
                               float lambda_sparsity, float *d_loss_sparsity, void *stream) {
    plx_status st = check_grid(grid);
    if (st == PLX_OK) st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (n < 0 || n >= (int64_t(1) << 36)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_origins || !d_dirs || !d_grad_rgb || !d_grad_rows)) return fail(PLX_EINVAL, "NULL buffer");
    if (d_grad_rows && !aligned(d_grad_rows, 16)) return fail(PLX_EINVAL, "d_grad_rows must be 16-byte aligned");
    if (!(lambda_sparsity >= 0.0f) || !std::isfinite(lambda_sparsity))
        return fail(PLX_EINVAL, "lambda_sparsity must be finite and >= 0");
    if (d_loss_sparsity && !aligned(d_loss_sparsity, 4)) return fail(PLX_EINVAL, "d_loss_sparsity must be 4-byte aligned");
    plx::RenderParams p = make_params(grid, opts);
    p.lam_s = lambda_sparsity;
    p.loss_s = d_loss_sparsity;
    if (p.max_chunks > 256)
        return fail(PLX_EUNSUPPORTED, "rays of up to %d samples exceed the backward's 8192-sample limit; raise step_vox",
                    p.max_chunks * 32);
    return cuda_status(plx::launch_render_backward(grid->view, d_origins, d_dirs, n, p, d_grad_rgb, d_grad_rows,
                                                   static_cast<cudaStream_t>(stream)), "plx_render_backward");
}

size_t plx_march_state_bytes(const plx_grid *grid, int64_t n, const plx_render_opts *opts) {
    if (!grid || check_opts(opts) != PLX_OK || n < 0 || n >= (int64_t(1) << 31)) return 0;
    const plx::RenderParams p = make_params(grid, opts);
    return plx::MarchLayout::make(n, p.max_chunks).total;
}

namespace {

// Validates a march-state buffer for n rays and fills the pointers and the header it must carry.
plx_status march_state(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                       const plx_render_opts *opts, const plx::RenderParams &p, void *d_state, size_t state_bytes,
                       plx::MarchPtrs *ptrs, plx::MarchHeader *hdr) {
    if (!d_state) return fail(PLX_EINVAL, "d_state is NULL");
    if (!aligned(d_state, 16)) return fail(PLX_EINVAL, "d_state must be 16-byte aligned");
    if (n * (int64_t)p.max_chunks >= (int64_t(1) << 31))
        return fail(PLX_EINVAL, "n x chunks per ray (%lld x %d) exceeds the work-item limit 2^31; split the batch",
                    (long long)n, p.max_chunks);
    const plx::MarchLayout L = plx::MarchLayout::make(n, p.max_chunks);
    if (state_bytes < L.total)
        return fail(PLX_EINVAL, "d_state holds %zu bytes, plx_march_state_bytes gives %zu", state_bytes, L.total);
    char *b = static_cast<char *>(d_state);
    ptrs->hdr = reinterpret_cast<plx::MarchHeader *>(b + L.hdr_off);
    ptrs->n_occ = reinterpret_cast<int32_t *>(b + L.nocc_off);
    ptrs->done = reinterpret_cast<int32_t *>(b + L.done_off);
    ptrs->range = reinterpret_cast<int2 *>(b + L.first_off);
    ptrs->items = reinterpret_cast<int2 *>(b + L.items_off);
    ptrs->part = reinterpret_cast<float4 *>(b + L.part_off);
    ptrs->live = reinterpret_cast<uint8_t *>(b + L.live_off);
    ptrs->samp = plx::MarchLayout::store_samples(p.max_chunks) ? reinterpret_cast<uint16_t *>(b + L.samp_off) : nullptr;
    ptrs->vals = plx::MarchLayout::store_samples(p.max_chunks) ? reinterpret_cast<float4 *>(b + L.vals_off) : nullptr;
    ptrs->setup = b + L.setup_off;
    ptrs->max_chunks = p.max_chunks;
    std::memset(hdr, 0, sizeof(*hdr));
    hdr->magic = plx::kMarchMagic;
    hdr->max_chunks = p.max_chunks;
    hdr->n = n;
    hdr->total_items = 0;
    hdr->R = grid->desc.reso;
    hdr->M = grid->desc.n_rows;
    hdr->delta = p.delta;
    hdr->delta_lo = p.delta_lo;
    hdr->stop = p.stop;
    hdr->mode = opts->stop_thresh > 0.0f ? plx::kMarchRecompute : plx::kMarchChunked;
    hdr->ro = d_origins;
    hdr->rd = d_dirs;
    hdr->rows = grid->rows ? static_cast<const void *>(grid->rows) : static_cast<const void *>(grid->rows_h);
    return PLX_OK;
}

}  // namespace

plx_status plx_render_train(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                            const plx_render_opts *opts, float *d_rgb, float *d_T_end, void *d_state,
                            size_t state_bytes, void *stream) {
    plx_status st = check_grid(grid);
    if (st == PLX_OK) st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_origins || !d_dirs || !d_rgb)) return fail(PLX_EINVAL, "NULL ray or output buffer");
    if (grid->desc.sh_form == PLX_SH_F32 && grid->desc.n_rows > 0 && !grid->rows) return fail(PLX_EINVAL, "grid has no F32 rows");
    const plx::RenderParams p = make_params(grid, opts);
    plx::MarchPtrs ptrs;
    plx::MarchHeader hdr;
    st = march_state(grid, d_origins, d_dirs, n, opts, p, d_state, state_bytes, &ptrs, &hdr);
    if (st != PLX_OK) return st;
    return cuda_status(plx::launch_render_train(grid->view, d_origins, d_dirs, n, p, ptrs, hdr, d_rgb, d_T_end,
                                                static_cast<cudaStream_t>(stream)), "plx_render_train");
}

plx_status plx_march_plan(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                          const plx_render_opts *opts, void *d_state, size_t state_bytes, void *stream) {
    plx_status st = check_grid(grid);
    if (st == PLX_OK) st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_origins || !d_dirs)) return fail(PLX_EINVAL, "NULL ray buffer");
    const plx::RenderParams p = make_params(grid, opts);
    plx::MarchPtrs ptrs;
    plx::MarchHeader hdr;
    st = march_state(grid, d_origins, d_dirs, n, opts, p, d_state, state_bytes, &ptrs, &hdr);
    if (st != PLX_OK) return st;
    return cuda_status(plx::launch_march_plan(grid->view, d_origins, d_dirs, n, p, ptrs, hdr,
                                              static_cast<cudaStream_t>(stream)), "plx_march_plan");
}

plx_status plx_render_planned(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                              const plx_render_opts *opts, float *d_rgb, float *d_T_end, void *d_state,
                              size_t state_bytes, void *stream) {
    plx_status st = check_grid(grid);
    if (st == PLX_OK) st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_origins || !d_dirs || !d_rgb)) return fail(PLX_EINVAL, "NULL ray or output buffer");
    if (grid->desc.sh_form == PLX_SH_F32 && grid->desc.n_rows > 0 && !grid->rows) return fail(PLX_EINVAL, "grid has no F32 rows");
    const plx::RenderParams p = make_params(grid, opts);
    plx::MarchPtrs ptrs;
    plx::MarchHeader hdr;
    st = march_state(grid, d_origins, d_dirs, n, opts, p, d_state, state_bytes, &ptrs, &hdr);
    if (st != PLX_OK) return st;
    return cuda_status(plx::launch_render_planned(grid->view, d_origins, d_dirs, n, p, ptrs, hdr, d_rgb, d_T_end,
                                                  nullptr, nullptr, nullptr, static_cast<cudaStream_t>(stream)),
                       "plx_render_planned");
}

plx_status plx_render_planned_mse(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                                  const plx_render_opts *opts, const float *d_target, float *d_rgb,
                                  float *d_grad_rgb, float *d_loss, void *d_state, size_t state_bytes, void *stream) {
    plx_status st = check_grid(grid);
    if (st == PLX_OK) st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_origins || !d_dirs || !d_rgb || !d_target || !d_grad_rgb))
        return fail(PLX_EINVAL, "NULL ray, target or output buffer");
    if (n > 0 && (d_grad_rgb == d_rgb || d_grad_rgb == d_target)) return fail(PLX_EINVAL, "d_grad_rgb aliases an input");
    if (grid->desc.sh_form == PLX_SH_F32 && grid->desc.n_rows > 0 && !grid->rows) return fail(PLX_EINVAL, "grid has no F32 rows");
    const plx::RenderParams p = make_params(grid, opts);
    plx::MarchPtrs ptrs;
    plx::MarchHeader hdr;
    st = march_state(grid, d_origins, d_dirs, n, opts, p, d_state, state_bytes, &ptrs, &hdr);
    if (st != PLX_OK) return st;
    return cuda_status(plx::launch_render_planned(grid->view, d_origins, d_dirs, n, p, ptrs, hdr, d_rgb, nullptr,
                                                  d_target, d_grad_rgb, d_loss, static_cast<cudaStream_t>(stream)),
                       "plx_render_planned_mse");
}

plx_status plx_render_backward_train(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                                     const plx_render_opts *opts, const float *d_grad_rgb, const void *d_state,
                                     size_t state_bytes, float *d_grad_rows, float lambda_sparsity,
                                     float *d_loss_sparsity, void *stream) {
    plx_status st = check_grid(grid);
    if (st == PLX_OK) st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_origins || !d_dirs || !d_grad_rgb || !d_grad_rows)) return fail(PLX_EINVAL, "NULL buffer");
    if (d_grad_rows && !aligned(d_grad_rows, 16)) return fail(PLX_EINVAL, "d_grad_rows must be 16-byte aligned");
    if (!(lambda_sparsity >= 0.0f) || !std::isfinite(lambda_sparsity))
        return fail(PLX_EINVAL, "lambda_sparsity must be finite and >= 0");
    if (d_loss_sparsity && !aligned(d_loss_sparsity, 4)) return fail(PLX_EINVAL, "d_loss_sparsity must be 4-byte aligned");
    plx::RenderParams p = make_params(grid, opts);
    p.lam_s = lambda_sparsity;
    p.loss_s = d_loss_sparsity;
    plx::MarchPtrs ptrs;
    plx::MarchHeader hdr;
    st = march_state(grid, d_origins, d_dirs, n, opts, p, const_cast<void *>(d_state), state_bytes, &ptrs, &hdr);
    if (st != PLX_OK) return st;
    if (hdr.mode == plx::kMarchRecompute && p.max_chunks > 256)
        return fail(PLX_EUNSUPPORTED, "rays of up to %d samples with stop_thresh > 0 exceed the backward's 8192-sample "
                    "limit; raise step_vox", p.max_chunks * 32);
    return cuda_status(plx::launch_render_backward_train(grid->view, d_origins, d_dirs, n, p, ptrs, hdr, d_grad_rgb,
                                                         d_grad_rows, static_cast<cudaStream_t>(stream)),
                       "plx_render_backward_train");
}

plx_status plx_render_tiles(const plx_grid *const *grids, int32_t n_grids, const float *d_cams, int32_t n_cams,
                            const plx_tile *d_tiles, int64_t n_tiles, const plx_render_opts *opts, void *stream) {
    plx_status st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (!grids || n_grids < 1 || n_grids > PLX_TILES_MAX_SCENES)
        return fail(PLX_EINVAL, "need 1..%d grids", PLX_TILES_MAX_SCENES);
    if (n_tiles < 0 || n_tiles >= (int64_t(1) << 30)) return fail(PLX_EINVAL, "n_tiles out of range");
    if (n_tiles > 0 && (!d_tiles || !d_cams || n_cams < 1)) return fail(PLX_EINVAL, "NULL tiles or cameras");
    if (n_tiles > 0 && !aligned(d_tiles, 8)) return fail(PLX_EINVAL, "d_tiles must be 8-byte aligned");
    plx::GridView views[PLX_TILES_MAX_SCENES];
    plx::RenderParams params[PLX_TILES_MAX_SCENES];
    for (int i = 0; i < n_grids; ++i) {
        const plx_grid *g = grids[i];
        if (!g) return fail(PLX_EINVAL, "grids[%d] is NULL", i);
        if (g->desc.sh_form != grids[0]->desc.sh_form) return fail(PLX_EINVAL, "grids of one call must share sh_form");
        if (g->desc.sh_form == PLX_SH_F32 && g->desc.n_rows > 0 && !g->rows)
            return fail(PLX_EINVAL, "grids[%d] has no F32 rows", i);
        views[i] = g->view;
        params[i] = make_params(g, opts);
    }
    return cuda_status(plx::launch_render_tiles(views, params, n_grids, d_cams, n_cams, d_tiles, n_tiles,
                                                static_cast<cudaStream_t>(stream)), "plx_render_tiles");
}

plx_status plx_count_nodes(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                           const plx_render_opts *opts, int64_t *d_counts, void *stream) {
    plx_status st = check_grid(grid);
    if (st == PLX_OK) st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (n < 0 || n >= (int64_t(1) << 36)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_origins || !d_dirs || !d_counts)) return fail(PLX_EINVAL, "NULL buffer");
    plx::RenderParams p = make_params(grid, opts);
    return cuda_status(plx::launch_count_nodes(grid->view, d_origins, d_dirs, n, p, d_counts,
                                               static_cast<cudaStream_t>(stream)), "plx_count_nodes");
}

plx_status plx_count_touched(const plx_grid *grid, int64_t *d_count, void *stream) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    if (!d_count || !aligned(d_count, 8)) return fail(PLX_EINVAL, "d_count must be non-NULL and 8-byte aligned");
    return cuda_status(plx::launch_count_touched(grid->view, d_count, static_cast<cudaStream_t>(stream)),
                       "plx_count_touched");
}

plx_status plx_max_weight(const plx_grid *grid, const float *d_origins, const float *d_dirs, int64_t n,
                          const plx_render_opts *opts, float *d_wmax, void *stream) {
    plx_status st = check_grid(grid);
    if (st == PLX_OK) st = check_opts(opts);
    if (st != PLX_OK) return st;
    if (n < 0 || n >= (int64_t(1) << 36)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_origins || !d_dirs)) return fail(PLX_EINVAL, "NULL ray buffer");
    if (grid->desc.n_rows > 0 && !d_wmax) return fail(PLX_EINVAL, "d_wmax is NULL");
    if (d_wmax && !aligned(d_wmax, 4)) return fail(PLX_EINVAL, "d_wmax must be 4-byte aligned");
    if (grid->desc.sh_form == PLX_SH_F32 && grid->desc.n_rows > 0 && !grid->rows) return fail(PLX_EINVAL, "grid has no F32 rows");
    plx::RenderParams p = make_params(grid, opts);
    return cuda_status(plx::launch_max_weight(grid->view, d_origins, d_dirs, n, p, d_wmax,
                                              static_cast<cudaStream_t>(stream)), "plx_max_weight");
}

plx_status plx_mse_grad(const float *d_rgb, const float *d_target, int64_t n, float *d_grad_rgb, float *d_loss,
                        void *stream) {
    if (n < 0 || n >= (int64_t(1) << 36)) return fail(PLX_EINVAL, "n out of range");
    if (n > 0 && (!d_rgb || !d_target || !d_grad_rgb)) return fail(PLX_EINVAL, "NULL buffer");
    if (n > 0 && (d_grad_rgb == d_rgb || d_grad_rgb == d_target)) return fail(PLX_EINVAL, "d_grad_rgb aliases an input");
    return cuda_status(plx::launch_mse_grad(d_rgb, d_target, n, d_grad_rgb, d_loss, static_cast<cudaStream_t>(stream)),
                       "plx_mse_grad");
}

plx_status plx_tv_grad(const plx_grid *grid, const int64_t *d_seg_start, const int64_t *d_seg_len, int64_t n_seg,
                       int64_t n_selected, float lambda_sigma, float lambda_sh, float *d_grad_rows, float *d_loss,
                       void *stream) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    if (n_seg < 0 || n_selected < 0) return fail(PLX_EINVAL, "negative segment count");
    if (n_seg == 0 || n_selected == 0) return PLX_OK;
    if (!d_seg_start || !d_seg_len || !d_grad_rows) return fail(PLX_EINVAL, "NULL buffer");
    if (grid->desc.n_rows > 0 && !grid->rows) return fail(PLX_EINVAL, "TV needs the grid's F32 rows");
    if (!std::isfinite(lambda_sigma) || !std::isfinite(lambda_sh)) return fail(PLX_EINVAL, "lambda not finite");
    const float ls = (float)((double)lambda_sigma / (double)n_selected);
    const float lh = (float)((double)lambda_sh / (double)n_selected);
    return cuda_status(plx::launch_tv(grid->view, d_seg_start, d_seg_len, n_seg, n_selected, ls, lh, d_grad_rows,
                                      d_loss, static_cast<cudaStream_t>(stream)), "plx_tv_grad");
}

plx_status plx_rmsprop_step(plx_grid *grid, float *d_grad_rows, float *d_v, float lr_sigma, float lr_sh, float beta,
                            float eps, int32_t sparse, void *stream) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    if (grid->desc.n_rows == 0) return PLX_OK;
    if (!grid->rows) return fail(PLX_EINVAL, "RMSProp needs the grid's F32 rows");
    if (!d_grad_rows || !d_v) return fail(PLX_EINVAL, "NULL gradient or state buffer");
    if (!(beta >= 0.0f && beta < 1.0f) || !(eps >= 0.0f) || !std::isfinite(lr_sigma) || !std::isfinite(lr_sh))
        return fail(PLX_EINVAL, "bad RMSProp hyper-parameters");
    if (sparse != 0 && sparse != 1) return fail(PLX_EINVAL, "sparse must be 0 or 1");
    // sparse calls alternate between the status block's two list lengths: each starts at zero (the
    // block is zeroed at creation) and the call that uses one zeroes the other for the next call
    plx::GridView v = grid->view;
    char *status = grid->ws + grid->layout.status_off;
    const size_t off[2] = {plx::WorkspaceLayout::kListCountOff, plx::WorkspaceLayout::kListCount2Off};
    v.tcount = reinterpret_cast<int *>(status + off[grid->rms_parity]);
    int *next = reinterpret_cast<int *>(status + off[grid->rms_parity ^ 1]);
    const plx_status r = cuda_status(plx::launch_rmsprop(v, grid->rows, grid->desc.sh_form == PLX_SH_BF16 ? grid->rows_h : nullptr,
                                                         d_grad_rows, d_v, lr_sigma, lr_sh, beta, eps, sparse,
                                                         sparse ? next : nullptr, static_cast<cudaStream_t>(stream)),
                                     "plx_rmsprop_step");
    if (r == PLX_OK && sparse) grid->rms_parity ^= 1;
    return r;
}

size_t plx_prune_workspace_bytes(int32_t reso) {
    if (reso < 2 || reso > 2048) return 0;
    return plx::prune_ws_bytes(reso);
}

size_t plx_upsample_workspace_bytes(int32_t new_reso) {
    if (new_reso < 2 || new_reso > 2048) return 0;
    return plx::upsample_ws_bytes(new_reso);
}

static plx_status prune_count(const plx_grid *grid, const float *d_key, float tau, int32_t dilate, void *d_ws,
                              int64_t *n_keep, void *stream, const char *who) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    if (!n_keep) return fail(PLX_EINVAL, "n_keep is NULL");
    if (!d_ws || !aligned(d_ws, 256)) return fail(PLX_EINVAL, "d_ws must be non-NULL and 256-byte aligned");
    if (grid->desc.n_rows > 0 && !grid->rows) return fail(PLX_EINVAL, "pruning needs the grid's F32 rows");
    if (std::isnan(tau)) return fail(PLX_EINVAL, "tau is NaN");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = plx::launch_prune_count(grid->view, d_key, tau, dilate ? 1 : 0, d_ws, s);
    int64_t count = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&count, static_cast<char *>(d_ws) + plx::kWsCountOff, sizeof(int64_t),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, who);
    *n_keep = count;
    return PLX_OK;
}

plx_status plx_grid_prune_count(const plx_grid *grid, float tau, int32_t dilate, void *d_ws, int64_t *n_keep,
                                void *stream) {
    return prune_count(grid, nullptr, tau, dilate, d_ws, n_keep, stream, "plx_grid_prune_count");
}

plx_status plx_grid_prune_count_key(const plx_grid *grid, const float *d_key, float tau, int32_t dilate, void *d_ws,
                                    int64_t *n_keep, void *stream) {
    if (grid && grid->desc.n_rows > 0 && !d_key) return fail(PLX_EINVAL, "d_key is NULL");
    return prune_count(grid, d_key, tau, dilate, d_ws, n_keep, stream, "plx_grid_prune_count_key");
}

plx_status plx_grid_prune_apply(const plx_grid *grid, const void *d_ws, int64_t n_keep, int32_t *d_idx_new,
                                float *d_rows_new, void *stream) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    if (!d_ws || !aligned(d_ws, 256) || !d_idx_new) return fail(PLX_EINVAL, "NULL or misaligned buffer");
    if (n_keep < 0 || n_keep > grid->desc.n_rows) return fail(PLX_EINVAL, "n_keep %lld out of range", (long long)n_keep);
    if (n_keep > 0 && !d_rows_new) return fail(PLX_EINVAL, "d_rows_new is NULL");
    if (d_rows_new && !aligned(d_rows_new, 16)) return fail(PLX_EINVAL, "d_rows_new must be 16-byte aligned");
    if (grid->desc.n_rows > 0 && !grid->rows) return fail(PLX_EINVAL, "pruning needs the grid's F32 rows");
    return cuda_status(plx::launch_prune_apply(grid->view, d_ws, n_keep, d_idx_new, d_rows_new,
                                               static_cast<cudaStream_t>(stream)), "plx_grid_prune_apply");
}

plx_status plx_grid_upsample_count(const plx_grid *grid, int32_t new_reso, void *d_ws, int64_t *n_rows_new, void *stream) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    if (new_reso < 2 || new_reso > 2048) return fail(PLX_EINVAL, "new_reso %d outside [2, 2048]", new_reso);
    if (!n_rows_new) return fail(PLX_EINVAL, "n_rows_new is NULL");
    if (!d_ws || !aligned(d_ws, 256)) return fail(PLX_EINVAL, "d_ws must be non-NULL and 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = plx::launch_upsample_count(grid->view, new_reso, d_ws, s);
    int64_t count = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&count, static_cast<char *>(d_ws) + plx::kWsCountOff, sizeof(int64_t),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "plx_grid_upsample_count");
    if (count >= (int64_t(1) << 31)) return fail(PLX_EUNSUPPORTED, "upsampled grid would have %lld rows", (long long)count);
    *n_rows_new = count;
    return PLX_OK;
}

plx_status plx_grid_upsample_apply(const plx_grid *grid, int32_t new_reso, const void *d_ws, int64_t n_rows_new,
                                   int32_t *d_idx_new, float *d_rows_new, void *stream) {
    plx_status st = check_grid(grid);
    if (st != PLX_OK) return st;
    if (new_reso < 2 || new_reso > 2048) return fail(PLX_EINVAL, "new_reso %d outside [2, 2048]", new_reso);
    if (!d_ws || !aligned(d_ws, 256) || !d_idx_new) return fail(PLX_EINVAL, "NULL or misaligned buffer");
    if (n_rows_new < 0 || n_rows_new >= (int64_t(1) << 31)) return fail(PLX_EINVAL, "n_rows_new out of range");
    if (n_rows_new > 0 && !d_rows_new) return fail(PLX_EINVAL, "d_rows_new is NULL");
    if (d_rows_new && !aligned(d_rows_new, 16)) return fail(PLX_EINVAL, "d_rows_new must be 16-byte aligned");
    if (grid->desc.n_rows > 0 && !grid->rows) return fail(PLX_EINVAL, "upsampling needs the grid's F32 rows");
    return cuda_status(plx::launch_upsample_apply(grid->view, new_reso, d_ws, n_rows_new, d_idx_new, d_rows_new,
                                                  static_cast<cudaStream_t>(stream)), "plx_grid_upsample_apply");
}

}  // extern "C"
