// plx_noalloc.cu -- density pruning in one call that allocates nothing.
//
// Who needs this: callers that cannot, or may not, allocate device memory
// while they run.  A renderer plugged into a host application works inside
// a fixed memory budget that the host hands out at start-up; a real-time
// loop cannot afford cudaMalloc, which may synchronise the whole device; and
// some embedders have no allocator of their own to give us a workspace.
// plx_grid_prune_count/apply need a caller workspace; this variant instead
// keeps the same scratch (keep bit maps, per-block counts and offsets) in a
// file-scope device array of fixed size, and writes the output into buffers
// the caller sized in advance (pruning never adds rows, so n_rows rows are
// always enough).
//
// The array is a single shared buffer per device:
//   * it holds PLX_PRUNE_NOALLOC_SCRATCH_BYTES on every GPU that loads the
//     library, until the process exits;
//   * it serves grids of up to PLX_PRUNE_NOALLOC_MAX_RESO nodes per axis;
//   * every call reuses it and it keeps the last call's contents; each call
//     overwrites all of it that it later reads, so nothing has to start at
//     zero;
//   * two calls whose work overlaps on the GPU (different streams, or
//     different host threads on one device) race on it.
#include "plx_internal.cuh"

namespace {

constexpr size_t kScratchBytes = PLX_PRUNE_NOALLOC_SCRATCH_BYTES;

__device__ __align__(256) unsigned char g_prune_scratch[kScratchBytes];

// Device address of g_prune_scratch on the current device.  In host code the symbol names a
// host-side shadow, not device memory, so only the address from cudaGetSymbolAddress may be
// passed to a kernel.  It is looked up on every call (no allocation, no stream work), so an
// address never outlives the context it came from: after a device reset the module is
// reloaded, possibly elsewhere, and the next call sees the new address.
cudaError_t scratch_for_current_device(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_prune_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" plx_status plx_grid_prune_noalloc(const plx_grid *grid, float tau, int32_t dilate, int32_t *d_idx_new,
                                             float *d_rows_new, int64_t *n_keep, void *stream) {
    const plx::GridView *v = plx::grid_view(grid);
    if (!v) return plx::set_error(PLX_EINVAL, "grid is NULL");
    if (!n_keep) return plx::set_error(PLX_EINVAL, "n_keep is NULL");
    if (!d_idx_new) return plx::set_error(PLX_EINVAL, "d_idx_new is NULL");
    if (v->M > 0 && (!d_rows_new || !v->rows))
        return plx::set_error(PLX_EINVAL, "pruning needs the grid's F32 rows and an output of n_rows rows");
    if (d_rows_new && (reinterpret_cast<uintptr_t>(d_rows_new) & 15u))
        return plx::set_error(PLX_EINVAL, "d_rows_new must be 16-byte aligned");
    if (tau != tau) return plx::set_error(PLX_EINVAL, "tau is NaN");
    if (v->R > PLX_PRUNE_NOALLOC_MAX_RESO || plx::prune_ws_bytes(v->R) > kScratchBytes)
        return plx::set_error(PLX_EUNSUPPORTED,
                              "plx_grid_prune_noalloc serves grids of at most 256^3 nodes (its fixed scratch); "
                              "use plx_grid_prune_count/apply with a workspace");
    void *ws = nullptr;
    cudaError_t e = scratch_for_current_device(&ws);
    if (e != cudaSuccess) return plx::set_error(PLX_ECUDA, cudaGetErrorString(e));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = plx::launch_prune_count(*v, nullptr, tau, dilate ? 1 : 0, ws, s);
    int64_t count = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&count, static_cast<char *>(ws) + plx::kWsCountOff, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && (count < 0 || count > v->M)) return plx::set_error(PLX_EDEVICE, "kept-row count out of range");
    if (e == cudaSuccess) e = plx::launch_prune_apply(*v, ws, count, d_idx_new, d_rows_new, s);
    if (e != cudaSuccess) return plx::set_error(PLX_ECUDA, cudaGetErrorString(e));
    *n_keep = count;
    return PLX_OK;
}
