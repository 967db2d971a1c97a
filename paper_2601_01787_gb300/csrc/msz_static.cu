// msz_static.cu -- msz_correct without a caller-provided workspace.
//
// Some callers cannot call cudaMalloc: a plugin whose host application owns
// every device allocation, code that runs where a device allocation would
// block or synchronize the device (a latency-critical loop, a host callback),
// or a program that must not grow its memory footprint after start-up.  For
// them this file keeps the correction's scratch memory in a file-scope
// __device__ array and passes its address to the unchanged msz_correct path.
//
// The array is fixed at compile time: every GPU that loads the library holds
// it until the process exits, and every call shares it.  msz_correct clears
// the part that must start at zero (control block, sweep log, bitmaps) at the
// start of each call; the rest is overwritten before it is read.  Calls that
// overlap on the GPU (different streams, different host threads) would share
// the array and race: serialize them.
#include <cuda_runtime.h>
#include <stdint.h>

#include "msz.h"
#include "msz_workspace.h"

namespace {

constexpr size_t kStaticBytes = msz::layout_for((uint64_t)MSZ_STATIC_MAX_VERTICES).total;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// The array's device address, looked up on every call with the caller's
// device current (host code cannot use the array's name as a device address).
// The lookup is cheap once the module is loaded, and a cached address would go
// stale if the context were torn down and re-created (cudaDeviceReset), which
// reloads the module at a possibly different address.
msz_status static_scratch(void **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return MSZ_ERR_CUDA;
    *out = p;
    return MSZ_OK;
}

}  // namespace

extern "C" msz_status msz_correct_static(const float *d_f, const float *d_fhat, float xi, msz_grid grid,
                                         float *d_out, uint32_t *d_edit_idx, float *d_edit_delta,
                                         int64_t edit_capacity, int64_t *h_edit_count, const msz_options *opt,
                                         msz_stats *h_stats, msz_stream_t stream) {
    msz::GridDev G;
    const msz_status gst = msz::make_grid(grid, G);
    if (gst != MSZ_OK) return gst;
    if ((int64_t)G.n > (int64_t)MSZ_STATIC_MAX_VERTICES) return MSZ_ERR_WORKSPACE;
    void *scratch = nullptr;
    const msz_status st = static_scratch(&scratch);
    if (st != MSZ_OK) return st;
    return msz_correct(d_f, d_fhat, xi, grid, d_out, d_edit_idx, d_edit_delta, edit_capacity, h_edit_count, opt,
                       h_stats, scratch, kStaticBytes, stream);
}
