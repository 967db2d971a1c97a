// msz_segment.cu -- Morse-Smale segmentation labels by pointer jumping and the
// verification counts (pMSz, arXiv 2601.01787, Sec. III-A and Sec. V-C).
//
// Sec. III-A: the integral line of a vertex follows the steepest neighbour
// until an extremum; the ascending (descending) segmentation groups vertices
// by the maximum (minimum) reached.  Labels start as the one-step pointers of
// the codes and jump in place, lab[i] <- lab[lab[i]], inside one cooperative
// kernel until a round changes nothing.  Every value a thread can observe is
// a vertex on the same integral line, so the in-place rounds converge to the
// unique fixed point: the extremum at the end of the line.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_workspace.h"

namespace msz {

constexpr int kSegThreads = 512;
constexpr uint32_t kErrCodes = 4u;  // a code names a slot outside the grid, or codes form a cycle
constexpr uint32_t kMaxRounds = 40;

template <int NDIM>
__global__ void __launch_bounds__(256) k_seg_init(const uint8_t *codes, __grid_constant__ const GridDev G,
                                                 int32_t *min_lab, int32_t *max_lab, Ctrl *C) {
    const uint32_t stride = gridDim.x * blockDim.x;
    constexpr uint32_t ns = NDIM == 2 ? 6 : 14;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += stride) {
        uint32_t x, y, z;
        coords_of(G, i, x, y, z);
        const uint8_t c = codes[i];
        const uint32_t up = c & 15u, dn = c >> 4;
        bool bad = false;
        int32_t mx = (int32_t)i, mn = (int32_t)i;
        if (up != kSelf) {
            if (up < ns && slot_in_domain(G, (int)up, x, y, z)) mx = (int32_t)((int64_t)i + G.off[up]);
            else bad = true;
        }
        if (dn != kSelf) {
            if (dn < ns && slot_in_domain(G, (int)dn, x, y, z)) mn = (int32_t)((int64_t)i + G.off[dn]);
            else bad = true;
        }
        if (bad) atomicOr(&C->error, kErrCodes);
        if (max_lab) max_lab[i] = mx;
        if (min_lab) min_lab[i] = mn;
    }
}

__global__ void __launch_bounds__(kSegThreads) k_seg_jump(uint32_t n, int32_t *min_lab, int32_t *max_lab,
                                                          Ctrl *C, uint32_t *flags) {
    const uint32_t stride = gridDim.x * blockDim.x;
    // Integral lines are at most n vertices long, so in-place jumping is done
    // within 32 rounds; more rounds mean the codes hold a cycle (codes not
    // computed from a field), reported instead of looping.
    for (uint32_t round = 0;; ++round) {
        if (round == kMaxRounds) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&C->error, kErrCodes);
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[(round + 1) % 3] = 0;
        bool changed = false;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            if (max_lab) {
                const int32_t a = max_lab[i];
                const int32_t b = max_lab[a];
                if (b != a) { max_lab[i] = b; changed = true; }
            }
            if (min_lab) {
                const int32_t a = min_lab[i];
                const int32_t b = min_lab[a];
                if (b != a) { min_lab[i] = b; changed = true; }
            }
        }
        if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&flags[round % 3], 1u);
        if (!grid_barrier(&C->bar_count, &C->bar_gen, &C->error)) return;
        if (ld_relaxed(&flags[round % 3]) == 0) return;
    }
}

__global__ void __launch_bounds__(256) k_compare(const uint8_t *cf, const uint8_t *cg, const int32_t *mnf,
                                                 const int32_t *mxf, const int32_t *mng, const int32_t *mxg,
                                                 uint64_t n, Ctrl *C) {
    uint32_t c[6] = {0, 0, 0, 0, 0, 0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint8_t a = cf[i], b = cg[i];
        c[0] += (mnf[i] != mng[i] || mxf[i] != mxg[i]);
        const bool maxf = (a & 15u) == kSelf, maxg = (b & 15u) == kSelf;
        const bool minf = (a >> 4) == kSelf, ming = (b >> 4) == kSelf;
        c[1] += maxg && !maxf;
        c[2] += maxf && !maxg;
        c[3] += ming && !minf;
        c[4] += minf && !ming;
        c[5] += a != b;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        uint32_t v = c[q];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(kFull, v, d);
        if (lane_id() == 0 && v) atomicAdd(&C->counts[q], (unsigned long long)v);
    }
}

static std::mutex g_seg_mu;

static msz_status seg_blocks(const DeviceInfo &d, int &blocks) {
    static int cache[64];
    std::lock_guard<std::mutex> lk(g_seg_mu);
    if (!cache[d.device]) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_seg_jump, kSegThreads, 0) != cudaSuccess)
            return MSZ_ERR_CUDA;
        if (per < 1) return MSZ_ERR_UNSUPPORTED;
        int b = per * d.sms;
        if (b > (int)kMaxBlocks) b = (int)kMaxBlocks;
        cache[d.device] = b;
    }
    blocks = cache[d.device];
    return MSZ_OK;
}

}  // namespace msz

using namespace msz;

extern "C" msz_status msz_segment(const uint8_t *d_codes, msz_grid grid, int32_t *d_min_label, int32_t *d_max_label,
                                  void *d_workspace, size_t workspace_bytes, msz_stream_t stream) {
    if (!d_codes || (!d_min_label && !d_max_label)) return MSZ_ERR_INVALID_ARG;
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    if (!d_workspace || workspace_bytes < MSZ_SMALL_WORKSPACE) return MSZ_ERR_WORKSPACE;
    if ((uintptr_t)d_workspace % kAlign) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Ctrl *C = (Ctrl *)d_workspace;
    uint32_t *flags = (uint32_t *)((char *)d_workspace + align_up(sizeof(Ctrl)));
    if (cudaMemsetAsync(d_workspace, 0, align_up(sizeof(Ctrl)) + kAlign, s) != cudaSuccess) return MSZ_ERR_CUDA;
    const int blocks = dev.sms * 8;
    if (G.ndim == 3)
        k_seg_init<3><<<blocks, 256, 0, s>>>(d_codes, G, d_min_label, d_max_label, C);
    else
        k_seg_init<2><<<blocks, 256, 0, s>>>(d_codes, G, d_min_label, d_max_label, C);
    if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
    int jb = 0;
    if ((st = seg_blocks(dev, jb)) != MSZ_OK) return st;
    uint32_t n = G.n;
    void *args[] = {(void *)&n, (void *)&d_min_label, (void *)&d_max_label, (void *)&C, (void *)&flags};
    if (cudaLaunchCooperativeKernel((const void *)k_seg_jump, dim3(jb), dim3(kSegThreads), args, 0, s) != cudaSuccess)
        return MSZ_ERR_CUDA;
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, &C->error, sizeof err, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (err & kErrCodes) return MSZ_ERR_INVALID_ARG;
    if (err & kErrTimeout) return MSZ_ERR_TIMEOUT;
    return MSZ_OK;
}

extern "C" msz_status msz_compare(const uint8_t *d_codes_f, const uint8_t *d_codes_g, const int32_t *d_min_f,
                                  const int32_t *d_max_f, const int32_t *d_min_g, const int32_t *d_max_g, int64_t n,
                                  int64_t h_counts[6], void *d_workspace, size_t workspace_bytes,
                                  msz_stream_t stream) {
    if (!d_codes_f || !d_codes_g || !d_min_f || !d_max_f || !d_min_g || !d_max_g || !h_counts || n < 0)
        return MSZ_ERR_INVALID_ARG;
    if (!d_workspace || workspace_bytes < MSZ_SMALL_WORKSPACE) return MSZ_ERR_WORKSPACE;
    if ((uintptr_t)d_workspace % kAlign) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    msz_status st = current_device(dev);
    if (st != MSZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Ctrl *C = (Ctrl *)d_workspace;
    if (cudaMemsetAsync(d_workspace, 0, sizeof(Ctrl), s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (n > 0) {
        k_compare<<<dev.sms * 8, 256, 0, s>>>(d_codes_f, d_codes_g, d_min_f, d_max_f, d_min_g, d_max_g, (uint64_t)n, C);
        if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
    }
    unsigned long long c[8];
    if (cudaMemcpyAsync(c, C->counts, sizeof c, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    for (int q = 0; q < 6; ++q) h_counts[q] = (int64_t)c[q];
    return MSZ_OK;
}
