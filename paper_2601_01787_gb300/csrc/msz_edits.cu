// msz_edits.cu -- encoding of the edit list (the storage of the edits that the
// pMSz paper, arXiv 2601.01787, counts as its storage overhead in Sec. V).
//
// An edit is (i, m): vertex i where g and fhat differ bitwise and its ulp
// distance m = (ord(fhat_i) - ord(g_i)) mod 2^32 (ord: a float's bits as an
// unsigned key in value order).  The list is cut into blocks of
// MSZ_EDIT_BLOCK edits; each block stores its first index and bit-packs the
// index gaps and the ulp distances at the widths its own largest values need.
// Blocks are independent once their payload offsets are known, so encoding
// is three launches (widths, a scan of the block sizes, packing) and
// decoding two (a check of the whole stream, then the edits applied) with one
// warp per block.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_workspace.h"

namespace msz {
namespace edits {

constexpr uint32_t B = MSZ_EDIT_BLOCK;
constexpr uint32_t PER_LANE = B / 32;  // 8 edits per lane, contiguous
constexpr int kWarps = 8;              // warps (blocks of the stream) per thread block
constexpr uint32_t kErrArg = 1u;
constexpr uint32_t kErrCap = 2u;  // the stream would exceed the output buffer (nothing written)

struct Ctrl {
    uint32_t error;
    uint32_t pad;
    unsigned long long total_words;
};

// The number of edits: count_cap, or, when d_count is given (an encode queued
// behind the correction that lists them), min(*d_count, count_cap).
__device__ __forceinline__ uint64_t edit_count(const unsigned long long *d_count, uint64_t count_cap) {
    if (!d_count) return count_cap;
    const unsigned long long c = *d_count;
    return c < count_cap ? c : count_cap;
}

__device__ __forceinline__ uint32_t ord_key(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float float_of_key(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ uint32_t bit_len(uint32_t v) { return v ? 32u - (uint32_t)__clz(v) : 0u; }

__host__ __device__ inline uint64_t section_words(uint32_t c, uint32_t w) { return ((uint64_t)c * w + 31u) / 32u; }

// Byte offsets of the stream's parts for nb blocks.
struct Layout {
    uint64_t first, start, wd, wm, payload;
};
__host__ __device__ inline Layout layout_of(uint64_t nb) {
    Layout L;
    L.first = 16;
    L.start = L.first + 4 * nb;
    L.wd = L.start + 4 * nb;
    L.wm = L.wd + nb;
    L.payload = (L.wm + nb + 3) / 4 * 4;
    return L;
}

// Word t of a section of c values packed w bits each (vals in shared memory).
__device__ __forceinline__ uint32_t packed_word(const uint32_t *vals, uint32_t c, uint32_t w, uint32_t t) {
    const uint32_t lo = 32u * t;
    const uint32_t j0 = lo / w;
    const uint32_t j1 = min(c - 1u, (lo + 31u) / w);
    uint32_t word = 0;
    for (uint32_t j = j0; j <= j1; ++j) {
        const int64_t pos = (int64_t)j * w - lo;
        const uint64_t v = vals[j];
        word |= (uint32_t)(pos >= 0 ? v << pos : v >> -pos);
    }
    return word;
}

// Value j of a section packed w bits each starting at word pointer sec.
__device__ __forceinline__ uint32_t unpacked(const uint32_t *sec, uint32_t w, uint32_t j) {
    if (w == 0) return 0u;
    const uint64_t pos = (uint64_t)j * w;
    const uint32_t wi = (uint32_t)(pos >> 5), sh = (uint32_t)(pos & 31u);
    uint64_t v = sec[wi] >> sh;
    if (sh + w > 32u) v |= (uint64_t)sec[wi + 1] << (32u - sh);
    return (uint32_t)(w == 32u ? v : v & ((1ull << w) - 1ull));
}

// ---- encode 1: per block, gaps and distances, their widths and word count
__global__ void __launch_bounds__(kWarps * 32) k_widths(const float *fhat, const float *g, uint32_t n,
                                                        const uint32_t *idx, const unsigned long long *d_count,
                                                        uint64_t count_cap, uint32_t *words, uint8_t *wd_out,
                                                        uint8_t *wm_out, Ctrl *C) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t count = edit_count(d_count, count_cap);
    const uint64_t nb = (count + B - 1) / B;
    for (uint64_t k = ((uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5)); k < nb; k += (uint64_t)gridDim.x * kWarps) {
        const uint64_t base = k * B;
        const uint32_t c = (uint32_t)(count - base < B ? count - base : B);
        uint32_t dmax = 0, mmax = 0;
        bool bad = false;
        for (uint32_t e = 0; e < PER_LANE; ++e) {
            const uint32_t j = lane * PER_LANE + e;
            if (j >= c) break;
            const uint32_t i = idx[base + j];
            if (i >= n) { bad = true; continue; }
            if (base + j > 0) {
                const uint32_t p = idx[base + j - 1];
                if (i <= p) { bad = true; continue; }
                if (j > 0) dmax = max(dmax, i - p - 1u);
            }
            mmax = max(mmax, ord_key(fhat[i]) - ord_key(g[i]) - 1u);
        }
        if (bad) atomicOr(&C->error, kErrArg);
        dmax = __reduce_max_sync(kFull, dmax);
        mmax = __reduce_max_sync(kFull, mmax);
        if (lane == 0) {
            const uint32_t wd = bit_len(dmax), wm = bit_len(mmax);
            wd_out[k] = (uint8_t)wd;
            wm_out[k] = (uint8_t)wm;
            words[k] = (uint32_t)(section_words(c, wd) + section_words(c, wm));
        }
    }
}

// ---- encode 2: exclusive scan of the block word counts (one thread block)
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_scan(const uint32_t *words, const unsigned long long *d_count,
                                                      uint64_t count_cap, uint32_t *start, Ctrl *C) {
    const uint64_t nb = (edit_count(d_count, count_cap) + B - 1) / B;
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_carry;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const uint64_t k = b0 + threadIdx.x;
        const unsigned long long v = k < nb ? words[k] : 0ull;
        unsigned long long x = v;  // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = s_warp[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kFull, t, o);
                if (lane >= (uint32_t)o) t += y;
            }
            s_warp[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        const unsigned long long before = s_carry + (warp ? s_warp[warp - 1] : 0ull) + x - v;
        if (k < nb) start[k] = (uint32_t)before;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[kScanThreads / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) C->total_words = s_carry;
}

// ---- encode 3: header, table and payload
__global__ void __launch_bounds__(kWarps * 32) k_pack(const float *fhat, const float *g, const uint32_t *idx,
                                                      const unsigned long long *d_count, uint64_t count_cap,
                                                      const uint32_t *start, const uint8_t *wd_in,
                                                      const uint8_t *wm_in, uint8_t *out, uint64_t capacity,
                                                      Ctrl *C) {
    __shared__ uint32_t s_d[kWarps][B], s_m[kWarps][B];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t count = edit_count(d_count, count_cap);
    const uint64_t nb = (count + B - 1) / B;
    const Layout L = layout_of(nb);
    // an error found by the widths pass, or a stream longer than the buffer:
    // nothing is written
    if (ld_relaxed(&C->error) || L.payload + 4ull * C->total_words > capacity) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && !C->error) atomicOr(&C->error, kErrCap);
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t *h = reinterpret_cast<uint32_t *>(out);
        h[0] = MSZ_EDIT_MAGIC;
        h[1] = B;
        h[2] = (uint32_t)count;
        h[3] = (uint32_t)(count >> 32);
        for (uint64_t q = L.wm + nb; q < L.payload; ++q) out[q] = 0;
    }
    uint32_t *pay = reinterpret_cast<uint32_t *>(out + L.payload);
    for (uint64_t k = ((uint64_t)blockIdx.x * kWarps + warp); k < nb; k += (uint64_t)gridDim.x * kWarps) {
        const uint64_t base = k * B;
        const uint32_t c = (uint32_t)(count - base < B ? count - base : B);
        for (uint32_t e = 0; e < PER_LANE; ++e) {
            const uint32_t j = lane * PER_LANE + e;
            if (j >= c) break;
            const uint32_t i = idx[base + j];
            s_d[warp][j] = j ? i - idx[base + j - 1] - 1u : 0u;
            s_m[warp][j] = ord_key(fhat[i]) - ord_key(g[i]) - 1u;
        }
        __syncwarp();
        const uint32_t wd = wd_in[k], wm = wm_in[k];
        const uint32_t nd = (uint32_t)section_words(c, wd), nm = (uint32_t)section_words(c, wm);
        uint32_t *dst = pay + start[k];
        for (uint32_t t = lane; t < nd; t += 32) dst[t] = packed_word(s_d[warp], c, wd, t);
        for (uint32_t t = lane; t < nm; t += 32) dst[nd + t] = packed_word(s_m[warp], c, wm, t);
        if (lane == 0) {
            reinterpret_cast<uint32_t *>(out + L.first)[k] = idx[base];
            reinterpret_cast<uint32_t *>(out + L.start)[k] = start[k];
            out[L.wd + k] = (uint8_t)wd;
            out[L.wm + k] = (uint8_t)wm;
        }
        __syncwarp();
    }
}

// ---- decode 1: every block's table entry and indices checked; last index
// of each block recorded
__global__ void __launch_bounds__(kWarps * 32) k_check(const uint8_t *in, uint64_t payload_words, uint64_t count,
                                                       uint32_t n, uint32_t *last, Ctrl *C) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nb = (count + B - 1) / B;
    const Layout L = layout_of(nb);
    const uint32_t *pay = reinterpret_cast<const uint32_t *>(in + L.payload);
    for (uint64_t k = ((uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5)); k < nb; k += (uint64_t)gridDim.x * kWarps) {
        const uint32_t c = (uint32_t)(count - k * B < B ? count - k * B : B);
        const uint32_t first = reinterpret_cast<const uint32_t *>(in + L.first)[k];
        const uint32_t s = reinterpret_cast<const uint32_t *>(in + L.start)[k];
        const uint32_t wd = in[L.wd + k], wm = in[L.wm + k];
        bool ok = wd <= 32u && wm <= 32u && first < n;
        ok = ok && (uint64_t)s + section_words(c, wd) + section_words(c, wm) <= payload_words;
        // index of the lane's last edit: first + sum of (d_j + 1) over j >= 1
        unsigned long long sum = 0;
        if (ok) {
            for (uint32_t e = 0; e < PER_LANE; ++e) {
                const uint32_t j = lane * PER_LANE + e;
                if (j >= c || j == 0) continue;
                sum += (unsigned long long)unpacked(pay + s, wd, j) + 1ull;
            }
        }
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);  // < 2^41: no wrap
        if (lane == 0) {
            const unsigned long long li = (unsigned long long)first + sum;
            if (!ok || li >= n) atomicOr(&C->error, kErrArg);
            last[k] = li < 0xffffffffull ? (uint32_t)li : 0xffffffffu;
        }
    }
}

// ---- decode 2: blocks in ascending order (first index past the previous
// block's last)
__global__ void k_order(const uint8_t *in, uint64_t count, const uint32_t *last, Ctrl *C) {
    const uint64_t nb = (count + B - 1) / B;
    const Layout L = layout_of(nb);
    const uint32_t *first = reinterpret_cast<const uint32_t *>(in + L.first);
    for (uint64_t k = 1 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += (uint64_t)gridDim.x * blockDim.x)
        if (first[k] <= last[k - 1]) atomicOr(&C->error, kErrArg);
}

// ---- decode 3: the edits applied, g_i = ord^-1(ord(fhat_i) - m_i)
__global__ void __launch_bounds__(kWarps * 32) k_apply(const uint8_t *in, uint64_t count, float *field) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nb = (count + B - 1) / B;
    const Layout L = layout_of(nb);
    const uint32_t *pay = reinterpret_cast<const uint32_t *>(in + L.payload);
    for (uint64_t k = ((uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5)); k < nb; k += (uint64_t)gridDim.x * kWarps) {
        const uint32_t c = (uint32_t)(count - k * B < B ? count - k * B : B);
        const uint32_t first = reinterpret_cast<const uint32_t *>(in + L.first)[k];
        const uint32_t s = reinterpret_cast<const uint32_t *>(in + L.start)[k];
        const uint32_t wd = in[L.wd + k], wm = in[L.wm + k];
        const uint32_t nd = (uint32_t)section_words(c, wd);
        // the lane's 8 edits are contiguous: its indices are the warp's
        // exclusive prefix of gap sums plus a running sum
        uint32_t d[PER_LANE], local = 0;
        for (uint32_t e = 0; e < PER_LANE; ++e) {
            const uint32_t j = lane * PER_LANE + e;
            d[e] = (j < c && j > 0) ? unpacked(pay + s, wd, j) + 1u : 0u;
            local += d[e];
        }
        uint32_t incl = local;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        uint32_t i = first + incl - local;
        for (uint32_t e = 0; e < PER_LANE; ++e) {
            const uint32_t j = lane * PER_LANE + e;
            if (j >= c) break;
            i += d[e];
            const uint32_t m = unpacked(pay + s + nd, wm, j) + 1u;
            field[i] = float_of_key(ord_key(field[i]) - m);
        }
    }
}

__host__ __device__ inline uint64_t blocks_of(int64_t count) { return ((uint64_t)count + B - 1) / B; }

struct Work {
    Ctrl *ctrl;
    uint32_t *words;   // encode: words per block; decode: last index per block
    uint32_t *start;
    uint8_t *wd, *wm;
};

inline size_t work_bytes(uint64_t nb) { return 256 + align_up(4 * nb) * 2 + align_up(nb) * 2; }

inline Work work_of(void *ws, uint64_t nb) {
    uint8_t *p = static_cast<uint8_t *>(ws);
    Work w;
    w.ctrl = reinterpret_cast<Ctrl *>(p);
    p += 256;
    w.words = reinterpret_cast<uint32_t *>(p);
    p += align_up(4 * nb);
    w.start = reinterpret_cast<uint32_t *>(p);
    p += align_up(4 * nb);
    w.wd = p;
    p += align_up(nb);
    w.wm = p;
    return w;
}

inline int grid_for(const DeviceInfo &dev, uint64_t nb) {
    const uint64_t want = (nb + kWarps - 1) / kWarps, cap = (uint64_t)dev.sms * 16;
    return (int)(want < 1 ? 1 : want > cap ? cap : want);
}

}  // namespace edits

// The encode queued on a stream behind the correction that lists the edits
// (the pipeline's encoded output): the count is read on the device from
// d_count (capped at count_cap); no host synchronization.  The workspace's
// first 16 bytes then hold {error, pad, total_words}: the stream is
// encoded_length(count, total_words) bytes unless error is set.
size_t encode_async_workspace(uint64_t count_cap) { return edits::work_bytes(edits::blocks_of((int64_t)count_cap)); }

uint64_t encoded_length(uint64_t count, uint64_t total_words) {
    return edits::layout_of(edits::blocks_of((int64_t)count)).payload + 4ull * total_words;
}

msz_status encode_async(const float *d_fhat, const float *d_g, uint32_t n, const uint32_t *d_idx,
                        const unsigned long long *d_count, uint64_t count_cap, uint8_t *d_stream, size_t capacity,
                        void *d_ws, const DeviceInfo &dev, cudaStream_t s) {
    const uint64_t nb = edits::blocks_of((int64_t)count_cap);
    const edits::Work w = edits::work_of(d_ws, nb);
    if (cudaMemsetAsync(w.ctrl, 0, sizeof(edits::Ctrl), s) != cudaSuccess) return MSZ_ERR_CUDA;
    const int grid = edits::grid_for(dev, nb);
    edits::k_widths<<<grid, edits::kWarps * 32, 0, s>>>(d_fhat, d_g, n, d_idx, d_count, count_cap, w.words, w.wd,
                                                        w.wm, w.ctrl);
    edits::k_scan<<<1, edits::kScanThreads, 0, s>>>(w.words, d_count, count_cap, w.start, w.ctrl);
    edits::k_pack<<<grid, edits::kWarps * 32, 0, s>>>(d_fhat, d_g, d_idx, d_count, count_cap, w.start, w.wd, w.wm,
                                                      d_stream, capacity, w.ctrl);
    return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

namespace edits {
// The stream into host memory the device addresses (stream_out_async): a
// grid-stride copy, 16 bytes a thread where both ends are 16-byte aligned.
__global__ void k_stream_out(const uint8_t *src, const Ctrl *ctrl, const unsigned long long *d_count,
                             uint64_t count_cap, uint8_t *dst, uint64_t capacity) {
    const uint64_t count = edit_count(d_count, count_cap);
    const uint64_t len = layout_of(blocks_of((int64_t)count)).payload + 4ull * ctrl->total_words;
    if (ctrl->error || len > capacity) return;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
    const bool vec = (((uintptr_t)src | (uintptr_t)dst) & 15u) == 0;
    const uint64_t nv = vec ? len / 16 : 0;
    for (uint64_t i = tid; i < nv; i += stride)
        reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
    for (uint64_t i = 16 * nv + tid; i < len; i += stride) dst[i] = src[i];
}
}  // namespace edits

msz_status stream_out_async(const uint8_t *d_stream, const void *d_ws, const unsigned long long *d_count,
                            uint64_t count_cap, uint8_t *h_dst, size_t capacity, cudaStream_t s) {
    const edits::Work w = edits::work_of(const_cast<void *>(d_ws), edits::blocks_of((int64_t)count_cap));
    edits::k_stream_out<<<64, 256, 0, s>>>(d_stream, w.ctrl, d_count, count_cap, h_dst, (uint64_t)capacity);
    return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

}  // namespace msz

using namespace msz;

extern "C" size_t msz_edits_encoded_bound(int64_t count) {
    if (count < 0) return 0;
    const uint64_t nb = edits::blocks_of(count);
    return (size_t)(edits::layout_of(nb).payload + 8ull * (uint64_t)count);
}

extern "C" size_t msz_edits_workspace_size(int64_t count) {
    if (count < 0) return 0;
    return edits::work_bytes(edits::blocks_of(count));
}

extern "C" msz_status msz_edits_encode(const float *d_fhat, const float *d_g, int64_t n, const uint32_t *d_idx,
                                       int64_t count, uint8_t *d_stream, size_t capacity, size_t *h_bytes,
                                       void *d_workspace, size_t workspace_bytes, msz_stream_t stream) {
    if (!d_fhat || !d_g || !d_stream || !h_bytes || n < 0 || n > MSZ_MAX_VERTICES || count < 0 || count > n)
        return MSZ_ERR_INVALID_ARG;
    if (count > 0 && !d_idx) return MSZ_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_stream) % 4 != 0) return MSZ_ERR_INVALID_ARG;
    const uint64_t nb = edits::blocks_of(count);
    if (!d_workspace || workspace_bytes < edits::work_bytes(nb)) return MSZ_ERR_WORKSPACE;
    DeviceInfo dev;
    msz_status st = current_device(dev);
    if (st != MSZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const edits::Work w = edits::work_of(d_workspace, nb);
    const edits::Layout L = edits::layout_of(nb);
    if (cudaMemsetAsync(w.ctrl, 0, sizeof(edits::Ctrl), s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (nb > 0) {
        edits::k_widths<<<edits::grid_for(dev, nb), edits::kWarps * 32, 0, s>>>(
            d_fhat, d_g, (uint32_t)n, d_idx, nullptr, (uint64_t)count, w.words, w.wd, w.wm, w.ctrl);
        edits::k_scan<<<1, edits::kScanThreads, 0, s>>>(w.words, nullptr, (uint64_t)count, w.start, w.ctrl);
    }
    edits::Ctrl hc;
    if (cudaMemcpyAsync(&hc, w.ctrl, sizeof hc, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (hc.error) return MSZ_ERR_INVALID_ARG;
    const uint64_t bytes = L.payload + 4ull * hc.total_words;
    *h_bytes = (size_t)bytes;
    if (bytes > capacity) return MSZ_ERR_CAPACITY;
    edits::k_pack<<<edits::grid_for(dev, nb), edits::kWarps * 32, 0, s>>>(
        d_fhat, d_g, d_idx, nullptr, (uint64_t)count, w.start, w.wd, w.wm, d_stream, capacity, w.ctrl);
    if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(s));
}

extern "C" msz_status msz_edits_decode(const uint8_t *d_stream, size_t bytes, float *d_field, int64_t n,
                                       int64_t *h_count, void *d_workspace, size_t workspace_bytes,
                                       msz_stream_t stream) {
    if (!d_stream || !d_field || !h_count || n < 0 || n > MSZ_MAX_VERTICES || bytes < 16) return MSZ_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_stream) % 4 != 0) return MSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t head[4];
    if (cudaMemcpyAsync(head, d_stream, sizeof head, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    const uint64_t count = (uint64_t)head[2] | ((uint64_t)head[3] << 32);
    if (head[0] != MSZ_EDIT_MAGIC || head[1] != edits::B || count > (uint64_t)n) return MSZ_ERR_INVALID_ARG;
    const uint64_t nb = edits::blocks_of((int64_t)count);
    const edits::Layout L = edits::layout_of(nb);
    if (bytes < L.payload) return MSZ_ERR_INVALID_ARG;
    *h_count = (int64_t)count;
    if (count == 0) return MSZ_OK;
    if (!d_workspace || workspace_bytes < edits::work_bytes(nb)) return MSZ_ERR_WORKSPACE;
    DeviceInfo dev;
    msz_status st = current_device(dev);
    if (st != MSZ_OK) return st;
    const edits::Work w = edits::work_of(d_workspace, nb);
    if (cudaMemsetAsync(w.ctrl, 0, sizeof(edits::Ctrl), s) != cudaSuccess) return MSZ_ERR_CUDA;
    const int grid = edits::grid_for(dev, nb);
    edits::k_check<<<grid, edits::kWarps * 32, 0, s>>>(d_stream, (bytes - L.payload) / 4, count, (uint32_t)n, w.words,
                                                      w.ctrl);
    edits::k_order<<<grid, 256, 0, s>>>(d_stream, count, w.words, w.ctrl);
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, &w.ctrl->error, sizeof err, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (err) return MSZ_ERR_INVALID_ARG;
    edits::k_apply<<<grid, edits::kWarps * 32, 0, s>>>(d_stream, count, d_field);
    if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(s));
}
