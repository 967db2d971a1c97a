// msz_learned.cu -- the learned initial-edit proposal (a small 3D conv net
// that predicts, per vertex, how many value edits the correction will apply
// to it), trained and run on sm_103a.  The exact correction loop always
// finishes from the proposed start, so results stay exact.
//
//   features   16 channels per vertex (BF16): (fhat - f)/xi, the forward
//              differences of f and of fhat / (4 xi) (clamped to +-1), the
//              extremum flags of f and fhat, the first sweep's mismatch and
//              target flags, and the fraction of tied neighbours in f;
//   conv3d     4 layers of 3x3x3 cross-correlations with zero padding,
//              16->32->32->32->16 channels, ReLU between, as implicit
//              GEMMs on tcgen05 (BF16 operands in shared memory, FP32
//              accumulators in TMEM);
//   head       16 logits per vertex, one per class k = 0..15: the number of
//              HALVE edits the plain loop applies to the vertex (15: fifteen
//              or more); the proposed start g0 is fhat edited k times by the
//              same rule, so a right class reproduces the plain loop's value
//              bit for bit;
//   training   softmax cross-entropy against the plain loop's classes;
//              backward-data through the same tcgen05 kernel with mirrored
//              weights, weight gradients on CUDA cores (FP32), Adam in FP32.
//
// Conv kernel layout.  Activations are channels-last BF16 ([z][y][x][C]).  A
// tile is 128 consecutive x of 2 rows (y) of 2 planes (z); its input is the
// 4 x 4 (y, z) lines of 130 voxels around it, staged by one TMA box per
// 8-channel slab ([z][y][x][8 channels], 16 bytes per voxel).  In that
// canonical no-swizzle K-major layout the voxels of a slab are uniformly 16
// bytes apart, so the operand of every one of the 27 kernel offsets is the
// same staged data with a shifted descriptor start: nothing is loaded twice.
// A stage holds one K = 16 slab pair; two stages in a ring let the TMA load
// of the next pair run under the MMAs of the current one.  One thread issues
// the MMAs (M = 128 voxels, N = output channels, K = 16 channels), four warps
// drain the double-buffered TMEM accumulators.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_workspace.h"

namespace msz {
namespace learned {

constexpr int kConvThreads = 192;  // warp 0: TMA producer, warp 1: MMA issuer, warps 2..5: epilogue
constexpr int kRows = 130;         // staged voxels of a line (x0-1 .. x0+128)
constexpr int kLines = 16;         // staged (y, z) lines: 4 x 4 around a 2 x 2 block of output rows
constexpr int kLineBytes = kRows * 16;            // one line of one 8-channel slab
constexpr int kSlabBytes = kLines * kLineBytes;   // one slab of a tile (one TMA box)
constexpr int kStageBytes = 2 * kSlabBytes;       // a K = 16 slab pair
constexpr int kStages = 2;
constexpr int kTmemCols = 256;
constexpr uint64_t kWaitNs = 2000000000ull;

enum { MODE_RELU = 0, MODE_HEAD = 1, MODE_DGRAD = 2, MODE_RAW = 3 };
constexpr int kClasses = 16;       // edit-count classes 0..15 of the head
constexpr uint32_t kErrWait = 1u;  // a bounded wait ran out

struct ConvParams {
    uint32_t nx, ny, nz;
    uint32_t tiles_x, tiles_y, tiles;
    const uint16_t *wimg;  // BF16 weight image (canonical layout)
    const float *bias;     // COUT entries (MODE_RELU, MODE_HEAD, MODE_RAW: may be null)
    uint16_t *out_bf16;    // MODE_RELU / MODE_DGRAD: channels-last output
    float *out_f32;        // MODE_RAW: channels-last f32; MODE_HEAD: the class used
    const uint16_t *mask;  // MODE_DGRAD: activation whose positive entries pass the gradient
    const float *f;        // MODE_HEAD
    const float *fhat;
    float *g0;
    float xi;
    int shift;             // MODE_HEAD: added to every nonzero class (then clamped to 1..15)
    uint32_t *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    // start address, leading (K-direction) and stride (M/N-direction) byte
    // offsets of 8 x 16-byte core matrices, all in 16-byte units; version 1
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// Bounded wait for the phase of the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, uint32_t *err) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 255u) {
            const uint64_t now = global_ns();
            if (!t0) t0 = now;
            else if (now - t0 > kWaitNs) {
                atomicOr(err, kErrWait);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

template <int N>
__device__ __forceinline__ void tmem_load(uint32_t taddr, uint32_t (&r)[N]);
template <>
__device__ __forceinline__ void tmem_load<32>(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
template <>
__device__ __forceinline__ void tmem_load<16>(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float bf16_to_f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t f_to_bf16(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Weight image: one strip per (slab pair sp, dx, dz) of 2 K halves x 5 dy
// blocks x COUT output channels x 8 input channels (BF16, 16 bytes a row):
// block b holds the weights of offset dy = 2 - b, blocks 0 and 4 (dy = +-2)
// are zero.  An MMA takes two neighbouring blocks as one B operand of N =
// 2 COUT rows, so that one staged input line (the A operand) feeds both output
// rows of a plane pair: block 3 - dyl for the tile's row y0 (dy = dyl - 1)
// and the next for row y0 + 1 (dy = dyl - 2); a zero block stands for the
// offset that reaches past the kernel.
constexpr int kDyBlocks = 5;
__host__ __device__ constexpr int img_strip_bytes(int cout) { return 2 * kDyBlocks * cout * 16; }
__host__ __device__ constexpr int img_bytes(int cin, int cout) { return (cin / 16) * 9 * img_strip_bytes(cout); }

template <int CIN, int COUT>
struct ConvShape {
    static constexpr int KG = CIN / 8;                        // 8-channel slabs per voxel
    static constexpr int NP = KG / 2;                         // K = 16 slab pairs per tile (1 or 2)
    static constexpr int WBYTES = img_bytes(CIN, COUT);       // weight image
    static constexpr int WAL = (WBYTES + 1023) / 1024 * 1024;
    static constexpr int SMEM = WAL + kStages * kStageBytes;
    // kind::f16: FP32 accumulator (bit 4), BF16 A and B (bits 7, 10), K-major,
    // N >> 3 at bit 17, M >> 4 at bit 24 (M = 128); N = 2 COUT (two output rows)
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * COUT) >> 3) << 17) |
                                      ((uint32_t)(128 >> 4) << 24);
    static_assert(SMEM + 1024 <= 227 * 1024, "weight image and stages must fit one block's shared memory");
};

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(kConvThreads, 1)
    k_conv(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ ConvParams P) {
    using S = ConvShape<CIN, COUT>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kStages], bar_free[kStages], bar_done[2], bar_acc[2], bar_end;
    __shared__ uint32_t tmem_slot;
    // the launch asks for S::SMEM + 1024 bytes: align the operand area here
    // rather than rely on the placement of the dynamic window
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *wsm = smem;
    unsigned char *stg = smem + S::WAL;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;

    for (uint32_t i = tid; i < (uint32_t)S::WBYTES / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(wsm)[i] = reinterpret_cast<const uint4 *>(P.wimg)[i];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            mbar_init(smem_u32(&bar_full[q]), 1);
            mbar_init(smem_u32(&bar_free[q]), 1);
        }
        mbar_init(smem_u32(&bar_done[0]), 1);
        mbar_init(smem_u32(&bar_done[1]), 1);
        mbar_init(smem_u32(&bar_acc[0]), 4);
        mbar_init(smem_u32(&bar_acc[1]), 4);
        mbar_init(smem_u32(&bar_end), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t tiles_xy = P.tiles_x * P.tiles_y;

    if (warp == 0) {
        if (lane == 0) {  // ---- TMA producer: one stage = one slab pair of one tile
            uint32_t q = 0;
            bool ok = true;
            for (uint32_t t = blockIdx.x; ok && t < P.tiles; t += gridDim.x) {
                const int x0 = (int)(t % P.tiles_x) * 128, y0 = (int)((t / P.tiles_x) % P.tiles_y) * 2,
                          z0 = (int)(t / tiles_xy) * 2;
                for (int sp = 0; sp < S::NP; ++sp, ++q) {
                    const uint32_t st = q % kStages, use = q / kStages;
                    if (use > 0 && !mbar_wait(smem_u32(&bar_free[st]), (use - 1) & 1u, P.err)) {
                        ok = false;
                        break;
                    }
                    unsigned char *dst = stg + st * kStageBytes;
                    mbar_expect_tx(smem_u32(&bar_full[st]), kStageBytes);
                    tma_load_4d(smem_u32(dst), &tmx, sp * 16, x0 - 1, y0 - 1, z0 - 1, smem_u32(&bar_full[st]));
                    tma_load_4d(smem_u32(dst + kSlabBytes), &tmx, sp * 16 + 8, x0 - 1, y0 - 1, z0 - 1,
                                smem_u32(&bar_full[st]));
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer
            uint32_t it = 0, q = 0;
            const uint32_t sstg = smem_u32(stg), swsm = smem_u32(wsm);
            bool issued = false, ok = true;
            for (uint32_t t = blockIdx.x; ok && t < P.tiles; t += gridDim.x, ++it) {
                const uint32_t buf = it & 1u;
                if (it >= 2 && !mbar_wait(smem_u32(&bar_acc[buf]), ((it >> 1) - 1) & 1u, P.err)) break;
                for (int sp = 0; sp < S::NP; ++sp, ++q) {
                    const uint32_t st = q % kStages, use = q / kStages;
                    if (!mbar_wait(smem_u32(&bar_full[st]), use & 1u, P.err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // descriptors of the first line of this stage and of this slab
                    // pair's first strip; every MMA adds a compile-time start offset
                    // (in 16-byte units: the start field stays below 2^14 for
                    // addresses under 256 KB)
                    const uint64_t a0 = sdesc(sstg + st * kStageBytes, kSlabBytes, 128);
                    const uint64_t b0 = sdesc(swsm + sp * 9 * img_strip_bytes(COUT), kDyBlocks * COUT * 16, 128);
                    const uint32_t first = sp > 0 ? 1u : 0u;
                    // plane rz of the tile: accumulators r = 2 rz (row y0) and
                    // 2 rz + 1 (row y0 + 1) side by side, N = 2 COUT; input line
                    // (dyl, dzl) of the staged 4 x 4 for kernel offsets (dx, dz)
#pragma unroll
                    for (int rz = 0; rz < 2; ++rz) {
#pragma unroll
                        for (int i = 0; i < 36; ++i) {
                            const int dx = i % 3 - 1, dyl = (i / 3) % 4, dz = i / 12 - 1;
                            const int L = (rz + 1 + dz) * 4 + dyl;
                            const uint64_t a = a0 + (uint64_t)((L * kLineBytes + (1 + dx) * 16) >> 4);
                            const int strip = (dx + 1) * 3 + (dz + 1);
                            const uint64_t b =
                                b0 + (uint64_t)((strip * img_strip_bytes(COUT) + (3 - dyl) * COUT * 16) >> 4);
                            mma_bf16(tmem + (buf * 4 + 2 * rz) * COUT, a, b, S::IDESC, i > 0 ? 1u : first);
                        }
                    }
                    mma_commit(smem_u32(&bar_free[st]));
                    issued = true;
                }
                if (!ok) break;
                mma_commit(smem_u32(&bar_done[buf]));
            }
            // every MMA this block issued completes before TMEM is released
            if (issued) {
                mma_commit(smem_u32(&bar_end));
                mbar_wait(smem_u32(&bar_end), 0, P.err);
            }
        }
    } else {  // ---- epilogue: warps 2..5 own TMEM lanes 32*(warp % 4) ..
        const uint32_t q = warp & 3u;
        const uint32_t i = 32u * q + lane;  // voxel of the 128-row tile
        uint32_t it = 0;
        for (uint32_t t = blockIdx.x; t < P.tiles; t += gridDim.x, ++it) {
            const uint32_t buf = it & 1u;
            if (!mbar_wait(smem_u32(&bar_done[buf]), (it >> 1) & 1u, P.err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t x0 = (t % P.tiles_x) * 128, y0 = ((t / P.tiles_x) % P.tiles_y) * 2,
                           z0 = (t / tiles_xy) * 2;
            for (int r = 0; r < 4; ++r) {
                uint32_t acc[COUT];
                tmem_load<COUT>(tmem + ((32u * q) << 16) + (buf * 4 + r) * COUT, acc);
                const uint32_t x = x0 + i, y = y0 + (r & 1), z = z0 + (r >> 1);
                if (x >= P.nx || y >= P.ny || z >= P.nz) continue;
                const size_t v = ((size_t)z * P.ny + y) * P.nx + x;
                if (MODE == MODE_RELU || MODE == MODE_DGRAD) {
                    uint32_t packed[COUT / 2];
#pragma unroll
                    for (int c = 0; c < COUT; c += 2) {
                        float a0 = __uint_as_float(acc[c]), a1 = __uint_as_float(acc[c + 1]);
                        if (MODE == MODE_RELU) {
                            a0 = fmaxf(a0 + P.bias[c], 0.0f);
                            a1 = fmaxf(a1 + P.bias[c + 1], 0.0f);
                        } else {
                            const uint32_t m = reinterpret_cast<const uint32_t *>(P.mask + v * COUT)[c / 2];
                            if (!(bf16_to_f((uint16_t)(m & 0xffffu)) > 0.0f)) a0 = 0.0f;
                            if (!(bf16_to_f((uint16_t)(m >> 16)) > 0.0f)) a1 = 0.0f;
                        }
                        packed[c / 2] = (uint32_t)f_to_bf16(a0) | ((uint32_t)f_to_bf16(a1) << 16);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(P.out_bf16 + v * COUT);
#pragma unroll
                    for (int c = 0; c < COUT / 8; ++c)
                        dst[c] = make_uint4(packed[4 * c], packed[4 * c + 1], packed[4 * c + 2], packed[4 * c + 3]);
                } else if (MODE == MODE_HEAD) {
                    // class = argmax of the logits (the lowest class on ties)
                    int k = 0;
                    float best = __uint_as_float(acc[0]) + P.bias[0];
#pragma unroll
                    for (int c = 1; c < COUT; ++c) {
                        const float zc = __uint_as_float(acc[c]) + P.bias[c];
                        if (zc > best) {
                            best = zc;
                            k = c;
                        }
                    }
                    if (k > 0) k = min(max(k + P.shift, 1), kClasses - 1);
                    if (P.out_f32) P.out_f32[v] = (float)k;
                    if (P.g0) {
                        const float L = floor_bound(P.f[v], P.xi);
                        float g = P.fhat[v];
                        for (int e = 0; e < k; ++e) {
                            float h;
                            if (!edit_value(g, L, MSZ_RULE_HALVE, h)) break;
                            g = h;
                        }
                        P.g0[v] = g;
                    }
                } else {
                    float4 *dst = reinterpret_cast<float4 *>(P.out_f32 + v * COUT);
#pragma unroll
                    for (int c = 0; c < COUT; c += 4) {
                        float4 o4;
                        o4.x = __uint_as_float(acc[c]) + (P.bias ? P.bias[c] : 0.0f);
                        o4.y = __uint_as_float(acc[c + 1]) + (P.bias ? P.bias[c + 1] : 0.0f);
                        o4.z = __uint_as_float(acc[c + 2]) + (P.bias ? P.bias[c + 2] : 0.0f);
                        o4.w = __uint_as_float(acc[c + 3]) + (P.bias ? P.bias[c + 3] : 0.0f);
                        dst[c / 4] = o4;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_acc[buf]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ------------------------------------------------------------- features
// 16 channels per vertex (BF16).  codes_f / codes_h: the steepest-neighbour
// codes of f and fhat (3D slots).
//   0      (fhat - f) / xi                    clamped to [-1, 1]
//   1..3   forward differences of f / (4 xi)  along x, y, z, clamped to [-1, 1]
//   4, 5   f has a maximum / a minimum here
//   6, 7   fhat's ascending / descending code differs from f's
//   8, 9   the vertex is the target of an ascending / descending mismatch in
//          the first sweep (the correction's target rule applied to g = fhat)
//   10, 11 fhat has a maximum / a minimum here
//   12..14 forward differences of fhat / (4 xi), clamped to [-1, 1]
//   15     the fraction of the 14 neighbours whose f value equals this one's
__global__ void __launch_bounds__(256) k_features(const float *f, const float *fhat, const uint8_t *codes_f,
                                                 const uint8_t *codes_h, const GridDev G, float xi, uint16_t *out) {
    const size_t n = (size_t)G.n;
    const uint32_t nx = G.nx, ny = G.ny, nz = G.nz;
    const float inv = xi > 0.0f ? 1.0f / xi : 0.0f;
    const float inv4 = xi > 0.0f ? 0.25f / xi : 0.0f;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        uint32_t x, y, z;
        coords_of(G, (uint32_t)v, x, y, z);
        const float fv = f[v], hv = fhat[v];
        float ch[16];
        ch[0] = fminf(fmaxf((hv - fv) * inv, -1.0f), 1.0f);
        ch[1] = x + 1 < nx ? fminf(fmaxf((f[v + 1] - fv) * inv4, -1.0f), 1.0f) : 0.0f;
        ch[2] = y + 1 < ny ? fminf(fmaxf((f[v + nx] - fv) * inv4, -1.0f), 1.0f) : 0.0f;
        ch[3] = z + 1 < nz ? fminf(fmaxf((f[v + (size_t)G.nxy] - fv) * inv4, -1.0f), 1.0f) : 0.0f;
        const uint32_t cf = codes_f[v], cg = codes_h[v];
        ch[4] = (cf & 15u) == kSelf ? 1.0f : 0.0f;
        ch[5] = (cf >> 4) == kSelf ? 1.0f : 0.0f;
        ch[6] = (cf & 15u) != (cg & 15u) ? 1.0f : 0.0f;
        ch[7] = (cf >> 4) != (cg >> 4) ? 1.0f : 0.0f;
        // a mismatched vertex j targets itself (ascending: when fhat makes it a
        // maximum; descending: when f makes it a minimum), else its steepest
        // neighbour (ascending: in fhat; descending: in f)
        bool at = (cf & 15u) != (cg & 15u) && (cg & 15u) == kSelf;
        bool dt = (cf >> 4) != (cg >> 4) && (cf >> 4) == kSelf;
        int ties = 0;
        for (int sl = 0; sl < 14; ++sl) {
            if (!slot_in_domain(G, sl, x, y, z)) continue;
            const size_t j = (size_t)((int64_t)v + G.off[sl]);
            const uint32_t back = (uint32_t)(sl < 7 ? sl + 7 : sl - 7);  // slot of v seen from j
            const uint32_t jf = codes_f[j], jg = codes_h[j];
            at = at || ((jf & 15u) != (jg & 15u) && (jg & 15u) == back);
            dt = dt || ((jf >> 4) != (jg >> 4) && (jf >> 4) == back);
            ties += f[j] == fv ? 1 : 0;
        }
        ch[8] = at ? 1.0f : 0.0f;
        ch[9] = dt ? 1.0f : 0.0f;
        ch[10] = (cg & 15u) == kSelf ? 1.0f : 0.0f;
        ch[11] = (cg >> 4) == kSelf ? 1.0f : 0.0f;
        ch[12] = x + 1 < nx ? fminf(fmaxf((fhat[v + 1] - hv) * inv4, -1.0f), 1.0f) : 0.0f;
        ch[13] = y + 1 < ny ? fminf(fmaxf((fhat[v + nx] - hv) * inv4, -1.0f), 1.0f) : 0.0f;
        ch[14] = z + 1 < nz ? fminf(fmaxf((fhat[v + (size_t)G.nxy] - hv) * inv4, -1.0f), 1.0f) : 0.0f;
        ch[15] = (float)ties / 14.0f;
        uint32_t p[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) p[c] = (uint32_t)f_to_bf16(ch[2 * c]) | ((uint32_t)f_to_bf16(ch[2 * c + 1]) << 16);
        uint4 *dst = reinterpret_cast<uint4 *>(out + v * 16);
        dst[0] = make_uint4(p[0], p[1], p[2], p[3]);
        dst[1] = make_uint4(p[4], p[5], p[6], p[7]);
    }
}

// ------------------------------------------------------------ weights
// FP32 weights w[o][cout][cin] (cout < cout_real, cin < cin_real) -> BF16 image
// of a conv with CIN >= cin_real input and COUT >= cout_real output channels
// (zero padding), in strips (see img_strip_bytes): byte offset
// (((sp * 3 + dx + 1) * 3 + dz + 1) * 2 + h) * 5 * COUT * 16 + (b * COUT + n) * 16
// + 2 k8 holds input channel 16 sp + 8 h + k8 of output channel n at offset
// (dx, dy = 2 - b, dz); offset o = (dz + 1) * 9 + (dy + 1) * 3 + dx + 1.
// mirror: the backward-data image, i.e. the conv of the gradient with
// w[26 - o] and input / output channels swapped.
__global__ void k_weight_image(const float *w, int cout_real, int cin_real, int CIN, int COUT, int mirror,
                               uint16_t *img) {
    const int NP = CIN / 16;
    const int total = NP * 9 * 2 * kDyBlocks * COUT * 8;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int k8 = e & 7, n = (e >> 3) % COUT, bl = (e >> 3) / COUT % kDyBlocks;
        const int h = (e >> 3) / COUT / kDyBlocks % 2, sdz = (e >> 3) / COUT / kDyBlocks / 2;
        const int dz = sdz % 3 - 1, dx = sdz / 3 % 3 - 1, sp = sdz / 9;
        const int dy = 2 - bl;
        float v = 0.0f;
        if (dy >= -1 && dy <= 1) {
            const int o = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
            const int kin = sp * 16 + h * 8 + k8;  // input channel of this image's conv
            if (!mirror) {
                if (n < cout_real && kin < cin_real) v = w[((size_t)o * cout_real + n) * cin_real + kin];
            } else {
                // image conv: input = gradient channels (= forward cout), output = forward cin
                if (kin < cout_real && n < cin_real) v = w[((size_t)(26 - o) * cout_real + kin) * cin_real + n];
            }
        }
        img[e] = f_to_bf16(v);
    }
}

// --------------------------------------------------------- head / loss
// Softmax cross-entropy of the 16 head logits (the RAW head output, bias
// included) against the class k of each vertex: loss += logsumexp(z) - z_k
// (summed in double); the gradient with respect to the logits,
// scale * (softmax(z) - onehot(k)), is written as the BF16 input of the last
// layer's backward-data conv.
__global__ void k_head_grad(const float *z, const float *target, size_t n, float scale, uint16_t *dz16,
                            double *loss_sum) {
    double acc = 0.0;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        float zc[kClasses];
        const float4 *src = reinterpret_cast<const float4 *>(z + v * kClasses);
#pragma unroll
        for (int q = 0; q < kClasses / 4; ++q) {
            const float4 t4 = src[q];
            zc[4 * q] = t4.x;
            zc[4 * q + 1] = t4.y;
            zc[4 * q + 2] = t4.z;
            zc[4 * q + 3] = t4.w;
        }
        const int k = min(max((int)target[v], 0), kClasses - 1);
        float m = zc[0];
#pragma unroll
        for (int c = 1; c < kClasses; ++c) m = fmaxf(m, zc[c]);
        float sum = 0.0f, zk = 0.0f;
#pragma unroll
        for (int c = 0; c < kClasses; ++c) {
            zk = c == k ? zc[c] : zk;
            zc[c] = expf(zc[c] - m);
            sum += zc[c];
        }
        acc += (double)(m + logf(sum) - zk);
        const float inv = scale / sum;
        uint32_t p[kClasses / 2];
#pragma unroll
        for (int c = 0; c < kClasses; c += 2) {
            const float g0 = zc[c] * inv - (c == k ? scale : 0.0f);
            const float g1 = zc[c + 1] * inv - (c + 1 == k ? scale : 0.0f);
            p[c / 2] = (uint32_t)f_to_bf16(g0) | ((uint32_t)f_to_bf16(g1) << 16);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(dz16 + v * kClasses);
        dst[0] = make_uint4(p[0], p[1], p[2], p[3]);
        dst[1] = make_uint4(p[4], p[5], p[6], p[7]);
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(kFull, acc, d);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, acc);
}

// ------------------------------------------------------------- targets
// Training class of a vertex: how many HALVE edits take fhat to the corrected
// value g (g lies on that chain when g is the plain loop's result), capped at
// 15; 0 for an unedited vertex.
__global__ void k_target(const float *f, const float *fhat, const float *g, float xi, size_t n, float *t) {
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const float L = floor_bound(f[v], xi);
        const float gv = g[v];
        float h = fhat[v];
        int k = 0;
        while (k < kClasses - 1 && h > gv) {
            float nh;
            if (!edit_value(h, L, MSZ_RULE_HALVE, nh)) break;
            h = nh;
            ++k;
        }
        t[v] = (float)k;
    }
}

// ------------------------------------------------------ weight gradient
// dw[o][cout][cin] += sum_v dz[v][cout] * x[v + d_o][cin] and db[cout] +=
// sum_v dz[v][cout] on CUDA cores (FP32).  A block takes rows of 128 voxels
// (x) at one (y, z), stages dz and the 9 (y, z) neighbour lines of x in shared
// memory, and each thread accumulates 27 offsets x 4 input channels of one
// output channel in registers.  Each thread then writes its partial sums to
// its own slot of the workspace (no atomics), and k_wgrad_reduce adds the
// slots in a fixed order: the gradient is the same bit for bit on every run.
// CIN in {16, 32} (x channels), COUT in {16, 32} (dz channels), cin_real /
// cout_real the channels that carry weights.
constexpr int kWgradBlocks = 304;  // fixed, so the summation order is too

template <int CIN, int COUT>
struct WgradShape {
    static constexpr int PAIRS = COUT * (CIN / 4);  // (cout, cin group) pairs
    static constexpr int NREP = 256 / PAIRS;        // threads per pair (each a share of the voxels)
    static constexpr int SLOT = 27 * COUT * CIN + COUT;  // floats of one partial: weights, then biases
    static constexpr size_t BYTES = (size_t)kWgradBlocks * NREP * SLOT * sizeof(float);
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_wgrad(const uint16_t *x, const uint16_t *dz, uint32_t nx, uint32_t ny,
                                               uint32_t nz, float *part) {
    constexpr int CG = CIN / 4;              // groups of 4 input channels
    constexpr int PAIRS = COUT * CG;         // (cout, cin group) pairs
    extern __shared__ __align__(16) unsigned char wsmem[];
    auto sx = reinterpret_cast<uint16_t (*)[130][CIN]>(wsmem);                     // [9][130][CIN]
    auto sz = reinterpret_cast<uint16_t (*)[COUT]>(wsmem + 9 * 130 * CIN * 2);      // [128][COUT]
    const uint32_t tid = threadIdx.x;
    const int pair = (int)tid % PAIRS, rep = (int)tid / PAIRS;  // threads beyond PAIRS split the voxels
    const int nrep = 256 / PAIRS;
    const int co = pair / CG, cg = pair % CG;
    float acc[27][4];
#pragma unroll
    for (int o = 0; o < 27; ++o)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[o][c] = 0.0f;
    float bacc = 0.0f;
    const uint32_t tx = (nx + 127) / 128, rows = tx * ny * nz;
    for (uint32_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const uint32_t x0 = (row % tx) * 128, y = (row / tx) % ny, z = row / (tx * ny);
        __syncthreads();
        for (uint32_t e = tid; e < 9u * 130u * (CIN / 8); e += blockDim.x) {
            const uint32_t c8 = e % (CIN / 8), xi_ = (e / (CIN / 8)) % 130, l = e / (CIN / 8) / 130;
            const int xx = (int)x0 - 1 + (int)xi_, yy = (int)y + (int)(l % 3) - 1, zz = (int)z + (int)(l / 3) - 1;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (xx >= 0 && xx < (int)nx && yy >= 0 && yy < (int)ny && zz >= 0 && zz < (int)nz)
                val = reinterpret_cast<const uint4 *>(x + (((size_t)zz * ny + yy) * nx + xx) * CIN)[c8];
            reinterpret_cast<uint4 *>(&sx[l][xi_][0])[c8] = val;
        }
        for (uint32_t e = tid; e < 128u * (COUT / 8); e += blockDim.x) {
            const uint32_t c8 = e % (COUT / 8), xi_ = e / (COUT / 8);
            uint4 val = make_uint4(0, 0, 0, 0);
            if (x0 + xi_ < nx)
                val = reinterpret_cast<const uint4 *>(dz + (((size_t)z * ny + y) * nx + x0 + xi_) * COUT)[c8];
            reinterpret_cast<uint4 *>(&sz[xi_][0])[c8] = val;
        }
        __syncthreads();
        for (int i = rep; i < 128; i += nrep) {
            const float d = bf16_to_f(sz[i][co]);
            if (d == 0.0f) continue;
            bacc += d;
#pragma unroll
            for (int o = 0; o < 27; ++o) {
                const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dzz = o / 9 - 1;
                const int l = (dzz + 1) * 3 + (dy + 1);
                const uint2 xv = *reinterpret_cast<const uint2 *>(&sx[l][i + 1 + dx][cg * 4]);
                acc[o][0] = fmaf(d, bf16_to_f((uint16_t)(xv.x & 0xffffu)), acc[o][0]);
                acc[o][1] = fmaf(d, bf16_to_f((uint16_t)(xv.x >> 16)), acc[o][1]);
                acc[o][2] = fmaf(d, bf16_to_f((uint16_t)(xv.y & 0xffffu)), acc[o][2]);
                acc[o][3] = fmaf(d, bf16_to_f((uint16_t)(xv.y >> 16)), acc[o][3]);
            }
        }
    }
    using S = WgradShape<CIN, COUT>;
    float *slot = part + ((size_t)blockIdx.x * S::NREP + rep) * S::SLOT;
#pragma unroll
    for (int o = 0; o < 27; ++o)
        *reinterpret_cast<float4 *>(&slot[((size_t)o * COUT + co) * CIN + cg * 4]) =
            make_float4(acc[o][0], acc[o][1], acc[o][2], acc[o][3]);
    if (cg == 0) slot[27 * COUT * CIN + co] = bacc;
}

// dw[o][co][ci] (real channel counts) += the partials of every block and
// share, added in slot order; db likewise.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_wgrad_reduce(const float *part, int cin_real, int cout_real, float *dw,
                                                      float *db) {
    using S = WgradShape<CIN, COUT>;
    const int nw = 27 * cout_real * cin_real, total = nw + cout_real;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x) {
        int src;
        if (j < nw) {
            const int o = j / (cout_real * cin_real), co = (j / cin_real) % cout_real, ci = j % cin_real;
            src = (o * COUT + co) * CIN + ci;
        } else {
            src = 27 * COUT * CIN + (j - nw);
        }
        float sum = 0.0f;
        for (int p = 0; p < kWgradBlocks * S::NREP; ++p) sum += part[(size_t)p * S::SLOT + src];
        if (j < nw) dw[j] += sum;
        else db[j - nw] += sum;
    }
}

// ---------------------------------------------------------------- Adam
__global__ void k_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ----------------------------------------------------------------- host
std::mutex g_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

msz_status encoder(PFN_cuTensorMapEncodeTiled_v12000 &fn) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_encode) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return MSZ_ERR_CUDA;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    fn = g_encode;
    return MSZ_OK;
}

// Tensor map of a channels-last BF16 activation [nz][ny][nx][C]: boxes of 8
// channels x 130 x 4 x 4 voxels (one slab of a tile's 16 lines); out-of-grid
// voxels read as zero.
msz_status act_map(const uint16_t *x, int C, uint32_t nx, uint32_t ny, uint32_t nz, CUtensorMap &map) {
    PFN_cuTensorMapEncodeTiled_v12000 enc;
    msz_status st = encoder(enc);
    if (st != MSZ_OK) return st;
    if (((uintptr_t)x & 15u) != 0) return MSZ_ERR_INVALID_ARG;
    cuuint64_t dims[4] = {(cuuint64_t)C, nx, ny, nz};
    cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * nx, (cuuint64_t)C * 2 * nx * ny};
    cuuint32_t box[4] = {8, (cuuint32_t)kRows, 4, 4};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)x, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return MSZ_ERR_CUDA;
    return MSZ_OK;
}

template <int CIN, int COUT, int MODE>
msz_status launch_conv(const uint16_t *x, const ConvParams &P0, int sms, cudaStream_t s) {
    using S = ConvShape<CIN, COUT>;
    static bool attr_set[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr_set[dev & 63]) {
        if (cudaFuncSetAttribute(k_conv<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 S::SMEM + 1024) != cudaSuccess)
            return MSZ_ERR_CUDA;
        attr_set[dev & 63] = true;
    }
    CUtensorMap map;
    msz_status st = act_map(x, CIN, P0.nx, P0.ny, P0.nz, map);
    if (st != MSZ_OK) return st;
    ConvParams P = P0;
    P.tiles_x = (P.nx + 127) / 128;
    P.tiles_y = (P.ny + 1) / 2;
    P.tiles = P.tiles_x * P.tiles_y * ((P.nz + 1) / 2);
    const int blocks = (int)(P.tiles < (uint32_t)sms ? P.tiles : (uint32_t)sms);
    k_conv<CIN, COUT, MODE><<<blocks, kConvThreads, S::SMEM + 1024, s>>>(map, P);
    return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

template <int CIN, int COUT>
msz_status launch_wgrad(const uint16_t *x, const uint16_t *dz, const GridDev &G, int cin_real, int cout_real,
                        float *dw, float *db, void *ws, size_t ws_bytes, cudaStream_t s) {
    if (!ws || ws_bytes < WgradShape<CIN, COUT>::BYTES || ((uintptr_t)ws & 15u)) return MSZ_ERR_WORKSPACE;
    const int smem = 9 * 130 * CIN * 2 + 128 * COUT * 2;
    // the attribute belongs to the current context: set it on every call
    if (cudaFuncSetAttribute(k_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return MSZ_ERR_CUDA;
    k_wgrad<CIN, COUT><<<kWgradBlocks, 256, smem, s>>>(x, dz, G.nx, G.ny, G.nz, (float *)ws);
    k_wgrad_reduce<CIN, COUT><<<64, 256, 0, s>>>((const float *)ws, cin_real, cout_real, dw, db);
    return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

}  // namespace learned
}  // namespace msz

using namespace msz;
using namespace msz::learned;

extern "C" msz_status msz_learned_features(const float *d_f, const float *d_fhat, float xi, msz_grid grid,
                                           const uint8_t *d_codes_f, const uint8_t *d_codes_fhat, uint16_t *d_x,
                                           msz_stream_t stream) {
    if (!d_f || !d_fhat || !d_codes_f || !d_codes_fhat || !d_x || !(xi >= 0.0f)) return MSZ_ERR_INVALID_ARG;
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    if (grid.ndim != 3 || ((uintptr_t)d_x & 15u)) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    k_features<<<dev.sms * 8, 256, 0, (cudaStream_t)stream>>>(d_f, d_fhat, d_codes_f, d_codes_fhat, G, xi, d_x);
    return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

extern "C" msz_status msz_learned_weight_image(const float *d_w, int32_t cout_real, int32_t cin_real, int32_t cin,
                                               int32_t cout, int32_t mirror, uint16_t *d_img, msz_stream_t stream) {
    if (!d_w || !d_img || cin % 16 || cout % 16 || cin < 16 || cout < 16 || cin > 32 || cout > 32 ||
        cout_real < 1 || cin_real < 1)
        return MSZ_ERR_INVALID_ARG;
    if (!mirror && (cout_real > cout || cin_real > cin)) return MSZ_ERR_INVALID_ARG;
    if (mirror && (cout_real > cin || cin_real > cout)) return MSZ_ERR_INVALID_ARG;
    k_weight_image<<<64, 256, 0, (cudaStream_t)stream>>>(d_w, cout_real, cin_real, cin, cout, mirror, d_img);
    return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

extern "C" size_t msz_learned_weight_image_size(int32_t cin, int32_t cout) {
    if (cin % 16 || cout % 16 || cin < 16 || cout < 16 || cin > 32 || cout > 32) return 0;
    return (size_t)img_bytes(cin, cout);
}

// Channel combinations each conv mode is built for.
static bool conv_supported(int mode, int cin, int cout) {
    switch (mode) {
        case MODE_RELU:
        case MODE_DGRAD: return (cin == 16 || cin == 32) && cout == 32;
        case MODE_HEAD: return cin == 32 && cout == 16;
        case MODE_RAW: return (cin == 16 && cout == 32) || (cin == 32 && (cout == 32 || cout == 16));
    }
    return false;
}

extern "C" msz_status msz_learned_conv(const uint16_t *d_x, int32_t cin, int32_t cout, int32_t mode, msz_grid grid,
                                       const uint16_t *d_img, const float *d_bias, uint16_t *d_out_bf16,
                                       float *d_out_f32, const uint16_t *d_mask, const float *d_f,
                                       const float *d_fhat, float xi, int32_t shift, float *d_g0,
                                       uint32_t *d_err, msz_stream_t stream) {
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    if (grid.ndim != 3 || !d_x || !d_img || !d_err || !conv_supported(mode, cin, cout)) return MSZ_ERR_INVALID_ARG;
    if (((uintptr_t)d_x & 15u) || ((uintptr_t)d_img & 15u)) return MSZ_ERR_INVALID_ARG;
    switch (mode) {
        case MODE_RELU:
            if (!d_bias || !d_out_bf16 || ((uintptr_t)d_out_bf16 & 15u)) return MSZ_ERR_INVALID_ARG;
            break;
        case MODE_DGRAD:
            if (!d_mask || !d_out_bf16 || ((uintptr_t)d_out_bf16 & 15u) || ((uintptr_t)d_mask & 3u))
                return MSZ_ERR_INVALID_ARG;
            break;
        case MODE_HEAD:
            if (!d_bias || (!d_out_f32 && !d_g0) || (d_g0 && (!d_f || !d_fhat || !(xi >= 0.0f))))
                return MSZ_ERR_INVALID_ARG;
            break;
        case MODE_RAW:
            if (!d_out_f32 || ((uintptr_t)d_out_f32 & 15u)) return MSZ_ERR_INVALID_ARG;
            break;
    }
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    ConvParams P{};
    P.nx = G.nx;
    P.ny = G.ny;
    P.nz = G.nz;
    P.wimg = d_img;
    P.bias = d_bias;
    P.out_bf16 = d_out_bf16;
    P.out_f32 = d_out_f32;
    P.mask = d_mask;
    P.f = d_f;
    P.fhat = d_fhat;
    P.g0 = d_g0;
    P.xi = xi;
    P.shift = shift;
    P.err = d_err;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = dev.sms;
    switch (mode) {
        case MODE_RELU:
            if (cin == 16) return launch_conv<16, 32, MODE_RELU>(d_x, P, sms, s);
            return launch_conv<32, 32, MODE_RELU>(d_x, P, sms, s);
        case MODE_DGRAD:
            if (cin == 16) return launch_conv<16, 32, MODE_DGRAD>(d_x, P, sms, s);
            return launch_conv<32, 32, MODE_DGRAD>(d_x, P, sms, s);
        case MODE_HEAD:
            return launch_conv<32, 16, MODE_HEAD>(d_x, P, sms, s);
        default:
            if (cin == 16) return launch_conv<16, 32, MODE_RAW>(d_x, P, sms, s);
            if (cout == 32) return launch_conv<32, 32, MODE_RAW>(d_x, P, sms, s);
            return launch_conv<32, 16, MODE_RAW>(d_x, P, sms, s);
    }
}

extern "C" msz_status msz_learned_head_grad(const float *d_z, const float *d_target, int64_t n, float scale,
                                            uint16_t *d_dz16, double *d_loss_sum, msz_stream_t stream) {
    if (!d_z || !d_target || !d_dz16 || !d_loss_sum || n < 0) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    msz_status st = current_device(dev);
    if (st != MSZ_OK) return st;
    k_head_grad<<<dev.sms * 8, 256, 0, (cudaStream_t)stream>>>(d_z, d_target, (size_t)n, scale, d_dz16, d_loss_sum);
    return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

extern "C" msz_status msz_learned_target(const float *d_f, const float *d_fhat, const float *d_g, float xi, int64_t n,
                                         float *d_target, msz_stream_t stream) {
    if (!d_f || !d_fhat || !d_g || !d_target || n < 0 || !(xi >= 0.0f)) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    msz_status st = current_device(dev);
    if (st != MSZ_OK) return st;
    if (n == 0) return MSZ_OK;
    k_target<<<dev.sms * 8, 256, 0, (cudaStream_t)stream>>>(d_f, d_fhat, d_g, xi, (size_t)n, d_target);
    return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

extern "C" size_t msz_learned_wgrad_workspace_size(int32_t cin, int32_t cout) {
    if (cin == 16 && cout == 32) return WgradShape<16, 32>::BYTES;
    if (cin == 32 && cout == 32) return WgradShape<32, 32>::BYTES;
    if (cin == 32 && cout == 16) return WgradShape<32, 16>::BYTES;
    return 0;
}

extern "C" msz_status msz_learned_wgrad(const uint16_t *d_x, int32_t cin, const uint16_t *d_dz, int32_t cout,
                                        msz_grid grid, int32_t cin_real, int32_t cout_real, float *d_dw, float *d_db,
                                        void *d_workspace, size_t workspace_bytes, msz_stream_t stream) {
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    if (grid.ndim != 3 || !d_x || !d_dz || !d_dw || !d_db) return MSZ_ERR_INVALID_ARG;
    const bool shape_ok = (cin == 16 && cout == 32) || (cin == 32 && (cout == 32 || cout == 16));
    if (!shape_ok || cin_real < 1 || cin_real > cin || cout_real < 1 || cout_real > cout) return MSZ_ERR_INVALID_ARG;
    if (((uintptr_t)d_x & 15u) || ((uintptr_t)d_dz & 15u)) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    void *w = d_workspace;
    const size_t wb = workspace_bytes;
    if (cin == 16) return launch_wgrad<16, 32>(d_x, d_dz, G, cin_real, cout_real, d_dw, d_db, w, wb, s);
    if (cout == 32) return launch_wgrad<32, 32>(d_x, d_dz, G, cin_real, cout_real, d_dw, d_db, w, wb, s);
    return launch_wgrad<32, 16>(d_x, d_dz, G, cin_real, cout_real, d_dw, d_db, w, wb, s);
}

extern "C" msz_status msz_learned_adam(float *d_p, const float *d_g, float *d_m, float *d_v, int64_t n, float lr,
                                       float beta1, float beta2, float eps, int64_t step, msz_stream_t stream) {
    if (!d_p || !d_g || !d_m || !d_v || n < 0 || step < 1) return MSZ_ERR_INVALID_ARG;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<256, 256, 0, (cudaStream_t)stream>>>(d_p, d_g, d_m, d_v, (size_t)n, lr, beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}
