// msz_correct.cu -- steepest-neighbour codes and the correction loop of pMSz
// (arXiv 2601.01787) on sm_103a.
//
// msz_correct is one cooperative persistent kernel (k_correct) with bounded
// grid barriers between its phases:
//   sweep 0   one pass over the grid: codes of f (Sec. IV-A n_min / n_max,
//             Sec. III-A extrema), g = fhat, the input bound check, and sweep
//             0's detection (which vertices are distorted, which targets to
//             edit).  3D grids go through shared-memory tiles (msz_tile.cuh).
//   sweep k   edit phase: Eq. 1 applied once to every distinct target of
//             sweep k (Jacobi); detection phase of sweep k+1 over either the
//             worklist (closed neighbourhoods of the vertices changed in sweep
//             k plus the vertices distorted in sweep k) or, when that set
//             would be large, the whole grid -- both give the same g^(k+1).
//   end       stops when nothing is distorted (or STUCK / MAX_SWEEPS), then
//             writes the sorted edit list from the edited-vertex bitmap.
// Target sets and worklists are bitmaps marked with fire-and-forget
// reductions (duplicates merge for free, no warp waits on an atomic); the
// edit and sparse detection phases walk their set bits word by word.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_edits_async.h"
#include "msz_phases.cuh"
#include "msz_tile.cuh"
#include "msz_workspace.h"

namespace msz {

constexpr int kThreads = tile::THREADS;  // 256 per block of the persistent kernel
#ifndef MSZ_MIN_BLOCKS
#define MSZ_MIN_BLOCKS 3
#endif
constexpr int kMinBlocks = MSZ_MIN_BLOCKS;  // resident blocks per SM the register budget aims at
constexpr uint32_t kDenseFactor = 6;        // worklist estimate: 6 x distorted vertices
constexpr int kListRounds = 4;              // edit-list rounds whose loads a warp issues together
static_assert(kListRounds == 4, "the edit list's round group is written out for four rounds");
#ifndef MSZ_DETECT_TILE_Z
#define MSZ_DETECT_TILE_Z 16
#endif
// planes per tile of the whole-grid TMA detection (measured on the 512^3
// peak field: 4, 8, 16 and 32 planes within 1.5 % of one another; 16 best)
constexpr uint32_t kDetectTileZ = MSZ_DETECT_TILE_Z;
// a sweep keeps chunk flags when its worklist is bounded by this many
// vertices (measured on the 512^3 peak field, kernel time with bounds of
// 2^10, 2^13, 2^16, 2^19, 2^22: 16.0, 15.4, 15.2, 15.2, 15.3 ms; 16.2 ms
// without flags)
#ifndef MSZ_SPARSE_WORKLIST
#define MSZ_SPARSE_WORKLIST (1ull << 19)
#endif
constexpr unsigned long long kSparseWorklist = MSZ_SPARSE_WORKLIST;

struct Problem {
    CUtensorMap map_f;  // TMA maps of f, of the start field and of g (the TMA passes only)
    CUtensorMap map_s;
    CUtensorMap map_g;
    FieldView F;
    uint32_t *stb;     // chunk flags of F.tb, F.dm[0], F.dm[1] (kept in sparse sweeps)
    uint32_t *sdm[2];
    Ctrl *ctrl;
    SweepRec *log;
    uint32_t *bsum;
    uint32_t *edit_idx;
    float *edit_delta;
    unsigned long long edit_cap;
    uint32_t max_sweeps;
    long long dense_min;  // < 0: never scan densely after sweep 0
    uint32_t test_fault;  // test hooks: 1: block 0 does not arrive at the first grid barrier;
                          // 2: block 0 of the TMA code pass withholds its first plane copy
    uint32_t detect_tile_z;  // planes per tile of the whole-grid TMA detection
};

// ------------------------------------------------ sweep 0's pass over a 3D grid
// The codes of f with their certification, g = start, the bound check and
// sweep 0's detection, in a kernel of its own: its staging ring is the
// largest shared-memory user of the correction, and as a separate launch it
// leaves the loop kernel's L1 (which its gathering phases need) alone.  The
// kernel boundary orders its writes before the loop kernel.
template <bool TMA>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_codes(__grid_constant__ const Problem P) {
    extern __shared__ __align__(16) float smem[];
    const FieldView &F = P.F;
    Ctrl *C = P.ctrl;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        C->t_start = global_ns();
        P.log[0].worklist = F.G.n;
        C->examined = F.G.n;
        C->dense_sweeps = 1;
    }
    uint32_t distorted = 0;
    if (TMA)
        first_tiled_tma<true>(F, &P.map_f, &P.map_s, &P.log[0].tile_next, smem, &C->error, distorted,
                              P.test_fault == 2);
    else first_tiled<true, true>(F, &P.log[0].tile_next, smem, &C->error, distorted);
    warp_add(distorted, &P.log[0].distorted);
}

// ------------------------------------------------------ the persistent kernel
template <int NDIM, bool TMA>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_correct(__grid_constant__ const Problem P) {
    extern __shared__ __align__(16) float smem[];
    const FieldView &F = P.F;
    const GridDev &G = F.G;
    Ctrl *C = P.ctrl;
    __shared__ uint32_t sm[40];
    __shared__ uint32_t s_rq[kThreads / 32][kRoundCap];  // each warp's round queue (sparse walks)
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    const bool leader = gtid == 0;

    // ---- sweep 0: codes of f with their certification, g = start, bound
    // check, and the detection of sweep 0 (only uncertified vertices can be
    // distorted).  On 3D grids k_codes ran it (tiles detect their own
    // uncertified vertices from the staged start field); 2D grids take it
    // here, the detection in a second phase.
    bool ok;
    if (NDIM == 3) {
        ok = ld_relaxed(&C->error) == 0;  // every block reads k_codes' verdict
        if (ok && P.test_fault == 1)
            ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error, kTestBarrierNs, blockIdx.x == 0);
        if (leader) C->t_codes = global_ns();
    } else {
        if (leader) {
            C->t_start = global_ns();
            P.log[0].worklist = G.n;
            C->examined = G.n;
            C->dense_sweeps = 1;
        }
        first_generic<NDIM>(F, &C->error);
        ok = P.test_fault == 1
                 ? grid_barrier(&C->bar_count, &C->bar_gen, &C->error, kTestBarrierNs, blockIdx.x == 0)
                 : grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
        if (leader) C->t_codes = global_ns();
        if (ok) {
            Emitter E{F.dm[1], 0};
            uint32_t seen = 0;
            walk_bits_pairs<false>(F.ub, nullptr, G, seen, [&](bool h1, uint32_t v1, bool h2, uint32_t v2) {
                detect_vertex2<NDIM>(F, E, h1, v1, h2, v2);
            });
            warp_add(E.distorted, &P.log[0].distorted);
        }
        ok = ok && grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
    }
    if (leader) P.log[0].t_detect = global_ns();
    // Chunk flags are kept only in sparse sweeps (a dense sweep would store
    // them millions of times over for no walk that skips anything).
    // sum_k: the phases of sweep k keep them -- decided before sweep k's
    // detection from a bound on its worklist (15 x changed + distorted of
    // sweep k-1), so that every mark into sweep k's targets and into the next
    // worklist sets its chunk's flag whenever a walk relies on it.
    bool sum_k = false;  // sweep 0 keeps none
    uint32_t k = 0;
    while (ok) {
        const uint32_t m = ld_relaxed(&P.log[k].distorted);
        if (m == 0) {
            if (leader) { C->status = MSZ_OK; C->sweeps = k; }
            break;
        }
        if (k >= P.max_sweeps) {
            // count the distinct targets this sweep found, for the record
            uint32_t nt = 0;
            if (!sum_k) walk_bits<true>(F.tb, nullptr, G, nt, [&](bool, uint32_t) {});
            else walk_flagged<true, false>(F.tb, P.stb, nullptr, G, nt, s_rq[threadIdx.x >> 5], [&](bool, uint32_t) {});
            warp_add(nt, &P.log[k].targets);
            if (leader) { C->status = MSZ_ERR_MAX_SWEEPS; C->sweeps = k; C->left = m; }
            ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
            break;
        }
        const bool dense_next =
            P.dense_min >= 0 && (unsigned long long)m * kDenseFactor >= (unsigned long long)P.dense_min;
        // ---- edit phase of sweep k (Eq. 1), one application per distinct target.
        // In a sparse sweep the targets and the next worklist carry chunk
        // flags, so the walks visit only the chunks that may hold set bits.
        {
            uint32_t *dnext = F.dm[(k + 1) & 1];
            uint32_t targets = 0, changed_here = 0;
            if (!sum_k) {
                walk_bits<true>(
                    F.tb, nullptr, G, targets,
                    [&](bool has, uint32_t t) {
                        if (has && apply_target<NDIM>(F, t, dense_next, dnext)) ++changed_here;
                    },
                    s_rq[threadIdx.x >> 5]);
            } else {
                uint32_t *dsum = P.sdm[(k + 1) & 1];
                walk_flagged<true, false>(F.tb, P.stb, nullptr, G, targets, s_rq[threadIdx.x >> 5], [&](bool has, uint32_t t) {
                    if (has && apply_target<NDIM>(F, t, dense_next, dnext, dsum)) ++changed_here;
                });
            }
            if (TMA && dense_next) tma::fence_proxy_async_global();  // g is read by TMA next
            warp_add(targets, &P.log[k].targets);
            warp_add(changed_here, &P.log[k].changed);
        }
        ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
        if (!ok) break;
        if (leader) P.log[k].t_edit = global_ns();
        const uint32_t changed_k = ld_relaxed(&P.log[k].changed);
        if (changed_k == 0) {
            if (leader) { C->status = MSZ_STUCK; C->sweeps = k + 1; C->left = m; }
            break;
        }
        if (leader) C->edits += changed_k;
        const bool sum_k1 = 15ull * changed_k + m <= kSparseWorklist;
        // ---- detection phase of sweep k + 1
        // Detection of sweep k1 keeps flags of its targets and of the next
        // worklist when sum_k1; the current worklist has them when sweep k
        // kept them (sum_k).
        const uint32_t k1 = k + 1;
        Emitter E{F.dm[(k1 + 1) & 1], 0, sum_k1 ? P.sdm[(k1 + 1) & 1] : nullptr, sum_k1 ? P.stb : nullptr};
        uint32_t *dcur = F.dm[k1 & 1];
        uint32_t *dcur_sum = sum_k ? P.sdm[k1 & 1] : nullptr;
        uint32_t seen = 0;
        if (dense_next) {
            // whole grid: every uncertified vertex
            if (leader) {
                P.log[k1].worklist = G.n;
                C->examined += G.n;
                C->dense_sweeps += 1;
            }
            for (uint32_t w = gtid; w < G.words; w += stride) dcur[w] = 0;
            if (dcur_sum)
                for (uint32_t w = gtid; w < (uint32_t)chunk_count(G.words); w += stride) dcur_sum[w] = 0;
            if (TMA) {
                detect_tiled_tma(F, P.detect_tile_z, &P.map_g, &P.log[k1].tile_next, smem, &C->error, E.dnext,
                                 E.distorted, E.dsum, E.tsum);
            } else if (NDIM == 3) {
                detect_tiled_cp(F, P.detect_tile_z, &P.log[k1].tile_next, smem, E.dnext, E.distorted, E.dsum,
                                E.tsum);
            } else {
                walk_bits_pairs<false>(F.ub, nullptr, G, seen, [&](bool h1, uint32_t v1, bool h2, uint32_t v2) {
                    detect_vertex2<NDIM>(F, E, h1, v1, h2, v2);
                });
            }
        } else if (dcur_sum) {
            // the worklist, restricted to uncertified vertices, flagged chunk by flagged chunk
            walk_flagged<true, true>(dcur, dcur_sum, F.ub, G, seen, s_rq[threadIdx.x >> 5], [&](bool h1, uint32_t v1, bool h2, uint32_t v2) {
                detect_vertex2<NDIM>(F, E, h1, v1, h2, v2);
            });
            warp_add(seen, &P.log[k1].worklist);
        } else {
            // a worklist without flags (sweep 1's, built by sweep 0, and a dense sweep's)
            walk_bits_pairs<true>(
                dcur, F.ub, G, seen,
                [&](bool h1, uint32_t v1, bool h2, uint32_t v2) { detect_vertex2<NDIM>(F, E, h1, v1, h2, v2); },
                AllWords(), s_rq[threadIdx.x >> 5]);
            warp_add(seen, &P.log[k1].worklist);
        }
        warp_add(E.distorted, &P.log[k1].distorted);
        ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
        if (leader) {
            P.log[k1].t_detect = global_ns();
            if (!dense_next) C->examined += P.log[k1].worklist;
        }
        k = k1;
        sum_k = sum_k1;
    }
    if (!ok) return;

    // ---- edit list: every vertex of the edited bitmap, ascending index.
    // Each warp owns a contiguous range of bitmap words; a block scan of the
    // warps' counts and a grid-wide prefix over the blocks give each warp its
    // first output position, and the warp then writes its range 32 words at
    // a time with warp scans only.
    const uint32_t W = G.words;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const uint32_t nwarps = gridDim.x * wpb;
    const uint32_t per = (W + nwarps - 1) / nwarps;
    const uint32_t gw = blockIdx.x * wpb + warp;
    const uint32_t w0 = min(gw * per, W), w1 = min(w0 + per, W);
    uint32_t cnt = 0, unc = 0;
#pragma unroll 4
    for (uint32_t w = w0 + lane; w < w1; w += 32) {
        cnt += __popc(F.eb[w]);
        unc += __popc(F.ub[w]);
    }
    warp_add(unc, &C->uncertified);
    uint32_t tot;
    const uint32_t wcnt = __reduce_add_sync(kFull, cnt);
    const uint32_t wpre = block_exclusive_scan(lane == 0 ? wcnt : 0u, sm, tot);
    const uint32_t warp_pre = __shfl_sync(kFull, wpre, 0);  // this warp's offset in its block
    if (threadIdx.x == 0) P.bsum[blockIdx.x] = tot;
    if (!grid_barrier(&C->bar_count, &C->bar_gen, &C->error)) return;
    uint32_t pre = 0, all = 0;
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const uint32_t s = ld_relaxed(&P.bsum[b]);
        all += s;
        if (b < blockIdx.x) pre += s;
    }
    uint32_t bpre;
    block_exclusive_scan(pre, sm, bpre);
    block_exclusive_scan(all, sm, all);
    if (leader) C->edit_count = all;
    unsigned long long prefix = (unsigned long long)bpre + warp_pre;
    // Rounds of 32 words; a round's edits go to the lanes in index order
    // (ChunkBits), so its stores coalesce.  kListRounds rounds at a time: their
    // words are loaded together, then the first 32 edits of each gathered (g
    // and fhat) before any is stored, and the next group's words are loaded
    // before this group's stores -- a warp's chain of dependent loads is one
    // link per group instead of one per round.
    constexpr int R = kListRounds;
    auto word_at = [&](uint32_t w) -> uint32_t { return w < w1 ? F.eb[w] : 0u; };
    uint32_t wd[R];
#pragma unroll
    for (int q = 0; q < R; ++q) wd[q] = word_at(w0 + 32u * q + lane);
    for (uint32_t r = w0; r < w1; r += 32u * R) {
        ChunkBits cb[R] = {ChunkBits(r, wd[0]), ChunkBits(r + 32u, wd[1]), ChunkBits(r + 64u, wd[2]),
                           ChunkBits(r + 96u, wd[3])};
        bool h[R];
        uint32_t v[R];
        float gv[R], fv[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            cb[q].pick(lane, h[q], v[q]);
            gv[q] = h[q] ? F.g[v[q]] : 0.f;
            fv[q] = h[q] ? __ldg(&F.fhat[v[q]]) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) wd[q] = word_at(r + 32u * (R + q) + lane);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (h[q] && prefix + lane < P.edit_cap) {
                P.edit_idx[prefix + lane] = v[q];
                P.edit_delta[prefix + lane] = __fsub_rn(gv[q], fv[q]);
            }
            // a chunk with more than 32 edits (clustered edits): the rest
            // four rounds at a time, gathers first
            for (uint32_t j0 = 32u; j0 < cb[q].total; j0 += 32u * R) {
                bool hj[R];
                uint32_t vj[R];
                float gj[R], fj[R];
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    cb[q].pick(j0 + 32u * u + lane, hj[u], vj[u]);
                    gj[u] = hj[u] ? F.g[vj[u]] : 0.f;
                    fj[u] = hj[u] ? __ldg(&F.fhat[vj[u]]) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    const unsigned long long pos = prefix + j0 + 32u * u + lane;
                    if (hj[u] && pos < P.edit_cap) {
                        P.edit_idx[pos] = vj[u];
                        P.edit_delta[pos] = __fsub_rn(gj[u], fj[u]);
                    }
                }
            }
            prefix += cb[q].total;
        }
    }
    if (!grid_barrier(&C->bar_count, &C->bar_gen, &C->error)) return;
    if (leader) C->t_end = global_ns();
}

// --------------------------------------------------------- codes of a field
template <int NDIM>
__global__ void __launch_bounds__(256) k_directions(const float *v, __grid_constant__ const GridDev G, uint8_t *codes) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < G.n; i += stride) {
        uint32_t x, y, z;
        coords_of(G, i, x, y, z);
        codes[i] = code_global<NDIM>(v, G, i, x, y, z);
    }
}

// ------------------------------------------------------------- host helpers
static std::mutex g_mu;

msz_status current_device(DeviceInfo &info) {
    static DeviceInfo cache[64];
    static bool have[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MSZ_ERR_CUDA;
    if (dev < 0 || dev >= 64) return MSZ_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!have[dev]) {
        DeviceInfo d{};
        d.device = dev;
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
            return MSZ_ERR_CUDA;
        cache[dev] = d;
        have[dev] = true;
    }
    info = cache[dev];
    if (info.major != 10 || info.minor != 3) return MSZ_ERR_UNSUPPORTED;
    return MSZ_OK;
}

// Dynamic shared memory: the loop kernel stages one field for its whole-grid
// detection (TMA, or the cp.async ring on other 3D grids); k_codes stages f
// and the start field.
template <int NDIM, bool TMA>
static size_t correct_smem() {
    return NDIM == 3 ? (TMA ? tile::tma_ring_bytes(tile::kDetectSlots, 1) : tile::kRingBytes) : 0;
}
template <bool TMA>
static size_t codes_smem() {
    return TMA ? tile::tma_ring_bytes(tile::kCodeSlots, 2) : tile::kPairRingBytes;
}

// Resident blocks of kernel fn with sm bytes of dynamic shared memory, times
// the SM count (the persistent grid).  The attribute belongs to the current
// context, so it is set on every call (a context re-created after
// cudaDeviceReset starts without it); the occupancy it allows is a property of
// the device and is cached in *cache.
template <class K>
static msz_status persistent_blocks(K fn, size_t sm, const DeviceInfo &d, int *cache, int &blocks) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (sm > 48 * 1024 && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return MSZ_ERR_CUDA;
    if (!cache[d.device]) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kThreads, sm) != cudaSuccess) return MSZ_ERR_CUDA;
        if (per < 1) return MSZ_ERR_UNSUPPORTED;
        int b = per * d.sms;
        if (b > (int)kMaxBlocks) b = (int)kMaxBlocks;
        cache[d.device] = b;
    }
    blocks = cache[d.device];
    return MSZ_OK;
}

template <int NDIM, bool TMA>
static msz_status correct_blocks(const DeviceInfo &d, int &blocks) {
    static int cache[64];
    return persistent_blocks(k_correct<NDIM, TMA>, correct_smem<NDIM, TMA>(), d, cache, blocks);
}

template <bool TMA>
static msz_status codes_blocks(const DeviceInfo &d, int &blocks) {
    static int cache[64];
    return persistent_blocks(k_codes<TMA>, codes_smem<TMA>(), d, cache, blocks);
}

// Default planes per tile of the code pass: the deepest of kTileZ (24), 16,
// 8 that still gives every block of the persistent grid two tiles or more
// (deeper tiles re-read fewer halo planes; more tiles balance the blocks'
// work).
static uint32_t default_tile_z(const GridDev &G, int blocks) {
    for (const uint32_t tz : {kTileZ, 16u})
        if ((uint64_t)tile::tile_geom(G.nx, G.ny, G.nz, tz).count >= 2ull * (uint64_t)blocks) return tz;
    return 8;
}

// The TMA ring stages planes of the whole staged width: 3D grids whose x
// extent is a multiple of 4 (row strides of whole 16-byte units) and at least
// one box wide, at least one box high, with 16-byte aligned arrays.
static bool tma_eligible(const FieldView &F) {
    const GridDev &G = F.G;
    auto al = [](const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    return G.ndim == 3 && G.nx % 4 == 0 && G.nx >= (uint32_t)tile::PW && G.ny >= (uint32_t)tile::ROWS && al(F.f) &&
           al(F.fhat) && al(F.ginit) && al(F.g);
}

static PFN_cuTensorMapEncodeTiled_v12000 plane_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// Tensor map of one float field for the code pass: boxes of PW x ROWS x 1
// (x, y, z), positions outside the grid read as NaN.
static bool plane_map(const float *v, const GridDev &G, CUtensorMap &map) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = plane_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[3] = {G.nx, G.ny, G.nz};
    cuuint64_t strides[2] = {(cuuint64_t)G.nx * 4u, (cuuint64_t)G.nxy * 4u};
    cuuint32_t box[3] = {(cuuint32_t)tile::PW, (cuuint32_t)tile::ROWS, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)v, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA) == CUDA_SUCCESS;
}

// Records the caller's timing event ev (if any) on the stream.
static msz_status record(void *ev, cudaStream_t stream) {
    return !ev || cudaEventRecord((cudaEvent_t)ev, stream) == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

template <int NDIM, bool TMA>
static msz_status launch_correct(Problem &P, const DeviceInfo &dev, cudaStream_t stream, void *const *ev) {
    int blocks = 0;
    msz_status st = correct_blocks<NDIM, TMA>(dev, blocks);
    if (st != MSZ_OK) return st;
    if ((st = record(ev[0], stream)) != MSZ_OK) return st;
    if (NDIM == 3) {
        // sweep 0's pass first, as its own persistent launch (no grid-wide
        // wait inside it: an ordinary launch)
        int cblocks = 0;
        if ((st = codes_blocks<TMA>(dev, cblocks)) != MSZ_OK) return st;
        if (P.F.tile_z == 0) P.F.tile_z = default_tile_z(P.F.G, cblocks);
        k_codes<TMA><<<cblocks, kThreads, codes_smem<TMA>(), stream>>>(P);
        if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
    }
    if ((st = record(ev[1], stream)) != MSZ_OK) return st;
    void *args[] = {(void *)&P};
    if (cudaLaunchCooperativeKernel((const void *)k_correct<NDIM, TMA>, dim3(blocks), dim3(kThreads), args,
                                    correct_smem<NDIM, TMA>(), stream) != cudaSuccess)
        return MSZ_ERR_CUDA;
    return record(ev[2], stream);
}

// Default whole-grid detection rule (P.dense_min == 0).  A tiled whole-grid
// pass (g staged by TMA, or by cp.async on grids the TMA ring cannot stage)
// costs about one code pass without the certification; the worklist walk,
// which hands each chunk's vertices to the lanes in index order, is as fast
// or faster down to the largest worklists: measured at 512^3, dense while
// 6 x distorted >= N/4, N/16 or N takes the peak field 18.4, 24.2 or 16.2 ms
// (never dense: 16.3 ms; TMA) and leaves the Perlin field on worklists.  The
// default is N: the whole-grid pass only when nearly every vertex is on the
// worklist anyway.  2D grids keep worklists (their whole-grid walk gathers).
template <int NDIM>
static msz_status run_correct(Problem &P, const DeviceInfo &dev, cudaStream_t stream, void *const *ev) {
    if constexpr (NDIM == 3) {
        if (tma_eligible(P.F) && plane_map(P.F.f, P.F.G, P.map_f) &&
            plane_map(P.F.ginit ? P.F.ginit : P.F.fhat, P.F.G, P.map_s) && plane_map(P.F.g, P.F.G, P.map_g)) {
            if (P.dense_min == 0) P.dense_min = (long long)P.F.G.n;
            return launch_correct<3, true>(P, dev, stream, ev);
        }
    }
    if (P.dense_min == 0) P.dense_min = NDIM == 3 ? (long long)P.F.G.n : -1;
    return launch_correct<NDIM, false>(P, dev, stream, ev);
}

}  // namespace msz

using namespace msz;

extern "C" size_t msz_workspace_size(msz_grid grid) {
    GridDev G;
    if (make_grid(grid, G) != MSZ_OK) return 0;
    return layout_for(G.n).total;
}

extern "C" size_t msz_workspace_size_rule(msz_grid grid, int32_t rule) {
    GridDev G;
    if (make_grid(grid, G) != MSZ_OK) return 0;
    if (rule == MSZ_RULE_HALVE || rule == MSZ_RULE_SNAP) return layout_for(G.n).total;
    if (rule == MSZ_RULE_BELOW_REFERENCE) return layout_for(G.n).total + cand_bytes(G.n);
    return 0;
}

extern "C" msz_status msz_directions(const float *d_v, msz_grid grid, uint8_t *d_codes, msz_stream_t stream) {
    if (!d_v || !d_codes) return MSZ_ERR_INVALID_ARG;
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    const int blocks = dev.sms * 8;
    if (G.ndim == 3)
        k_directions<3><<<blocks, 256, 0, (cudaStream_t)stream>>>(d_v, G, d_codes);
    else
        k_directions<2><<<blocks, 256, 0, (cudaStream_t)stream>>>(d_v, G, d_codes);
    return cuda_status(cudaGetLastError());
}

namespace msz {

// msz_correct in three steps, shared with the pipeline below: the argument
// checks and the kernel's problem, the launch, and the results from the
// control block read back after it.
static msz_status prepare_correct(const float *d_f, const float *d_fhat, float xi, msz_grid grid, float *d_out,
                                  uint32_t *d_edit_idx, float *d_edit_delta, int64_t edit_capacity,
                                  const msz_options *opt, void *d_workspace, size_t workspace_bytes, Problem &P,
                                  msz_options &o) {
    if (!d_f || !d_fhat || !d_out) return MSZ_ERR_INVALID_ARG;
    if (edit_capacity < 0 || (edit_capacity > 0 && (!d_edit_idx || !d_edit_delta))) return MSZ_ERR_INVALID_ARG;
    if (!(xi >= 0.0f) || isinf(xi)) return MSZ_ERR_INVALID_ARG;
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    o = msz_options{};
    if (opt) o = *opt;
    if (o.rule != MSZ_RULE_HALVE && o.rule != MSZ_RULE_SNAP && o.rule != MSZ_RULE_BELOW_REFERENCE)
        return MSZ_ERR_INVALID_ARG;
    if (o.test_fault < 0 || o.test_fault > 2) return MSZ_ERR_INVALID_ARG;
    if (o.max_sweeps > MSZ_MAX_SWEEPS_LIMIT || o.dense_min_items < -1 || o.log_capacity < 0 || o.tile_z < 0 ||
        o.tile_z > 1024 ||
        (o.log_capacity > 0 && !o.h_sweep_log))
        return MSZ_ERR_INVALID_ARG;
    const Layout L = layout_for(G.n);
    const bool below = o.rule == MSZ_RULE_BELOW_REFERENCE;
    if (!d_workspace || workspace_bytes < L.total + (below ? cand_bytes(G.n) : 0)) return MSZ_ERR_WORKSPACE;
    if ((uintptr_t)d_workspace % kAlign) return MSZ_ERR_INVALID_ARG;

    char *ws = (char *)d_workspace;
    P = Problem{};
    FieldView &F = P.F;
    F.G = G;
    F.f = d_f;
    F.fhat = d_fhat;
    F.ginit = o.d_g_init;
    F.g = d_out;
    F.codes_f = (uint8_t *)(ws + L.codes);
    F.tb = (uint32_t *)(ws + L.tb);
    F.dm[0] = (uint32_t *)(ws + L.d0);
    F.dm[1] = (uint32_t *)(ws + L.d1);
    F.eb = (uint32_t *)(ws + L.eb);
    F.ub = (uint32_t *)(ws + L.ub);
    F.cand = below ? (uint32_t *)(ws + L.total) : nullptr;  // after the shared layout
    F.xi = xi;
    F.two_xi = 2.0f * xi;  // exact (power-of-two scaling), +inf on overflow
    F.rule = o.rule;
    F.tile_z = o.tile_z > 0 ? (uint32_t)o.tile_z : 0u;  // 0: chosen from the grid and the launch
    P.stb = (uint32_t *)(ws + L.stb);
    P.sdm[0] = (uint32_t *)(ws + L.sd0);
    P.sdm[1] = (uint32_t *)(ws + L.sd1);
    P.ctrl = (Ctrl *)(ws + L.ctrl);
    P.log = (SweepRec *)(ws + L.log);
    P.bsum = (uint32_t *)(ws + L.bsum);
    P.edit_idx = d_edit_idx;
    P.edit_delta = d_edit_delta;
    P.edit_cap = (unsigned long long)edit_capacity;
    P.max_sweeps = o.max_sweeps <= 0 ? (uint32_t)MSZ_MAX_SWEEPS_LIMIT : (uint32_t)o.max_sweeps;
    // default (0): decided with the staging in run_correct
    P.dense_min = o.dense_min_items == 0 ? 0LL : (long long)o.dense_min_items;
    P.test_fault = (uint32_t)o.test_fault;
    P.detect_tile_z = kDetectTileZ;
    return MSZ_OK;
}

// ev: the caller's three timing events (entries may be null), or null.
static msz_status enqueue_correct(Problem &P, const DeviceInfo &dev, cudaStream_t s, void *const *ev = nullptr) {
    static void *const kNoEvents[3] = {nullptr, nullptr, nullptr};
    if (!ev) ev = kNoEvents;
    if (cudaMemsetAsync(P.ctrl, 0, layout_for(P.F.G.n).zero_bytes, s) != cudaSuccess) return MSZ_ERR_CUDA;
    // BELOW_REFERENCE: no candidate yet anywhere (all-ones keys)
    if (P.F.cand && cudaMemsetAsync(P.F.cand, 0xff, (size_t)P.F.G.n * 4u, s) != cudaSuccess) return MSZ_ERR_CUDA;
    return P.F.G.ndim == 3 ? run_correct<3>(P, dev, s, ev) : run_correct<2>(P, dev, s, ev);
}

// Status, edit count and stats from the control block and the record of
// sweep 0 read back after the kernel.
static msz_status finish_correct(const Ctrl &hc, const SweepRec &r0, int64_t edit_capacity, int64_t *h_edit_count,
                                 msz_stats *h_stats) {
    if (hc.error & kErrInput) return MSZ_ERR_INPUT_BOUND;
    if (hc.error & kErrTimeout) return MSZ_ERR_TIMEOUT;
    *h_edit_count = (int64_t)hc.edit_count;
    if (h_stats) {
        *h_stats = msz_stats{};
        h_stats->sweeps = hc.sweeps;
        h_stats->edits = (int64_t)hc.edits;
        h_stats->edited = (int64_t)hc.edit_count;
        h_stats->first_distorted = r0.distorted;
        h_stats->left = hc.left;
        h_stats->examined = (int64_t)hc.examined;
        h_stats->dense_sweeps = hc.dense_sweeps;
        h_stats->kernel_ns = hc.t_end > hc.t_start ? (int64_t)(hc.t_end - hc.t_start) : 0;
        h_stats->codes_ns = hc.t_codes > hc.t_start ? (int64_t)(hc.t_codes - hc.t_start) : 0;
        h_stats->uncertified = hc.uncertified;
    }
    const msz_status loop = (msz_status)hc.status;
    if (loop == MSZ_OK && (int64_t)hc.edit_count > edit_capacity) return MSZ_ERR_CAPACITY;
    return loop;
}

}  // namespace msz

extern "C" msz_status msz_correct(const float *d_f, const float *d_fhat, float xi, msz_grid grid, float *d_out,
                                  uint32_t *d_edit_idx, float *d_edit_delta, int64_t edit_capacity,
                                  int64_t *h_edit_count, const msz_options *opt, msz_stats *h_stats,
                                  void *d_workspace, size_t workspace_bytes, msz_stream_t stream) {
    if (!h_edit_count) return MSZ_ERR_INVALID_ARG;
    Problem P;
    msz_options o;
    msz_status st = prepare_correct(d_f, d_fhat, xi, grid, d_out, d_edit_idx, d_edit_delta, edit_capacity, opt,
                                    d_workspace, workspace_bytes, P, o);
    if (st != MSZ_OK) return st;
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = enqueue_correct(P, dev, s, o.phase_events)) != MSZ_OK) return st;
    // the control block and sweep 0's record in one read-back (the log
    // follows the control block in the workspace)
    static_assert(offsetof(Layout, ctrl) == 0, "layout order");
    const size_t head = (size_t)((const char *)P.log - (const char *)P.ctrl) + sizeof(SweepRec);
    alignas(16) unsigned char hb[1024];
    static_assert(sizeof(Ctrl) + sizeof(SweepRec) <= sizeof hb, "read-back buffer");
    if (head > sizeof hb) return MSZ_ERR_CUDA;
    if (cudaMemcpyAsync(hb, P.ctrl, head, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    Ctrl hc;
    SweepRec r0;
    memcpy(&hc, hb, sizeof hc);
    memcpy(&r0, hb + (head - sizeof(SweepRec)), sizeof r0);
    st = finish_correct(hc, r0, edit_capacity, h_edit_count, h_stats);
    if (st == MSZ_ERR_INPUT_BOUND || st == MSZ_ERR_TIMEOUT) return st;
    if (o.log_capacity > 0) {
        const int64_t nrec = (int64_t)hc.sweeps + 1 < o.log_capacity ? (int64_t)hc.sweeps + 1 : o.log_capacity;
        SweepRec tmp[256];
        for (int64_t b = 0; b < nrec; b += 256) {
            const int64_t c = nrec - b < 256 ? nrec - b : 256;
            if (cudaMemcpy(tmp, P.log + b, (size_t)c * sizeof(SweepRec), cudaMemcpyDeviceToHost) != cudaSuccess)
                return MSZ_ERR_CUDA;
            for (int64_t q = 0; q < c; ++q) {
                if (o.h_timeline) {
                    const unsigned long long td = tmp[q].t_detect, te = tmp[q].t_edit;
                    o.h_timeline[2 * (b + q) + 0] = td ? (int64_t)(td - hc.t_start) : -1;
                    o.h_timeline[2 * (b + q) + 1] = te ? (int64_t)(te - hc.t_start) : -1;
                }
                o.h_sweep_log[4 * (b + q) + 0] = tmp[q].worklist;
                o.h_sweep_log[4 * (b + q) + 1] = tmp[q].distorted;
                o.h_sweep_log[4 * (b + q) + 2] = tmp[q].targets;
                o.h_sweep_log[4 * (b + q) + 3] = tmp[q].changed;
            }
        }
    }
    return st;
}

extern "C" size_t msz_host_workspace_size(msz_grid grid, int64_t edit_capacity) {
    GridDev G;
    if (make_grid(grid, G) != MSZ_OK || edit_capacity < 0) return 0;
    const size_t fld = align_up((size_t)G.n * 4);
    const size_t cap = align_up((size_t)edit_capacity * 4);
    return layout_for(G.n).total + 3 * fld + 2 * cap;
}

extern "C" msz_status msz_correct_host(const float *h_f, const float *h_fhat, float xi, msz_grid grid,
                                       float *h_out, uint32_t *h_edit_idx, float *h_edit_delta,
                                       int64_t edit_capacity, int64_t *h_edit_count, const msz_options *opt,
                                       msz_stats *h_stats, void *d_workspace, size_t workspace_bytes,
                                       msz_stream_t stream) {
    if (!h_f || !h_fhat || !h_out || !h_edit_count) return MSZ_ERR_INVALID_ARG;
    if (edit_capacity < 0 || (edit_capacity > 0 && (!h_edit_idx || !h_edit_delta))) return MSZ_ERR_INVALID_ARG;
    if (opt && opt->d_g_init) return MSZ_ERR_INVALID_ARG;  // host entry takes no device start
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    const size_t need = msz_host_workspace_size(grid, edit_capacity);
    if (!d_workspace || workspace_bytes < need) return MSZ_ERR_WORKSPACE;
    if ((uintptr_t)d_workspace % kAlign) return MSZ_ERR_INVALID_ARG;
    const size_t base = layout_for(G.n).total, fld = align_up((size_t)G.n * 4),
                 cap = align_up((size_t)edit_capacity * 4);
    char *ws = (char *)d_workspace;
    float *d_f = (float *)(ws + base), *d_fhat = (float *)(ws + base + fld), *d_out = (float *)(ws + base + 2 * fld);
    uint32_t *d_idx = (uint32_t *)(ws + base + 3 * fld);
    float *d_del = (float *)(ws + base + 3 * fld + cap);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)G.n * 4;
    if (cudaMemcpyAsync(d_f, h_f, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaMemcpyAsync(d_fhat, h_fhat, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return MSZ_ERR_CUDA;
    int64_t count = 0;
    st = msz_correct(d_f, d_fhat, xi, grid, d_out, edit_capacity ? d_idx : nullptr, edit_capacity ? d_del : nullptr,
                     edit_capacity, &count, opt, h_stats, d_workspace, base, stream);
    *h_edit_count = count;
    if (st != MSZ_OK && st != MSZ_ERR_CAPACITY && st != MSZ_STUCK && st != MSZ_ERR_MAX_SWEEPS) return st;
    if (cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    const int64_t ne = count < edit_capacity ? count : edit_capacity;
    if (ne > 0) {
        if (cudaMemcpyAsync(h_edit_idx, d_idx, (size_t)ne * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return MSZ_ERR_CUDA;
        if (cudaMemcpyAsync(h_edit_delta, d_del, (size_t)ne * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return MSZ_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    return st;
}

// ------------------------------------------------------------ pipeline
// Two slots of device buffers (f, fhat, g, edit list, correction workspace,
// and for an encoded pipeline the edit-list stream and its workspace) and
// three streams: inputs up, correction, result down.  Field k+1's inputs go
// up while field k is corrected and field k-1's result comes down; events
// order each slot's reuse.
struct msz_pipeline {
    msz_grid grid;
    GridDev G;
    int64_t cap;
    bool encoded;  // results: the edit list's stream (msz_edits_encode format) instead of g
    char *ws;
    size_t slot_bytes, fld, capb, base, stream_cap;
    cudaStream_t s_in, s_comp, s_out;
    struct Slot {
        cudaEvent_t in_done, comp_done, out_done;
        bool used;
        bool stream_dev;  // the encoded stream went to the host buffer from the device (stream_out_async)
        bool field_dev;   // g and the edit list went to the host buffers from the device (k_field_out)
        float *h_out;
        uint32_t *h_idx;
        float *h_del;
        uint8_t *h_stream;
        size_t h_stream_cap;
        Problem P;
    } slot[2];
    struct EncCtrl {
        uint32_t error, pad;
        unsigned long long total_words;
    };
    // pinned and mapped: the control block, sweep-0 record and encoder state
    // of each slot, written by k_readback (the d_ pointers: their device
    // addresses)
    msz::Ctrl *h_ctrl;
    msz::SweepRec *h_rec;
    EncCtrl *h_enc;
    msz::Ctrl *d_hctrl;
    msz::SweepRec *d_hrec;
    EncCtrl *d_henc;
    int head, tail, pending;
};

namespace msz {
// Bytes of one slot: correction workspace, f, fhat, g, the edit list, and
// when encoded the stream and its workspace.
static size_t pipeline_slot_bytes(const GridDev &G, int64_t cap, bool encoded, size_t *stream_cap = nullptr) {
    size_t b = layout_for(G.n).total + 3 * align_up((size_t)G.n * 4) + 2 * align_up((size_t)cap * 4);
    const size_t sc = encoded ? align_up(msz_edits_encoded_bound(cap)) : 0;
    if (stream_cap) *stream_cap = sc;
    if (encoded) b += sc + align_up(encode_async_workspace((uint64_t)cap));
    return b;
}

static msz_status pipeline_create(msz_grid grid, int64_t edit_capacity, bool encoded, void *d_workspace,
                                  size_t workspace_bytes, msz_pipeline **out) {
    if (!out || edit_capacity < 0) return MSZ_ERR_INVALID_ARG;
    *out = nullptr;
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    const size_t need = 2 * pipeline_slot_bytes(G, edit_capacity, encoded);
    if (!d_workspace || workspace_bytes < need) return MSZ_ERR_WORKSPACE;
    if ((uintptr_t)d_workspace % kAlign) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    msz_pipeline *pl = new msz_pipeline{};
    pl->grid = grid;
    pl->G = G;
    pl->cap = edit_capacity;
    pl->encoded = encoded;
    pl->ws = (char *)d_workspace;
    pl->slot_bytes = pipeline_slot_bytes(G, edit_capacity, encoded, &pl->stream_cap);
    pl->base = layout_for(G.n).total;
    pl->fld = align_up((size_t)G.n * 4);
    pl->capb = align_up((size_t)edit_capacity * 4);
    bool ok = cudaStreamCreateWithFlags(&pl->s_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&pl->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&pl->s_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaHostAlloc((void **)&pl->h_ctrl, 2 * sizeof(Ctrl), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc((void **)&pl->h_rec, 2 * sizeof(SweepRec), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc((void **)&pl->h_enc, 2 * sizeof(msz_pipeline::EncCtrl), cudaHostAllocMapped) ==
                  cudaSuccess &&
              cudaHostGetDevicePointer((void **)&pl->d_hctrl, pl->h_ctrl, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&pl->d_hrec, pl->h_rec, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&pl->d_henc, pl->h_enc, 0) == cudaSuccess;
    for (int k = 0; ok && k < 2; ++k)
        ok = cudaEventCreateWithFlags(&pl->slot[k].in_done, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&pl->slot[k].comp_done, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&pl->slot[k].out_done, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        msz_pipeline_destroy(pl);
        return MSZ_ERR_CUDA;
    }
    *out = pl;
    return MSZ_OK;
}

// The device buffers of slot k.
struct SlotBufs {
    float *f, *fhat, *g;
    uint32_t *idx;
    float *del;
    uint8_t *stream;
    void *enc_ws;
};
static SlotBufs slot_bufs(const msz_pipeline *pl, int k) {
    char *w = pl->ws + (size_t)k * pl->slot_bytes;
    SlotBufs b;
    b.f = (float *)(w + pl->base);
    b.fhat = (float *)(w + pl->base + pl->fld);
    b.g = (float *)(w + pl->base + 2 * pl->fld);
    b.idx = (uint32_t *)(w + pl->base + 3 * pl->fld);
    b.del = (float *)(w + pl->base + 3 * pl->fld + pl->capb);
    b.stream = (uint8_t *)(w + pl->base + 3 * pl->fld + 2 * pl->capb);
    b.enc_ws = (void *)(w + pl->base + 3 * pl->fld + 2 * pl->capb + pl->stream_cap);
    return b;
}

// The small results of a slot's correction -- the control block, sweep 0's
// record and, when encoded, the encoder's state -- written by a kernel into
// mapped pinned host memory.  A download on the correction's stream would
// sit in a copy engine's queue waiting for the correction, and the next
// field's upload, queued behind it, would wait too: the link would idle
// while each field is corrected.
__global__ void k_readback(const uint32_t *ctrl, uint32_t *h_ctrl, const uint32_t *rec, uint32_t *h_rec,
                           const uint32_t *enc, uint32_t *h_enc) {
    constexpr uint32_t nc = sizeof(Ctrl) / 4, nr = sizeof(SweepRec) / 4;
    constexpr uint32_t ne = sizeof(msz_pipeline::EncCtrl) / 4;
    static_assert(sizeof(Ctrl) % 4 == 0 && sizeof(SweepRec) % 4 == 0, "word copies");
    for (uint32_t i = threadIdx.x; i < nc + nr + ne; i += blockDim.x) {
        if (i < nc) h_ctrl[i] = ctrl[i];
        else if (i < nc + nr) h_rec[i - nc] = rec[i - nc];
        else if (enc) h_enc[i - nc - nr] = enc[i - nc - nr];
    }
}

// The corrected field and the edit list into host memory the device
// addresses (pipelined, field results): a grid-stride copy of g (16 bytes a
// thread where both ends are aligned), then of the first min(count, cap)
// entries of the edit list, the count read on the device.  A copy engine's
// download queued on another stream would wait for the correction in the
// engine's queue and hold up the next field's upload behind it.
__global__ void k_field_out(float *h_g, const float *g, uint32_t n, uint32_t *h_idx, float *h_del,
                            const uint32_t *idx, const float *del, const unsigned long long *count, uint64_t cap) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(h_g) | reinterpret_cast<uintptr_t>(g)) & 15u) == 0;
    const uint64_t nv = vec ? n / 4u : 0u;
    for (uint64_t i = tid; i < nv; i += stride)
        reinterpret_cast<float4 *>(h_g)[i] = reinterpret_cast<const float4 *>(g)[i];
    for (uint64_t i = 4u * nv + tid; i < n; i += stride) h_g[i] = g[i];
    const uint64_t c = *count, m = c < cap ? c : cap;
    for (uint64_t i = tid; i < m; i += stride) {
        h_idx[i] = idx[i];
        h_del[i] = del[i];
    }
}

// The device address of host buffer p when the device can write it (pinned
// or registered memory), else null.
static void *device_view(void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();  // pageable memory on older runtimes: not an error here
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Queues one field into the head slot: inputs up, the correction (and, when
// encoded, the edit list's stream), the result down.
static msz_status pipeline_submit(msz_pipeline *pl, const float *h_f, const float *h_fhat, float xi, float *h_out,
                                  uint32_t *h_idx, float *h_del, uint8_t *h_stream, size_t h_stream_cap,
                                  const msz_options *opt) {
    if (pl->pending == 2) return MSZ_ERR_INVALID_ARG;  // collect the oldest field first
    if (opt && (opt->d_g_init || opt->h_sweep_log || opt->log_capacity || opt->test_fault)) return MSZ_ERR_INVALID_ARG;
    const int k = pl->head;
    msz_pipeline::Slot &sl = pl->slot[k];
    const SlotBufs b = slot_bufs(pl, k);
    char *w = pl->ws + (size_t)k * pl->slot_bytes;
    msz_options o;
    msz_status st = prepare_correct(b.f, b.fhat, xi, pl->grid, b.g, pl->cap ? b.idx : nullptr,
                                    pl->cap ? b.del : nullptr, pl->cap, opt, w, pl->base, sl.P, o);
    if (st != MSZ_OK) return st;
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    const size_t bytes = (size_t)pl->G.n * 4;
    // inputs up, once the slot's previous correction has read its inputs
    if (sl.used && cudaStreamWaitEvent(pl->s_in, sl.comp_done, 0) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaMemcpyAsync(b.f, h_f, bytes, cudaMemcpyHostToDevice, pl->s_in) != cudaSuccess ||
        cudaMemcpyAsync(b.fhat, h_fhat, bytes, cudaMemcpyHostToDevice, pl->s_in) != cudaSuccess ||
        cudaEventRecord(sl.in_done, pl->s_in) != cudaSuccess)
        return MSZ_ERR_CUDA;
    // the correction, once the inputs are up and the slot's previous result
    // has come down
    if (cudaStreamWaitEvent(pl->s_comp, sl.in_done, 0) != cudaSuccess) return MSZ_ERR_CUDA;
    if (sl.used && cudaStreamWaitEvent(pl->s_comp, sl.out_done, 0) != cudaSuccess) return MSZ_ERR_CUDA;
    if ((st = enqueue_correct(sl.P, dev, pl->s_comp)) != MSZ_OK) return st;
    sl.stream_dev = false;
    sl.field_dev = false;
    if (!pl->encoded) {
        // g and the edit list into the caller's buffers from the device when
        // it can address all three, else by copies (g queued below, the edit
        // list at collect, when its length is known on the host)
        float *ho = (float *)device_view(h_out);
        uint32_t *hi = pl->cap ? (uint32_t *)device_view(h_idx) : nullptr;
        float *hd = pl->cap ? (float *)device_view(h_del) : nullptr;
        if (ho && (!pl->cap || (hi && hd))) {
            k_field_out<<<dev.sms * 2, 256, 0, pl->s_comp>>>(ho, b.g, pl->G.n, hi, hd, b.idx, b.del,
                                                            &sl.P.ctrl->edit_count, (uint64_t)pl->cap);
            if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
            sl.field_dev = true;
        }
    }
    if (pl->encoded) {
        st = encode_async(b.fhat, b.g, pl->G.n, b.idx, &sl.P.ctrl->edit_count, (uint64_t)pl->cap, b.stream,
                          pl->stream_cap, b.enc_ws, dev, pl->s_comp);
        if (st != MSZ_OK) return st;
        // the stream into the caller's buffer from the device when it can
        // (its length is known there), else by a copy at collect
        if (uint8_t *hs = (uint8_t *)device_view(h_stream)) {
            st = stream_out_async(b.stream, b.enc_ws, &sl.P.ctrl->edit_count, (uint64_t)pl->cap, hs, h_stream_cap,
                                  pl->s_comp);
            if (st != MSZ_OK) return st;
            sl.stream_dev = true;
        }
    }
    k_readback<<<1, 64, 0, pl->s_comp>>>((const uint32_t *)sl.P.ctrl, (uint32_t *)&pl->d_hctrl[k],
                                         (const uint32_t *)sl.P.log, (uint32_t *)&pl->d_hrec[k],
                                         pl->encoded ? (const uint32_t *)b.enc_ws : nullptr,
                                         (uint32_t *)&pl->d_henc[k]);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(sl.comp_done, pl->s_comp) != cudaSuccess)
        return MSZ_ERR_CUDA;
    // the corrected field down (an encoded pipeline's stream comes down at
    // collect, when its length is known)
    if (cudaStreamWaitEvent(pl->s_out, sl.comp_done, 0) != cudaSuccess) return MSZ_ERR_CUDA;
    if (!pl->encoded && !sl.field_dev &&
        cudaMemcpyAsync(h_out, b.g, bytes, cudaMemcpyDeviceToHost, pl->s_out) != cudaSuccess)
        return MSZ_ERR_CUDA;
    if (cudaEventRecord(sl.out_done, pl->s_out) != cudaSuccess) return MSZ_ERR_CUDA;
    sl.used = true;
    sl.h_out = h_out;
    sl.h_idx = h_idx;
    sl.h_del = h_del;
    sl.h_stream = h_stream;
    sl.h_stream_cap = h_stream_cap;
    pl->head ^= 1;
    pl->pending += 1;
    return MSZ_OK;
}

// The results of dequeued slot k: status, edit count, stats, (encoded) stream
// length, and the downloads whose length is known only now, queued behind
// the field's own download.
static msz_status pipeline_results(msz_pipeline *pl, int k, int64_t *h_edit_count, size_t *h_stream_bytes,
                                   msz_stats *h_stats) {
    msz_pipeline::Slot &sl = pl->slot[k];
    if (cudaEventSynchronize(sl.comp_done) != cudaSuccess) return MSZ_ERR_CUDA;
    int64_t count = 0;
    msz_status st = finish_correct(pl->h_ctrl[k], pl->h_rec[k], pl->cap, &count, h_stats);
    *h_edit_count = count;
    const bool listed = st != MSZ_ERR_INPUT_BOUND && st != MSZ_ERR_TIMEOUT;
    const SlotBufs b = slot_bufs(pl, k);
    if (pl->encoded) {
        if (h_stream_bytes) *h_stream_bytes = 0;
        if (listed && st != MSZ_ERR_CAPACITY) {
            const msz_pipeline::EncCtrl e = pl->h_enc[k];
            const uint64_t len = encoded_length((uint64_t)count, e.total_words);
            if (h_stream_bytes) *h_stream_bytes = (size_t)len;
            if (e.error & 1u) return MSZ_ERR_INVALID_ARG;  // not expected: the loop lists edits in order
            if (e.error || len > sl.h_stream_cap) {
                st = MSZ_ERR_CAPACITY;
            } else if (!sl.stream_dev &&
                       (cudaMemcpyAsync(sl.h_stream, b.stream, (size_t)len, cudaMemcpyDeviceToHost, pl->s_out) !=
                            cudaSuccess ||
                        cudaEventRecord(sl.out_done, pl->s_out) != cudaSuccess)) {
                return MSZ_ERR_CUDA;
            }
        }
    } else {
        const int64_t ne = count < pl->cap ? count : pl->cap;
        if (ne > 0 && listed && !sl.field_dev) {
            // the edit list down, behind the field (its length is known now)
            if (cudaMemcpyAsync(sl.h_idx, b.idx, (size_t)ne * 4, cudaMemcpyDeviceToHost, pl->s_out) != cudaSuccess ||
                cudaMemcpyAsync(sl.h_del, b.del, (size_t)ne * 4, cudaMemcpyDeviceToHost, pl->s_out) != cudaSuccess ||
                cudaEventRecord(sl.out_done, pl->s_out) != cudaSuccess)
                return MSZ_ERR_CUDA;
        }
    }
    return st;
}

// Waits for the oldest field: its status, edit count, stats and (encoded)
// stream length.  Its host buffers are complete, and no copy into them is
// still in flight, on every return, errors included.
static msz_status pipeline_collect(msz_pipeline *pl, int64_t *h_edit_count, size_t *h_stream_bytes,
                                   msz_stats *h_stats) {
    if (pl->pending == 0) return MSZ_ERR_INVALID_ARG;
    const int k = pl->tail;
    pl->tail ^= 1;
    pl->pending -= 1;
    msz_status st = pipeline_results(pl, k, h_edit_count, h_stream_bytes, h_stats);
    if (cudaEventSynchronize(pl->slot[k].out_done) != cudaSuccess && st == MSZ_OK) st = MSZ_ERR_CUDA;
    return st;
}
}  // namespace msz

extern "C" size_t msz_pipeline_workspace_size(msz_grid grid, int64_t edit_capacity) {
    GridDev G;
    if (make_grid(grid, G) != MSZ_OK || edit_capacity < 0) return 0;
    return 2 * pipeline_slot_bytes(G, edit_capacity, false);
}

extern "C" size_t msz_pipeline_workspace_size_encoded(msz_grid grid, int64_t edit_capacity) {
    GridDev G;
    if (make_grid(grid, G) != MSZ_OK || edit_capacity < 0) return 0;
    return 2 * pipeline_slot_bytes(G, edit_capacity, true);
}

extern "C" msz_status msz_pipeline_create(msz_grid grid, int64_t edit_capacity, void *d_workspace,
                                          size_t workspace_bytes, msz_pipeline **out) {
    return pipeline_create(grid, edit_capacity, false, d_workspace, workspace_bytes, out);
}

extern "C" msz_status msz_pipeline_create_encoded(msz_grid grid, int64_t edit_capacity, void *d_workspace,
                                                  size_t workspace_bytes, msz_pipeline **out) {
    return pipeline_create(grid, edit_capacity, true, d_workspace, workspace_bytes, out);
}

extern "C" msz_status msz_pipeline_submit(msz_pipeline *pl, const float *h_f, const float *h_fhat, float xi,
                                          float *h_out, uint32_t *h_edit_idx, float *h_edit_delta,
                                          const msz_options *opt) {
    if (!pl || pl->encoded || !h_f || !h_fhat || !h_out) return MSZ_ERR_INVALID_ARG;
    if (pl->cap > 0 && (!h_edit_idx || !h_edit_delta)) return MSZ_ERR_INVALID_ARG;
    return pipeline_submit(pl, h_f, h_fhat, xi, h_out, h_edit_idx, h_edit_delta, nullptr, 0, opt);
}

extern "C" msz_status msz_pipeline_submit_encoded(msz_pipeline *pl, const float *h_f, const float *h_fhat, float xi,
                                                  uint8_t *h_stream, size_t stream_capacity,
                                                  const msz_options *opt) {
    if (!pl || !pl->encoded || !h_f || !h_fhat || !h_stream) return MSZ_ERR_INVALID_ARG;
    return pipeline_submit(pl, h_f, h_fhat, xi, nullptr, nullptr, nullptr, h_stream, stream_capacity, opt);
}

extern "C" msz_status msz_pipeline_collect(msz_pipeline *pl, int64_t *h_edit_count, msz_stats *h_stats) {
    if (!pl || pl->encoded || !h_edit_count) return MSZ_ERR_INVALID_ARG;
    return pipeline_collect(pl, h_edit_count, nullptr, h_stats);
}

extern "C" msz_status msz_pipeline_collect_encoded(msz_pipeline *pl, int64_t *h_edit_count, size_t *h_stream_bytes,
                                                   msz_stats *h_stats) {
    if (!pl || !pl->encoded || !h_edit_count || !h_stream_bytes) return MSZ_ERR_INVALID_ARG;
    return pipeline_collect(pl, h_edit_count, h_stream_bytes, h_stats);
}

extern "C" void msz_pipeline_destroy(msz_pipeline *pl) {
    if (!pl) return;
    if (pl->s_in) cudaStreamSynchronize(pl->s_in);
    if (pl->s_comp) cudaStreamSynchronize(pl->s_comp);
    if (pl->s_out) cudaStreamSynchronize(pl->s_out);
    for (auto &sl : pl->slot) {
        if (sl.in_done) cudaEventDestroy(sl.in_done);
        if (sl.comp_done) cudaEventDestroy(sl.comp_done);
        if (sl.out_done) cudaEventDestroy(sl.out_done);
    }
    if (pl->s_in) cudaStreamDestroy(pl->s_in);
    if (pl->s_comp) cudaStreamDestroy(pl->s_comp);
    if (pl->s_out) cudaStreamDestroy(pl->s_out);
    if (pl->h_ctrl) cudaFreeHost(pl->h_ctrl);
    if (pl->h_rec) cudaFreeHost(pl->h_rec);
    if (pl->h_enc) cudaFreeHost(pl->h_enc);
    delete pl;
}

extern "C" const char *msz_status_str(msz_status status) {
    switch (status) {
        case MSZ_OK: return "MSZ_OK";
        case MSZ_ERR_INVALID_ARG: return "MSZ_ERR_INVALID_ARG";
        case MSZ_ERR_INPUT_BOUND: return "MSZ_ERR_INPUT_BOUND";
        case MSZ_ERR_CAPACITY: return "MSZ_ERR_CAPACITY";
        case MSZ_ERR_WORKSPACE: return "MSZ_ERR_WORKSPACE";
        case MSZ_ERR_CUDA: return "MSZ_ERR_CUDA";
        case MSZ_ERR_MAX_SWEEPS: return "MSZ_ERR_MAX_SWEEPS";
        case MSZ_ERR_TIMEOUT: return "MSZ_ERR_TIMEOUT";
        case MSZ_STUCK: return "MSZ_STUCK";
        case MSZ_ERR_UNSUPPORTED: return "MSZ_ERR_UNSUPPORTED";
    }
    return "MSZ_UNKNOWN_STATUS";
}
