// msz_relaxed.cu -- the relaxed synchronization of pMSz (Sec. IV-B) emulated
// on one GB300: the paper's per-process blocks become tiles of 32 x 8 x 8
// vertices worked on by one thread block each, the ghost layer becomes the
// one-vertex ring around a tile, and the ghost exchange becomes a merge by
// minimum in global memory.
//
// One cooperative persistent kernel (k_relaxed) with bounded grid barriers:
//   sweep 0   the tiled code pass of msz_correct: codes of f and their
//             certification, g = fhat, the input bound check;
//   iteration k
//     detect  every examined vertex whose code in g^k differs from f's
//             marks its tile active (iteration 0 examines every uncertified
//             vertex, later ones a worklist);  none: done;
//     tiles   each active tile loads g^k over the tile and its ring into
//             shared memory and runs synchronous sweeps on that copy alone
//             (its own vertices are examined through a worklist, targets may
//             lie on the ring, Eq. 1 once per distinct target and sweep)
//             until no own vertex is distorted, a sweep changes nothing or
//             local_cap sweeps; every value below g^k is proposed to a
//             per-vertex minimum (IEEE totalOrder key, atomicMin);
//     merge   g^(k+1) = the proposals; no decrease at all: STUCK;
//   end       the sorted edit list, as in msz_correct.
// Tiles read g^k only and the merge is a minimum, so the result does not
// depend on which block runs which tile when: it equals the CPU oracle's
// orc_correct_relaxed bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_phases.cuh"
#include "msz_tile.cuh"
#include "msz_workspace.h"

namespace msz {
namespace relaxed {

constexpr int TX = MSZ_RELAXED_TILE_X, TY = MSZ_RELAXED_TILE_Y, TZ = MSZ_RELAXED_TILE_Z;
static_assert(TX == 32, "one interior row of a tile is one 32-bit word");
constexpr int RX = TX + 2, RY = TY + 2, RZ = TZ + 2;  // the tile with its ring
constexpr int RN = RX * RY * RZ;                      // 3400 ring-extended positions
constexpr int IW = TY * TZ;                           // interior rows (words)
constexpr int TW = (RN + 31) / 32;                    // words of a bitmap over the ring-extended box
constexpr int kThreads = tile::THREADS;
#ifndef MSZ_MIN_BLOCKS
#define MSZ_MIN_BLOCKS 3
#endif
constexpr int kMinBlocks = MSZ_MIN_BLOCKS;

struct Problem {
    FieldView F;
    Ctrl *ctrl;
    SweepRec *log;     // per iteration: tile runs, distorted, local sweeps, decreased values
    uint32_t *bsum;
    uint32_t *prop;    // merge proposals (totalOrder keys); all ones between iterations
    uint32_t *active;  // tiles holding a distorted vertex (bitmap)
    uint32_t *changed; // vertices with a proposal (bitmap)
    uint32_t *wl[2];   // detection worklists by iteration parity (after iteration 0)
    uint32_t ntx, nty, ntz, ntiles;
    uint32_t max_iters, local_cap;
    uint32_t *edit_idx;
    float *edit_delta;
    unsigned long long edit_cap;
};

// Shared memory of one tile run.
struct TileSmem {
    float loc[RN];               // the copy of g over the ring-extended box (NaN outside the grid)
    uint8_t cf[TX * TY * TZ];    // codes of f of the tile's own vertices
    uint32_t uw[IW];             // uncertified own vertices, one word per row
    uint32_t w[2][IW];           // worklists by local-sweep parity
    uint32_t tb[TW];             // targets of the current sweep (box positions)
    uint32_t ed[TW];             // box positions this run decreased
    uint32_t n_dist[2], n_changed[2];
};
static_assert(sizeof(TileSmem) <= tile::kRingBytes, "a tile run reuses the code pass's shared memory");

__device__ __forceinline__ uint32_t tkey(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float tval(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k ^ 0x80000000u) : ~k);
}

// Offset in the ring-extended box of the neighbour in slot s.
__device__ __forceinline__ int box_offset(int s) {
    int dx, dy, dz;
    slot_delta(3, s, dx, dy, dz);
    return dx + RX * dy + RX * RY * dz;
}

// Marks own vertex (x, y, z) (box coordinates 1..T) in a row bitmap.
__device__ __forceinline__ void mark_own(uint32_t *rows, int bx, int by, int bz) {
    if (bx < 1 || bx > TX || by < 1 || by > TY || bz < 1 || bz > TZ) return;
    atomicOr(&rows[(by - 1) + TY * (bz - 1)], 1u << (bx - 1));
}

// One run of tile t (block-collective).  Returns the local sweeps made.
// Two block barriers per local sweep: worklists and counters alternate by
// the sweep's parity, so a sweep clears what the next one will fill.
__device__ uint32_t run_tile(const Problem &P, uint32_t t, TileSmem &S) {
    const FieldView &F = P.F;
    const GridDev &G = F.G;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const int x0 = (int)(t % P.ntx) * TX, y0 = (int)((t / P.ntx) % P.nty) * TY, z0 = (int)(t / (P.ntx * P.nty)) * TZ;
    const float qnan = __int_as_float(0x7fffffff);
    auto global_of = [&](int q) {
        const int bx = q % RX, by = (q / RX) % RY, bz = q / (RX * RY);
        return (size_t)(x0 - 1 + bx) + (size_t)G.nx * ((size_t)(y0 - 1 + by) + (size_t)G.ny * (z0 - 1 + bz));
    };
    for (int q = (int)tid; q < RN; q += kThreads) {
        const int bx = q % RX, by = (q / RX) % RY, bz = q / (RX * RY);
        const int gx = x0 - 1 + bx, gy = y0 - 1 + by, gz = z0 - 1 + bz;
        const bool in = gx >= 0 && gx < (int)G.nx && gy >= 0 && gy < (int)G.ny && gz >= 0 && gz < (int)G.nz;
        S.loc[q] = in ? F.g[global_of(q)] : qnan;
    }
    for (int i = (int)tid; i < TX * TY * TZ; i += kThreads) {
        const int gx = x0 + i % TX, gy = y0 + (i / TX) % TY, gz = z0 + i / (TX * TY);
        uint8_t c = 0;
        if (gx < (int)G.nx && gy < (int)G.ny && gz < (int)G.nz)
            c = __ldg(&F.codes_f[(size_t)gx + (size_t)G.nx * ((size_t)gy + (size_t)G.ny * gz)]);
        S.cf[i] = c;
    }
    for (int r = (int)tid; r < IW; r += kThreads) {
        const int gy = y0 + r % TY, gz = z0 + r / TY;
        uint32_t bits = 0;
        if (gy < (int)G.ny && gz < (int)G.nz) {
            // uncertified bits of the row's vertices x0 .. x0+31 (possibly across two words)
            const uint32_t v0 = (uint32_t)x0 + G.nx * ((uint32_t)gy + G.ny * (uint32_t)gz);
            const uint32_t wi = v0 >> 5, sh = v0 & 31u;
            const uint32_t lo = F.ub[wi];
            const uint32_t hi = (sh && wi + 1 < G.words) ? F.ub[wi + 1] : 0u;
            bits = sh ? (lo >> sh) | (hi << (32u - sh)) : lo;
            const int valid = (int)G.nx - x0;
            if (valid < 32) bits &= (1u << valid) - 1u;
        }
        S.uw[r] = bits;
        S.w[0][r] = bits;
        S.w[1][r] = 0u;
    }
    for (int q = (int)tid; q < TW; q += kThreads) {
        S.tb[q] = 0u;
        S.ed[q] = 0u;
    }
    if (tid < 2) {
        S.n_dist[tid] = 0;
        S.n_changed[tid] = 0;
    }
    __syncthreads();
    uint32_t sweeps = 0, p = 0;
    for (uint32_t ls = 0; ls < P.local_cap; ++ls, p ^= 1u) {
        // detection on the copy: warp w takes rows w, w + 8, ..., lane = x
        uint32_t nd = 0;
        for (int r = (int)warp; r < IW; r += kThreads / 32) {
            if (!((S.w[p][r] & S.uw[r]) >> lane & 1u)) continue;
            const int by = r % TY + 1, bz = r / TY + 1, bx = (int)lane + 1;
            const int q = bx + RX * (by + RY * bz);
            float c[15];
            c[0] = S.loc[q - 1 - RX - RX * RY];
            c[1] = S.loc[q - RX - RX * RY];
            c[2] = S.loc[q - 1 - RX * RY];
            c[3] = S.loc[q - RX * RY];
            c[4] = S.loc[q - 1 - RX];
            c[5] = S.loc[q - RX];
            c[6] = S.loc[q - 1];
            c[7] = S.loc[q];
            c[8] = S.loc[q + 1];
            c[9] = S.loc[q + RX];
            c[10] = S.loc[q + 1 + RX];
            c[11] = S.loc[q + RX * RY];
            c[12] = S.loc[q + 1 + RX * RY];
            c[13] = S.loc[q + RX + RX * RY];
            c[14] = S.loc[q + 1 + RX + RX * RY];
            const uint32_t cg = code_of_closed<3>(c);
            const uint32_t cf = S.cf[lane + TX * r];
            if (cg == cf) continue;
            ++nd;
            // the targets of the correction's rule, as box positions
            const uint32_t asc_f = cf & 15u, asc_g = cg & 15u, desc_f = cf >> 4, desc_g = cg >> 4;
            if (asc_g != asc_f) {
                const int tq = asc_g == kSelf ? q : q + box_offset((int)asc_g);
                atomicOr(&S.tb[tq >> 5], 1u << (tq & 31));
            }
            if (desc_g != desc_f) {
                const int tq = desc_f == kSelf ? q : q + box_offset((int)desc_f);
                atomicOr(&S.tb[tq >> 5], 1u << (tq & 31));
            }
            atomicOr(&S.w[p ^ 1u][r], 1u << lane);  // a distorted vertex stays in the worklist
        }
        nd = __reduce_add_sync(kFull, nd);
        if (lane == 0 && nd) atomicAdd(&S.n_dist[p], nd);
        __syncthreads();
        if (S.n_dist[p] == 0) break;
        ++sweeps;
        // Eq. 1 once per distinct target; a changed target adds its closed
        // neighbourhood (own vertices only) to the next worklist.  This
        // sweep's worklist and the other parity's counters are cleared for
        // the sweep after next.
        uint32_t nc = 0;
        for (int wq = (int)tid; wq < TW; wq += kThreads) {
            uint32_t bits = S.tb[wq];
            S.tb[wq] = 0u;
            while (bits) {
                const int q = wq * 32 + (__ffs(bits) - 1);
                bits &= bits - 1u;
                float h;
                if (!edit_value(S.loc[q], floor_bound(__ldg(&F.f[global_of(q)]), F.xi), F.rule, h)) continue;
                S.loc[q] = h;
                atomicOr(&S.ed[wq], 1u << (q & 31));
                ++nc;
                const int bx = q % RX, by = (q / RX) % RY, bz = q / (RX * RY);
                mark_own(S.w[p ^ 1u], bx, by, bz);
                for (int s = 0; s < 14; ++s) {
                    int dx, dy, dz;
                    slot_delta(3, s, dx, dy, dz);
                    mark_own(S.w[p ^ 1u], bx + dx, by + dy, bz + dz);
                }
            }
        }
        for (int r = (int)tid; r < IW; r += kThreads) S.w[p][r] = 0u;
        if (tid == 0) {
            S.n_dist[p ^ 1u] = 0;
            S.n_changed[p ^ 1u] = 0;
        }
        nc = __reduce_add_sync(kFull, nc);
        if (lane == 0 && nc) atomicAdd(&S.n_changed[p], nc);
        __syncthreads();
        if (S.n_changed[p] == 0) break;
    }
    // propose every value this run decreased (all below g^k) to the merge
    for (int wq = (int)tid; wq < TW; wq += kThreads) {
        uint32_t bits = S.ed[wq];
        while (bits) {
            const int q = wq * 32 + (__ffs(bits) - 1);
            bits &= bits - 1u;
            const size_t v = global_of(q);
            atomicMin(&P.prop[v], tkey(S.loc[q]));
            red_or(&P.changed[v >> 5], 1u << (v & 31u));
        }
    }
    __syncthreads();
    return sweeps;
}

__global__ void __launch_bounds__(kThreads, kMinBlocks) k_relaxed(__grid_constant__ const Problem P) {
    extern __shared__ __align__(16) float smem[];
    const FieldView &F = P.F;
    const GridDev &G = F.G;
    Ctrl *C = P.ctrl;
    __shared__ uint32_t sm[40];
    __shared__ uint32_t s_t;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    const bool leader = gtid == 0;
    if (leader) C->t_start = global_ns();

    // ---- sweep 0: codes of f with their certification, g = fhat, bound check
    uint32_t unused = 0;
    first_tiled<false>(F, &P.log[0].tile_next, smem, &C->error, unused);
    bool ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
    if (leader) C->t_codes = global_ns();
    uint32_t k = 0;
    while (ok) {
        // ---- detection: active tiles.  Iteration 0 examines every
        // uncertified vertex; later ones the worklist (the closed
        // neighbourhoods of the values the last merge decreased, and the
        // vertices distorted before) -- any other vertex keeps its code.
        uint32_t seen = 0, nd = 0;
        uint32_t *wnext = P.wl[(k + 1) & 1u];
        auto detect = [&](bool h1, uint32_t v1, bool h2, uint32_t v2) {
            float a[15], b[15];
            gather_closed<3>(F.g, G, h1, v1, a);
            gather_closed<3>(F.g, G, h2, v2, b);
            const uint32_t c1 = h1 ? code_of_closed<3>(a) : 0u, c2 = h2 ? code_of_closed<3>(b) : 0u;
            const bool d1 = h1 && c1 != __ldg(&F.codes_f[v1]);
            const bool d2 = h2 && c2 != __ldg(&F.codes_f[v2]);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const bool d = e ? d2 : d1;
                if (!d) continue;
                ++nd;
                const uint32_t v = e ? v2 : v1;
                red_or(&wnext[v >> 5], 1u << (v & 31u));
                uint32_t x, y, z;
                coords_of(G, v, x, y, z);
                const uint32_t tt = x / TX + P.ntx * (y / TY + P.nty * (z / TZ));
                red_or(&P.active[tt >> 5], 1u << (tt & 31u));
            }
        };
        if (k == 0) walk_bits_pairs<false>(F.ub, nullptr, G, seen, detect);
        else walk_bits_pairs<true>(P.wl[k & 1u], F.ub, G, seen, detect);
        warp_add(nd, &P.log[k].distorted);
        ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
        if (!ok) break;
        if (leader) P.log[k].t_detect = global_ns();
        const uint32_t m = ld_relaxed(&P.log[k].distorted);
        if (m == 0) {
            if (leader) { C->status = MSZ_OK; C->sweeps = k; }
            break;
        }
        if (k >= P.max_iters) {
            if (leader) { C->status = MSZ_ERR_MAX_SWEEPS; C->sweeps = k; C->left = m; }
            break;
        }
        // ---- local sweeps of the active tiles on copies of g^k
        {
            TileSmem &S = *reinterpret_cast<TileSmem *>(smem);
            uint32_t runs = 0, lsw = 0;
            for (;;) {
                __syncthreads();
                if (threadIdx.x == 0) s_t = atomicAdd(&P.log[k + 1].tile_next, 1u);
                __syncthreads();
                const uint32_t t = s_t;
                if (t >= P.ntiles) break;
                if (!((ld_relaxed(&P.active[t >> 5]) >> (t & 31u)) & 1u)) continue;
                lsw += run_tile(P, t, S);
                ++runs;
            }
            if (threadIdx.x == 0) {
                if (runs) atomicAdd(&P.log[k].worklist, runs);
                if (lsw) atomicAdd(&P.log[k].targets, lsw);
            }
        }
        ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
        if (!ok) break;
        // ---- merge: the proposals become g^(k+1); the active tiles are cleared
        {
            uint32_t decreased = 0, seen2 = 0;
            walk_bits<true>(P.changed, nullptr, G, seen2, [&](bool has, uint32_t v) {
                if (!has) return;
                const uint32_t key = P.prop[v];
                P.prop[v] = 0xffffffffu;
                F.g[v] = tval(key);
                red_or(&F.eb[v >> 5], 1u << (v & 31u));
                mark_closed<3>(G, v, P.wl[(k + 1) & 1u]);
                ++decreased;
            });
            warp_add(decreased, &P.log[k].changed);
            for (uint32_t w = gtid; w < (P.ntiles + 31) / 32; w += stride) P.active[w] = 0u;
        }
        ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
        if (!ok) break;
        if (leader) P.log[k].t_edit = global_ns();
        if (ld_relaxed(&P.log[k].changed) == 0) {
            if (leader) { C->status = MSZ_STUCK; C->sweeps = k; C->left = m; }
            break;
        }
        k += 1;
    }
    if (!ok) return;

    // ---- edit list: every vertex of the edited bitmap, ascending index
    const uint32_t W = G.words;
    const uint32_t per = (W + gridDim.x - 1) / gridDim.x;
    const uint32_t w0 = min(blockIdx.x * per, W), w1 = min(w0 + per, W);
    uint32_t cnt = 0, unc = 0;
    for (uint32_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        cnt += __popc(F.eb[w]);
        unc += __popc(F.ub[w]);
    }
    warp_add(unc, &C->uncertified);
    uint32_t tot;
    block_exclusive_scan(cnt, sm, tot);
    if (threadIdx.x == 0) P.bsum[blockIdx.x] = tot;
    if (!grid_barrier(&C->bar_count, &C->bar_gen, &C->error)) return;
    uint32_t pre = 0, all = 0;
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const uint32_t s = ld_relaxed(&P.bsum[b]);
        all += s;
        if (b < blockIdx.x) pre += s;
    }
    uint32_t prefix;
    block_exclusive_scan(pre, sm, prefix);
    block_exclusive_scan(all, sm, all);
    if (leader) C->edit_count = all;
    for (uint32_t r = w0; r < w1; r += blockDim.x) {
        const uint32_t w = r + threadIdx.x;
        const uint32_t word = w < w1 ? F.eb[w] : 0u;
        uint32_t rt;
        const uint32_t ex = block_exclusive_scan((uint32_t)__popc(word), sm, rt);
        unsigned long long pos = (unsigned long long)prefix + ex;
        uint32_t bits = word;
        while (bits) {
            const uint32_t b = (uint32_t)(__ffs(bits) - 1);
            bits &= bits - 1;
            const uint32_t i = w * 32u + b;
            if (pos < P.edit_cap) {
                P.edit_idx[pos] = i;
                P.edit_delta[pos] = __fsub_rn(F.g[i], __ldg(&F.fhat[i]));
            }
            ++pos;
        }
        prefix += rt;
    }
    if (!grid_barrier(&C->bar_count, &C->bar_gen, &C->error)) return;
    if (leader) C->t_end = global_ns();
}

std::mutex g_mu;

msz_status relaxed_blocks(const DeviceInfo &d, int &blocks) {
    static int cache[64];
    std::lock_guard<std::mutex> lk(g_mu);
    const size_t sm = tile::kRingBytes;
    // the attribute belongs to the current context, so it is set on every
    // call (a context re-created after cudaDeviceReset starts without it);
    // the occupancy it allows is a property of the device and is cached
    if (cudaFuncSetAttribute(k_relaxed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return MSZ_ERR_CUDA;
    if (!cache[d.device]) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_relaxed, kThreads, sm) != cudaSuccess)
            return MSZ_ERR_CUDA;
        if (per < 1) return MSZ_ERR_UNSUPPORTED;
        int b = per * d.sms;
        if (b > (int)kMaxBlocks) b = (int)kMaxBlocks;
        cache[d.device] = b;
    }
    blocks = cache[d.device];
    return MSZ_OK;
}

// Workspace: the correction's layout, then the proposals (4 bytes per
// vertex) and a second worklist bitmap.
size_t relaxed_bytes(const GridDev &G, size_t &prop_off, size_t &wl_off) {
    const Layout L = layout_for(G.n);
    prop_off = L.total;
    wl_off = prop_off + align_up((size_t)G.n * 4);
    return wl_off + align_up((size_t)G.words * 4);
}

}  // namespace relaxed
}  // namespace msz

using namespace msz;
using namespace msz::relaxed;

extern "C" size_t msz_relaxed_workspace_size(msz_grid grid) {
    GridDev G;
    if (grid.ndim != 3 || make_grid(grid, G) != MSZ_OK) return 0;
    size_t off, woff;
    return relaxed_bytes(G, off, woff);
}

extern "C" msz_status msz_correct_relaxed(const float *d_f, const float *d_fhat, float xi, msz_grid grid,
                                          float *d_out, uint32_t *d_edit_idx, float *d_edit_delta,
                                          int64_t edit_capacity, int64_t *h_edit_count, const msz_options *opt,
                                          msz_stats *h_stats, void *d_workspace, size_t workspace_bytes,
                                          msz_stream_t stream) {
    if (!d_f || !d_fhat || !d_out || !h_edit_count) return MSZ_ERR_INVALID_ARG;
    if (edit_capacity < 0 || (edit_capacity > 0 && (!d_edit_idx || !d_edit_delta))) return MSZ_ERR_INVALID_ARG;
    if (!(xi >= 0.0f) || isinf(xi)) return MSZ_ERR_INVALID_ARG;
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    if (grid.ndim != 3) return MSZ_ERR_INVALID_ARG;
    msz_options o{};
    if (opt) o = *opt;
    if (o.rule != MSZ_RULE_HALVE && o.rule != MSZ_RULE_SNAP) return MSZ_ERR_INVALID_ARG;
    if (o.d_g_init || o.test_fault || o.max_sweeps > MSZ_MAX_SWEEPS_LIMIT || o.log_capacity < 0 || o.tile_z < 0 ||
        o.tile_z > 1024 || o.local_cap < 0 || (o.log_capacity > 0 && !o.h_sweep_log))
        return MSZ_ERR_INVALID_ARG;
    size_t prop_off, wl_off;
    const size_t need = relaxed_bytes(G, prop_off, wl_off);
    if (!d_workspace || workspace_bytes < need) return MSZ_ERR_WORKSPACE;
    if ((uintptr_t)d_workspace % kAlign) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const Layout L = layout_for(G.n);
    char *ws = (char *)d_workspace;
    Problem P{};
    FieldView &F = P.F;
    F.G = G;
    F.f = d_f;
    F.fhat = d_fhat;
    F.ginit = nullptr;
    F.g = d_out;
    F.codes_f = (uint8_t *)(ws + L.codes);
    F.tb = (uint32_t *)(ws + L.tb);
    F.dm[0] = (uint32_t *)(ws + L.d0);
    F.dm[1] = (uint32_t *)(ws + L.d1);
    F.eb = (uint32_t *)(ws + L.eb);
    F.ub = (uint32_t *)(ws + L.ub);
    F.xi = xi;
    F.two_xi = 2.0f * xi;
    F.rule = o.rule;
    F.tile_z = o.tile_z > 0 ? (uint32_t)o.tile_z : kTileZ;
    P.ctrl = (Ctrl *)(ws + L.ctrl);
    P.log = (SweepRec *)(ws + L.log);
    P.bsum = (uint32_t *)(ws + L.bsum);
    P.prop = (uint32_t *)(ws + prop_off);
    P.active = (uint32_t *)(ws + L.d0);   // one bit per tile
    P.changed = (uint32_t *)(ws + L.tb);  // one bit per vertex
    P.wl[0] = (uint32_t *)(ws + L.d1);
    P.wl[1] = (uint32_t *)(ws + wl_off);
    P.ntx = (G.nx + TX - 1) / TX;
    P.nty = (G.ny + TY - 1) / TY;
    P.ntz = (G.nz + TZ - 1) / TZ;
    P.ntiles = P.ntx * P.nty * P.ntz;
    P.max_iters = o.max_sweeps <= 0 ? (uint32_t)MSZ_MAX_SWEEPS_LIMIT : (uint32_t)o.max_sweeps;
    P.local_cap = o.local_cap <= 0 ? 65536u : (uint32_t)o.local_cap;
    P.edit_idx = d_edit_idx;
    P.edit_delta = d_edit_delta;
    P.edit_cap = (unsigned long long)edit_capacity;

    if (cudaMemsetAsync(ws, 0, L.zero_bytes, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaMemsetAsync(P.prop, 0xff, (size_t)G.n * 4, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaMemsetAsync(P.wl[1], 0, (size_t)G.words * 4, s) != cudaSuccess) return MSZ_ERR_CUDA;
    int blocks = 0;
    if ((st = relaxed_blocks(dev, blocks)) != MSZ_OK) return st;
    void *args[] = {(void *)&P};
    if (cudaLaunchCooperativeKernel((const void *)k_relaxed, dim3(blocks), dim3(kThreads), args, tile::kRingBytes,
                                    s) != cudaSuccess)
        return MSZ_ERR_CUDA;
    Ctrl hc;
    if (cudaMemcpyAsync(&hc, P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (hc.error & kErrInput) return MSZ_ERR_INPUT_BOUND;
    if (hc.error & kErrTimeout) return MSZ_ERR_TIMEOUT;
    *h_edit_count = (int64_t)hc.edit_count;
    // per-iteration records: [tile runs, distorted, local sweeps, decreased values]
    const int64_t nrec = (int64_t)hc.sweeps + 1;
    int64_t runs = 0, lsw = 0, first = 0;
    SweepRec tmp[256];
    for (int64_t b = 0; b < nrec; b += 256) {
        const int64_t c = nrec - b < 256 ? nrec - b : 256;
        if (cudaMemcpy(tmp, P.log + b, (size_t)c * sizeof(SweepRec), cudaMemcpyDeviceToHost) != cudaSuccess)
            return MSZ_ERR_CUDA;
        for (int64_t q = 0; q < c; ++q) {
            if (b + q == 0) first = tmp[q].distorted;
            runs += tmp[q].worklist;
            lsw += tmp[q].targets;
            if (b + q < o.log_capacity) {
                o.h_sweep_log[4 * (b + q) + 0] = tmp[q].worklist;
                o.h_sweep_log[4 * (b + q) + 1] = tmp[q].distorted;
                o.h_sweep_log[4 * (b + q) + 2] = tmp[q].targets;
                o.h_sweep_log[4 * (b + q) + 3] = tmp[q].changed;
                if (o.h_timeline) {
                    const unsigned long long td = tmp[q].t_detect, te = tmp[q].t_edit;
                    o.h_timeline[2 * (b + q) + 0] = td ? (int64_t)(td - hc.t_start) : -1;
                    o.h_timeline[2 * (b + q) + 1] = te ? (int64_t)(te - hc.t_start) : -1;
                }
            }
        }
    }
    if (h_stats) {
        memset(h_stats, 0, sizeof *h_stats);
        h_stats->sweeps = hc.sweeps;
        h_stats->edited = (int64_t)hc.edit_count;
        h_stats->first_distorted = first;
        h_stats->left = hc.left;
        h_stats->local_sweeps = lsw;
        h_stats->tile_runs = runs;
        h_stats->kernel_ns = hc.t_end > hc.t_start ? (int64_t)(hc.t_end - hc.t_start) : 0;
        h_stats->codes_ns = hc.t_codes > hc.t_start ? (int64_t)(hc.t_codes - hc.t_start) : 0;
        h_stats->uncertified = hc.uncertified;
    }
    const msz_status loop = (msz_status)hc.status;
    if (loop == MSZ_OK && (int64_t)hc.edit_count > edit_capacity) return MSZ_ERR_CAPACITY;
    return loop;
}
