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
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_tile.cuh"
#include "msz_workspace.h"

namespace msz {

constexpr int kThreads = tile::THREADS;  // 256 per block of the persistent kernel
constexpr uint32_t kTileZ = 32;          // planes per tile of a whole-grid pass
#ifndef MSZ_MIN_BLOCKS
#define MSZ_MIN_BLOCKS 3
#endif
constexpr int kMinBlocks = MSZ_MIN_BLOCKS;  // resident blocks per SM the register budget aims at
constexpr uint32_t kDenseFactor = 6;        // worklist estimate: 6 x distorted vertices
constexpr int kDenseWord = 6;               // set bits from which a bitmap word is walked by the whole warp

struct Problem {
    GridDev G;
    const float *f;
    const float *fhat;
    const float *ginit;
    float *g;
    uint8_t *codes_f;
    uint32_t *tb;      // targets of the current sweep
    uint32_t *dm[2];   // worklist of a sweep, by sweep parity
    uint32_t *eb;      // edited vertices
    uint32_t *ub;      // uncertified vertices: the only ones that can ever be distorted
    Ctrl *ctrl;
    SweepRec *log;
    uint32_t *bsum;
    uint32_t *edit_idx;
    float *edit_delta;
    unsigned long long edit_cap;
    float xi;
    float two_xi;      // 2 xi rounded up: the certification margin
    int rule;
    uint32_t max_sweeps;
    long long dense_min;  // < 0: never scan densely after sweep 0
};

// Where a detection phase records: the targets (P.tb) and the worklist of the
// next sweep (dnext); distorted vertices are counted per thread and added to
// the sweep's record when the phase ends.
struct Emitter {
    uint32_t *dnext;
    uint32_t distorted;
};

// Warp-collective: vertex v (valid lanes) with codes cf in f and cg in g; a
// distorted vertex marks its targets and, unless the caller marks whole words
// itself (self_marked), itself for the next worklist.
__device__ __forceinline__ bool report(const Problem &P, Emitter &E, bool valid, uint32_t v, uint32_t cf,
                                       uint32_t cg, bool self_marked = false) {
    const bool dist = valid && cf != cg;
    if (!__any_sync(kFull, dist)) return false;
    if (dist) {
        uint32_t t0, t1;
        const int nt = targets_of(P.G, v, (uint8_t)cf, (uint8_t)cg, t0, t1);
        red_or(&P.tb[t0 >> 5], 1u << (t0 & 31u));
        if (nt > 1) red_or(&P.tb[t1 >> 5], 1u << (t1 & 31u));
        if (!self_marked) red_or(&E.dnext[v >> 5], 1u << (v & 31u));
        E.distorted += 1;
    }
    return dist;
}

// Warp-collective walk over the set bits of a bitmap: each warp takes 32
// consecutive words (1024 vertices) at a time, grid-stride.  CLEAR zeroes the
// visited words; `seen` counts their set bits; a non-null filter restricts the
// calls to the vertices also set there.  fn(valid, v) runs once per round
// with one vertex per lane.
template <bool CLEAR, class F>
__device__ __forceinline__ void walk_bits(uint32_t *bm, const uint32_t *filter, const GridDev &G, uint32_t &seen,
                                          F &&fn) {
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t base = gw * 32u; base < G.words; base += nw * 32u) {
        const uint32_t wi = base + lane;
        uint32_t bits = 0;
        if (wi < G.words) {
            bits = bm[wi];
            if (CLEAR && bits) bm[wi] = 0u;
            seen += (uint32_t)__popc(bits);
            if (filter && bits) bits &= filter[wi];
        }
        // words with many set bits: the whole warp takes one word at a time,
        // lane l on vertex 32*word + l, so neighbour loads coalesce
        const bool dense = __popc(bits) >= kDenseWord;
        uint32_t dm = __ballot_sync(kFull, dense);
        while (dm) {
            const int j = __ffs(dm) - 1;
            dm &= dm - 1u;
            const uint32_t word = __shfl_sync(kFull, bits, j);
            fn(((word >> lane) & 1u) != 0u, (base + (uint32_t)j) * 32u + lane);
        }
        if (dense) bits = 0u;
        // the remaining sparse words: each lane walks its own word's bits
        while (__any_sync(kFull, bits != 0u)) {
            const bool has = bits != 0u;
            uint32_t v = 0;
            if (has) {
                v = wi * 32u + (uint32_t)(__ffs(bits) - 1);
                bits &= bits - 1u;
            }
            fn(has, v);
        }
    }
}

// Detection of one vertex in the current g (warp-collective).
template <int NDIM>
__device__ __forceinline__ void detect_vertex(const Problem &P, Emitter &E, bool has, uint32_t v) {
    uint32_t cf = 0, cg = 0;
    if (has) {
        uint32_t x, y, z;
        coords_of(P.G, v, x, y, z);
        cg = code_global<NDIM>(P.g, P.G, v, x, y, z);
        cf = __ldg(&P.codes_f[v]);
    }
    report(P, E, has, v, cf, cg);
}

// ------------------------------------------------ generic (2D) codes of f
template <int NDIM>
__device__ void first_generic(const Problem &P) {
    const GridDev &G = P.G;
    const uint32_t lane = lane_id();
    const uint32_t stride = gridDim.x * blockDim.x;
    bool bad = false;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < G.n; base += stride) {
        const uint32_t i = base + lane;
        const bool valid = i < G.n;
        bool differs = false, uncert = false;
        if (valid) {
            uint32_t x, y, z;
            coords_of(G, i, x, y, z);
            const float fi = P.f[i], fh = P.fhat[i];
            const float gs = P.ginit ? P.ginit[i] : fh;
            const float L = floor_bound(fi, P.xi), U = ceil_bound(fi, P.xi);
            bad = bad || !(isfinite(fi) && isfinite(fh) && fh >= L && fh <= U);
            if (P.ginit) {
                bad = bad || !(isfinite(gs) && gs >= L && gs <= U);
                differs = __float_as_uint(gs) != __float_as_uint(fh);
            }
            bool cert;
            P.codes_f[i] = code_global_cert<NDIM>(P.f, G, i, x, y, z, P.two_xi, cert);
            uncert = !cert;
            P.g[i] = gs;
        }
        // base is a multiple of 32: this warp owns whole bitmap words
        const uint32_t um = __ballot_sync(kFull, uncert);
        if (lane == 0) P.ub[base >> 5] = um;
        if (P.ginit) {
            const uint32_t m = __ballot_sync(kFull, differs);
            if (lane == 0 && m) P.eb[base >> 5] = m;
        }
    }
    if (bad) atomicOr(&P.ctrl->error, kErrInput);
}

// ------------------------------------------------ tiled (3D) codes of f
// Codes of f with their certification, g = start value, bound check.
__device__ void first_tiled(const Problem &P, uint32_t *tile_next, float *smem) {
    using namespace tile;
    const GridDev &G = P.G;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const TileGeom tg = tile_geom(G.nx, G.ny, G.nz, kTileZ);
    __shared__ uint32_t s_tile;
    bool bad = false;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_tile = atomicAdd(tile_next, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= tg.count) break;
        const uint32_t txi = t % tg.tx, tyi = (t / tg.tx) % tg.ty, tzi = t / (tg.tx * tg.ty);
        const int x0 = (int)(txi * BX), y0 = (int)(tyi * BY);
        const int zb = (int)(tzi * tg.bz);
        const int ze = min(zb + (int)tg.bz, (int)G.nz);

        // copy slots of this thread: element e = tid + j*THREADS of the
        // ROWS x LOADW staged region; bit j of inm / ownm = in the grid / in
        // the tile interior.
        uint32_t inm = 0, ownm = 0;
#pragma unroll
        for (int j = 0; j < PER_THREAD; ++j) {
            const int e = (int)tid + j * THREADS;
            const int r = e / LOADW, c = e - r * LOADW;
            const int gx = x0 - 1 + c, gy = y0 - 1 + r;
            const bool in = e < ELEMS && gx >= 0 && gx < (int)G.nx && gy >= 0 && gy < (int)G.ny;
            inm |= (uint32_t)in << j;
            ownm |= (uint32_t)(in && r >= 1 && r <= BY && c >= 1 && c <= BX) << j;
        }
        const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
        const int gbase = (y0 - 1) * (int)G.nx + (x0 - 1);  // plane offset of staged element 0
        const float qnan = __int_as_float(0x7fffffff);
        // Positions outside the grid hold NaN: a NaN candidate never wins a
        // comparison, so the codes need no domain masks (it only withholds the
        // certification of vertices on the grid boundary, which is safe).
#pragma unroll
        for (int j = 0; j < PER_THREAD; ++j) {
            const int e = (int)tid + j * THREADS;
            if (e >= ELEMS || (inm >> j & 1u)) continue;
            const int r = e / LOADW, c = e - r * LOADW;
            for (int sl = 0; sl < NSLOT; ++sl) smem[sl * SLOT + r * PW + c + 3] = qnan;
        }
        // asynchronous copy of plane p (f over the staged region, fhat over the
        // owned region) into its ring slot; planes outside the grid become NaN
        auto issue = [&](int p) {
            if (p >= 0 && p <= ze) {
                const int slot = (p - zb + 1) % NSLOT;
                const bool inside = p < (int)G.nz;
                const size_t pb = (size_t)p * G.nxy;
#pragma unroll
                for (int j = 0; j < PER_THREAD; ++j) {
                    if (!(inm >> j & 1u)) continue;
                    const int e = (int)tid + j * THREADS;
                    const int r = e / LOADW, c = e - r * LOADW;
                    const uint32_t so = (uint32_t)(slot * SLOT + r * PW + c + 3);
                    if (!inside) {
                        smem[so] = qnan;
                        continue;
                    }
                    const size_t gi = pb + (size_t)(gbase + r * (int)G.nx + c);
                    cp_async4(sbase + 4u * so, P.f + gi);
                    if (ownm >> j & 1u) cp_async4(sbase + 4u * (so + (uint32_t)PLANE), P.fhat + gi);
                }
            } else if (p < 0) {
                const int slot = (p - zb + 1) % NSLOT;
#pragma unroll
                for (int j = 0; j < PER_THREAD; ++j) {
                    if (!(inm >> j & 1u)) continue;
                    const int e = (int)tid + j * THREADS;
                    const int r = e / LOADW, c = e - r * LOADW;
                    smem[slot * SLOT + r * PW + c + 3] = qnan;
                }
            }
            cp_async_commit();
        };
        // owned vertices of plane p: bound check and g = start value
        auto own = [&](int p) {
            const int slot = (p - zb + 1) % NSLOT;
            const size_t pb = (size_t)p * G.nxy;
#pragma unroll
            for (int j = 0; j < PER_THREAD; ++j) {
                if (!(ownm >> j & 1u)) continue;
                const int e = (int)tid + j * THREADS;
                const int r = e / LOADW, c = e - r * LOADW;
                const int so = slot * SLOT + r * PW + c + 3;
                const float fi = smem[so], fh = smem[so + PLANE];
                const size_t gi = pb + (size_t)(gbase + r * (int)G.nx + c);
                const float gs = P.ginit ? P.ginit[gi] : fh;
                const float L = floor_bound(fi, P.xi), U = ceil_bound(fi, P.xi);
                bool ok = isfinite(fi) && isfinite(fh) && fh >= L && fh <= U;
                if (P.ginit) {
                    ok = ok && isfinite(gs) && gs >= L && gs <= U;
                    if (__float_as_uint(fh) != __float_as_uint(gs)) red_or(&P.eb[gi >> 5], 1u << (gi & 31u));
                }
                bad = bad || !ok;
                P.g[gi] = gs;
            }
        };
        issue(zb - 1);
        issue(zb);
        issue(zb + 1);
        issue(zb + 2);
        const int y = y0 + (int)warp, r = (int)warp + 1;
        const int xl = x0 + 4 * (int)lane;
        for (int z = zb; z < ze; ++z) {
            cp_async_wait<1>();  // planes up to z+1 of this thread have landed (z+2 may be in flight)
            __syncthreads();     // ... of every thread; the slot of z-2 is free
            issue(z + 3);
            own(z);
            if (y >= (int)G.ny) continue;
            auto plane = [&](int p) { return smem + ((p - zb + 1) % NSLOT) * SLOT; };
            uint32_t cf[4], cert;
            tile::codes4_cert(plane(z - 1), plane(z), plane(z + 1), r, lane, P.two_xi, cf, cert);
            const size_t rowbase = (size_t)z * G.nxy + (size_t)y * G.nx;
            const size_t i0 = rowbase + xl;
            if (xl + 3 < (int)G.nx && (i0 & 3) == 0) {
                *reinterpret_cast<uint32_t *>(P.codes_f + i0) = cf[0] | cf[1] << 8 | cf[2] << 16 | cf[3] << 24;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (xl + e < (int)G.nx) P.codes_f[i0 + e] = (uint8_t)cf[e];
            }
            // uncertified bits of this lane's vertices (outside the grid: 0)
            uint32_t nib = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) nib |= (uint32_t)(xl + e < (int)G.nx && !((cert >> e) & 1u)) << e;
            const bool words_ok = ((rowbase + (size_t)x0) & 31u) == 0 && x0 + BX <= (int)G.nx;
            if (words_ok) {
                // the warp's 128 vertices are 4 whole bitmap words
                uint32_t w = nib << (4u * (lane & 7u));
                w |= __shfl_xor_sync(kFull, w, 1);
                w |= __shfl_xor_sync(kFull, w, 2);
                w |= __shfl_xor_sync(kFull, w, 4);
                if ((lane & 7u) == 0) P.ub[(i0) >> 5] = w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if ((nib >> e) & 1u) red_or(&P.ub[(i0 + e) >> 5], 1u << ((i0 + e) & 31u));
            }
        }
        cp_async_wait<0>();
    }
    if (bad) atomicOr(&P.ctrl->error, kErrInput);
}

// ------------------------------------------------------ the persistent kernel
template <int NDIM>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_correct(__grid_constant__ const Problem P) {
    extern __shared__ __align__(16) float smem[];
    const GridDev &G = P.G;
    Ctrl *C = P.ctrl;
    __shared__ uint32_t sm[40];
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    const bool leader = gtid == 0;
    if (leader) C->t_start = global_ns();

    // ---- sweep 0: codes of f with their certification, g = start, bound check
    if (NDIM == 3) first_tiled(P, &P.log[0].tile_next, smem);
    else first_generic<NDIM>(P);
    bool ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
    if (leader) C->t_codes = global_ns();
    // ---- detection of sweep 0: only uncertified vertices can be distorted
    if (ok) {
        Emitter E{P.dm[1], 0};
        uint32_t seen = 0;
        walk_bits<false>(P.ub, nullptr, G, seen, [&](bool has, uint32_t v) { detect_vertex<NDIM>(P, E, has, v); });
        warp_add(E.distorted, &P.log[0].distorted);
    }
    if (leader) {
        P.log[0].worklist = G.n;
        C->examined = G.n;
        C->dense_sweeps = 1;
    }
    ok = ok && grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
    if (leader) P.log[0].t_detect = global_ns();
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
            walk_bits<true>(P.tb, nullptr, G, nt, [&](bool, uint32_t) {});
            warp_add(nt, &P.log[k].targets);
            if (leader) { C->status = MSZ_ERR_MAX_SWEEPS; C->sweeps = k; C->left = m; }
            ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
            break;
        }
        const bool dense_next =
            P.dense_min >= 0 && (unsigned long long)m * kDenseFactor >= (unsigned long long)P.dense_min;
        // ---- edit phase of sweep k (Eq. 1), one application per distinct target
        {
            uint32_t *dnext = P.dm[(k + 1) & 1];
            uint32_t targets = 0, changed_here = 0;
            walk_bits<true>(P.tb, nullptr, G, targets, [&](bool has, uint32_t t) {
                if (!has) return;
                const float gt = P.g[t];
                const float L = floor_bound(__ldg(&P.f[t]), P.xi);
                float h;
                if (!edit_value(gt, L, P.rule, h)) return;
                P.g[t] = h;
                ++changed_here;
                red_or(&P.eb[t >> 5], 1u << (t & 31u));
                if (dense_next) return;
                red_or(&dnext[t >> 5], 1u << (t & 31u));
                uint32_t x, y, z;
                coords_of(G, t, x, y, z);
                constexpr int ns = NDIM == 2 ? 6 : 14;
#pragma unroll
                for (int s = 0; s < ns; ++s) {
                    if (!slot_in_domain(G, s, x, y, z)) continue;
                    const uint32_t j = (uint32_t)((int64_t)t + G.off[s]);
                    red_or(&dnext[j >> 5], 1u << (j & 31u));
                }
            });
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
        // ---- detection phase of sweep k + 1
        const uint32_t k1 = k + 1;
        Emitter E{P.dm[(k1 + 1) & 1], 0};
        uint32_t *dcur = P.dm[k1 & 1];
        uint32_t seen = 0;
        if (dense_next) {
            // whole grid: every uncertified vertex
            if (leader) {
                P.log[k1].worklist = G.n;
                C->examined += G.n;
                C->dense_sweeps += 1;
            }
            for (uint32_t w = gtid; w < G.words; w += stride) dcur[w] = 0;
            walk_bits<false>(P.ub, nullptr, G, seen, [&](bool has, uint32_t v) { detect_vertex<NDIM>(P, E, has, v); });
        } else {
            // the worklist, restricted to uncertified vertices
            walk_bits<true>(dcur, P.ub, G, seen, [&](bool has, uint32_t v) { detect_vertex<NDIM>(P, E, has, v); });
            warp_add(seen, &P.log[k1].worklist);
        }
        warp_add(E.distorted, &P.log[k1].distorted);
        ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
        if (leader) {
            P.log[k1].t_detect = global_ns();
            if (!dense_next) C->examined += P.log[k1].worklist;
        }
        k = k1;
    }
    if (!ok) return;

    // ---- edit list: every vertex of the edited bitmap, ascending index
    const uint32_t W = G.words;
    const uint32_t per = (W + gridDim.x - 1) / gridDim.x;
    const uint32_t w0 = min(blockIdx.x * per, W), w1 = min(w0 + per, W);
    uint32_t cnt = 0;
    for (uint32_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) cnt += __popc(P.eb[w]);
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
        const uint32_t word = w < w1 ? P.eb[w] : 0u;
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
                P.edit_delta[pos] = __fsub_rn(P.g[i], __ldg(&P.fhat[i]));
            }
            ++pos;
        }
        prefix += rt;
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

template <int NDIM>
static size_t correct_smem() { return NDIM == 3 ? tile::kRingBytes : 0; }

template <int NDIM>
static msz_status correct_blocks(const DeviceInfo &d, int &blocks) {
    static int cache[64];
    std::lock_guard<std::mutex> lk(g_mu);
    if (!cache[d.device]) {
        const size_t sm = correct_smem<NDIM>();
        if (sm > 48 * 1024 &&
            cudaFuncSetAttribute(k_correct<NDIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return MSZ_ERR_CUDA;
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_correct<NDIM>, kThreads, sm) != cudaSuccess)
            return MSZ_ERR_CUDA;
        if (per < 1) return MSZ_ERR_UNSUPPORTED;
        int b = per * d.sms;
        if (b > (int)kMaxBlocks) b = (int)kMaxBlocks;
        cache[d.device] = b;
    }
    blocks = cache[d.device];
    return MSZ_OK;
}

template <int NDIM>
static msz_status run_correct(Problem &P, const DeviceInfo &dev, cudaStream_t stream) {
    int blocks = 0;
    msz_status st = correct_blocks<NDIM>(dev, blocks);
    if (st != MSZ_OK) return st;
    void *args[] = {(void *)&P};
    if (cudaLaunchCooperativeKernel((const void *)k_correct<NDIM>, dim3(blocks), dim3(kThreads), args,
                                    correct_smem<NDIM>(), stream) != cudaSuccess)
        return MSZ_ERR_CUDA;
    return MSZ_OK;
}

}  // namespace msz

using namespace msz;

extern "C" size_t msz_workspace_size(msz_grid grid) {
    GridDev G;
    if (make_grid(grid, G) != MSZ_OK) return 0;
    return layout_for(G.n).total;
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

extern "C" msz_status msz_correct(const float *d_f, const float *d_fhat, float xi, msz_grid grid, float *d_out,
                                  uint32_t *d_edit_idx, float *d_edit_delta, int64_t edit_capacity,
                                  int64_t *h_edit_count, const msz_options *opt, msz_stats *h_stats,
                                  void *d_workspace, size_t workspace_bytes, msz_stream_t stream) {
    if (!d_f || !d_fhat || !d_out || !h_edit_count) return MSZ_ERR_INVALID_ARG;
    if (edit_capacity < 0 || (edit_capacity > 0 && (!d_edit_idx || !d_edit_delta))) return MSZ_ERR_INVALID_ARG;
    if (!(xi >= 0.0f) || isinf(xi)) return MSZ_ERR_INVALID_ARG;
    GridDev G;
    msz_status st = make_grid(grid, G);
    if (st != MSZ_OK) return st;
    msz_options o{};
    if (opt) o = *opt;
    if (o.rule != MSZ_RULE_HALVE && o.rule != MSZ_RULE_SNAP) return MSZ_ERR_INVALID_ARG;
    if (o.max_sweeps > MSZ_MAX_SWEEPS_LIMIT || o.dense_min_items < -1 || o.log_capacity < 0 ||
        (o.log_capacity > 0 && !o.h_sweep_log))
        return MSZ_ERR_INVALID_ARG;
    const Layout L = layout_for(G.n);
    if (!d_workspace || workspace_bytes < L.total) return MSZ_ERR_WORKSPACE;
    if ((uintptr_t)d_workspace % kAlign) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    if ((st = current_device(dev)) != MSZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    char *ws = (char *)d_workspace;
    Problem P{};
    P.G = G;
    P.f = d_f;
    P.fhat = d_fhat;
    P.ginit = o.d_g_init;
    P.g = d_out;
    P.codes_f = (uint8_t *)(ws + L.codes);
    P.tb = (uint32_t *)(ws + L.tb);
    P.dm[0] = (uint32_t *)(ws + L.d0);
    P.dm[1] = (uint32_t *)(ws + L.d1);
    P.eb = (uint32_t *)(ws + L.eb);
    P.ub = (uint32_t *)(ws + L.ub);
    P.ctrl = (Ctrl *)(ws + L.ctrl);
    P.log = (SweepRec *)(ws + L.log);
    P.bsum = (uint32_t *)(ws + L.bsum);
    P.edit_idx = d_edit_idx;
    P.edit_delta = d_edit_delta;
    P.edit_cap = (unsigned long long)edit_capacity;
    P.xi = xi;
    P.two_xi = 2.0f * xi;  // exact (power-of-two scaling), +inf on overflow
    P.rule = o.rule;
    P.max_sweeps = o.max_sweeps <= 0 ? (uint32_t)MSZ_MAX_SWEEPS_LIMIT : (uint32_t)o.max_sweeps;
    P.dense_min = o.dense_min_items == 0 ? (long long)(G.n / 16 > 0 ? G.n / 16 : 1) : (long long)o.dense_min_items;

    if (cudaMemsetAsync(ws, 0, L.zero_bytes, s) != cudaSuccess) return MSZ_ERR_CUDA;
    st = G.ndim == 3 ? run_correct<3>(P, dev, s) : run_correct<2>(P, dev, s);
    if (st != MSZ_OK) return st;
    Ctrl hc;
    if (cudaMemcpyAsync(&hc, P.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (hc.error & kErrInput) return MSZ_ERR_INPUT_BOUND;
    if (hc.error & kErrTimeout) return MSZ_ERR_TIMEOUT;
    *h_edit_count = (int64_t)hc.edit_count;
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
    if (h_stats) {
        SweepRec r0;
        if (cudaMemcpy(&r0, P.log, sizeof r0, cudaMemcpyDeviceToHost) != cudaSuccess) return MSZ_ERR_CUDA;
        h_stats->sweeps = hc.sweeps;
        h_stats->edits = (int64_t)hc.edits;
        h_stats->edited = (int64_t)hc.edit_count;
        h_stats->first_distorted = r0.distorted;
        h_stats->left = hc.left;
        h_stats->examined = (int64_t)hc.examined;
        h_stats->dense_sweeps = hc.dense_sweeps;
        h_stats->kernel_ns = hc.t_end > hc.t_start ? (int64_t)(hc.t_end - hc.t_start) : 0;
        h_stats->codes_ns = hc.t_codes > hc.t_start ? (int64_t)(hc.t_codes - hc.t_start) : 0;
    }
    const msz_status loop = (msz_status)hc.status;
    if (loop == MSZ_OK && (int64_t)hc.edit_count > edit_capacity) return MSZ_ERR_CAPACITY;
    return loop;
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
