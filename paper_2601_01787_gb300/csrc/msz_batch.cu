// msz_batch.cu -- many fields of uneven sizes corrected by one cooperative
// persistent launch (msz_correct_batch).
//
// The fields sit side by side in one virtual index space (field k owns
// vertices [base_k, base_k + n_k), bases aligned to 1024 vertices).  The
// workspace bitmaps and codes span that space; each field's FieldView holds
// windows into them, so the per-field phases of msz_phases.cuh run unchanged.
//   - codes pass: one tile queue over every field's tiles;
//   - every later phase walks the shared bitmaps; a set bit is mapped to its
//     field by binary search over the bases;
//   - each (sweep, field) pair gets its own record (worklist, distorted,
//     targets, changed), accumulated in shared memory per block;
//   - a field stops taking part once it is done (no distortion), stuck or
//     capped; the launch ends when every field has stopped;
//   - the edit list is split per field into the caller's arrays.
// Every field's sweeps are the same Jacobi sweeps as a separate msz_correct
// call, so its g, edit list and per-sweep records are identical.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_phases.cuh"
#include "msz_tile.cuh"
#include "msz_workspace.h"

namespace msz {
namespace {

constexpr int kThreads = tile::THREADS;
constexpr int kMinBlocksB = 3;
constexpr uint32_t kDenseFactorB = 6;
constexpr int kListRoundsB = 4;  // edit-list rounds whose loads are grouped
static_assert(kListRoundsB == 4, "the edit list's round group is written out for four rounds");
// a sweep keeps chunk flags when its worklist is bounded by the larger of
// this and 1/256 of the batch's vertices (the walks they spare read every
// bitmap word of every field)
constexpr unsigned long long kSparseWorklistB = 1ull << 19;

struct FieldDev {
    FieldView F;
    uint32_t base;       // first vertex in the shared index space (multiple of 1024)
    uint32_t tile_base;  // first tile in the shared tile queue
    uint32_t *edit_idx;
    float *edit_delta;
    unsigned long long edit_cap;
};

struct BatchRec {
    uint32_t worklist, distorted, targets, changed;
    uint32_t dense;  // the detection of this sweep scanned every uncertified vertex
    // field 0's record only: [0] the tile counter of a whole-field detection;
    // [1] / [2] device time (ns from the code pass's start, 0: none) at the
    // end of this sweep's detection / edit phase
    uint32_t pad[3];
};

// Nanoseconds since t0 for a timeline record (0 is kept for "none").
__device__ __forceinline__ uint32_t stamp_since(uint64_t t0) {
    const uint64_t d = global_ns() - t0;
    return d >= 0xffffffffull ? 0xffffffffu : d == 0 ? 1u : (uint32_t)d;
}

struct FieldRes {
    unsigned long long edit_count;
    uint32_t error;
    uint32_t uncertified;  // vertices the code pass could not certify
};

struct BatchProblem {
    const FieldDev *fields;
    uint32_t nfields;
    uint32_t ntiles;
    GridDev all;  // the shared index space (only n, words used)
    Ctrl *ctrl;
    BatchRec *log;  // [sweep][field]
    uint32_t *stb, *sdm[2];          // chunk flags of tb, dm[0], dm[1] (kept in sparse sweeps)
    uint32_t *cpre;                  // per chunk: its first edit's position in the shared order
    unsigned long long sparse_max;   // worklist bound of a sweep that keeps them
    FieldRes *res;
    uint32_t *bsum;
    uint32_t max_sweeps;
    long long dense_min;             // < 0: never scan whole fields after sweep 0; 0: a field scans
                                     // whole when 6 x its distorted >= its vertices; > 0: >= this
    uint32_t *tb, *dm[2], *eb, *ub;  // shared bitmaps (global words)
    const uint8_t *bfield;           // field of each 1024-vertex block
};

struct BatchLayout {
    size_t ctrl, fields, log, res, bsum, tb, d0, d1, eb, ub, stb, sd0, sd1, codes, bfield, cpre, total, zero_bytes;
};

BatchLayout batch_layout(uint32_t nfields, uint64_t ntot, uint32_t max_sweeps) {
    BatchLayout L{};
    const uint64_t words = ntot / 32;
    size_t o = 0;
    L.ctrl = o;   o = align_up(o + sizeof(Ctrl));
    L.res = o;    o = align_up(o + nfields * sizeof(FieldRes));
    L.log = o;    o = align_up(o + (size_t)(max_sweeps + 2) * nfields * sizeof(BatchRec));
    L.bsum = o;   o = align_up(o + kMaxBlocks * sizeof(uint32_t));
    L.tb = o;     o = align_up(o + words * 4);
    L.d0 = o;     o = align_up(o + words * 4);
    L.d1 = o;     o = align_up(o + words * 4);
    L.eb = o;     o = align_up(o + words * 4);
    L.ub = o;     o = align_up(o + words * 4);
    L.stb = o;    o = align_up(o + ntot / 1024 * 4);
    L.sd0 = o;    o = align_up(o + ntot / 1024 * 4);
    L.sd1 = o;    o = align_up(o + ntot / 1024 * 4);
    L.zero_bytes = o;
    L.fields = o; o = align_up(o + nfields * sizeof(FieldDev));
    L.codes = o;  o = align_up(o + ntot);
    L.bfield = o; o = align_up(o + ntot / 1024);
    L.cpre = o;   o = align_up(o + ntot / 1024 * 4);
    L.total = o;
    return L;
}

// Field of vertex v of the shared space: field bases are 1024-aligned, so one
// byte per 1024 vertices names it.
static_assert(MSZ_BATCH_MAX_FIELDS <= 256, "field indices are stored in one byte");
__device__ __forceinline__ uint32_t field_of(const uint8_t *bfield, uint32_t v) { return __ldg(&bfield[v >> 10]); }

// Field of a vertex (or tile) of the shared space: the last k with tab[k] <= v.
__device__ __forceinline__ uint32_t find_field(const uint32_t *tab, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;  // tab[lo] <= v < tab[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (tab[mid] <= v) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Block-local per-field counters, flushed to the (sweep, field) record.
__device__ __forceinline__ void flush_counts(uint32_t (*cnt)[4], uint32_t nf, BatchRec *rec) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nf * 4; i += blockDim.x) {
        const uint32_t k = i >> 2, c = i & 3;
        const uint32_t v = cnt[k][c];
        if (v) {
            uint32_t *dst = c == 0 ? &rec[k].worklist : c == 1 ? &rec[k].distorted : c == 2 ? &rec[k].targets
                                                                                        : &rec[k].changed;
            atomicAdd(dst, v);
            cnt[k][c] = 0;
        }
    }
    __syncthreads();
}

// A tile's field view, staged in shared memory by the whole block: the tile
// passes read its members many times a row, and global loads of them miss the
// L1 that the plane rings leave small.  Block-collective; the caller has
// synchronized the block since the last use of buf.
constexpr uint32_t kFieldWords = (uint32_t)(sizeof(FieldView) / 4);
static_assert(sizeof(FieldView) % 4 == 0 && alignof(FieldView) <= 16, "FieldView is copied as aligned words");
__device__ __forceinline__ void stage_field(uint32_t *buf, const FieldView &src) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(&src);
    for (uint32_t i = threadIdx.x; i < kFieldWords; i += blockDim.x) buf[i] = w[i];
    __syncthreads();
}

// Eq. 1 on target t of field F (HALVE or SNAP, the rules a batch takes)
// with its current value gt and f_t already loaded: as apply_target.
__device__ __forceinline__ bool edit_loaded(const FieldView &F, uint32_t t, float gt, float ft, bool dense_next,
                                            uint32_t *dnext, uint32_t *dsum) {
    float h;
    if (!edit_value(gt, floor_bound(ft, F.xi), F.rule, h)) return false;
    F.g[t] = h;
    red_or(&F.eb[t >> 5], 1u << (t & 31u));
    if (!dense_next) mark_closed<3>(F.G, t, dnext, dsum);
    return true;
}

// A field's view of shared-space chunk flags (null stays null): field bases
// are 1024-aligned, so a field-local vertex v has chunk (base >> 10) + (v >> 10).
__device__ __forceinline__ uint32_t *field_flags(uint32_t *flags, uint32_t base) {
    return flags ? flags + (base >> 10) : nullptr;
}

// walk_words_pairs over the chunks (32 words) whose flags are set, clearing
// the flags: the bits of word w are finish(w, fetch(w)), the next flagged
// chunk's words loaded before the current one is queued; chunk c belongs to
// warp c mod (warps of the grid), a warp reading 32 of its flags at once.
// rq: the warp's kRoundCap entries of shared memory.
template <class FE, class FI, class F>
__device__ __forceinline__ void walk_flagged_words(uint32_t *flags, const GridDev &G, FE &&fetch, FI &&finish,
                                                   uint32_t *rq, F &&fn) {
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t chunks = (G.words + 31u) / 32u;
    RoundQueue<true> Q{rq};
    for (uint32_t c0 = gw; c0 < chunks; c0 += 32u * nw) {
        const uint32_t mine = c0 + lane * nw;  // this lane's chunk of the round
        const bool set = mine < chunks && flags[mine] != 0u;
        if (set) flags[mine] = 0u;
        uint32_t marks = __ballot_sync(kFull, set);
        if (!marks) continue;
        uint32_t c = c0 + (uint32_t)(__ffs(marks) - 1) * nw;
        marks &= marks - 1u;
        uint32_t nxt = c * 32u + lane < G.words ? fetch(c * 32u + lane) : 0u;
        for (;;) {
            const uint32_t base = c * 32u;
            const uint32_t wi = base + lane;
            const uint32_t raw = nxt;
            const bool more = marks != 0u;
            if (more) {
                c = c0 + (uint32_t)(__ffs(marks) - 1) * nw;
                marks &= marks - 1u;
                nxt = c * 32u + lane < G.words ? fetch(c * 32u + lane) : 0u;
            }
            const uint32_t bits = wi < G.words ? finish(wi, raw) : 0u;
            Q.push_chunk(base, bits, fn);
            if (!more) break;
        }
    }
    Q.flush(fn);
}

// Detection of two vertices per lane of the shared index space (each may lie
// in a different field): the neighbour loads of both are issued before either
// code is formed; distorted vertices are counted per field in s_cnt[f][1].
// sums: the marks also set the chunk flags of the targets and of the next
// worklist.
template <class Alive>
__device__ __forceinline__ void detect_pair(const BatchProblem &P, const uint32_t *s_base, uint32_t nf,
                                            uint32_t (*s_cnt)[4], uint32_t next_parity, bool sums, Alive &&alive,
                                            bool h1, uint32_t v1, bool h2, uint32_t v2) {
    const uint32_t f1 = h1 ? field_of(P.bfield, v1) : 0u, f2 = h2 ? field_of(P.bfield, v2) : 0u;
    const bool l1 = h1 && alive(f1), l2 = h2 && alive(f2);
    const FieldView &F1 = P.fields[f1].F;
    const FieldView &F2 = P.fields[f2].F;
    const uint32_t i1 = l1 ? v1 - s_base[f1] : 0u, i2 = l2 ? v2 - s_base[f2] : 0u;
    float a[15], b[15];
    gather_closed<3>(F1.g, F1.G, l1, i1, a);
    gather_closed<3>(F2.g, F2.G, l2, i2, b);
    const uint32_t cf1 = l1 ? __ldg(&F1.codes_f[i1]) : 0u;
    const uint32_t cf2 = l2 ? __ldg(&F2.codes_f[i2]) : 0u;
    uint32_t *const dsum = sums ? P.sdm[next_parity] : nullptr, *const tsum = sums ? P.stb : nullptr;
    Emitter E1{F1.dm[next_parity], 0, field_flags(dsum, s_base[f1]), field_flags(tsum, s_base[f1])};
    report(F1, E1, l1, i1, cf1, code_of_closed<3>(a));
    Emitter E2{F2.dm[next_parity], 0, field_flags(dsum, s_base[f2]), field_flags(tsum, s_base[f2])};
    report(F2, E2, l2, i2, cf2, code_of_closed<3>(b));
    // distorted counts per field, aggregated over the warp's lanes of one field
    const uint32_t lane = lane_id();
    const uint32_t p1 = __match_any_sync(kFull, E1.distorted ? f1 : 0xffffffffu);
    if (E1.distorted && lane == (uint32_t)(__ffs(p1) - 1)) atomicAdd(&s_cnt[f1][1], (uint32_t)__popc(p1));
    const uint32_t p2 = __match_any_sync(kFull, E2.distorted ? f2 : 0xffffffffu);
    if (E2.distorted && lane == (uint32_t)(__ffs(p2) - 1)) atomicAdd(&s_cnt[f2][1], (uint32_t)__popc(p2));
}

// ---- sweep 0: codes of every field and the detection of sweep 0 over
// their uncertified vertices, one shared tile queue, as an ordinary launch
// of its own (its paired-row ring is the largest shared-memory user of the
// batch; the kernel boundary orders its writes before k_batch)
__global__ void __launch_bounds__(kThreads, kMinBlocksB) k_batch_codes(__grid_constant__ const BatchProblem P) {
    extern __shared__ __align__(16) float smem[];
    __shared__ uint32_t s_tile[MSZ_BATCH_MAX_FIELDS + 1];
    __shared__ uint32_t s_cnt[MSZ_BATCH_MAX_FIELDS][4];
    __shared__ uint32_t s_next;
    __shared__ __align__(16) uint32_t s_F[kFieldWords];  // the current tile's field view
    const FieldView &F = *reinterpret_cast<const FieldView *>(s_F);
    uint32_t staged = 0xffffffffu;                      // its field (block-uniform)
    const uint32_t nf = P.nfields;
    Ctrl *C = P.ctrl;
    for (uint32_t k = threadIdx.x; k <= nf; k += blockDim.x) s_tile[k] = k < nf ? P.fields[k].tile_base : P.ntiles;
    for (uint32_t i = threadIdx.x; i < nf * 4; i += blockDim.x) s_cnt[i >> 2][i & 3] = 0;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) C->t_start = global_ns();
    bool bad = false;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_next = atomicAdd(&C->flag, 1u);
        __syncthreads();
        const uint32_t t = s_next;
        if (t >= P.ntiles) break;
        const uint32_t k = find_field(s_tile, nf, t);
        if (k != staged) {
            stage_field(s_F, P.fields[k].F);
            staged = k;
        }
        const tile::TileGeom tg = tile::tile_geom(F.G.nx, F.G.ny, F.G.nz, F.tile_z);
        const uint32_t lt = t - s_tile[k];
        const uint32_t txi = lt % tg.tx, tyi = (lt / tg.tx) % tg.ty, tzi = lt / (tg.tx * tg.ty);
        const int zb = (int)(tzi * tg.bz);
        bool fb = false;
        uint32_t dist = 0;
        first_tile<true, true>(F, (int)(txi * tile::BX), (int)(tyi * tile::BY), zb,
                               min(zb + (int)tg.bz, (int)F.G.nz), smem, fb, dist);
        warp_add(dist, &s_cnt[k][1]);
        if (fb) atomicOr(&P.res[k].error, kErrInput);
        bad = bad || fb;
    }
    if (bad) atomicOr(&C->error, kErrInput);
    flush_counts(s_cnt, nf, P.log);
}

// ---- the later sweeps and the edit lists (cooperative, persistent)
__global__ void __launch_bounds__(kThreads, kMinBlocksB) k_batch(__grid_constant__ const BatchProblem P) {
    extern __shared__ __align__(16) float smem[];
    __shared__ uint32_t s_base[MSZ_BATCH_MAX_FIELDS + 1];
    __shared__ uint32_t s_tile[MSZ_BATCH_MAX_FIELDS + 1];
    __shared__ uint32_t s_cnt[MSZ_BATCH_MAX_FIELDS][4];
    __shared__ uint32_t s_alive[(MSZ_BATCH_MAX_FIELDS + 31) / 32];
    __shared__ uint32_t s_dense[(MSZ_BATCH_MAX_FIELDS + 31) / 32];  // fields whose next detection scans whole
    __shared__ uint32_t s_dtile[MSZ_BATCH_MAX_FIELDS + 1];          // prefix of those fields' tile counts
    __shared__ uint32_t s_next;
    __shared__ unsigned long long s_sum, s_chg;
    __shared__ uint32_t sm[40];
    __shared__ uint32_t s_rq[kThreads / 32][kRoundCap];  // each warp's round queue
    __shared__ __align__(16) uint32_t s_F[kFieldWords];   // the current tile's field view (whole-field scans)
    uint32_t *rq = s_rq[threadIdx.x >> 5];
    const uint32_t nf = P.nfields;
    Ctrl *C = P.ctrl;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    for (uint32_t k = threadIdx.x; k <= nf; k += blockDim.x) {
        s_base[k] = k < nf ? P.fields[k].base : P.all.n;
        s_tile[k] = k < nf ? P.fields[k].tile_base : P.ntiles;
    }
    for (uint32_t i = threadIdx.x; i < nf * 4; i += blockDim.x) s_cnt[i >> 2][i & 3] = 0;
    for (uint32_t i = threadIdx.x; i < (nf + 31) / 32; i += blockDim.x) s_alive[i] = 0xffffffffu;
    __syncthreads();
    auto alive = [&](uint32_t k) { return (s_alive[k >> 5] >> (k & 31u)) & 1u; };
    auto dense = [&](uint32_t k) { return (s_dense[k >> 5] >> (k & 31u)) & 1u; };
    bool ok = ld_relaxed(&C->error) == 0;  // every block reads k_batch_codes' verdict
    if (leader) C->t_codes = global_ns();
    // Chunk flags are kept only in sparse sweeps.  sum_k: the phases of
    // sweep k keep them -- decided before sweep k's detection from a bound on
    // its worklist (15 x changed + distorted of sweep k-1, over all fields),
    // so that every mark into sweep k's targets and into the next worklist
    // sets its chunk's flag whenever a walk relies on it.  Sweep 0 keeps none.
    bool sum_k = false;
    uint32_t k = 0;
    while (ok) {
        BatchRec *rec = P.log + (size_t)k * nf;
        // every block derives the same verdicts from the same records
        if (threadIdx.x == 0) s_sum = s_chg = 0;
        for (uint32_t i = threadIdx.x; i < (nf + 31) / 32; i += blockDim.x) s_dense[i] = 0u;
        __syncthreads();
        unsigned long long m_all = 0;
        for (uint32_t f = threadIdx.x; f < nf; f += blockDim.x) {
            if (!alive(f)) continue;
            const uint32_t m = ld_relaxed(&rec[f].distorted);
            if (m == 0) atomicAnd(&s_alive[f >> 5], ~(1u << (f & 31u)));  // done
            m_all += m;
            // whole-field scans for this field's next sweep, as msz_correct
            // decides them for the field alone
            const unsigned long long lim = P.dense_min > 0 ? (unsigned long long)P.dense_min
                                                           : (unsigned long long)P.fields[f].F.G.n;
            if (m && P.dense_min >= 0 && (unsigned long long)m * kDenseFactorB >= lim)
                atomicOr(&s_dense[f >> 5], 1u << (f & 31u));
        }
        if (m_all) atomicAdd(&s_sum, m_all);
        __syncthreads();
        const unsigned long long m_tot = s_sum;
        __syncthreads();
        if (m_tot == 0) {
            if (leader) { C->status = MSZ_OK; C->sweeps = k; }
            break;
        }
        if (k >= P.max_sweeps) {
            uint32_t nt = 0;
            auto count = [&](bool has, uint32_t t) {
                if (has) {
                    const uint32_t f = field_of(P.bfield, t);
                    if (alive(f)) atomicAdd(&s_cnt[f][2], 1u);
                }
            };
            if (!sum_k) walk_bits<true>(P.tb, nullptr, P.all, nt, count);
            else walk_flagged<true, false>(P.tb, P.stb, nullptr, P.all, nt, rq, count);
            flush_counts(s_cnt, nf, rec);
            if (leader) { C->status = MSZ_ERR_MAX_SWEEPS; C->sweeps = k; }
            ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
            break;
        }
        // ---- edit phase of sweep k (targets of a field whose next detection
        // scans whole mark no worklist)
        {
            uint32_t targets = 0;
            uint32_t *const dsum = sum_k ? P.sdm[(k + 1) & 1] : nullptr;
            // counts per field, aggregated over the warp's lanes of one field
            auto count = [&](bool live, uint32_t f, bool changed) {
                const uint32_t peers = __match_any_sync(kFull, live ? f : 0xffffffffu);
                const uint32_t nch = (uint32_t)__popc(peers & __ballot_sync(kFull, changed));
                if (live && lane_id() == (uint32_t)(__ffs(peers) - 1)) {
                    atomicAdd(&s_cnt[f][2], (uint32_t)__popc(peers));
                    if (nch) atomicAdd(&s_cnt[f][3], nch);
                }
            };
            // two targets a lane: both loads in flight before either edit
            auto edit2 = [&](bool h1, uint32_t t1, bool h2, uint32_t t2) {
                const uint32_t f1 = h1 ? field_of(P.bfield, t1) : 0u, f2 = h2 ? field_of(P.bfield, t2) : 0u;
                const bool l1 = h1 && alive(f1), l2 = h2 && alive(f2);
                const FieldView &F1 = P.fields[f1].F;
                const FieldView &F2 = P.fields[f2].F;
                const uint32_t i1 = l1 ? t1 - s_base[f1] : 0u, i2 = l2 ? t2 - s_base[f2] : 0u;
                const float g1 = l1 ? F1.g[i1] : 0.f, v1 = l1 ? __ldg(&F1.f[i1]) : 0.f;
                const float g2 = l2 ? F2.g[i2] : 0.f, v2 = l2 ? __ldg(&F2.f[i2]) : 0.f;
                const bool c1 = l1 && edit_loaded(F1, i1, g1, v1, dense(f1) != 0u, F1.dm[(k + 1) & 1],
                                                  field_flags(dsum, s_base[f1]));
                const bool c2 = l2 && edit_loaded(F2, i2, g2, v2, dense(f2) != 0u, F2.dm[(k + 1) & 1],
                                                  field_flags(dsum, s_base[f2]));
                count(l1, f1, c1);
                count(l2, f2, c2);
            };
            if (!sum_k) walk_bits_pairs<true>(P.tb, nullptr, P.all, targets, edit2, AllWords(), rq);
            else walk_flagged<true, true>(P.tb, P.stb, nullptr, P.all, targets, rq, edit2);
            (void)targets;
            flush_counts(s_cnt, nf, rec);
        }
        ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
        if (!ok) break;
        if (leader) rec[0].pad[2] = stamp_since(C->t_start);
        // fields whose targets were all at their floor are stuck
        uint32_t any_changed = 0;
        unsigned long long chg = 0;
        for (uint32_t f = threadIdx.x; f < nf; f += blockDim.x) {
            if (!alive(f)) continue;
            const uint32_t c = ld_relaxed(&rec[f].changed);
            if (c == 0) atomicAnd(&s_alive[f >> 5], ~(1u << (f & 31u)));
            else any_changed = 1;
            chg += c;
        }
        if (chg) atomicAdd(&s_chg, chg);
        if (!__syncthreads_or(any_changed)) {
            if (leader) { C->status = MSZ_STUCK; C->sweeps = k + 1; }
            break;
        }
        const bool sum_k1 = 15ull * s_chg + m_tot <= P.sparse_max;
        // ---- detection phase of sweep k + 1: its marks keep the flags of its
        // targets and of the next worklist when sum_k1; the current worklist
        // has them when sweep k kept them (sum_k)
        const uint32_t k1 = k + 1;
        BatchRec *rec1 = P.log + (size_t)k1 * nf;
        uint32_t *dcur = P.dm[k1 & 1];
        uint32_t *const dsum1 = sum_k1 ? P.sdm[(k1 + 1) & 1] : nullptr, *const tsum1 = sum_k1 ? P.stb : nullptr;
        {
            const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
            for (uint32_t f = gtid; f < nf; f += stride)
                if (alive(f) && dense(f)) {
                    rec1[f].worklist = P.fields[f].F.G.n;
                    rec1[f].dense = 1;
                }
            // whole-field scans: every uncertified vertex of each live field
            // that scans whole, tile by tile over a queue of those fields'
            // tiles (g staged in shared memory)
            {
                const uint32_t f = threadIdx.x;
                const uint32_t tc = f < nf && alive(f) && dense(f) ? s_tile[f + 1] - s_tile[f] : 0u;
                uint32_t total;
                const uint32_t ex = block_exclusive_scan(tc, sm, total);
                if (f < nf) s_dtile[f] = ex;
                if (f == 0) s_dtile[nf] = total;
                __syncthreads();
            }
            const uint32_t dtiles = s_dtile[nf];
            if (dtiles) {
                uint32_t *counter = &rec1[0].pad[0];
                const FieldView &F = *reinterpret_cast<const FieldView *>(s_F);
                uint32_t staged = 0xffffffffu;  // the field of s_F (block-uniform)
                for (;;) {
                    __syncthreads();
                    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1u);
                    __syncthreads();
                    const uint32_t t = s_next;
                    if (t >= dtiles) break;
                    const uint32_t f = find_field(s_dtile, nf, t);
                    if (f != staged) {
                        stage_field(s_F, P.fields[f].F);
                        staged = f;
                    }
                    const tile::TileGeom tg = tile::tile_geom(F.G.nx, F.G.ny, F.G.nz, F.tile_z);
                    const uint32_t lt = t - s_dtile[f];
                    const uint32_t txi = lt % tg.tx, tyi = (lt / tg.tx) % tg.ty, tzi = lt / (tg.tx * tg.ty);
                    const int zb = (int)(tzi * tg.bz);
                    uint32_t dist = 0;
                    detect_tile_cp(F, (int)(txi * tile::BX), (int)(tyi * tile::BY), zb,
                                   min(zb + (int)tg.bz, (int)F.G.nz), smem, F.dm[(k1 + 1) & 1], dist,
                                   field_flags(dsum1, s_base[f]), field_flags(tsum1, s_base[f]));
                    warp_add(dist, &s_cnt[f][1]);
                }
            }
            // the other live fields: per word, the uncertified vertices of
            // the worklist.  Every word is cleared as it is read (dead fields
            // and fields that scanned whole contribute nothing; a word never
            // straddles two fields: bases are 1024-aligned).
            auto fetch = [&](uint32_t wi) -> uint32_t { return dcur[wi]; };
            auto finish = [&](uint32_t wi, uint32_t wl) -> uint32_t {
                if (!wl) return 0u;
                dcur[wi] = 0u;
                const uint32_t f = field_of(P.bfield, wi * 32u);
                if (!alive(f) || dense(f)) return 0u;
                atomicAdd(&s_cnt[f][0], (uint32_t)__popc(wl));
                return wl & P.ub[wi];
            };
            auto detect = [&](bool h1, uint32_t v1, bool h2, uint32_t v2) {
                detect_pair(P, s_base, nf, s_cnt, (k1 + 1) & 1, sum_k1, alive, h1, v1, h2, v2);
            };
            if (sum_k) walk_flagged_words(P.sdm[k1 & 1], P.all, fetch, finish, rq, detect);
            else walk_words_pairs(P.all, fetch, finish, detect, rq);
        }
        flush_counts(s_cnt, nf, rec1);
        ok = grid_barrier(&C->bar_count, &C->bar_gen, &C->error);
        if (leader) rec1[0].pad[1] = stamp_since(C->t_start);
        k = k1;
        sum_k = sum_k1;
    }
    if (!ok) return;

    // ---- edit lists, split per field, ascending index, chunk (32 words,
    // 1024 vertices, one field) by chunk.  (1) Each warp counts the edits of
    // a contiguous range of chunks, recording each chunk's count; a block
    // scan of the warps' totals and a grid-wide prefix over the blocks turn
    // the counts into each chunk's first position in the shared order, and a
    // field's list starts at the edits of the fields before it (fields lie
    // in the shared space in order).  (2) Warps then take chunks from a
    // shared queue, kListRoundsB at a time, so that the densely edited
    // regions spread over the grid instead of the warps that own them; a
    // chunk's edits go to the lanes in index order (ChunkBits), 32 a round,
    // so that the stores coalesce.
    const uint32_t CH = P.all.words / 32u;  // chunks of the shared space
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const uint32_t nwarps = gridDim.x * wpb;
    const uint32_t per = (CH + nwarps - 1) / nwarps;
    const uint32_t gw = blockIdx.x * wpb + warp;
    const uint32_t c0 = min(gw * per, CH), c1 = min(c0 + per, CH);
    uint32_t cnt = 0;  // the warp's edits so far (warp-uniform)
    {
        uint32_t cur = 0xffffffffu, ac = 0, au = 0;  // lane 0: per-field counts of the current field
#pragma unroll 4
        for (uint32_t c = c0; c < c1; ++c) {
            const uint32_t e = __reduce_add_sync(kFull, (uint32_t)__popc(P.eb[c * 32u + lane]));
            const uint32_t u = __reduce_add_sync(kFull, (uint32_t)__popc(P.ub[c * 32u + lane]));
            if (lane == 0) {
                P.cpre[c] = cnt;  // warp-local for now
                if (e | u) {
                    const uint32_t f = field_of(P.bfield, c * 1024u);
                    if (f != cur) {
                        if (ac) atomicAdd(&s_cnt[cur][0], ac);
                        if (au) atomicAdd(&s_cnt[cur][1], au);
                        cur = f;
                        ac = au = 0;
                    }
                    ac += e;
                    au += u;
                }
            }
            cnt += e;
        }
        if (lane == 0) {
            if (ac) atomicAdd(&s_cnt[cur][0], ac);
            if (au) atomicAdd(&s_cnt[cur][1], au);
        }
    }
    uint32_t tot;
    const uint32_t wpre = block_exclusive_scan(lane == 0 ? cnt : 0u, sm, tot);
    const uint32_t warp_pre = __shfl_sync(kFull, wpre, 0);  // this warp's offset in its block
    if (threadIdx.x == 0) P.bsum[blockIdx.x] = tot;
    __syncthreads();
    for (uint32_t f = threadIdx.x; f < nf; f += blockDim.x) {
        if (s_cnt[f][0]) {
            atomicAdd(&P.res[f].edit_count, (unsigned long long)s_cnt[f][0]);
            s_cnt[f][0] = 0;
        }
        if (s_cnt[f][1]) {
            atomicAdd(&P.res[f].uncertified, s_cnt[f][1]);
            s_cnt[f][1] = 0;
        }
    }
    if (!grid_barrier(&C->bar_count, &C->bar_gen, &C->error)) return;
    uint32_t pre = 0;
    for (uint32_t b = threadIdx.x; b < blockIdx.x; b += blockDim.x) pre += ld_relaxed(&P.bsum[b]);
    uint32_t bpre;
    block_exclusive_scan(pre, sm, bpre);
    {
        const uint32_t base = bpre + warp_pre;
        for (uint32_t c = c0 + lane; c < c1; c += 32u) P.cpre[c] += base;
    }
    // s_tile reused: exclusive prefix of the per-field edit counts (one a
    // thread: nf <= blockDim.x; every count and their sum fit 32 bits)
    static_assert(MSZ_BATCH_MAX_FIELDS <= kThreads, "one field a thread in the edit-count scan");
    {
        const uint32_t ec = threadIdx.x < nf ? (uint32_t)((volatile FieldRes *)P.res)[threadIdx.x].edit_count : 0u;
        uint32_t all_edits;
        const uint32_t ex = block_exclusive_scan(ec, sm, all_edits);
        if (threadIdx.x < nf) s_tile[threadIdx.x] = ex;
    }
    if (!grid_barrier(&C->bar_count, &C->bar_gen, &C->error)) return;
    // edit j of a chunk (lane-picked vertex v, shared index): its field's
    // list position and value
    auto emit = [&](bool h, uint32_t v, uint32_t pos, float gv, float fv, uint32_t f) {
        if (!h) return;
        const FieldDev &D = P.fields[f];
        const unsigned long long q = (unsigned long long)(pos - s_tile[f]);
        if (q < D.edit_cap) {
            D.edit_idx[q] = v - s_base[f];
            D.edit_delta[q] = __fsub_rn(gv, fv);
        }
    };
    auto gather = [&](bool h, uint32_t v, uint32_t f, float &gv, float &fv) {
        const FieldView &F = P.fields[f].F;
        const uint32_t i = h ? v - s_base[f] : 0u;
        gv = h ? F.g[i] : 0.f;
        fv = h ? __ldg(&F.fhat[i]) : 0.f;
    };
    constexpr int R = kListRoundsB;
    uint32_t *const queue = &C->tcount[0];
    uint32_t next = 0;
    if (lane == 0) next = atomicAdd(queue, (uint32_t)R);
    next = __shfl_sync(kFull, next, 0);
    while (next < CH) {
        const uint32_t g0 = next;
        // the words and first positions of this grab's chunks, and the next
        // grab, requested together
        uint32_t wd[R], pos[R], fq[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const uint32_t c = g0 + (uint32_t)q;
            wd[q] = c < CH ? P.eb[c * 32u + lane] : 0u;
            pos[q] = c < CH ? P.cpre[c] : 0u;
            fq[q] = c < CH ? field_of(P.bfield, c * 1024u) : 0u;
        }
        if (lane == 0) next = atomicAdd(queue, (uint32_t)R);
        next = __shfl_sync(kFull, next, 0);
        ChunkBits cb[R] = {ChunkBits((g0 + 0u) * 32u, wd[0]), ChunkBits((g0 + 1u) * 32u, wd[1]),
                           ChunkBits((g0 + 2u) * 32u, wd[2]), ChunkBits((g0 + 3u) * 32u, wd[3])};
        // the first 32 edits of every chunk gathered before any is stored
        bool h[R];
        uint32_t v[R];
        float gv[R], fv[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            cb[q].pick(lane, h[q], v[q]);
            gather(h[q], v[q], fq[q], gv[q], fv[q]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            emit(h[q], v[q], pos[q] + lane, gv[q], fv[q], fq[q]);
            // a chunk with more than 32 edits: the rest four rounds at a
            // time, gathers first
            for (uint32_t j0 = 32u; j0 < cb[q].total; j0 += 32u * R) {
                bool hj[R];
                uint32_t vj[R];
                float gj[R], sj[R];
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    cb[q].pick(j0 + 32u * u + lane, hj[u], vj[u]);
                    gather(hj[u], vj[u], fq[q], gj[u], sj[u]);
                }
#pragma unroll
                for (int u = 0; u < R; ++u) emit(hj[u], vj[u], pos[q] + j0 + 32u * u + lane, gj[u], sj[u], fq[q]);
            }
        }
    }
    if (!grid_barrier(&C->bar_count, &C->bar_gen, &C->error)) return;
    if (leader) C->t_end = global_ns();
}

std::mutex g_batch_mu;

// Resident blocks of kernel fn with sm bytes of dynamic shared memory, times
// the SM count.  The attribute belongs to the current context, so it is set
// on every call (a context re-created after cudaDeviceReset starts without
// it); the occupancy it allows is a property of the device and is cached.
template <class K>
msz_status resident_blocks(K fn, size_t sm, const DeviceInfo &d, int *cache, int &blocks) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
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

// the loop kernel (its dense detection stages g on the cp.async ring) and
// the code pass (f and fhat on the paired-row ring)
msz_status batch_blocks(const DeviceInfo &d, int &blocks) {
    static int cache[64];
    return resident_blocks(k_batch, tile::kRingBytes, d, cache, blocks);
}
msz_status batch_codes_blocks(const DeviceInfo &d, int &blocks) {
    static int cache[64];
    return resident_blocks(k_batch_codes, tile::kPairRingBytes, d, cache, blocks);
}

// Shared index space of the fields: per-field base (1024-aligned) and total.
uint32_t field_tile_z(const msz_field &f, const msz_options *opt) {
    if (f.tile_z > 0) return (uint32_t)f.tile_z;
    if (opt && opt->tile_z > 0) return (uint32_t)opt->tile_z;
    return kTileZ;
}

bool plan(int32_t n, const msz_field *fields, const msz_options *opt, std::vector<GridDev> &grids,
          std::vector<uint32_t> &bases, uint64_t &ntot, uint32_t &ntiles, std::vector<uint32_t> &tile_bases) {
    grids.resize(n);
    bases.resize(n);
    tile_bases.resize(n);
    ntot = 0;
    uint64_t tiles = 0;
    for (int32_t k = 0; k < n; ++k) {
        if (fields[k].grid.ndim != 3 || make_grid(fields[k].grid, grids[k]) != MSZ_OK) return false;
        bases[k] = (uint32_t)ntot;
        ntot += ((uint64_t)grids[k].n + 1023) / 1024 * 1024;
        tile_bases[k] = (uint32_t)tiles;
        const uint32_t tz = field_tile_z(fields[k], opt);
        if (tz < 1 || tz > 1024) return false;
        tiles += tile::tile_geom(grids[k].nx, grids[k].ny, grids[k].nz, tz).count;
        if (ntot > (uint64_t)MSZ_MAX_VERTICES || tiles > 0xffffffffull) return false;
    }
    ntiles = (uint32_t)tiles;
    return true;
}

size_t batch_workspace_bytes(int32_t n, const msz_field *fields, int64_t max_sweeps) {
    if (n < 1 || n > MSZ_BATCH_MAX_FIELDS || !fields) return 0;
    if (max_sweeps <= 0) max_sweeps = MSZ_BATCH_MAX_SWEEPS;
    if (max_sweeps > MSZ_BATCH_MAX_SWEEPS) return 0;
    std::vector<GridDev> grids;
    std::vector<uint32_t> bases, tile_bases;
    uint64_t ntot;
    uint32_t ntiles;
    if (!plan(n, fields, nullptr, grids, bases, ntot, ntiles, tile_bases)) return 0;
    return batch_layout((uint32_t)n, ntot, (uint32_t)max_sweeps).total;
}

// A prepared batch: everything the launch needs, kept on the host.
struct BatchPlanImpl {
    int32_t n;
    uint32_t max_sweeps;
    int blocks;
    int codes_blocks;
    int device;
    char *ws;
    BatchLayout L;
    BatchProblem P;
    std::vector<GridDev> grids;
    int64_t *h_timeline;  // the options' timeline (2 * timeline_cap int64) or NULL
    int64_t timeline_cap;
};

}  // namespace
}  // namespace msz

struct msz_batch_plan {
    msz::BatchPlanImpl impl;
};

using namespace msz;

extern "C" size_t msz_batch_workspace_size(int32_t n, const msz_field *fields, int64_t max_sweeps) {
    return batch_workspace_bytes(n, fields, max_sweeps);
}

extern "C" msz_status msz_batch_plan_create(int32_t n, const msz_field *fields, const msz_options *opt,
                                            void *d_workspace, size_t workspace_bytes, msz_stream_t stream,
                                            msz_batch_plan **out_plan) {
    if (!out_plan) return MSZ_ERR_INVALID_ARG;
    *out_plan = nullptr;
    if (n < 1 || n > MSZ_BATCH_MAX_FIELDS || !fields) return MSZ_ERR_INVALID_ARG;
    msz_options o{};
    if (opt) o = *opt;
    if (o.rule != MSZ_RULE_HALVE && o.rule != MSZ_RULE_SNAP) return MSZ_ERR_INVALID_ARG;
    if (o.d_g_init || o.test_fault || o.max_sweeps > MSZ_BATCH_MAX_SWEEPS || o.dense_min_items < -1)
        return MSZ_ERR_INVALID_ARG;
    const uint32_t max_sweeps = o.max_sweeps <= 0 ? (uint32_t)MSZ_BATCH_MAX_SWEEPS : (uint32_t)o.max_sweeps;
    for (int32_t k = 0; k < n; ++k) {
        const msz_field &F = fields[k];
        if (!F.d_f || !F.d_fhat || !F.d_out || F.edit_capacity < 0 ||
            (F.edit_capacity > 0 && (!F.d_edit_idx || !F.d_edit_delta)) || !(F.xi >= 0.0f) || isinf(F.xi))
            return MSZ_ERR_INVALID_ARG;
    }
    std::vector<GridDev> grids;
    std::vector<uint32_t> bases, tile_bases;
    uint64_t ntot;
    uint32_t ntiles;
    if (!plan(n, fields, &o, grids, bases, ntot, ntiles, tile_bases)) return MSZ_ERR_INVALID_ARG;
    const BatchLayout L = batch_layout((uint32_t)n, ntot, max_sweeps);
    if (!d_workspace || workspace_bytes < L.total) return MSZ_ERR_WORKSPACE;
    if ((uintptr_t)d_workspace % kAlign) return MSZ_ERR_INVALID_ARG;
    DeviceInfo dev;
    msz_status st = current_device(dev);
    if (st != MSZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)d_workspace;

    std::vector<FieldDev> tab(n);
    for (int32_t k = 0; k < n; ++k) {
        FieldDev &D = tab[k];
        memset(&D, 0, sizeof D);
        FieldView &F = D.F;
        const uint32_t wb = bases[k] / 32;
        F.G = grids[k];
        F.f = fields[k].d_f;
        F.fhat = fields[k].d_fhat;
        F.ginit = nullptr;
        F.g = fields[k].d_out;
        F.codes_f = (uint8_t *)(ws + L.codes) + bases[k];
        F.tb = (uint32_t *)(ws + L.tb) + wb;
        F.dm[0] = (uint32_t *)(ws + L.d0) + wb;
        F.dm[1] = (uint32_t *)(ws + L.d1) + wb;
        F.eb = (uint32_t *)(ws + L.eb) + wb;
        F.ub = (uint32_t *)(ws + L.ub) + wb;
        F.xi = fields[k].xi;
        F.two_xi = 2.0f * fields[k].xi;
        F.rule = o.rule;
        F.tile_z = field_tile_z(fields[k], &o);
        D.base = bases[k];
        D.tile_base = tile_bases[k];
        D.edit_idx = fields[k].d_edit_idx;
        D.edit_delta = fields[k].d_edit_delta;
        D.edit_cap = (unsigned long long)fields[k].edit_capacity;
    }
    BatchProblem P{};
    P.fields = (const FieldDev *)(ws + L.fields);
    P.nfields = (uint32_t)n;
    P.ntiles = ntiles;
    P.all.n = (uint32_t)ntot;
    P.all.words = (uint32_t)(ntot / 32);
    P.ctrl = (Ctrl *)(ws + L.ctrl);
    P.log = (BatchRec *)(ws + L.log);
    P.res = (FieldRes *)(ws + L.res);
    P.bsum = (uint32_t *)(ws + L.bsum);
    P.max_sweeps = max_sweeps;
    // default: each field scans whole while 6 x its distorted vertices >=
    // its vertex count, the rule msz_correct applies to it alone
    P.dense_min = (long long)o.dense_min_items;
    P.tb = (uint32_t *)(ws + L.tb);
    P.dm[0] = (uint32_t *)(ws + L.d0);
    P.dm[1] = (uint32_t *)(ws + L.d1);
    P.eb = (uint32_t *)(ws + L.eb);
    P.ub = (uint32_t *)(ws + L.ub);
    P.stb = (uint32_t *)(ws + L.stb);
    P.sdm[0] = (uint32_t *)(ws + L.sd0);
    P.sdm[1] = (uint32_t *)(ws + L.sd1);
    P.cpre = (uint32_t *)(ws + L.cpre);
    P.sparse_max = ntot / 256 > kSparseWorklistB ? ntot / 256 : kSparseWorklistB;
    P.bfield = (const uint8_t *)(ws + L.bfield);
    std::vector<uint8_t> bfield(ntot / 1024, 0);
    for (int32_t k = 0; k < n; ++k)
        for (uint64_t b = bases[k] / 1024; b < (bases[k] + (uint64_t)grids[k].n + 1023) / 1024; ++b)
            bfield[b] = (uint8_t)k;
    int blocks = 0, cblocks = 0;
    if ((st = batch_blocks(dev, blocks)) != MSZ_OK) return st;
    if ((st = batch_codes_blocks(dev, cblocks)) != MSZ_OK) return st;
    // the descriptor table is uploaded once; launches only clear the control
    // block and bitmaps, so a captured launch can be replayed
    if (cudaMemcpyAsync(ws + L.fields, tab.data(), n * sizeof(FieldDev), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MSZ_ERR_CUDA;
    if (!bfield.empty() &&
        cudaMemcpyAsync(ws + L.bfield, bfield.data(), bfield.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    msz_batch_plan *p = new (std::nothrow) msz_batch_plan;
    if (!p) return MSZ_ERR_WORKSPACE;
    p->impl.n = n;
    p->impl.max_sweeps = max_sweeps;
    p->impl.blocks = blocks;
    p->impl.codes_blocks = cblocks;
    p->impl.device = dev.device;
    p->impl.ws = ws;
    p->impl.L = L;
    p->impl.P = P;
    p->impl.grids = std::move(grids);
    p->impl.h_timeline = o.log_capacity > 0 ? o.h_timeline : nullptr;
    p->impl.timeline_cap = o.log_capacity;
    *out_plan = p;
    return MSZ_OK;
}

extern "C" msz_status msz_batch_launch(const msz_batch_plan *plan, msz_stream_t stream) {
    if (!plan) return MSZ_ERR_INVALID_ARG;
    const BatchPlanImpl &B = plan->impl;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != B.device) return MSZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(B.ws, 0, B.L.zero_bytes, s) != cudaSuccess) return MSZ_ERR_CUDA;
    k_batch_codes<<<B.codes_blocks, kThreads, tile::kPairRingBytes, s>>>(B.P);
    if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(B.blocks);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = tile::kRingBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BatchProblem P = B.P;
    if (cudaLaunchKernelEx(&cfg, k_batch, P) != cudaSuccess) return MSZ_ERR_CUDA;
    return MSZ_OK;
}

extern "C" msz_status msz_batch_collect(const msz_batch_plan *plan, msz_field *fields, int64_t *h_sweep_log,
                                        int64_t log_capacity, msz_stream_t stream) {
    if (!plan || !fields || log_capacity < 0 || (log_capacity > 0 && !h_sweep_log)) return MSZ_ERR_INVALID_ARG;
    const BatchPlanImpl &B = plan->impl;
    const int32_t n = B.n;
    const BatchLayout &L = B.L;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = B.ws;
    Ctrl hc;
    std::vector<FieldRes> res(n);
    if (cudaMemcpyAsync(&hc, ws + L.ctrl, sizeof hc, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (cudaMemcpyAsync(res.data(), ws + L.res, n * sizeof(FieldRes), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (hc.error & kErrTimeout) return MSZ_ERR_TIMEOUT;
    if (hc.error & kErrInput) {
        for (int32_t k = 0; k < n; ++k) fields[k].status = res[k].error ? MSZ_ERR_INPUT_BOUND : MSZ_ERR_INVALID_ARG;
        return MSZ_ERR_INPUT_BOUND;
    }
    // per-field records, then each field's own termination rule
    const uint32_t S = hc.sweeps;  // last sweep index the launch reached
    std::vector<BatchRec> log((size_t)(S + 1) * n);
    if (cudaMemcpy(log.data(), ws + L.log, log.size() * sizeof(BatchRec), cudaMemcpyDeviceToHost) != cudaSuccess)
        return MSZ_ERR_CUDA;
    const int64_t kernel_ns = hc.t_end > hc.t_start ? (int64_t)(hc.t_end - hc.t_start) : 0;
    const int64_t codes_ns = hc.t_codes > hc.t_start ? (int64_t)(hc.t_codes - hc.t_start) : 0;
    if (B.h_timeline) {
        // sweep 0's detection ends with the code pass; later stamps are field 0's records
        for (int64_t q = 0; q < B.timeline_cap; ++q) {
            int64_t td = -1, te = -1;
            if (q <= (int64_t)S) {
                const BatchRec &r = log[(size_t)q * n];
                td = q == 0 ? (codes_ns ? codes_ns : -1) : r.pad[1] ? (int64_t)r.pad[1] : -1;
                te = r.pad[2] ? (int64_t)r.pad[2] : -1;
            }
            B.h_timeline[2 * q] = td;
            B.h_timeline[2 * q + 1] = te;
        }
    }
    for (int32_t k = 0; k < n; ++k) {
        msz_field &F = fields[k];
        msz_stats &stt = F.stats;
        memset(&stt, 0, sizeof stt);
        stt.first_distorted = log[k].distorted;
        stt.kernel_ns = kernel_ns;
        stt.codes_ns = codes_ns;
        msz_status fs = MSZ_ERR_MAX_SWEEPS;
        for (uint32_t q = 0; q <= S; ++q) {
            const BatchRec &r = log[(size_t)q * n + k];
            const int64_t wl = q == 0 ? (int64_t)B.grids[k].n : (int64_t)r.worklist;
            stt.examined += wl;
            stt.dense_sweeps += (q == 0 || r.dense) ? 1 : 0;
            if (h_sweep_log && q < (uint64_t)log_capacity) {
                int64_t *row = h_sweep_log + 4 * ((size_t)k * log_capacity + q);
                row[0] = wl;
                row[1] = r.distorted;
                row[2] = r.targets;
                row[3] = r.changed;
            }
            if (r.distorted == 0) { fs = MSZ_OK; stt.sweeps = q; break; }
            if (q >= B.max_sweeps) { fs = MSZ_ERR_MAX_SWEEPS; stt.sweeps = q; stt.left = r.distorted; break; }
            if (r.changed == 0) { fs = MSZ_STUCK; stt.sweeps = q + 1; stt.left = r.distorted; break; }
            stt.edits += r.changed;
        }
        F.edit_count = (int64_t)res[k].edit_count;
        stt.edited = F.edit_count;
        stt.uncertified = res[k].uncertified;
        if (fs == MSZ_OK && F.edit_count > F.edit_capacity) fs = MSZ_ERR_CAPACITY;
        F.status = fs;
    }
    return MSZ_OK;
}

extern "C" void msz_batch_plan_destroy(msz_batch_plan *plan) { delete plan; }

extern "C" msz_status msz_correct_batch(int32_t n, msz_field *fields, const msz_options *opt,
                                        int64_t *h_sweep_log, int64_t log_capacity, void *d_workspace,
                                        size_t workspace_bytes, msz_stream_t stream) {
    if (log_capacity < 0 || (log_capacity > 0 && !h_sweep_log)) return MSZ_ERR_INVALID_ARG;
    msz_batch_plan *plan = nullptr;
    msz_status st = msz_batch_plan_create(n, fields, opt, d_workspace, workspace_bytes, stream, &plan);
    if (st != MSZ_OK) return st;
    st = msz_batch_launch(plan, stream);
    if (st == MSZ_OK) st = msz_batch_collect(plan, fields, h_sweep_log, log_capacity, stream);
    msz_batch_plan_destroy(plan);
    return st;
}
