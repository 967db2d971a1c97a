// msz_phases.cuh -- the phases of the correction loop for one field,
// shared by the single-field and the batched persistent kernels.
//
// A FieldView is one field's slice of the work: its grid, data pointers, and
// its windows into the workspace bitmaps (targets, worklists, edited,
// uncertified) and codes, all indexed by the field's own linear index.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_tile.cuh"
#include "msz_tma.cuh"
#include "msz_workspace.h"

namespace msz {

// default planes per tile of the code pass (512^3 Perlin field, two planes a
// step: 8, 16, 24, 32, 48, 64 -> 1.548, 1.551, 1.541, 1.574, 1.550, 1.658 ms)
constexpr uint32_t kTileZ = 24;
#ifndef MSZ_WALK_AHEAD
#define MSZ_WALK_AHEAD 4
#endif
constexpr int kAhead = MSZ_WALK_AHEAD;  // bitmap chunks a walking warp has loaded ahead

struct FieldView {
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
    uint32_t *cand;    // BELOW_REFERENCE only (else null): per vertex, the totalOrder key of
                       // the smallest value requested for it in this sweep (all ones: none)
    float xi;
    float two_xi;      // 2 xi (exact): the certification margin
    int rule;
    uint32_t tile_z;   // planes per tile of the code pass
};

// Where a detection phase records: the targets (P.tb) and the worklist of the
// next sweep (dnext); distorted vertices are counted per thread and added to
// the sweep's record when the phase ends.
// A phase that keeps chunk flags (one word per chunk of 32 bitmap words,
// 1024 vertices, nonzero when the chunk may hold a set bit) sets them through
// dsum (the next worklist's) and tsum (the targets').
struct Emitter {
    uint32_t *dnext;
    uint32_t distorted;
    uint32_t *dsum = nullptr;  // chunk flags of dnext, or null
    uint32_t *tsum = nullptr;  // chunk flags of P.tb, or null
};

// Sets the flag of the chunk (32 words, 1024 vertices) holding vertex v of a
// bitmap: a plain store of 1 (every writer stores the same value).
__device__ __forceinline__ void mark_chunk(uint32_t *sum, uint32_t v) { st_relaxed(&sum[v >> 10], 1u); }

// BELOW_REFERENCE: the value target t asks for to fall below reference r
// (value vr of this sweep) in the (value, index) order -- vr when r has the
// larger index, else the float just below vr -- recorded as the minimum, in
// IEEE totalOrder, over every request of the sweep.
__device__ __forceinline__ void request_below(const FieldView &P, uint32_t t, uint32_t r, float vr) {
    const float c = r > t ? vr : float_below(vr);
    atomicMin(&P.cand[t], total_key(c));
}

// Warp-collective: vertex v (valid lanes) with codes cf in f and cg in g; a
// distorted vertex marks its targets and, unless the caller marks whole words
// itself (self_marked), itself for the next worklist.  sweep0: the pass that
// runs sweep 0's detection while it writes g, where g of the sweep is still
// the start field (BELOW_REFERENCE reads its reference values there).
__device__ __forceinline__ bool report(const FieldView &P, Emitter &E, bool valid, uint32_t v, uint32_t cf,
                                       uint32_t cg, bool self_marked = false, bool sweep0 = false) {
    const bool dist = valid && cf != cg;
    if (!__any_sync(kFull, dist)) return false;
    if (dist) {
        uint32_t t0, t1;
        const int nt = targets_of(P.G, v, (uint8_t)cf, (uint8_t)cg, t0, t1);
        red_or(&P.tb[t0 >> 5], 1u << (t0 & 31u));
        if (nt > 1) red_or(&P.tb[t1 >> 5], 1u << (t1 & 31u));
        if (E.tsum) {
            mark_chunk(E.tsum, t0);
            if (nt > 1) mark_chunk(E.tsum, t1);
        }
        if (P.cand) {
            uint32_t r0, r1;
            references_of(P.G, v, (uint8_t)cf, (uint8_t)cg, r0, r1);
            const float *gk = sweep0 ? (P.ginit ? P.ginit : P.fhat) : P.g;
            request_below(P, t0, r0, gk[r0]);
            if (nt > 1) request_below(P, t1, r1, gk[r1]);
        }
        if (!self_marked) {
            red_or(&E.dnext[v >> 5], 1u << (v & 31u));
            if (E.dsum) mark_chunk(E.dsum, v);
        }
        E.distorted += 1;
    }
    return dist;
}

// The set bits of one chunk of 32 bitmap words (lane l holds word base + l
// in `bits`), handed out to the warp's lanes in index order: the chunk's
// j-th set bit goes to lane j mod 32.  pick(j, has, v) gives the vertex of
// the j-th bit (warp-collective: every lane calls it, with its own j).
struct ChunkBits {
    uint32_t base, bits, cnt, incl, total;
    __device__ __forceinline__ ChunkBits(uint32_t b, uint32_t w) : base(b), bits(w) {
        const uint32_t lane = lane_id();
        cnt = (uint32_t)__popc(w);
        if (!__any_sync(kFull, w != 0u)) {  // an empty chunk (most, in late sweeps)
            incl = 0u;
            total = 0u;
            return;
        }
        incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (lane >= (uint32_t)d) incl += y;
        }
        total = __shfl_sync(kFull, incl, 31);
    }
    __device__ __forceinline__ void pick(uint32_t j, bool &has, uint32_t &v) const {
        // the lane whose word holds bit j: the first whose inclusive count
        // exceeds j
        uint32_t owner = 0;
#pragma unroll
        for (uint32_t s = 16; s >= 1; s >>= 1) {
            const uint32_t c = __shfl_sync(kFull, incl, (int)(owner + s - 1u));
            if (c <= j) owner += s;
        }
        owner &= 31u;
        const uint32_t word = __shfl_sync(kFull, bits, (int)owner);
        const uint32_t before = __shfl_sync(kFull, incl - cnt, (int)owner);
        has = j < total;
        v = has ? (base + owner) * 32u + tile::nth_set(word, j - before) : 0u;
    }
};

// fn(has, v) once per round with one set bit of the chunk a lane.
template <class F>
__device__ __forceinline__ void chunk_each(uint32_t base, uint32_t bits, F &&fn) {
    const ChunkBits cb(base, bits);
    for (uint32_t j0 = 0; j0 < cb.total; j0 += 32u) {
        bool h;
        uint32_t v;
        cb.pick(j0 + lane_id(), h, v);
        fn(h, v);
    }
}

// fn(has1, v1, has2, v2) once per round with two set bits of the chunk a
// lane (bits j and j + 32 of a round of 64), so that each lane has the
// loads of both in flight at once.
template <class F>
__device__ __forceinline__ void chunk_pairs(uint32_t base, uint32_t bits, F &&fn) {
    const ChunkBits cb(base, bits);
    for (uint32_t j0 = 0; j0 < cb.total; j0 += 64u) {
        bool h1, h2;
        uint32_t v1, v2;
        cb.pick(j0 + lane_id(), h1, v1);
        cb.pick(j0 + 32u + lane_id(), h2, v2);
        fn(h1, v1, h2, v2);
    }
}

// Vertices of several chunks gathered into full rounds (warp-collective):
// the warp's buffer q (kRoundCap entries of shared memory) takes a chunk's
// set bits in index order, and whenever it holds a full round -- 64 vertices
// with PAIRS (two a lane), else 32 -- the round runs.  In a sparse sweep a
// chunk holds a few set bits, so a round per chunk would leave most lanes
// idle and put one dependent gather after another; a round over several
// chunks keeps the warp full.  The order of the calls does not matter to
// their callers (their effects are reductions and distinct targets).
constexpr uint32_t kRoundCap = 96;  // a full round plus one chunk round (< 32) carried over

template <bool PAIRS>
struct RoundQueue {
    static constexpr uint32_t R = PAIRS ? 64u : 32u;
    uint32_t *q;
    uint32_t n = 0;  // warp-uniform fill
    // runs the first cnt (<= R) queued vertices and moves the rest up
    template <class F>
    __device__ __forceinline__ void run(uint32_t cnt, F &fn) {
        const uint32_t lane = lane_id();
        __syncwarp();
        if constexpr (PAIRS) {
            const bool h1 = lane < cnt, h2 = lane + 32u < cnt;
            fn(h1, h1 ? q[lane] : 0u, h2, h2 ? q[lane + 32u] : 0u);
        } else {
            const bool h = lane < cnt;
            fn(h, h ? q[lane] : 0u);
        }
        const uint32_t rest = n - cnt;  // < 32
        const uint32_t mv = lane < rest ? q[cnt + lane] : 0u;
        __syncwarp();
        if (lane < rest) q[lane] = mv;
        __syncwarp();
        n = rest;
    }
    template <class F>
    __device__ __forceinline__ void push_chunk(uint32_t base, uint32_t bits, F &fn) {
        if (!__any_sync(kFull, bits != 0u)) return;
        const ChunkBits cb(base, bits);
        for (uint32_t j0 = 0; j0 < cb.total; j0 += 32u) {
            bool h;
            uint32_t v;
            cb.pick(j0 + lane_id(), h, v);  // lanes 0 .. take-1
            if (h) q[n + lane_id()] = v;
            n += min(32u, cb.total - j0);
            if (n >= R) run(R, fn);
        }
    }
    template <class F>
    __device__ __forceinline__ void flush(F &fn) {
        while (n) run(min(n, R), fn);
    }
};

// Warp-collective walk over the set bits of a bitmap: each warp takes 32
// consecutive words (1024 vertices) at a time, grid-stride.  CLEAR zeroes the
// visited words; `seen` counts their set bits; a non-null filter restricts the
// calls to the vertices also set there.  fn(valid, v) runs once per round
// with one vertex per lane, the chunk's bits handed out in index order
// (chunk_each), so that a round's loads are in flight together however the
// bits fall on the words; with rq (the warp's kRoundCap entries of shared
// memory) the bits go through a RoundQueue instead, rounds spanning chunks.
template <bool CLEAR, class F>
__device__ __forceinline__ void walk_bits(uint32_t *bm, const uint32_t *filter, const GridDev &G, uint32_t &seen,
                                          F &&fn, uint32_t *rq = nullptr) {
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t chunks = (G.words + 31u) / 32u;
    RoundQueue<false> Q{rq};
    // the words of the next kAhead chunks are loaded ahead (a sparse walk is
    // otherwise one dependent load after another)
    uint32_t pre[kAhead];
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
        const uint32_t wi = (gw + (uint32_t)u * nw) * 32u + lane;
        pre[u] = wi < G.words ? bm[wi] : 0u;
    }
    for (uint32_t c = gw; c < chunks; c += nw) {
        const uint32_t base = c * 32u;
        const uint32_t wi = base + lane;
        uint32_t bits = pre[0];
#pragma unroll
        for (int u = 0; u + 1 < kAhead; ++u) pre[u] = pre[u + 1];
        {
            const uint32_t wn = (c + (uint32_t)kAhead * nw) * 32u + lane;
            pre[kAhead - 1] = wn < G.words ? bm[wn] : 0u;
        }
        if (bits) {
            if (CLEAR) bm[wi] = 0u;
            seen += (uint32_t)__popc(bits);
            if (filter) bits &= filter[wi];
        }
        if (rq) Q.push_chunk(base, bits, fn);
        else chunk_each(base, bits, fn);
    }
    if (rq) Q.flush(fn);
}

// walk_bits for detection: two vertices per lane per round (chunk_pairs), so
// that each lane has the neighbour loads of both in flight at once.
// fn(has1, v1, has2, v2).  word_ok(w) false drops word w (after counting it
// in `seen`).  The filter's words are loaded one chunk ahead.  With rq (the
// warp's kRoundCap entries of shared memory) the set bits go through a
// RoundQueue, so rounds stay full where chunks hold few bits.
struct AllWords {
    __device__ __forceinline__ bool operator()(uint32_t) const { return true; }
};

template <bool CLEAR, class F, class W = AllWords>
__device__ __forceinline__ void walk_bits_pairs(uint32_t *bm, const uint32_t *filter, const GridDev &G,
                                                uint32_t &seen, F &&fn, W word_ok = W(), uint32_t *rq = nullptr) {
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t chunks = (G.words + 31u) / 32u;
    RoundQueue<true> Q{rq};
    uint32_t pre[kAhead];
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
        const uint32_t wi = (gw + (uint32_t)u * nw) * 32u + lane;
        pre[u] = wi < G.words ? bm[wi] : 0u;
    }
    uint32_t fnext = 0;  // the filter's word for the warp's next chunk
    if (filter) {
        const uint32_t wi = gw * 32u + lane;
        fnext = pre[0] && wi < G.words ? filter[wi] : 0u;
    }
    for (uint32_t c = gw; c < chunks; c += nw) {
        const uint32_t base = c * 32u;
        const uint32_t wi = base + lane;
        uint32_t bits = pre[0];
        const uint32_t fcur = fnext;
#pragma unroll
        for (int u = 0; u + 1 < kAhead; ++u) pre[u] = pre[u + 1];
        {
            const uint32_t wn = (c + (uint32_t)kAhead * nw) * 32u + lane;
            pre[kAhead - 1] = wn < G.words ? bm[wn] : 0u;
        }
        if (filter) {
            const uint32_t wn = (c + nw) * 32u + lane;
            fnext = pre[0] && wn < G.words ? filter[wn] : 0u;
        }
        if (bits) {
            if (CLEAR) bm[wi] = 0u;
            seen += (uint32_t)__popc(bits);
            if (filter) bits &= fcur;
            if (bits && !word_ok(wi)) bits = 0u;
        }
        if (rq) Q.push_chunk(base, bits, fn);
        else chunk_pairs(base, bits, fn);
    }
    if (rq) Q.flush(fn);
}

// walk_bits / walk_bits_pairs over the chunks (32 words) whose flags are
// set.  Chunk c belongs to warp c mod (warps of the grid), as in walk_bits,
// so that a cluster of flagged chunks spreads over many warps.  A warp reads
// the flags of 32 of its chunks at once (one per lane), then walks the
// flagged ones, loading the words of the next flagged chunk before the
// current one is queued; the set bits go through a RoundQueue (rq: the
// warp's kRoundCap entries of shared memory), so rounds are full.  CLEAR
// zeroes the visited words and flags.  PAIRS: fn(h1, v1, h2, v2), two
// vertices a lane; else fn(h, v).
template <bool CLEAR, bool PAIRS, class F>
__device__ __forceinline__ void walk_flagged(uint32_t *bm, uint32_t *flags, const uint32_t *filter, const GridDev &G,
                                             uint32_t &seen, uint32_t *rq, F &&fn) {
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t chunks = (G.words + 31u) / 32u;
    RoundQueue<PAIRS> Q{rq};
    for (uint32_t c0 = gw; c0 < chunks; c0 += 32u * nw) {
        const uint32_t mine = c0 + lane * nw;  // this lane's chunk of the round
        const bool set = mine < chunks && flags[mine] != 0u;
        if (CLEAR && set) flags[mine] = 0u;
        uint32_t marks = __ballot_sync(kFull, set);
        if (!marks) continue;
        uint32_t c = c0 + (uint32_t)(__ffs(marks) - 1) * nw;
        marks &= marks - 1u;
        uint32_t nxt = c * 32u + lane < G.words ? bm[c * 32u + lane] : 0u;
        for (;;) {
            const uint32_t base = c * 32u;
            const uint32_t wi = base + lane;
            uint32_t bits = nxt;
            const bool more = marks != 0u;
            if (more) {
                c = c0 + (uint32_t)(__ffs(marks) - 1) * nw;
                marks &= marks - 1u;
                nxt = c * 32u + lane < G.words ? bm[c * 32u + lane] : 0u;
            }
            if (bits) {
                if (CLEAR) bm[wi] = 0u;
                seen += (uint32_t)__popc(bits);
                if (filter) bits &= filter[wi];
            }
            Q.push_chunk(base, bits, fn);
            if (!more) break;
        }
    }
    Q.flush(fn);
}

// Like walk_bits_pairs, with the bits of word w given by finish(w, raw),
// where raw = fetch(w) is loaded kAhead chunks ahead (fetch only loads;
// finish may read, clear and count whatever else it needs).  rq: as in
// walk_bits_pairs.
template <class FE, class FI, class F>
__device__ __forceinline__ void walk_words_pairs(const GridDev &G, FE &&fetch, FI &&finish, F &&fn,
                                                 uint32_t *rq = nullptr) {
    const uint32_t lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t chunks = (G.words + 31u) / 32u;
    RoundQueue<true> Q{rq};
    uint32_t pre[kAhead];
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
        const uint32_t wi = (gw + (uint32_t)u * nw) * 32u + lane;
        pre[u] = wi < G.words ? fetch(wi) : 0u;
    }
    for (uint32_t c = gw; c < chunks; c += nw) {
        const uint32_t base = c * 32u;
        const uint32_t wi = base + lane;
        const uint32_t raw = pre[0];
#pragma unroll
        for (int u = 0; u + 1 < kAhead; ++u) pre[u] = pre[u + 1];
        {
            const uint32_t wn = (c + (uint32_t)kAhead * nw) * 32u + lane;
            pre[kAhead - 1] = wn < G.words ? fetch(wn) : 0u;
        }
        const uint32_t bits = wi < G.words ? finish(wi, raw) : 0u;
        if (rq) Q.push_chunk(base, bits, fn);
        else chunk_pairs(base, bits, fn);
    }
    if (rq) Q.flush(fn);
}

// Detection of two vertices per lane in the current g (warp-collective): all
// neighbour loads of both are issued before either code is formed.
template <int NDIM>
__device__ __forceinline__ void detect_vertex2(const FieldView &P, Emitter &E, bool h1, uint32_t v1, bool h2,
                                               uint32_t v2) {
    float a[15], b[15];
    gather_closed<NDIM>(P.g, P.G, h1, v1, a);
    gather_closed<NDIM>(P.g, P.G, h2, v2, b);
    const uint32_t cf1 = h1 ? __ldg(&P.codes_f[v1]) : 0u;
    const uint32_t cf2 = h2 ? __ldg(&P.codes_f[v2]) : 0u;
    report(P, E, h1, v1, cf1, code_of_closed<NDIM>(a));
    report(P, E, h2, v2, cf2, code_of_closed<NDIM>(b));
}

// Detection of one vertex in the current g (warp-collective).
template <int NDIM>
__device__ __forceinline__ void detect_vertex(const FieldView &P, Emitter &E, bool has, uint32_t v) {
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
__device__ void first_generic(const FieldView &P, uint32_t *err) {
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
    if (bad) atomicOr(err, kErrInput);
}

// One warp row of the code pass on the cp.async ring (warp-collective; the
// TMA ring takes two rows at once, tile_rows2): row r (1 .. BY) of the
// planes pm / p0 / pp staged at pitch PW (column c <-> x = x0 - 4 + c), the
// second field soff floats after each plane; rowbase = the linear index of
// (0, y, z).  Certifies the row's 128 vertices, marks the uncertified ones in
// P.ub and forms their exact codes of f (codes_f) and, when DETECT, of the
// second field, reporting sweep 0's distortions.
template <bool DETECT>
__device__ __forceinline__ void tile_row(const FieldView &P, const float *pm, const float *p0, const float *pp,
                                         int soff, int r, int x0, uint32_t rowbase, uint32_t &distorted) {
    using namespace tile;
    const GridDev &G = P.G;
    const uint32_t lane = lane_id();
    const int xl = x0 + 4 * (int)lane;
    const uint32_t cert = cert4(pm, p0, pp, r, lane, P.two_xi);
    const uint32_t i0 = rowbase + (uint32_t)xl;
    // uncertified bits of this lane's vertices (outside the grid: 0)
    uint32_t nib = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) nib |= (uint32_t)(xl + e < (int)G.nx && !((cert >> e) & 1u)) << e;
    // the row's 128 uncertified bits as 4 words: word q (lanes 8q .. 8q+7)
    // covers columns 32q .. 32q+31
    uint32_t w = nib << (4u * (lane & 7u));
    w |= __shfl_xor_sync(kFull, w, 1);
    w |= __shfl_xor_sync(kFull, w, 2);
    w |= __shfl_xor_sync(kFull, w, 4);
    const bool words_ok = ((rowbase + (uint32_t)x0) & 31u) == 0 && x0 + BX <= (int)G.nx;
    if (words_ok) {
        if ((lane & 7u) == 0) P.ub[i0 >> 5] = w;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if ((nib >> e) & 1u) red_or(&P.ub[(i0 + e) >> 5], 1u << ((i0 + e) & 31u));
    }
    // The row's uncertified vertices, 32 at a time in column order (lane j
    // takes the j-th one): the exact code in f, written to codes_f (the loop
    // reads codes_f at uncertified vertices only) and, when this pass
    // detects, the code in the second field, compared with it.
    const uint32_t w0 = __shfl_sync(kFull, w, 0), w1 = __shfl_sync(kFull, w, 8);
    const uint32_t w2 = __shfl_sync(kFull, w, 16), w3 = __shfl_sync(kFull, w, 24);
    const uint32_t c0 = (uint32_t)__popc(w0), c1 = c0 + (uint32_t)__popc(w1);
    const uint32_t c2 = c1 + (uint32_t)__popc(w2), total = c2 + (uint32_t)__popc(w3);
    Emitter E{P.dm[1], 0};
    for (uint32_t j0 = 0; j0 < total; j0 += 32u) {
        const uint32_t j = j0 + lane;
        const bool has = j < total;
        uint32_t col = 0, cf = 0, cg = 0;
        if (has) {
            const uint32_t q = j < c0 ? 0u : j < c1 ? 1u : j < c2 ? 2u : 3u;
            const uint32_t wq = q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : w3;
            const uint32_t before = q == 0 ? 0u : q == 1 ? c0 : q == 2 ? c1 : c2;
            col = 32u * q + nth_set(wq, j - before);
            cf = code1(pm, p0, pp, r, 4 + (int)col);
            P.codes_f[rowbase + (uint32_t)x0 + col] = (uint8_t)cf;
            if (DETECT) cg = code1(pm + soff, p0 + soff, pp + soff, r, 4 + (int)col);
        }
        if (DETECT) report(P, E, has, rowbase + (uint32_t)x0 + col, cf, cg, false, true);
    }
    distorted += E.distorted;
}

// The uncertified columns of one warp row, kept in three registers: the
// lane-distributed word w (lanes 8q .. 8q+7 hold word q: columns 32q ..
// 32q+31), the running counts of words 0, 0-1 and 0-2 (a byte each) and the
// total.
struct RowBits {
    uint32_t w, counts, total;
    __device__ __forceinline__ void from(uint32_t word) {
        w = word;
        const uint32_t c0 = (uint32_t)__popc(__shfl_sync(kFull, word, 0));
        const uint32_t c1 = c0 + (uint32_t)__popc(__shfl_sync(kFull, word, 8));
        const uint32_t c2 = c1 + (uint32_t)__popc(__shfl_sync(kFull, word, 16));
        total = c2 + (uint32_t)__popc(__shfl_sync(kFull, word, 24));
        counts = c0 | c1 << 8 | c2 << 16;
    }
};

// Which of the 4 words of a row (RowBits::counts) holds its j-th uncertified
// vertex, and how many come before that word.
__device__ __forceinline__ void row_word_of(uint32_t counts, uint32_t j, uint32_t &q, uint32_t &before) {
    const uint32_t c0 = counts & 0xffu, c1 = (counts >> 8) & 0xffu, c2 = counts >> 16;
    q = j < c0 ? 0u : j < c1 ? 1u : j < c2 ? 2u : 3u;
    before = q == 0 ? 0u : q == 1 ? c0 : q == 2 ? c1 : c2;
}

// Certification of one warp row (planes pm / p0 / pp, row r) on the warp's
// diagonal (tile::cert4_diag; cc and carried as there): marks its uncertified
// vertices in P.ub and returns them as RowBits.  rowbase = the linear index of
// (0, y, z).
__device__ __forceinline__ RowBits certify_row(const FieldView &P, const float *pm, const float *p0, const float *pp,
                                               int r, int x0, uint32_t rowbase, tile::CubeCarry &cc, bool carried) {
    using namespace tile;
    const GridDev &G = P.G;
    const uint32_t lane = lane_id();
    const int xl = x0 + 4 * (int)lane;
    const uint32_t cert = cert4_diag(pm, p0, pp, r, lane, P.two_xi, cc, carried);
    const uint32_t i0 = rowbase + (uint32_t)xl;
    uint32_t nib = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) nib |= (uint32_t)(xl + e < (int)G.nx && !((cert >> e) & 1u)) << e;
    uint32_t w = nib << (4u * (lane & 7u));
    w |= __shfl_xor_sync(kFull, w, 1);
    w |= __shfl_xor_sync(kFull, w, 2);
    w |= __shfl_xor_sync(kFull, w, 4);
    const bool words_ok = ((rowbase + (uint32_t)x0) & 31u) == 0 && x0 + BX <= (int)G.nx;
    if (words_ok) {
        if ((lane & 7u) == 0) P.ub[i0 >> 5] = w;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if ((nib >> e) & 1u) red_or(&P.ub[(i0 + e) >> 5], 1u << ((i0 + e) & 31u));
    }
    RowBits b;
    b.from(w);
    return b;
}

// The code pass on two consecutive rows of a warp's diagonal (warp-
// collective): row ra of plane z (staged planes pm / p0 / pp) when has_a, and
// row rb of plane z+1 (p0 / pp / pq) when has_b; rowbase_a / rowbase_b = the
// linear index of (0, y, z) of each; the second field soff floats after each
// plane.  carried: cc holds the unit cubes of row ra-1 of plane z-1; on
// return it says whether cc holds those of row rb of plane z+1.  Both rows
// are certified first; their uncertified vertices then share rounds of 32
// (one a lane), so a round's exact codes -- of f, written to codes_f, and,
// when DETECT, of the second field, compared with it -- serve up to 32
// vertices of either row instead of the dozen or so that one row of a smooth
// field holds.
template <bool DETECT>
__device__ __forceinline__ void tile_rows2(const FieldView &P, const float *pm, const float *p0, const float *pp,
                                           const float *pq, int soff, int ra, bool has_a, int rb, bool has_b, int x0,
                                           uint32_t rowbase_a, uint32_t rowbase_b, tile::CubeCarry &cc,
                                           bool &carried, uint32_t &distorted) {
    const uint32_t lane = lane_id();
    RowBits A, B;
    A.w = A.counts = A.total = 0u;
    B = A;
    if (has_a) A = certify_row(P, pm, p0, pp, ra, x0, rowbase_a, cc, carried);
    carried = has_a && rb == ra + 1;
    if (has_b) B = certify_row(P, p0, pp, pq, rb, x0, rowbase_b, cc, carried);
    carried = has_b;
    const uint32_t total = A.total + B.total;
    Emitter E{P.dm[1], 0};
    for (uint32_t j0 = 0; j0 < total; j0 += 32u) {
        const uint32_t j = j0 + lane;
        const bool has = j < total;
        const bool sec = j >= A.total;  // a vertex of the second row
        const uint32_t base = (sec ? rowbase_b : rowbase_a) + (uint32_t)x0;
        // the word of each row the lane's vertex would be in (every lane
        // shuffles both rows' words), then the one row's column
        uint32_t qa, ba, qb, bb;
        row_word_of(A.counts, j, qa, ba);
        row_word_of(B.counts, j - A.total, qb, bb);
        const uint32_t wa = __shfl_sync(kFull, A.w, (int)(8u * qa)), wb = __shfl_sync(kFull, B.w, (int)(8u * qb));
        uint32_t col = 0, cf = 0, cg = 0;
        if (has) {
            col = 32u * (sec ? qb : qa) + tile::nth_set(sec ? wb : wa, sec ? j - A.total - bb : j - ba);
            const float *qm = sec ? p0 : pm, *q0 = sec ? pp : p0, *qp = sec ? pq : pp;
            const int r = sec ? rb : ra;
            cf = tile::code1(qm, q0, qp, r, 4 + (int)col);
            P.codes_f[base + col] = (uint8_t)cf;
            if (DETECT) cg = tile::code1(qm + soff, q0 + soff, qp + soff, r, 4 + (int)col);
        }
        if (DETECT) report(P, E, has, base + col, cf, cg, false, true);
    }
    distorted += E.distorted;
}

// The warp's row of plane p0 in the cp.async ring (row r, x0 .. x0+127, any
// x extent): bound check and g = start value, 4 vertices a lane.  The
// second field (fhat, or the start field when DETECT) sits PLANE floats
// after f.
template <bool DETECT>
__device__ __forceinline__ void own_row_cp(const FieldView &P, const float *p0, int r, int x0, uint32_t rowbase,
                                           bool &bad) {
    using namespace tile;
    const uint32_t lane = lane_id();
    const int xl = x0 + 4 * (int)lane;
    if (xl >= (int)P.G.nx) return;
    const float4 f4 = *reinterpret_cast<const float4 *>(p0 + r * PW + 4 + 4 * (int)lane);
    const float4 s4 = *reinterpret_cast<const float4 *>(p0 + PLANE + r * PW + 4 + 4 * (int)lane);
    const float fv[4] = {f4.x, f4.y, f4.z, f4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (xl + e >= (int)P.G.nx) break;
        const uint32_t gi = rowbase + (uint32_t)(xl + e);
        float fh = sv[e], gs = sv[e];
        if (P.ginit) {
            if (DETECT) fh = P.fhat[gi];
            else gs = P.ginit[gi];
        }
        // with f finite, L and U are finite, so L <= v <= U rules out a NaN
        // or infinite v
        const float L = floor_bound(fv[e], P.xi), U = ceil_bound(fv[e], P.xi);
        bool ok = isfinite(fv[e]) && fh >= L && fh <= U;
        if (P.ginit) {
            ok = ok && gs >= L && gs <= U;
            if (__float_as_uint(fh) != __float_as_uint(gs)) red_or(&P.eb[gi >> 5], 1u << (gi & 31u));
        }
        bad = bad || !ok;
        P.g[gi] = gs;
    }
}

// ------------------------------------------------ tiled (3D) codes of f
// One tile (x0, y0, planes zb .. ze-1) of field P: certification of every
// vertex, codes of f at the uncertified ones, g = start value, bound check
// (bad is set on a violation).
// DETECT: also sweep 0's detection of the tile's uncertified vertices, whose
// codes in the start field come from the staged planes; they mark targets and
// the worklist P.dm[1], and add to `distorted`.
// Block-collective; the caller synchronizes the block before the next tile.
// PAIR: rows of two planes a step (tile_rows2) on a ring of kPairSlots
// planes (z-1 .. z+2 in use, z+3 and z+4 in flight; one block barrier per
// two planes), else one plane a step (tile_row) on NSLOT planes.
template <bool DETECT, bool PAIR = false>
__device__ __forceinline__ void first_tile(const FieldView &P, int x0, int y0, int zb, int ze, float *smem,
                                           bool &bad, uint32_t &distorted) {
    constexpr int NS = PAIR ? tile::kPairSlots : tile::NSLOT;
    using namespace tile;
    const GridDev &G = P.G;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
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
    // second staged field: the start field over the whole region when this
    // pass detects (it needs the start values of the halo), else fhat over the
    // owned region
    const uint32_t secm = DETECT ? inm : ownm;
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
        for (int sl = 0; sl < NS; ++sl) {
            smem[sl * SLOT + r * PW + c + 3] = qnan;
            if (DETECT) smem[sl * SLOT + PLANE + r * PW + c + 3] = qnan;
        }
    }
    // this thread's staged elements: shared-memory word within a slot and
    // offset within a grid plane, computed once a tile
    uint32_t soff[PER_THREAD], goff[PER_THREAD];
#pragma unroll
    for (int j = 0; j < PER_THREAD; ++j) {
        const int e = (int)tid + j * THREADS;
        const int r = e / LOADW, c = e - r * LOADW;
        soff[j] = (uint32_t)(r * PW + c + 3);
        goff[j] = (uint32_t)(gbase + r * (int)G.nx + c);
    }
    // asynchronous copy of plane p (f over the staged region, the second
    // field over its region) into its ring slot; planes outside the grid
    // become NaN
    auto issue = [&](int p) {
        if (p >= 0 && p <= ze) {
            const int slot = (p - zb + 1) % NS;
            const bool inside = p < (int)G.nz;
            const uint32_t pb = (uint32_t)p * G.nxy;
            const float *sec = DETECT && P.ginit ? P.ginit : P.fhat;
#pragma unroll
            for (int j = 0; j < PER_THREAD; ++j) {
                if (!(inm >> j & 1u)) continue;
                const uint32_t so = (uint32_t)(slot * SLOT) + soff[j];
                if (!inside) {
                    smem[so] = qnan;
                    if (DETECT) smem[so + PLANE] = qnan;
                    continue;
                }
                const uint32_t gi = pb + goff[j];
                cp_async4(sbase + 4u * so, P.f + gi);
                if (secm >> j & 1u) cp_async4(sbase + 4u * (so + (uint32_t)PLANE), sec + gi);
            }
        } else if (p < 0) {
            const int slot = (p - zb + 1) % NS;
#pragma unroll
            for (int j = 0; j < PER_THREAD; ++j) {
                if (!(inm >> j & 1u)) continue;
                const int e = (int)tid + j * THREADS;
                const int r = e / LOADW, c = e - r * LOADW;
                smem[slot * SLOT + r * PW + c + 3] = qnan;
                if (DETECT) smem[slot * SLOT + PLANE + r * PW + c + 3] = qnan;
            }
        }
        cp_async_commit();
    };
    issue(zb - 1);
    issue(zb);
    issue(zb + 1);
    issue(zb + 2);
    auto plane = [&](int p) { return smem + ((p - zb + 1) % NS) * SLOT; };
    if constexpr (PAIR) {
        // each warp walks a diagonal: row ra of plane z, then row rb = ra+1
        // of plane z+1 (tile::diag_row)
        tile::CubeCarry cc;
        bool carried = false;
        for (int z = zb; z < ze; z += 2) {
            cp_async_wait<0>();  // planes up to z+2 of this thread have landed
            __syncthreads();     // ... of every thread; the slots of z-3 and z-2 are free
            issue(z + 3);
            issue(z + 4);
            const bool two = z + 1 < ze;
            const int ra = diag_row(warp, z - zb), rb = ra == BY ? 1 : ra + 1;
            const int ya = y0 + ra - 1, yb = y0 + rb - 1;
            const bool has_a = ya < (int)G.ny, has_b = two && yb < (int)G.ny;
            if (ra == 1) carried = false;
            if (!has_a && !has_b) {
                carried = false;
                continue;
            }
            const uint32_t rba = (uint32_t)z * G.nxy + (uint32_t)ya * G.nx;
            const uint32_t rbb = (uint32_t)(z + 1) * G.nxy + (uint32_t)yb * G.nx;
            if (has_a) own_row_cp<DETECT>(P, plane(z), ra, x0, rba, bad);
            if (has_b) own_row_cp<DETECT>(P, plane(z + 1), rb, x0, rbb, bad);
            tile_rows2<DETECT>(P, plane(z - 1), plane(z), plane(z + 1), plane(z + 2), PLANE, ra, has_a, rb, has_b,
                               x0, rba, rbb, cc, carried, distorted);
        }
    } else {
        const int y = y0 + (int)warp, r = (int)warp + 1;
        for (int z = zb; z < ze; ++z) {
            cp_async_wait<1>();  // planes up to z+1 of this thread have landed (z+2 may be in flight)
            __syncthreads();     // ... of every thread; the slot of z-2 is free
            issue(z + 3);
            if (y >= (int)G.ny) continue;
            const uint32_t rowbase = (uint32_t)z * G.nxy + (uint32_t)y * G.nx;
            own_row_cp<DETECT>(P, plane(z), r, x0, rowbase, bad);
            tile_row<DETECT>(P, plane(z - 1), plane(z), plane(z + 1), PLANE, r, x0, rowbase, distorted);
        }
    }
    cp_async_wait<0>();
}

// ------------------------------------------- tiled whole-grid detection (cp.async)
// One tile (x0, y0, planes zb .. ze-1) of field P in a whole-grid detection
// of a later sweep, for grids the TMA ring cannot stage: g is staged plane by
// plane through the cp.async ring (NaN outside the grid; field slot 0 only),
// and each warp examines its row's uncertified vertices 32 at a time, their
// codes of g from shared memory and of f from codes_f.  Distorted vertices
// mark their targets and themselves in dnext and add to `distorted`.
// Block-collective; the caller synchronizes the block before the next tile.
__device__ __forceinline__ void detect_tile_cp(const FieldView &P, int x0, int y0, int zb, int ze, float *smem,
                                               uint32_t *dnext, uint32_t &distorted, uint32_t *dsum = nullptr,
                                               uint32_t *tsum = nullptr) {
    using namespace tile;
    const GridDev &G = P.G;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    uint32_t inm = 0, soff[PER_THREAD], goff[PER_THREAD];
    const int gbase = (y0 - 1) * (int)G.nx + (x0 - 1);
#pragma unroll
    for (int j = 0; j < PER_THREAD; ++j) {
        const int e = (int)tid + j * THREADS;
        const int r = e / LOADW, c = e - r * LOADW;
        const int gx = x0 - 1 + c, gy = y0 - 1 + r;
        inm |= (uint32_t)(e < ELEMS && gx >= 0 && gx < (int)G.nx && gy >= 0 && gy < (int)G.ny) << j;
        soff[j] = (uint32_t)(r * PW + c + 3);
        goff[j] = (uint32_t)(gbase + r * (int)G.nx + c);
    }
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const float qnan = __int_as_float(0x7fffffff);
#pragma unroll
    for (int j = 0; j < PER_THREAD; ++j) {
        const int e = (int)tid + j * THREADS;
        if (e >= ELEMS || (inm >> j & 1u)) continue;
        for (int sl = 0; sl < NSLOT; ++sl) smem[sl * SLOT + soff[j]] = qnan;
    }
    auto issue = [&](int p) {
        if (p >= 0 && p <= ze) {
            const uint32_t so0 = (uint32_t)(((p - zb + 1) % NSLOT) * SLOT);
            const bool inside = p < (int)G.nz;
            const uint32_t pb = (uint32_t)p * G.nxy;
#pragma unroll
            for (int j = 0; j < PER_THREAD; ++j) {
                if (!(inm >> j & 1u)) continue;
                if (!inside) smem[so0 + soff[j]] = qnan;
                else cp_async4(sbase + 4u * (so0 + soff[j]), P.g + pb + goff[j]);
            }
        } else if (p < 0) {
            const uint32_t so0 = (uint32_t)(((p - zb + 1) % NSLOT) * SLOT);
#pragma unroll
            for (int j = 0; j < PER_THREAD; ++j)
                if (inm >> j & 1u) smem[so0 + soff[j]] = qnan;
        }
        cp_async_commit();
    };
    issue(zb - 1);
    issue(zb);
    issue(zb + 1);
    issue(zb + 2);
    const int y = y0 + (int)warp, r = (int)warp + 1;
    const int xl = x0 + 4 * (int)lane;
    const bool in = y < (int)G.ny && xl < (int)G.nx;
    const uint32_t valid = !in ? 0u : (int)G.nx - xl >= 4 ? 15u : (1u << ((int)G.nx - xl)) - 1u;
    // this lane's 4 uncertified bits (they may straddle two words) and codes
    // of f, loaded one plane ahead as raw values and combined where used, so
    // that their latency overlaps the examination of the plane before
    uint32_t ua = 0, ua1 = 0, cb[4] = {0u, 0u, 0u, 0u};
    auto fetch = [&](int z) {
        ua = 0;
        ua1 = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) cb[e] = 0;
        if (!in || z >= ze) return;
        const uint32_t i0 = (uint32_t)z * G.nxy + (uint32_t)y * G.nx + (uint32_t)xl, wi = i0 >> 5;
        ua = __ldg(&P.ub[wi]);
        if ((i0 & 31u) > 28u && wi + 1u < G.words) ua1 = __ldg(&P.ub[wi + 1u]);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if ((valid >> e) & 1u) cb[e] = __ldg(&P.codes_f[i0 + e]);
    };
    fetch(zb);
    Emitter E{dnext, 0, dsum, tsum};
    for (int z = zb; z < ze; ++z) {
        cp_async_wait<1>();
        __syncthreads();
        issue(z + 3);
        if (y >= (int)G.ny) continue;
        auto plane = [&](int p) { return smem + ((p - zb + 1) % NSLOT) * SLOT; };
        const uint32_t rowbase = (uint32_t)z * G.nxy + (uint32_t)y * G.nx;
        uint32_t nib = 0, cfw = 0;
        if (in) {
            const uint32_t sh = (rowbase + (uint32_t)xl) & 31u;
            uint32_t bits = ua >> sh;
            if (sh > 28u) bits |= ua1 << (32u - sh);
            nib = bits & valid;
            // codes of certified vertices are never written and never used
            cfw = cb[0] | cb[1] << 8 | cb[2] << 16 | cb[3] << 24;
        }
        fetch(z + 1);
        uint32_t w = nib << (4u * (lane & 7u));
        w |= __shfl_xor_sync(kFull, w, 1);
        w |= __shfl_xor_sync(kFull, w, 2);
        w |= __shfl_xor_sync(kFull, w, 4);
        const uint32_t w0 = __shfl_sync(kFull, w, 0), w1 = __shfl_sync(kFull, w, 8);
        const uint32_t w2 = __shfl_sync(kFull, w, 16), w3 = __shfl_sync(kFull, w, 24);
        const uint32_t c0 = (uint32_t)__popc(w0), c1 = c0 + (uint32_t)__popc(w1);
        const uint32_t c2 = c1 + (uint32_t)__popc(w2), total = c2 + (uint32_t)__popc(w3);
        for (uint32_t j0 = 0; j0 < total; j0 += 32u) {
            const uint32_t j = j0 + lane;
            const bool has = j < total;
            uint32_t col = 0, cg = 0;
            if (has) {
                const uint32_t q = j < c0 ? 0u : j < c1 ? 1u : j < c2 ? 2u : 3u;
                const uint32_t wq = q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : w3;
                const uint32_t before = q == 0 ? 0u : q == 1 ? c0 : q == 2 ? c1 : c2;
                col = 32u * q + nth_set(wq, j - before);
                cg = code1(plane(z - 1), plane(z), plane(z + 1), r, 4 + (int)col);
            }
            const uint32_t cf = (__shfl_sync(kFull, cfw, (int)(col >> 2)) >> (8u * (col & 3u))) & 0xffu;
            report(P, E, has, rowbase + (uint32_t)x0 + col, cf, cg);
        }
    }
    cp_async_wait<0>();
    distorted += E.distorted;
}

// Whole-grid detection of a later sweep over the tiles of one field (the
// cp.async form; block-collective).
__device__ __forceinline__ void detect_tiled_cp(const FieldView &P, uint32_t tile_z, uint32_t *tile_next, float *smem,
                                                uint32_t *dnext, uint32_t &distorted, uint32_t *dsum = nullptr,
                                               uint32_t *tsum = nullptr) {
    using namespace tile;
    const GridDev &G = P.G;
    const TileGeom tg = tile_geom(G.nx, G.ny, G.nz, tile_z);
    __shared__ uint32_t s_tile;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_next, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= tg.count) break;
        const uint32_t txi = t % tg.tx, tyi = (t / tg.tx) % tg.ty, tzi = t / (tg.tx * tg.ty);
        const int zb = (int)(tzi * tg.bz);
        detect_tile_cp(P, (int)(txi * BX), (int)(tyi * BY), zb, min(zb + (int)tg.bz, (int)G.nz), smem, dnext,
                       distorted, dsum, tsum);
    }
}

// Tiles of one field handed out by an atomic counter (block-collective).
// DETECT: the pass also runs sweep 0's detection (distorted vertices counted
// in `distorted`).  PAIR: the paired-row form of first_tile (its ring is
// kPairRingBytes of dynamic shared memory, else kRingBytes).
template <bool DETECT, bool PAIR = false>
__device__ __forceinline__ void first_tiled(const FieldView &P, uint32_t *tile_next, float *smem, uint32_t *err,
                                            uint32_t &distorted) {
    using namespace tile;
    const GridDev &G = P.G;
    const TileGeom tg = tile_geom(G.nx, G.ny, G.nz, P.tile_z);
    __shared__ uint32_t s_tile;
    bool bad = false;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_next, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= tg.count) break;
        const uint32_t txi = t % tg.tx, tyi = (t / tg.tx) % tg.ty, tzi = t / (tg.tx * tg.ty);
        const int zb = (int)(tzi * tg.bz);
        first_tile<DETECT, PAIR>(P, (int)(txi * BX), (int)(tyi * BY), zb, min(zb + (int)tg.bz, (int)G.nz), smem,
                                 bad, distorted);
    }
    if (bad) atomicOr(err, kErrInput);
}

// ------------------------------------------------ tiled (3D) codes, TMA ring
// The code pass with its planes staged by TMA (grids whose x extent is a
// multiple of 4 and at least PW, y extent at least ROWS, and whose arrays
// are 16-byte aligned).  A slot holds one plane of f and of the second field
// (map_s: the start field when DETECT, else fhat); a fill completes on the
// slot's mbarrier, and out-of-grid positions arrive as NaN from the maps'
// fill mode.  Warps never wait for one another inside a tile: each waits only
// for the planes it needs, and the last warp to finish with a plane refills
// its slot with the plane NS further on, so fast warps run ahead of slow
// ones by up to the planes in flight.  Every wait is bounded; a wait that runs out
// records kErrTimeout, stops the block's tiles and, before leaving, waits
// (bounded) for the block's copies still in flight.

// The warp's row of plane p0 (row r, x0 .. x0+127): bound check and g =
// start value, 4 vertices a lane (nx is a multiple of 4: all in or all out).
template <bool DETECT>
__device__ __forceinline__ void own_row_tma(const FieldView &P, const float *p0, int r, int x0, uint32_t rowbase,
                                            bool &bad) {
    using namespace tile;
    const uint32_t lane = lane_id();
    const int xl = x0 + 4 * (int)lane;
    if (xl >= (int)P.G.nx) return;
    const uint32_t gi = rowbase + (uint32_t)xl;
    const float4 f4 = *reinterpret_cast<const float4 *>(p0 + r * PW + 4 + 4 * (int)lane);
    const float4 s4 = *reinterpret_cast<const float4 *>(p0 + TFIELD + r * PW + 4 + 4 * (int)lane);
    float4 fh4 = s4, gs4 = s4;
    if (P.ginit) {
        if (DETECT) fh4 = *reinterpret_cast<const float4 *>(P.fhat + gi);
        else gs4 = *reinterpret_cast<const float4 *>(P.ginit + gi);
    }
    const float fv[4] = {f4.x, f4.y, f4.z, f4.w}, hv[4] = {fh4.x, fh4.y, fh4.z, fh4.w};
    const float gv[4] = {gs4.x, gs4.y, gs4.z, gs4.w};
    uint32_t differs = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        // with f finite, L and U are finite, so L <= v <= U already rules out
        // a NaN or infinite v
        const float L = floor_bound(fv[e], P.xi), U = ceil_bound(fv[e], P.xi);
        bool ok = isfinite(fv[e]) && hv[e] >= L && hv[e] <= U;
        if (P.ginit) {
            ok = ok && gv[e] >= L && gv[e] <= U;
            differs |= (uint32_t)(__float_as_uint(hv[e]) != __float_as_uint(gv[e])) << e;
        }
        bad = bad || !ok;
    }
    if (differs) red_or(&P.eb[gi >> 5], differs << (gi & 31u));  // gi is a multiple of 4: one word
    *reinterpret_cast<float4 *>(P.g + gi) = gs4;
}

// The TMA plane ring over the tiles of field P (block-collective): NBOX
// boxes a plane (maps[0..NBOX-1], each TFIELD floats after the previous one
// in a slot).  STEP 1: row(pm, p0, pp, pq, r, x0, rowbase, two) runs for
// every warp row inside the grid with the staged planes z-1, z, z+1 (two
// false, pq unused); STEP 2: once for the rows of planes z and z+1 (two
// true; rowbase the linear index of (0, y, z)), pq staging plane z+2, or for
// row z alone (two false) when the tile's last plane is z.  withhold (a test
// hook): block 0 never issues its first plane, so its waits run out after
// kTestWaitNs.  DIAG: the rows are the caller's to choose (each warp's
// diagonal): row(pm, p0, pp, pq, x0, y0, z, zb, two) runs for every warp and
// step, whether or not its rows lie in the grid.
template <int NBOX, int STEP, int NS, bool DIAG = false, class ROW>
__device__ __forceinline__ void tma_tiles(const FieldView &P, uint32_t tile_z, const CUtensorMap *map0,
                                          const CUtensorMap *map1, uint32_t *tile_next, float *smem_raw,
                                          uint32_t *err, ROW &&row, bool withhold = false) {
    using namespace tile;
    const GridDev &G = P.G;
    const TileGeom tg = tile_geom(G.nx, G.ny, G.nz, tile_z);
    constexpr uint32_t kWarps = THREADS / 32;
    __shared__ uint32_t s_tile;
    constexpr int TSLOT = NBOX * TFIELD;  // floats of one slot
    __shared__ __align__(8) uint64_t s_full[NS];
    __shared__ uint32_t s_rel[NS];
    __shared__ uint32_t s_pending[NS];
    __shared__ uint32_t s_dead;
    float *ring = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    __syncthreads();  // the ring's previous users are done with its barriers
    if (tid == 0) {
        for (int q = 0; q < NS; ++q) {
            tma::mbar_init(tma::smem_u32(&s_full[q]), 1);
            s_rel[q] = 0;
            s_pending[q] = 0;
        }
        s_dead = 0;
        tma::fence_mbarrier_init();
    }
    // g may have been written by generic stores earlier in this kernel (made
    // visible by a grid barrier); every thread that issues copies orders them
    // before its TMA reads
    tma::fence_proxy_async_global();
    __syncthreads();
    uint32_t ph = 0;  // bit q: parity of the next completion of slot q's barrier
    const uint64_t limit = withhold ? tma::kTestWaitNs : tma::kWaitNs;
    bool first_tile = true;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_tile = atomicAdd(tile_next, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= tg.count || s_dead) break;
        const uint32_t txi = t % tg.tx, tyi = (t / tg.tx) % tg.ty, tzi = t / (tg.tx * tg.ty);
        const int x0 = (int)(txi * BX), y0 = (int)(tyi * BY), zb = (int)(tzi * tg.bz);
        const int ze = min(zb + (int)tg.bz, (int)G.nz);
        auto slot_of = [&](int p) { return (p - zb + 1) % NS; };
        auto issue = [&](int p, int q) {
            const uint32_t bar = tma::smem_u32(&s_full[q]);
            const uint32_t dst = tma::smem_u32(ring + q * TSLOT);
            s_pending[q] = 1;
            tma::mbar_expect_tx(bar, (uint32_t)NBOX * kTboxBytes);
            tma::load_3d(dst, map0, x0 - 4, y0 - 1, p, bar);
            if (NBOX > 1) tma::load_3d(dst + 4u * TFIELD, map1, x0 - 4, y0 - 1, p, bar);
        };
        auto wait_plane = [&](int p) -> bool {
            const int q = slot_of(p);
            if (!tma::mbar_wait_bounded(tma::smem_u32(&s_full[q]), (ph >> q) & 1u, &s_dead, limit)) return false;
            ph ^= 1u << q;
            if (tid == 0) s_pending[q] = 0;
            return true;
        };
        // planes zb-1 .. ze; the first NS now, each later one when the plane
        // NS before it is released
        if (tid == 0) {
            tma::fence_proxy_async();  // the previous tile's reads of the ring come first
            for (int q = 0; q < NS && zb - 1 + q <= ze; ++q)
                if (!(withhold && first_tile && blockIdx.x == 0 && q == 0)) issue(zb - 1 + q, q);
        }
        first_tile = false;
        // this warp is done with plane p: the last warp to say so refills its
        // slot with plane p + NS
        auto release = [&](int p) {
            if (lane == 0) {
                const int q = slot_of(p);
                __threadfence_block();
                if (atomicAdd(&s_rel[q], 1u) == kWarps - 1u) {
                    s_rel[q] = 0;
                    __threadfence_block();
                    if (p + NS <= ze) {
                        tma::fence_proxy_async();
                        issue(p + NS, q);
                    }
                }
            }
        };
        bool alive = wait_plane(zb - 1) && wait_plane(zb);
        const int y = y0 + (int)warp, r = (int)warp + 1;
        for (int z = zb; alive && z < ze; z += STEP) {
            const bool two = STEP == 2 && z + 1 < ze;
            if (!wait_plane(z + 1) || (two && !wait_plane(z + 2))) {
                alive = false;
                break;
            }
            const float *pm = ring + slot_of(z - 1) * TSLOT, *p0 = ring + slot_of(z) * TSLOT;
            const float *pp = ring + slot_of(z + 1) * TSLOT;
            const float *pq = two ? ring + slot_of(z + 2) * TSLOT : pp;
            if constexpr (DIAG) row(pm, p0, pp, pq, x0, y0, z, zb, two);
            else if (y < (int)G.ny) row(pm, p0, pp, pq, r, x0, (uint32_t)z * G.nxy + (uint32_t)y * G.nx, two);
            __syncwarp();
            release(z - 1);
            if (two) release(z);
        }
        if (!alive) {
            atomicOr(err, kErrTimeout);
            s_dead = 1;
        }
    }
    if (s_dead && tid == 0) {
        // copies still in flight land before the block leaves (bounded)
        uint32_t none = 0;
        for (int q = 0; q < NS; ++q)
            if (s_pending[q]) tma::mbar_wait_bounded(tma::smem_u32(&s_full[q]), (ph >> q) & 1u, &none, limit);
    }
}

// The code pass (sweep 0) on the TMA ring: f and the second field (the start
// field when DETECT, else fhat) a plane, two planes a step (tile_rows2).
template <bool DETECT>
__device__ __forceinline__ void first_tiled_tma(const FieldView &P, const CUtensorMap *map_f, const CUtensorMap *map_s,
                                                uint32_t *tile_next, float *smem_raw, uint32_t *err,
                                                uint32_t &distorted, bool withhold = false) {
    bool bad = false;
    tile::CubeCarry cc;
    bool carried = false;
    tma_tiles<2, 2, tile::kCodeSlots, true>(
        P, P.tile_z, map_f, map_s, tile_next, smem_raw, err,
        [&](const float *pm, const float *p0, const float *pp, const float *pq, int x0, int y0, int z, int zb,
            bool two) {
            // each warp walks a diagonal: row ra of plane z, then row rb =
            // ra+1 of plane z+1 (tile::diag_row)
            const GridDev &G = P.G;
            const int ra = tile::diag_row(threadIdx.x >> 5, z - zb), rb = ra == tile::BY ? 1 : ra + 1;
            const int ya = y0 + ra - 1, yb = y0 + rb - 1;
            const bool has_a = ya < (int)G.ny, has_b = two && yb < (int)G.ny;
            if (z == zb || ra == 1) carried = false;
            if (!has_a && !has_b) {
                carried = false;
                return;
            }
            const uint32_t rba = (uint32_t)z * G.nxy + (uint32_t)ya * G.nx;
            const uint32_t rbb = (uint32_t)(z + 1) * G.nxy + (uint32_t)yb * G.nx;
            if (has_a) own_row_tma<DETECT>(P, p0, ra, x0, rba, bad);
            if (has_b) own_row_tma<DETECT>(P, pp, rb, x0, rbb, bad);
            tile_rows2<DETECT>(P, pm, p0, pp, pq, tile::TFIELD, ra, has_a, rb, has_b, x0, rba, rbb, cc, carried,
                               distorted);
        },
        withhold);
    if (bad) atomicOr(err, kErrInput);
}

// Whole-grid detection of a later sweep on the TMA ring (g a plane): every
// uncertified vertex gets its code in g from the staged planes and its code
// of f from codes_f; distorted ones mark their targets and themselves in
// dnext (the next sweep's worklist).  nx is a multiple of 4, so a lane's 4
// vertices have their 4 uncertified bits in one bitmap word and their codes
// of f in one aligned 32-bit word.  Both are loaded one plane ahead (the
// warp's row of plane z+1 while it examines plane z), so their latency
// overlaps the examination and the wait for the next staged plane.
__device__ __forceinline__ void detect_tiled_tma(const FieldView &P, uint32_t tile_z, const CUtensorMap *map_g,
                                                 uint32_t *tile_next, float *smem_raw, uint32_t *err,
                                                 uint32_t *dnext, uint32_t &distorted, uint32_t *dsum = nullptr,
                                               uint32_t *tsum = nullptr) {
    using namespace tile;
    const GridDev &G = P.G;
    // the prefetched row: index of the tile row's first vertex (x0, y, z),
    // this lane's raw bitmap word and codes
    uint32_t pf_row = 0xffffffffu, pf_ubw = 0, pf_cfw = 0;
    tma_tiles<1, 1, tile::kDetectSlots>(P, tile_z, map_g, nullptr, tile_next, smem_raw, err,
                    [&](const float *pm, const float *p0, const float *pp, const float *, int r, int x0,
                        uint32_t rowbase, bool) {
                     const uint32_t lane = lane_id();
                     const int xl = x0 + 4 * (int)lane;
                     const bool in = xl < (int)G.nx;
                     // the row's uncertified bits and codes of f (coalesced);
                     // a vertex's code of f then comes from the lane that
                     // loaded it
                     uint32_t ubw = 0, cfw = 0;
                     if (pf_row == rowbase + (uint32_t)x0) {
                         ubw = pf_ubw;
                         cfw = pf_cfw;
                     } else if (in) {
                         const uint32_t i0 = rowbase + (uint32_t)xl;
                         ubw = __ldg(&P.ub[i0 >> 5]);
                         cfw = __ldg(reinterpret_cast<const uint32_t *>(P.codes_f + i0));
                     }
                     // the same tile row of the next plane (a whole grid row
                     // lies in the grid when its first vertex does)
                     const uint32_t next = rowbase + G.nxy;
                     pf_row = next + (uint32_t)x0;
                     pf_ubw = 0;
                     pf_cfw = 0;
                     if (in && next < G.n) {
                         const uint32_t i1 = next + (uint32_t)xl;
                         pf_ubw = __ldg(&P.ub[i1 >> 5]);
                         pf_cfw = __ldg(reinterpret_cast<const uint32_t *>(P.codes_f + i1));
                     }
                     const uint32_t nib = in ? (ubw >> ((rowbase + (uint32_t)xl) & 31u)) & 15u : 0u;
                     uint32_t w = nib << (4u * (lane & 7u));
                     w |= __shfl_xor_sync(kFull, w, 1);
                     w |= __shfl_xor_sync(kFull, w, 2);
                     w |= __shfl_xor_sync(kFull, w, 4);
                     const uint32_t w0 = __shfl_sync(kFull, w, 0), w1 = __shfl_sync(kFull, w, 8);
                     const uint32_t w2 = __shfl_sync(kFull, w, 16), w3 = __shfl_sync(kFull, w, 24);
                     const uint32_t c0 = (uint32_t)__popc(w0), c1 = c0 + (uint32_t)__popc(w1);
                     const uint32_t c2 = c1 + (uint32_t)__popc(w2), total = c2 + (uint32_t)__popc(w3);
                     Emitter E{dnext, 0, dsum, tsum};
                     for (uint32_t j0 = 0; j0 < total; j0 += 32u) {
                         const uint32_t j = j0 + lane;
                         const bool has = j < total;
                         uint32_t col = 0, cg = 0;
                         if (has) {
                             const uint32_t q = j < c0 ? 0u : j < c1 ? 1u : j < c2 ? 2u : 3u;
                             const uint32_t wq = q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : w3;
                             const uint32_t before = q == 0 ? 0u : q == 1 ? c0 : q == 2 ? c1 : c2;
                             col = 32u * q + nth_set(wq, j - before);
                             cg = code1(pm, p0, pp, r, 4 + (int)col);
                         }
                         const uint32_t cf = (__shfl_sync(kFull, cfw, (int)(col >> 2)) >> (8u * (col & 3u))) & 0xffu;
                         report(P, E, has, rowbase + (uint32_t)x0 + col, cf, cg);
                     }
                     distorted += E.distorted;
                 });
}

// Sets the bits of up to 3 consecutive vertices j0, j0+1, j0+2 (bit k of m
// for vertex j0+k) with one reduction per bitmap word touched.
__device__ __forceinline__ void mark_run(uint32_t *bm, uint32_t j0, uint32_t m, uint32_t *sum = nullptr) {
    const uint32_t w = j0 >> 5, s = j0 & 31u;
    red_or(&bm[w], m << s);
    const bool spill = s && (m >> (32u - s));
    if (spill) red_or(&bm[w + 1], m >> (32u - s));
    if (sum) {
        mark_chunk(sum, j0);
        if (spill && ((w + 1u) >> 5) != (w >> 5)) mark_chunk(sum, j0 + 32u);
    }
}

// Marks vertex t and its neighbours in bitmap bm.  The closed neighbourhood
// lies on 7 grid rows in 3D (3 in 2D), each holding a run of 2 or 3
// consecutive vertices: (y, z) at x-1 .. x+1; (y-1, z), (y, z-1) and
// (y-1, z-1) at x-1, x; (y+1, z), (y, z+1) and (y+1, z+1) at x, x+1.  One
// reduction marks a run (two where it crosses a word).
template <int NDIM>
__device__ __forceinline__ void mark_closed(const GridDev &G, uint32_t t, uint32_t *bm, uint32_t *sum = nullptr) {
    uint32_t x, y, z;
    coords_of(G, t, x, y, z);
    // bit 0: x-1, bit 1: x, bit 2: x+1 -- dropped outside the grid
    const uint32_t xm = x > 0 ? 1u : 0u, xp = x + 1 < G.nx ? 4u : 0u;
    auto row = [&](uint32_t rt, uint32_t m) {
        m &= xm | 2u | xp;
        if (x == 0) mark_run(bm, rt, m >> 1, sum);
        else mark_run(bm, rt - 1u, m, sum);
    };
    const uint32_t nx = G.nx, nxy = G.nxy;
    row(t, 7u);
    if (y > 0) row(t - nx, 3u);
    if (y + 1 < G.ny) row(t + nx, 6u);
    if (NDIM == 3) {
        if (z > 0) {
            row(t - nxy, 3u);
            if (y > 0) row(t - nxy - nx, 3u);
        }
        if (z + 1 < G.nz) {
            row(t + nxy, 6u);
            if (y + 1 < G.ny) row(t + nxy + nx, 6u);
        }
    }
}

// Eq. 1 on target t of field P (once per sweep).  Returns whether g_t
// decreased.
__device__ __forceinline__ bool edit_target(const FieldView &P, uint32_t t) {
    const float gt = P.g[t];
    const float L = floor_bound(__ldg(&P.f[t]), P.xi);
    float h;
    if (P.cand) {
        // BELOW_REFERENCE: the smallest requested value, at or above the
        // floor; the record is reset for the next sweep
        const float c = from_total_key(P.cand[t]);
        P.cand[t] = 0xffffffffu;
        h = c < L ? L : c;
        if (!(h < gt)) return false;
    } else if (!edit_value(gt, L, P.rule, h)) {
        return false;
    }
    P.g[t] = h;
    return true;
}

// Eq. 1 on target t of field P (once per sweep); a changed target marks the
// edited bitmap and, unless the next sweep scans densely, its closed
// neighbourhood in the next worklist.  Returns whether g_t decreased.
template <int NDIM>
__device__ __forceinline__ bool apply_target(const FieldView &P, uint32_t t, bool dense_next, uint32_t *dnext,
                                             uint32_t *dsum = nullptr) {
    if (!edit_target(P, t)) return false;
    red_or(&P.eb[t >> 5], 1u << (t & 31u));
    if (dense_next) return true;
    mark_closed<NDIM>(P.G, t, dnext, dsum);
    return true;
}

}  // namespace msz
