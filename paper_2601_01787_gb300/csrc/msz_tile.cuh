// msz_tile.cuh -- shared-memory tiled dense pass over a 3D grid.
//
// A block of 256 threads (8 warps) owns a tile of 128 (x) x 8 (y) vertices
// and marches it through a range of z planes.  The field planes it needs
// (rows y0-1 .. y0+8, columns x0-1 .. x0+128) are staged through a ring of 5
// shared-memory slots filled by cp.async: planes z+2 and z+3 are in flight
// while plane z is computed from the slots of z-1, z and z+1.  Staged
// positions outside the grid hold NaN, which never wins a comparison.  Each
// lane certifies 4 consecutive vertices of a row from the two largest and
// two smallest values of their closed neighbourhoods: in the one-plane form
// (cert4) read as 7 row segments (one 16-byte shared-memory load plus one
// halo value passed by a warp shuffle each); in the two-plane forms of the
// code pass (cert4_diag) as two unit cubes, each warp walking a diagonal of
// the tile so that every cube serves two vertices.  The exact codes are then
// formed one vertex per lane, only for the vertices left uncertified.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "msz_device.cuh"

namespace msz {
namespace tile {

constexpr int BX = 128;          // vertices per warp row (32 lanes x 4)
constexpr int BY = 8;            // rows per tile (one per warp)
constexpr int THREADS = 256;
constexpr int ROWS = BY + 2;     // staged rows y0-1 .. y0+8
constexpr int PW = 136;          // staged row pitch: column c <-> x = x0 - 4 + c
constexpr int LOADW = BX + 2;    // loaded columns x0-1 .. x0+128 (c = 3 .. 132)
constexpr int PLANE = ROWS * PW; // floats per staged plane of one field
constexpr int NSLOT = 5;        // ring: planes z-1, z, z+1 in use, z+2 and z+3 in flight
constexpr int ELEMS = ROWS * LOADW;                       // loaded values per plane per field
constexpr int PER_THREAD = (ELEMS + THREADS - 1) / THREADS;  // 6

__device__ __forceinline__ void cp_async4(uint32_t saddr, const float *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One ring slot: the staged plane of f, then the plane of a second field with
// the same indexing (fhat over the owned region only, or the start field of
// the loop over the whole staged region when sweep 0's detection runs in the
// pass).
constexpr int SLOT = 2 * PLANE;
constexpr size_t kRingBytes = (size_t)NSLOT * SLOT * sizeof(float);
// The ring of the paired-row form (two planes a step): z-1 .. z+2 in use,
// z+3 and z+4 in flight.
constexpr int kPairSlots = 6;
constexpr size_t kPairRingBytes = (size_t)kPairSlots * SLOT * sizeof(float);

// The ring when TMA stages the planes: each slot holds two boxes of ROWS x PW
// floats (x0-4 .. x0+131, y0-1 .. y0+8: the same indexing as above), f first,
// then the second field TFIELD floats later; every box starts on a 128-byte
// boundary.
constexpr int TBOX = ROWS * PW;                                  // 1360 floats
constexpr int TFIELD = 1376;                                     // 5504 bytes
constexpr uint32_t kTboxBytes = (uint32_t)TBOX * sizeof(float);  // 5440
// Slots of the TMA rings.  The code pass takes two planes a step (rows z and
// z+1 use planes z-1 .. z+2) with two more in flight; it runs as a kernel of
// its own, so its ring does not shrink the L1 of the loop kernel, whose
// whole-grid detection stages one field a step with one plane in flight.
constexpr int kCodeSlots = 6;
constexpr int kDetectSlots = 5;
// ring bytes for `slots` slots of `nbox` boxes (+ alignment slack)
constexpr size_t tma_ring_bytes(int slots, int nbox) {
    return (size_t)slots * nbox * TFIELD * sizeof(float) + 128;
}
static_assert(TFIELD >= TBOX && (TFIELD * 4) % 128 == 0, "TMA boxes must start on 128-byte boundaries");

struct TileGeom {
    uint32_t tx, ty, tz;   // tiles along each axis
    uint32_t bz;           // planes per tile
    uint32_t count;
};

__host__ __device__ inline TileGeom tile_geom(uint32_t nx, uint32_t ny, uint32_t nz, uint32_t bz) {
    TileGeom t;
    t.tx = (nx + BX - 1) / BX;
    t.ty = (ny + BY - 1) / BY;
    t.bz = bz;
    t.tz = (nz + bz - 1) / bz;
    t.count = t.tx * t.ty * t.tz;
    return t;
}

// NaN-propagating min / max (PTX min.NaN / max.NaN): a NaN operand gives NaN.
__device__ __forceinline__ float fmin_nan(float a, float b) {
    float d;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float fmax_nan(float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
// Three-input max / min ignoring NaN operands (NaN only when all three are):
// one instruction, at the rate of the two-input form.
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Per-lane two largest and two smallest values of the closed neighbourhoods
// of 4 consecutive vertices (ties count twice: equal values give a zero
// margin).  The margins hv - h2 and l2 - lv decide whether a vertex can ever
// be distorted; the winners' slots are not tracked.
//
// Candidates come in pairs (a, b) of one row segment.  A NaN (a position
// outside the grid) must never make a vertex look certified; it may make one
// look uncertified, which only costs an examination:
//   - pair of two NaNs: hi = lo = NaN, and the NaN-propagating min against
//     the leader keeps every value unchanged;
//   - pair (NaN, w): hi = lo = w, so w counts twice -- a false tie at worst.
struct Top2x4 {
    float hv[4], h2[4], lv[4], l2[4];
    // the first pair: leader and runner-up in each direction (all NaN when
    // the pair is, which later pairs then replace)
    __device__ __forceinline__ void first2(int e, float a, float b) {
        const float hi = fmaxf(a, b), lo = fminf(a, b);
        hv[e] = hi;
        h2[e] = lo;
        lv[e] = lo;
        l2[e] = hi;
    }
    // 8 ops a pair (both directions): its larger value against the leader,
    // its smaller one straight into the runner-up, and the mirror image
    __device__ __forceinline__ void take2(int e, float a, float b) {
        const float hi = fmaxf(a, b), lo = fminf(a, b);
        h2[e] = fmax3(h2[e], lo, fmin_nan(hv[e], hi));
        hv[e] = fmaxf(hv[e], hi);
        l2[e] = fmin3(l2[e], hi, fmax_nan(lv[e], lo));
        lv[e] = fminf(lv[e], lo);
    }
    // one candidate; a NaN leaves every value unchanged
    __device__ __forceinline__ void take(int e, float w) {
        h2[e] = fmaxf(h2[e], fmin_nan(hv[e], w));
        hv[e] = fmaxf(hv[e], w);
        l2[e] = fminf(l2[e], fmax_nan(lv[e], w));
        lv[e] = fminf(lv[e], w);
    }
    // Certified: in f the winner beats the runner-up by more than 2 xi in both
    // directions (differences rounded down), so no g with |g - f| <= xi can
    // change either winner.  A NaN runner-up (a single value) never certifies.
    __device__ __forceinline__ bool certified(int e, float two_xi) const {
        return __fsub_rd(hv[e], h2[e]) > two_xi && __fsub_rd(l2[e], lv[e]) > two_xi;
    }
};

// Row segment x-1 .. x+3 (left type) or x .. x+4 (right type) of one staged row.
struct Seg {
    float v[5];
};

__device__ __forceinline__ Seg seg_left(const float *row, uint32_t lane) {
    const float4 q = *reinterpret_cast<const float4 *>(row + 4 + 4 * lane);
    float left = __shfl_up_sync(kFull, q.w, 1);
    if (lane == 0) left = row[3];
    Seg s;
    s.v[0] = left; s.v[1] = q.x; s.v[2] = q.y; s.v[3] = q.z; s.v[4] = q.w;
    return s;
}

__device__ __forceinline__ Seg seg_right(const float *row, uint32_t lane) {
    const float4 q = *reinterpret_cast<const float4 *>(row + 4 + 4 * lane);
    float right = __shfl_down_sync(kFull, q.x, 1);
    if (lane == 31) right = row[4 + BX];
    Seg s;
    s.v[0] = q.x; s.v[1] = q.y; s.v[2] = q.z; s.v[3] = q.w; s.v[4] = right;
    return s;
}

// Certification bits (bit e) of the 4 vertices of this lane in the field
// staged at pm / p0 / pp (planes z-1, z, z+1; each pointer at the start of the
// tile plane) for warp row r (1 .. BY).  The 15 values of a closed
// neighbourhood come from 7 row segments: (y-1,z-1) and (y,z-1) at x-1, x;
// (y-1,z) at x-1, x; (y,z) at x-1, x, x+1; (y+1,z), (y,z+1) and (y+1,z+1) at
// x, x+1.  Every staged position outside the grid holds NaN, so no domain
// mask is needed.
__device__ __forceinline__ uint32_t cert4(const float *pm, const float *p0, const float *pp, int r, uint32_t lane,
                                          float two_xi) {
    Top2x4 x;
    auto pair_left = [&](const float *row) {  // x-1 and x
        const Seg s = seg_left(row, lane);
#pragma unroll
        for (int e = 0; e < 4; ++e) x.take2(e, s.v[e], s.v[e + 1]);
    };
    auto pair_right = [&](const float *row) {  // x and x+1
        const Seg s = seg_right(row, lane);
#pragma unroll
        for (int e = 0; e < 4; ++e) x.take2(e, s.v[e], s.v[e + 1]);
    };
    {
        const Seg s = seg_left(pm + (r - 1) * PW, lane);  // (y-1, z-1): x-1, x
#pragma unroll
        for (int e = 0; e < 4; ++e) x.first2(e, s.v[e], s.v[e + 1]);
    }
    pair_left(pm + r * PW);
    pair_left(p0 + (r - 1) * PW);
    {
        const Seg s = seg_left(p0 + r * PW, lane);  // (y, z): x-1, x, x+1
        float right = __shfl_down_sync(kFull, s.v[1], 1);
        if (lane == 31) right = p0[r * PW + 4 + BX];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            x.take2(e, s.v[e], s.v[e + 1]);
            x.take(e, e < 3 ? s.v[e + 2] : right);
        }
    }
    pair_right(p0 + (r + 1) * PW);
    pair_right(pp + r * PW);
    pair_right(pp + (r + 1) * PW);
    uint32_t cert = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) cert |= (uint32_t)x.certified(e, two_xi) << e;
    return cert;
}

// ------------------------------------------- certification along the diagonal
// The closed Freudenthal neighbourhood of a vertex i is the union of two unit
// cubes: C(i) = i + {0,1}^3 (the vertex and its 7 positive offsets) and
// C(i - (1,1,1)) = i - {0,1}^3 (the vertex and its 7 negative offsets).  The
// forward cube of a vertex is therefore the backward cube of the vertex one
// step further along the main diagonal.  A warp that certifies row y of plane
// z and then row y+1 of plane z+1 forms each cube once and uses it twice,
// and a cube is itself the union of two 2 x 2 columns (fixed x, y..y+1,
// z..z+1), each shared by two neighbouring cubes of the row.  Merging these
// partial results costs about 40 ALU-pipe cycles a vertex against about 70
// for the 7 row segments of cert4.
//
// The vertex itself lies in both cubes.  Where it leads the union, the
// runner-up is taken from the two cubes' runners-up instead (cert4_diag), so
// that a strict local maximum or minimum is not held back by its own value
// counted twice.

// The two largest and two smallest values of a multiset (NaN: no value).
struct T2 {
    float h1, h2, l1, l2;
};

// The union of two multisets: the larger leader leads, the runner-up is the
// largest of the smaller leader and both runners-up (the leaders compared
// with NaN propagation, so an empty side adds nothing).
__device__ __forceinline__ T2 t2_merge(const T2 &a, const T2 &b) {
    T2 t;
    t.h1 = fmaxf(a.h1, b.h1);
    t.h2 = fmax3(fmin_nan(a.h1, b.h1), a.h2, b.h2);
    t.l1 = fminf(a.l1, b.l1);
    t.l2 = fmin3(fmax_nan(a.l1, b.l1), a.l2, b.l2);
    return t;
}

// T2 of a 2 x 2 column: the pairs (a, b) and (c, d).  A pair with one NaN
// counts its other value twice (a false tie at worst, which withholds a
// certification but never grants one); a pair of two NaNs counts nothing.
__device__ __forceinline__ T2 t2_quad(float a, float b, float c, float d) {
    const float hi1 = fmaxf(a, b), lo1 = fminf(a, b), hi2 = fmaxf(c, d), lo2 = fminf(c, d);
    T2 t;
    t.h1 = fmaxf(hi1, hi2);
    t.h2 = fmax3(fmin_nan(hi1, hi2), lo1, lo2);
    t.l1 = fminf(lo1, lo2);
    t.l2 = fmin3(fmax_nan(lo1, lo2), hi1, hi2);
    return t;
}

// One staged row at the lane's columns x-1 .. x-1+NV-1 (x = x0 + 4 lane;
// NV = 5 or 6): one 16-byte load, the outer columns passed by warp shuffles.
template <int NV>
__device__ __forceinline__ void row_vals(const float *row, uint32_t lane, float (&v)[NV]) {
    static_assert(NV == 5 || NV == 6, "columns x-1 .. x+3 or x+4");
    const float4 q = *reinterpret_cast<const float4 *>(row + 4 + 4 * lane);
    float left = __shfl_up_sync(kFull, q.w, 1);
    if (lane == 0) left = row[3];
    v[0] = left; v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
    if constexpr (NV == 6) {
        float right = __shfl_down_sync(kFull, q.x, 1);
        if (lane == 31) right = row[4 + BX];
        v[5] = right;
    }
}

// T2 of the unit cubes (c..c+1) x (y..y+1) x (z..z+1) at the lane's columns
// c = x-1 .. x-1+NC-1, from staged rows r (y) and r+1 of planes pa (z) and
// pb (z+1): each 2 x 2 column once, each cube the merge of two of them.
template <int NC>
__device__ __forceinline__ void unit_cubes(const float *pa, const float *pb, int r, uint32_t lane, T2 (&cb)[NC]) {
    float v0[NC + 1], v1[NC + 1], v2[NC + 1], v3[NC + 1];
    row_vals<NC + 1>(pa + r * PW, lane, v0);
    row_vals<NC + 1>(pa + (r + 1) * PW, lane, v1);
    row_vals<NC + 1>(pb + r * PW, lane, v2);
    row_vals<NC + 1>(pb + (r + 1) * PW, lane, v3);
    T2 prev = t2_quad(v0[0], v1[0], v2[0], v3[0]);
#pragma unroll
    for (int k = 1; k <= NC; ++k) {
        const T2 cur = t2_quad(v0[k], v1[k], v2[k], v3[k]);
        cb[k - 1] = t2_merge(prev, cur);
        prev = cur;
    }
}

// The backward cubes of the lane's 4 vertices in the next row on the
// diagonal: the unit cubes at columns x-1 .. x+2 of the row certified last.
struct CubeCarry {
    T2 c[4];
};

// Certification bits (bit e) of the lane's 4 vertices in warp row r of the
// plane staged at p0 (p1: plane z+1; pm: plane z-1, read only when !carried).
// carried: cc holds the unit cubes at (x-1 .., y-1, z-1), i.e. this warp
// certified row r-1 of plane z-1 last; otherwise they are formed here.  On
// return cc holds this row's cubes for row r+1 of plane z+1.  A vertex is
// certified when in f its winner beats the runner-up by more than 2 xi in
// both directions (differences rounded down), as in cert4.
__device__ __forceinline__ uint32_t cert4_diag(const float *pm, const float *p0, const float *p1, int r, uint32_t lane,
                                               float two_xi, CubeCarry &cc, bool carried) {
    if (!carried) unit_cubes<4>(pm, p0, r - 1, lane, cc.c);
    T2 fw[5];
    unit_cubes<5>(p0, p1, r, lane, fw);
    // the vertices' own values: both cubes hold them
    const float4 sv = *reinterpret_cast<const float4 *>(p0 + r * PW + 4 + 4 * lane);
    const float self[4] = {sv.x, sv.y, sv.z, sv.w};
    const float qnan = __int_as_float(0x7fffffff);
    uint32_t cert = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const T2 &a = fw[e + 1], &b = cc.c[e];
        // When the leader of the union is the vertex's own value, both cubes
        // lead with it (each holds the vertex), and the smaller leader is that
        // same vertex counted twice, not a runner-up: the runner-up is the
        // larger of the two cubes' runners-up (each the best of its cube
        // after one copy of the vertex; a neighbour tied with the vertex
        // still shows there).  Otherwise the plain union rule holds.
        const float h1 = fmaxf(a.h1, b.h1), l1 = fminf(a.l1, b.l1);
        const float mh = h1 == self[e] ? qnan : fmin_nan(a.h1, b.h1);
        const float ml = l1 == self[e] ? qnan : fmax_nan(a.l1, b.l1);
        const float h2 = fmax3(mh, a.h2, b.h2), l2 = fmin3(ml, a.l2, b.l2);
        cert |= (uint32_t)(__fsub_rd(h1, h2) > two_xi && __fsub_rd(l2, l1) > two_xi) << e;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) cc.c[e] = fw[e];
    return cert;
}

// Row of warp w on the diagonal at plane offset s = z - zb of a tile: row
// (w + s) mod BY, as a staged row index (1 .. BY).  Over a plane the BY warps
// cover every row once; from one plane to the next each warp moves one row
// up, wrapping from the last row to the first.
__device__ __forceinline__ int diag_row(uint32_t warp, int s) { return (int)((warp + (uint32_t)s) & (BY - 1)) + 1; }

// Position of the k-th set bit (k counted from 0) of w; k < popc(w).
__device__ __forceinline__ uint32_t nth_set(uint32_t w, uint32_t k) {
    uint32_t pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const uint32_t lo = (uint32_t)__popc(w & ((1u << s) - 1u));
        if (k >= lo) {
            k -= lo;
            w >>= s;
            pos += (uint32_t)s;
        }
    }
    return pos;
}

// Code (n_max slot | n_min slot << 4) of one vertex (staged column c, warp row
// r) in the field staged at pm / p0 / pp.  Candidates in ascending linear
// index order, the later one winning a tie for the maximum and the earlier
// one for the minimum; NaN (outside the grid) never wins.
__device__ __forceinline__ uint32_t code1(const float *pm, const float *p0, const float *pp, int r, int c) {
    float hv = -__int_as_float(0x7f800000), lv = __int_as_float(0x7f800000);
    uint32_t hs = kSelf, ls = kSelf;
    auto take = [&](float w, uint32_t s) {
        if (w >= hv) { hv = w; hs = s; }
        if (w < lv) { lv = w; ls = s; }
    };
    const int a = (r - 1) * PW + c, b = r * PW + c, d = (r + 1) * PW + c;
    take(pm[a - 1], 13); take(pm[a], 12);
    take(pm[b - 1], 11); take(pm[b], 9);
    take(p0[a - 1], 10); take(p0[a], 8);
    take(p0[b - 1], 7);  take(p0[b], kSelf); take(p0[b + 1], 0);
    take(p0[d], 1);      take(p0[d + 1], 3);
    take(pp[b], 2);      take(pp[b + 1], 4);
    take(pp[d], 5);      take(pp[d + 1], 6);
    return hs | (ls << 4);
}

}  // namespace tile
}  // namespace msz
