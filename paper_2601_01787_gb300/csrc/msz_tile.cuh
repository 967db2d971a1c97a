// msz_tile.cuh -- shared-memory tiled dense pass over a 3D grid.
//
// A block of 256 threads (8 warps) owns a tile of 128 (x) x 8 (y) vertices
// and marches it through a range of z planes.  The field planes it needs
// (rows y0-1 .. y0+8, columns x0-1 .. x0+128) are staged through a ring of 4
// shared-memory slots filled by cp.async: planes z+2 and z+3 are in flight
// while plane z is computed from the slots of z-1, z and z+1.  Staged
// positions outside the grid hold NaN, which never wins a comparison.  Each lane computes the
// codes of 4 consecutive vertices of its warp's row; the 15 candidates of a
// vertex come from 7 row segments (ascending linear index order), each read
// as one 16-byte shared-memory load plus one halo value passed by a warp
// shuffle.
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

// One ring slot: the staged plane of f, then fhat over the owned region (same
// indexing, only rows 1..BY and columns 1..BX are filled).
constexpr int SLOT = 2 * PLANE;
constexpr size_t kRingBytes = (size_t)NSLOT * SLOT * sizeof(float);

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

// Per-lane extremes of 4 consecutive vertices.
struct Ext4 {
    float hv[4], lv[4];
    uint32_t hs[4], ls[4];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            hv[e] = -__int_as_float(0x7f800000);
            lv[e] = __int_as_float(0x7f800000);
            hs[e] = kSelf;
            ls[e] = kSelf;
        }
    }
    template <bool MASK>
    __device__ __forceinline__ void take(int e, float w, uint32_t slot, bool ok) {
        if ((!MASK || ok) && w >= hv[e]) { hv[e] = w; hs[e] = slot; }
        if ((!MASK || ok) && w < lv[e]) { lv[e] = w; ls[e] = slot; }
    }
    __device__ __forceinline__ uint32_t code(int e) const { return hs[e] | (ls[e] << 4); }
};

// Per-lane extremes of 4 consecutive vertices with the runner-up values: the
// margins hv - h2 and l2 - lv decide whether a vertex can ever be distorted.
struct Ext4M {
    float hv[4], h2[4], lv[4], l2[4];
    uint32_t hs[4], ls[4];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            hv[e] = h2[e] = -__int_as_float(0x7f800000);
            lv[e] = l2[e] = __int_as_float(0x7f800000);
            hs[e] = kSelf;
            ls[e] = kSelf;
        }
    }
    template <bool MASK>
    __device__ __forceinline__ void take(int e, float w, uint32_t slot, bool ok) {
        if (!MASK || ok) {
            // a NaN candidate (outside the grid) fails both tests and leaves
            // every running value unchanged (fmaxf / fminf ignore NaN)
            const bool p = w >= hv[e];
            h2[e] = fmaxf(h2[e], p ? hv[e] : w);
            hv[e] = fmaxf(hv[e], w);
            hs[e] = p ? slot : hs[e];
            const bool q = w < lv[e];
            l2[e] = fminf(l2[e], q ? lv[e] : w);
            lv[e] = fminf(lv[e], w);
            ls[e] = q ? slot : ls[e];
        }
    }
    __device__ __forceinline__ uint32_t code(int e) const { return hs[e] | (ls[e] << 4); }
    // Certified: in f the winner beats the runner-up by more than 2 xi in both
    // directions (differences rounded down), so no g with |g - f| <= xi can
    // change either winner.
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

// Domain predicates of one lane's 4 vertices (used only on edge warps).
struct Dom {
    bool xm[4], xp[4];  // x-1 / x+1 inside
    bool ym, yp, zm, zp;
};

// Codes of the 4 vertices of this lane in the field staged at pm / p0 / pp
// (planes z-1, z, z+1; each pointer at the start of the tile plane) for warp
// row r (1 .. BY).  Candidates in ascending linear index order:
//   (y-1,z-1): 13 12   (y,z-1): 11 9   (y-1,z): 10 8   (y,z): 7 SELF 0
//   (y+1,z): 1 3       (y,z+1): 2 4    (y+1,z+1): 5 6
template <bool MASK, class EXT>
__device__ __forceinline__ void codes4_into(const float *pm, const float *p0, const float *pp, int r, uint32_t lane,
                                            const Dom &d, EXT &x) {
    x.init();
    {
        const Seg s = seg_left(pm + (r - 1) * PW, lane);  // (y-1, z-1): x-1, x
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            x.template take<MASK>(e, s.v[e], 13, d.xm[e] && d.ym && d.zm);
            x.template take<MASK>(e, s.v[e + 1], 12, d.ym && d.zm);
        }
    }
    {
        const Seg s = seg_left(pm + r * PW, lane);  // (y, z-1): x-1, x
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            x.template take<MASK>(e, s.v[e], 11, d.xm[e] && d.zm);
            x.template take<MASK>(e, s.v[e + 1], 9, d.zm);
        }
    }
    {
        const Seg s = seg_left(p0 + (r - 1) * PW, lane);  // (y-1, z): x-1, x
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            x.template take<MASK>(e, s.v[e], 10, d.xm[e] && d.ym);
            x.template take<MASK>(e, s.v[e + 1], 8, d.ym);
        }
    }
    {
        const Seg s = seg_left(p0 + r * PW, lane);  // (y, z): x-1, x
        float right = __shfl_down_sync(kFull, s.v[1], 1);
        if (lane == 31) right = p0[r * PW + 4 + BX];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            x.template take<MASK>(e, s.v[e], 7, d.xm[e]);
            x.template take<false>(e, s.v[e + 1], kSelf, true);
            x.template take<MASK>(e, e < 3 ? s.v[e + 2] : right, 0, d.xp[e]);
        }
    }
    {
        const Seg s = seg_right(p0 + (r + 1) * PW, lane);  // (y+1, z): x, x+1
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            x.template take<MASK>(e, s.v[e], 1, d.yp);
            x.template take<MASK>(e, s.v[e + 1], 3, d.xp[e] && d.yp);
        }
    }
    {
        const Seg s = seg_right(pp + r * PW, lane);  // (y, z+1): x, x+1
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            x.template take<MASK>(e, s.v[e], 2, d.zp);
            x.template take<MASK>(e, s.v[e + 1], 4, d.xp[e] && d.zp);
        }
    }
    {
        const Seg s = seg_right(pp + (r + 1) * PW, lane);  // (y+1, z+1): x, x+1
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            x.template take<MASK>(e, s.v[e], 5, d.yp && d.zp);
            x.template take<MASK>(e, s.v[e + 1], 6, d.xp[e] && d.yp && d.zp);
        }
    }
}

template <bool MASK>
__device__ __forceinline__ void codes4(const float *pm, const float *p0, const float *pp, int r, uint32_t lane,
                                       const Dom &d, uint32_t out[4]) {
    Ext4 x;
    codes4_into<MASK>(pm, p0, pp, r, lane, d, x);
#pragma unroll
    for (int e = 0; e < 4; ++e) out[e] = x.code(e);
}

// Codes plus the certification bit (bit e of cert) of the 4 vertices.  Every
// staged position outside the grid holds NaN, so no domain mask is needed.
__device__ __forceinline__ void codes4_cert(const float *pm, const float *p0, const float *pp, int r, uint32_t lane,
                                            float two_xi, uint32_t out[4], uint32_t &cert) {
    Ext4M x;
    const Dom d{};
    codes4_into<false>(pm, p0, pp, r, lane, d, x);
    cert = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        out[e] = x.code(e);
        cert |= (uint32_t)x.certified(e, two_xi) << e;
    }
}

}  // namespace tile
}  // namespace msz
