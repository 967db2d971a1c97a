// msz_device.cuh -- device-side building blocks of the correction engine
// (pMSz, arXiv 2601.01787) for sm_103a.
//
// Grid, neighbour slots, the index tie-break order and the packed
// steepest-neighbour code (Sec. III-A, Sec. IV-A); the exact float32 error
// bound and Eq. 1's edit; warp-aggregated worklist appends; a bounded grid
// barrier for cooperative launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "msz.h"

namespace msz {

constexpr uint32_t kSelf = MSZ_SELF;
constexpr uint32_t kFull = 0xffffffffu;

// error bits in Ctrl::error
constexpr uint32_t kErrInput = 1u;    // a value not finite or outside [L, U]
constexpr uint32_t kErrTimeout = 2u;  // a bounded wait ran out

// Division of an index n < 2^31 by a fixed d >= 1 without a divide: for d a
// power of two, n >> s; otherwise with s = ceil(log2 d) and
// m = ceil(2^(31+s) / d) < 2^32, floor(n / d) = umulhi(n, m) >> (s - 1),
// because n m / 2^(31+s) exceeds n / d by less than n / 2^(31+s) < 1/d, too
// little to reach the next integer.  m = 0 marks the power-of-two case.
struct FastDiv {
    uint32_t m, sh;
};

__host__ __device__ inline FastDiv fast_div(uint32_t d) {
    FastDiv f{0u, 0u};
    if ((d & (d - 1u)) == 0u) {
        while ((1u << f.sh) < d) ++f.sh;
        return f;
    }
    uint32_t s = 0;
    while (s < 32u && (1ull << s) < (unsigned long long)d) ++s;
    f.m = (uint32_t)(((1ull << (31u + s)) + d - 1ull) / d);
    f.sh = s - 1u;
    return f;
}

struct GridDev {
    int32_t ndim;
    uint32_t nx, ny, nz;
    uint32_t nxy;
    uint32_t n;
    uint32_t words;   // ceil(n / 32): bitmap words
    uint32_t blocks;  // ceil(n / 1024): top-level bits
    int32_t off[16];  // linear offset of each neighbour slot (14, 15 unused)
    FastDiv dx, dxy;  // division by nx and by nx * ny
};

__device__ __forceinline__ uint32_t div_fast(uint32_t n, FastDiv f) {
    return f.m ? (__umulhi(n, f.m) >> f.sh) : (n >> f.sh);
}

// Slot table (x, y, z) of the public header: positive offsets, then negatives.
__host__ __device__ __forceinline__ void slot_delta(int ndim, int s, int &dx, int &dy, int &dz) {
    if (ndim == 2) {
        const int t = s % 3, sg = s < 3 ? 1 : -1;
        dx = (t == 0 || t == 2) ? sg : 0;
        dy = (t == 1 || t == 2) ? sg : 0;
        dz = 0;
    } else {
        const int t = s % 7, sg = s < 7 ? 1 : -1;
        // 0 (1,0,0) 1 (0,1,0) 2 (0,0,1) 3 (1,1,0) 4 (1,0,1) 5 (0,1,1) 6 (1,1,1)
        dx = (t == 0 || t == 3 || t == 4 || t == 6) ? sg : 0;
        dy = (t == 1 || t == 3 || t == 5 || t == 6) ? sg : 0;
        dz = (t == 2 || t == 4 || t == 5 || t == 6) ? sg : 0;
    }
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void coords_of(const GridDev &G, uint32_t i, uint32_t &x, uint32_t &y, uint32_t &z) {
    z = div_fast(i, G.dxy);
    const uint32_t r = i - z * G.nxy;
    y = div_fast(r, G.dx);
    x = r - y * G.nx;
}

__device__ __forceinline__ bool slot_in_domain(const GridDev &G, int s, uint32_t x, uint32_t y, uint32_t z) {
    int dx, dy, dz;
    slot_delta(G.ndim, s, dx, dy, dz);
    const int X = (int)x + dx, Y = (int)y + dy, Z = (int)z + dz;
    return X >= 0 && X < (int)G.nx && Y >= 0 && Y < (int)G.ny && Z >= 0 && Z < (int)G.nz;
}

// Running extremes over the closed neighbourhood, visited in ascending linear
// index order: a later candidate with an equal value is above (wins the max),
// an earlier one is below (keeps the min).  Values are finite, so the
// sentinels +-inf are replaced by the first candidate.
struct Extremes {
    float hv, lv;
    uint32_t hs, ls;
    __device__ __forceinline__ void init() {
        hv = -__int_as_float(0x7f800000);
        lv = __int_as_float(0x7f800000);
        hs = kSelf;
        ls = kSelf;
    }
    __device__ __forceinline__ void take(float w, uint32_t slot) {
        if (w >= hv) { hv = w; hs = slot; }
        if (w < lv) { lv = w; ls = slot; }
    }
    __device__ __forceinline__ uint8_t code() const { return (uint8_t)(hs | (ls << 4)); }
};

// The 15 candidates of vertex i in ascending linear index order (3D; 7 in
// 2D), NaN where the neighbour is outside the grid or the lane has no vertex:
// a NaN candidate never wins a comparison.  Loads only, so that a caller can
// issue the loads of several vertices before using any of them.
template <int NDIM>
__device__ __forceinline__ void gather_closed(const float *v, const GridDev &G, bool has, uint32_t i, float (&w)[15]) {
    const float nan = __int_as_float(0x7fffffff);
#pragma unroll
    for (int k = 0; k < 15; ++k) w[k] = nan;
    if (!has) return;
    uint32_t x, y, z;
    coords_of(G, i, x, y, z);
    const bool xm = x > 0, xp = x + 1 < G.nx, ym = y > 0, yp = y + 1 < G.ny;
    const uint32_t nx = G.nx;
    if (NDIM == 3) {
        const bool zm = z > 0, zp = z + 1 < G.nz;
        const uint32_t nxy = G.nxy;
        if (xm && ym && zm) w[0] = v[i - 1 - nx - nxy];
        if (ym && zm) w[1] = v[i - nx - nxy];
        if (xm && zm) w[2] = v[i - 1 - nxy];
        if (zm) w[3] = v[i - nxy];
        if (xm && ym) w[4] = v[i - 1 - nx];
        if (ym) w[5] = v[i - nx];
        if (xm) w[6] = v[i - 1];
        w[7] = v[i];
        if (xp) w[8] = v[i + 1];
        if (yp) w[9] = v[i + nx];
        if (xp && yp) w[10] = v[i + 1 + nx];
        if (zp) w[11] = v[i + nxy];
        if (xp && zp) w[12] = v[i + 1 + nxy];
        if (yp && zp) w[13] = v[i + nx + nxy];
        if (xp && yp && zp) w[14] = v[i + 1 + nx + nxy];
    } else {
        if (xm && ym) w[0] = v[i - 1 - nx];
        if (ym) w[1] = v[i - nx];
        if (xm) w[2] = v[i - 1];
        w[3] = v[i];
        if (xp) w[4] = v[i + 1];
        if (yp) w[5] = v[i + nx];
        if (xp && yp) w[6] = v[i + 1 + nx];
    }
}

// Code from the candidates of gather_closed (slots in the same order).
template <int NDIM>
__device__ __forceinline__ uint8_t code_of_closed(const float (&w)[15]) {
    Extremes e;
    e.init();
    if (NDIM == 3) {
        constexpr uint8_t slot[15] = {13, 12, 11, 9, 10, 8, 7, kSelf, 0, 1, 3, 2, 4, 5, 6};
#pragma unroll
        for (int k = 0; k < 15; ++k) e.take(w[k], slot[k]);
    } else {
        constexpr uint8_t slot[7] = {5, 4, 3, kSelf, 0, 1, 2};
#pragma unroll
        for (int k = 0; k < 7; ++k) e.take(w[k], slot[k]);
    }
    return e.code();
}

// Code of vertex i (at x, y, z) of field v, reading neighbours from global
// memory with bounds checks.  v is read through the coherent path (no
// __restrict__): the loop kernel reads g while other blocks have written it.
// Ascending index order of the slots:
//   3D: 13 12 11 9 10 8 7 SELF 0 1 3 2 4 5 6      2D: 5 4 3 SELF 0 1 2
template <int NDIM>
__device__ __forceinline__ uint8_t code_global(const float *v, const GridDev &G, uint32_t i,
                                               uint32_t x, uint32_t y, uint32_t z) {
    Extremes e;
    e.init();
    const bool xm = x > 0, xp = x + 1 < G.nx, ym = y > 0, yp = y + 1 < G.ny;
    if (NDIM == 3) {
        const bool zm = z > 0, zp = z + 1 < G.nz;
        const uint32_t nx = G.nx, nxy = G.nxy;
        if (xm && ym && zm) e.take(v[i - 1 - nx - nxy], 13);
        if (ym && zm) e.take(v[i - nx - nxy], 12);
        if (xm && zm) e.take(v[i - 1 - nxy], 11);
        if (zm) e.take(v[i - nxy], 9);
        if (xm && ym) e.take(v[i - 1 - nx], 10);
        if (ym) e.take(v[i - nx], 8);
        if (xm) e.take(v[i - 1], 7);
        e.take(v[i], kSelf);
        if (xp) e.take(v[i + 1], 0);
        if (yp) e.take(v[i + nx], 1);
        if (xp && yp) e.take(v[i + 1 + nx], 3);
        if (zp) e.take(v[i + nxy], 2);
        if (xp && zp) e.take(v[i + 1 + nxy], 4);
        if (yp && zp) e.take(v[i + nx + nxy], 5);
        if (xp && yp && zp) e.take(v[i + 1 + nx + nxy], 6);
    } else {
        const uint32_t nx = G.nx;
        if (xm && ym) e.take(v[i - 1 - nx], 5);
        if (ym) e.take(v[i - nx], 4);
        if (xm) e.take(v[i - 1], 3);
        e.take(v[i], kSelf);
        if (xp) e.take(v[i + 1], 0);
        if (yp) e.take(v[i + nx], 1);
        if (xp && yp) e.take(v[i + 1 + nx], 2);
    }
    return e.code();
}

// Code of vertex i of field v plus its certification: the winner of each
// direction beats the runner-up by more than two_xi (rounded down), so that
// no field within xi of v can change the code.
template <int NDIM>
__device__ __forceinline__ uint8_t code_global_cert(const float *v, const GridDev &G, uint32_t i, uint32_t x,
                                                    uint32_t y, uint32_t z, float two_xi, bool &cert) {
    float hv = -__int_as_float(0x7f800000), h2 = hv, lv = __int_as_float(0x7f800000), l2 = lv;
    uint32_t hs = kSelf, ls = kSelf;
    auto take = [&](float w, uint32_t slot) {
        const bool p = w >= hv;
        h2 = fmaxf(h2, p ? hv : w);
        hv = fmaxf(hv, w);
        hs = p ? slot : hs;
        const bool q = w < lv;
        l2 = fminf(l2, q ? lv : w);
        lv = fminf(lv, w);
        ls = q ? slot : ls;
    };
    const bool xm = x > 0, xp = x + 1 < G.nx, ym = y > 0, yp = y + 1 < G.ny;
    if (NDIM == 3) {
        const bool zm = z > 0, zp = z + 1 < G.nz;
        const uint32_t nx = G.nx, nxy = G.nxy;
        if (xm && ym && zm) take(v[i - 1 - nx - nxy], 13);
        if (ym && zm) take(v[i - nx - nxy], 12);
        if (xm && zm) take(v[i - 1 - nxy], 11);
        if (zm) take(v[i - nxy], 9);
        if (xm && ym) take(v[i - 1 - nx], 10);
        if (ym) take(v[i - nx], 8);
        if (xm) take(v[i - 1], 7);
        take(v[i], kSelf);
        if (xp) take(v[i + 1], 0);
        if (yp) take(v[i + nx], 1);
        if (xp && yp) take(v[i + 1 + nx], 3);
        if (zp) take(v[i + nxy], 2);
        if (xp && zp) take(v[i + 1 + nxy], 4);
        if (yp && zp) take(v[i + nx + nxy], 5);
        if (xp && yp && zp) take(v[i + 1 + nx + nxy], 6);
    } else {
        const uint32_t nx = G.nx;
        if (xm && ym) take(v[i - 1 - nx], 5);
        if (ym) take(v[i - nx], 4);
        if (xm) take(v[i - 1], 3);
        take(v[i], kSelf);
        if (xp) take(v[i + 1], 0);
        if (yp) take(v[i + nx], 1);
        if (xp && yp) take(v[i + 1 + nx], 2);
    }
    cert = __fsub_rd(hv, h2) > two_xi && __fsub_rd(l2, lv) > two_xi;
    return (uint8_t)(hs | (ls << 4));
}

// L = smallest float32 >= f - xi and U = largest float32 <= f + xi: one
// directed-rounding subtraction / addition of the exact operands.
__device__ __forceinline__ float floor_bound(float f, float xi) { return __fsub_ru(f, xi); }
__device__ __forceinline__ float ceil_bound(float f, float xi) { return __fadd_rd(f, xi); }

// Eq. 1: one edit of a target whose value is gt and floor L.  Returns false
// (no change) when gt is already at its floor.  Intrinsics keep every step a
// single round-to-nearest operation (no contraction into an FMA).
__device__ __forceinline__ bool edit_value(float gt, float L, int rule, float &out) {
    if (!(gt > L)) return false;
    float h;
    if (rule == MSZ_RULE_SNAP) {
        h = L;
    } else {
        const float s = __fsub_rn(gt, L);
        const float half = __fmul_rn(0.5f, s);
        h = __fsub_rn(gt, half);
        if (h < L) h = L;
        if (!(h < gt)) h = L;
    }
    out = h;
    return true;
}

// Targets of a distorted vertex (Sec. III-B extremum rules, Sec. IV-A ordering
// rules).  Returns the number of targets (0..2) in t0 / t1.
__device__ __forceinline__ int targets_of(const GridDev &G, uint32_t i, uint8_t cf, uint8_t cg, uint32_t &t0,
                                          uint32_t &t1) {
    const uint32_t af = cf & 15u, ag = cg & 15u, df = cf >> 4, dg = cg >> 4;
    const bool ta = ag != af, td = dg != df;
    const uint32_t a = (ag == kSelf) ? i : (uint32_t)((int64_t)i + G.off[ag & 15u]);
    const uint32_t d = (df == kSelf) ? i : (uint32_t)((int64_t)i + G.off[df & 15u]);
    t0 = ta ? a : d;
    t1 = d;
    return (int)ta + (int)td;
}

// The vertices the targets of targets_of must fall below (BELOW_REFERENCE),
// in the same order: for an ascending mismatch, f's steepest ascent of i (i
// itself when f makes i a maximum); for a descending one, g's steepest
// descent of i (i itself when g makes i a minimum).
__device__ __forceinline__ void references_of(const GridDev &G, uint32_t i, uint8_t cf, uint8_t cg, uint32_t &r0,
                                              uint32_t &r1) {
    const uint32_t af = cf & 15u, ag = cg & 15u, dg = cg >> 4;
    const uint32_t a = (af == kSelf) ? i : (uint32_t)((int64_t)i + G.off[af & 15u]);
    const uint32_t d = (dg == kSelf) ? i : (uint32_t)((int64_t)i + G.off[dg & 15u]);
    r0 = ag != af ? a : d;
    r1 = d;
}

// IEEE totalOrder key of a float (unsigned comparison orders the floats, -0
// below +0) and its inverse.
__device__ __forceinline__ uint32_t total_key(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_total_key(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The next float below a finite v (towards -inf): one unit in the last place
// down in magnitude for v > 0, up for v < 0, and the negative subnormal of
// least magnitude for either zero.
__device__ __forceinline__ float float_below(float v) {
    const uint32_t b = __float_as_uint(v);
    if ((b & 0x7fffffffu) == 0u) return __uint_as_float(0x80000001u);
    return __uint_as_float((b & 0x80000000u) ? b + 1u : b - 1u);
}

// Set bit v of a bitmap; true when this call set it (first claimer).
__device__ __forceinline__ bool claim_bit(uint32_t *bm, uint32_t v) {
    const uint32_t bit = 1u << (v & 31u);
    return !(atomicOr(&bm[v >> 5], bit) & bit);
}

__device__ __forceinline__ void clear_bit(uint32_t *bm, uint32_t v) {
    atomicAnd(&bm[v >> 5], ~(1u << (v & 31u)));
}

// Warp-aggregated append.  Every lane of a fully converged warp calls it;
// lanes with take == true append value; one atomic per warp.
__device__ __forceinline__ void warp_append(bool take, uint32_t value, uint32_t *list, uint32_t *count) {
    const uint32_t m = __ballot_sync(kFull, take);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(count, (uint32_t)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (take) list[base + __popc(m & lanemask_lt())] = value;
}

// Fire-and-forget bitwise reductions on global words (no value returned, so
// the issuing warp does not wait for them).
__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_and(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.and.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Per-warp staging queue in shared memory.  Appends go to the warp's buffer;
// the warp moves the buffer to the global list with one atomicAdd whenever it
// holds more than 32 items (and at the end of a phase), so a list counter
// sees one atomic per >= 32 items instead of one per warp per append.
constexpr uint32_t kQueueCap = 64;

struct WarpQueue {
    uint32_t *buf;  // kQueueCap entries of this warp in shared memory
    uint32_t n;     // fill, warp-uniform
};

__device__ __forceinline__ void wq_flush(WarpQueue &q, uint32_t *list, uint32_t *count) {
    if (q.n == 0) return;
    __syncwarp();
    uint32_t base = 0;
    if (lane_id() == 0) base = atomicAdd(count, q.n);
    base = __shfl_sync(kFull, base, 0);
    for (uint32_t i = lane_id(); i < q.n; i += 32) list[base + i] = q.buf[i];
    __syncwarp();
    q.n = 0;
}

// Warp-collective: lanes with take == true append value.
__device__ __forceinline__ void wq_push(WarpQueue &q, bool take, uint32_t value, uint32_t *list, uint32_t *count) {
    const uint32_t m = __ballot_sync(kFull, take);
    if (!m) return;
    if (take) q.buf[q.n + __popc(m & lanemask_lt())] = value;
    q.n += __popc(m);
    if (q.n > kQueueCap - 32) wq_flush(q, list, count);
}

// Warp-collective: add the lanes' per-thread counts to a global counter.
__device__ __forceinline__ void warp_add(uint32_t v, uint32_t *counter) {
    const uint32_t t = __reduce_add_sync(kFull, v);
    if (lane_id() == 0 && t) atomicAdd(counter, t);
}

// Warp-aggregated counter increment.
__device__ __forceinline__ void warp_count(bool pred, uint32_t *counter) {
    const uint32_t m = __ballot_sync(kFull, pred);
    if (m && lane_id() == (uint32_t)(__ffs(m) - 1)) atomicAdd(counter, (uint32_t)__popc(m));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// wait is bounded: after timeout_ns the block records kErrTimeout and leaves.
// Returns false when any block has recorded an error.  skip_arrival (a test
// hook) makes this block wait without arriving, so that every block's wait
// runs out and every block returns false.
constexpr uint64_t kBarrierTimeoutNs = 4000000000ull;   // 4 s
constexpr uint64_t kTestBarrierNs = 250000000ull;       // 0.25 s, under the test hook

__device__ __forceinline__ bool grid_barrier(uint32_t *count, uint32_t *gen, uint32_t *err,
                                             uint64_t timeout_ns = kBarrierTimeoutNs, bool skip_arrival = false) {
    __shared__ uint32_t s_err;  // block-uniform verdict
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t g0 = ld_acquire(gen);
        const uint32_t arrived = skip_arrival ? 0u : atomicAdd(count, 1u);
        if (!skip_arrival && arrived == gridDim.x - 1) {
            *count = 0;
            __threadfence();
            st_release(gen, g0 + 1);
        } else {
            const uint64_t t0 = global_ns();
            while (ld_acquire(gen) == g0) {
                __nanosleep(32);
                if (global_ns() - t0 > timeout_ns) {
                    atomicOr(err, kErrTimeout);
                    break;
                }
            }
        }
        __threadfence();
        s_err = ld_relaxed(err);
    }
    __syncthreads();
    return s_err == 0;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x <= 1024,
// a multiple of 32).  Returns the exclusive prefix; *total gets the sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *smem32, uint32_t &total) {
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= (uint32_t)d) incl += y;
    }
    if (lane == 31) smem32[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nwarps ? smem32[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, wi, d);
            if (lane >= (uint32_t)d) wi += y;
        }
        if (lane < nwarps) smem32[lane] = wi - w;  // exclusive warp offsets
        if (lane == 31) smem32[32] = wi;           // block total
    }
    __syncthreads();
    const uint32_t res = smem32[warp] + incl - v;
    total = smem32[32];
    __syncthreads();
    return res;
}

}  // namespace msz
