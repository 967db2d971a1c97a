// msz_workspace.h -- layout of the caller-provided device workspace and the
// host-side helpers shared by the entry points.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "msz.h"
#include "msz_device.cuh"

namespace msz {

// One record per sweep k (device): worklist size, distorted vertices,
// distinct targets, targets whose value decreased.
struct SweepRec {
    uint32_t worklist, distorted, targets, changed;
    uint32_t tile_next;   // dynamic tile counter of a whole-grid pass in this sweep
    uint32_t pad;
    unsigned long long t_detect;  // %globaltimer when the detection phase of this sweep ended
    unsigned long long t_edit;    // ... when its edit phase ended
};

// Loop control block at the start of the workspace (device).
struct Ctrl {
    uint32_t bar_count, bar_gen;  // grid barrier
    uint32_t error;               // kErr* bits
    uint32_t status;              // final msz_status of the loop
    uint32_t sweeps;              // sweeps that applied edits
    uint32_t left;                // distorted vertices left on STUCK / MAX_SWEEPS
    uint32_t tcount[2];           // target-list fill, by sweep parity
    uint32_t wcount[2];           // worklist fill, by sweep parity
    uint32_t dense_sweeps;
    uint32_t flag;                // scratch flag (segment rounds)
    unsigned long long edits;     // total value decreases
    unsigned long long edit_count;
    unsigned long long examined;
    unsigned long long counts[8]; // compare counters
    unsigned long long t_start, t_end;  // %globaltimer at kernel start / edit list written
    unsigned long long t_codes;         // ... when the codes of f were complete
    uint32_t uncertified;               // vertices that sweep 0 could not certify
    uint32_t pad[15];
};

constexpr size_t kAlign = 256;
constexpr uint32_t kMaxBlocks = 4096;  // cooperative grid upper bound (block sums)
constexpr size_t kLogEntries = (size_t)MSZ_MAX_SWEEPS_LIMIT + 2;

constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Byte offsets of each region for a grid of n vertices (bitmaps: one bit per
// vertex).
struct Layout {
    size_t ctrl, log, bsum, tb, d0, d1, eb, ub, stb, sd0, sd1, codes, total;
    size_t zero_bytes;  // [0, zero_bytes) is cleared at the start of every call
};

// Chunk flags of a bitmap: one word per chunk of 32 bitmap words (1024
// vertices), nonzero when the chunk may hold a set bit.
__host__ __device__ constexpr uint64_t chunk_count(uint64_t words) { return (words + 31) / 32; }

constexpr Layout layout_for(uint64_t n) {
    Layout L{};
    const uint64_t words = (n + 31) / 32;
    size_t o = 0;
    L.ctrl = o;   o = align_up(o + sizeof(Ctrl));
    L.log = o;    o = align_up(o + kLogEntries * sizeof(SweepRec));
    L.bsum = o;   o = align_up(o + kMaxBlocks * sizeof(uint32_t));
    L.tb = o;     o = align_up(o + words * 4);
    L.d0 = o;     o = align_up(o + words * 4);
    L.d1 = o;     o = align_up(o + words * 4);
    L.eb = o;     o = align_up(o + words * 4);
    L.ub = o;     o = align_up(o + words * 4);
    L.stb = o;    o = align_up(o + chunk_count(words) * 4);
    L.sd0 = o;    o = align_up(o + chunk_count(words) * 4);
    L.sd1 = o;    o = align_up(o + chunk_count(words) * 4);
    L.zero_bytes = o;
    L.codes = o;  o = align_up(o + n);
    L.total = o;
    return L;
}

// BELOW_REFERENCE's candidate records (4 bytes a vertex), placed after the
// layout above.
constexpr size_t cand_bytes(uint64_t n) { return align_up(n * 4); }

// Validates a grid; fills G (offsets, sizes).  Returns MSZ_OK or INVALID_ARG.
inline msz_status make_grid(const msz_grid &g, GridDev &G) {
    if (g.ndim != 2 && g.ndim != 3) return MSZ_ERR_INVALID_ARG;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) return MSZ_ERR_INVALID_ARG;
    if (g.ndim == 2 && g.nz != 1) return MSZ_ERR_INVALID_ARG;
    if (g.nx > MSZ_MAX_VERTICES || g.ny > MSZ_MAX_VERTICES || g.nz > MSZ_MAX_VERTICES) return MSZ_ERR_INVALID_ARG;
    const double nd = (double)g.nx * (double)g.ny * (double)g.nz;
    if (nd > (double)MSZ_MAX_VERTICES) return MSZ_ERR_INVALID_ARG;
    G.ndim = g.ndim;
    G.nx = (uint32_t)g.nx;
    G.ny = (uint32_t)g.ny;
    G.nz = (uint32_t)g.nz;
    G.nxy = G.nx * G.ny;
    G.n = G.nxy * G.nz;
    G.words = (G.n + 31) / 32;
    G.blocks = (G.n + 1023) / 1024;
    const int ns = g.ndim == 2 ? 6 : 14;
    for (int s = 0; s < 16; ++s) {
        int dx = 0, dy = 0, dz = 0;
        if (s < ns) slot_delta(g.ndim, s, dx, dy, dz);
        G.off[s] = (int32_t)((int64_t)dx + (int64_t)G.nx * dy + (int64_t)G.nxy * dz);
    }
    G.dx = fast_div(G.nx);
    G.dxy = fast_div(G.nxy);
    return MSZ_OK;
}

struct DeviceInfo {
    int device;
    int sms;
    int major, minor;
};

// Current device; MSZ_ERR_CUDA / MSZ_ERR_UNSUPPORTED on failure.
msz_status current_device(DeviceInfo &info);

inline msz_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA; }

}  // namespace msz
