/*
 * msz_oracle.c -- CPU oracle for the pMSz correction loop (arXiv 2601.01787).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * restatement of what the paper's method computes.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference arm may load
 * it.  The CUDA product path shares no code, header, table or helper with it.
 *
 * Build: cc -std=c99 -O2 -ffp-contract=off -fPIC -shared (never -ffast-math,
 * never FMA contraction: every float operation below is one IEEE-754 binary32
 * operation rounded to nearest unless stated otherwise).
 *
 * Contents, in the order of the paper:
 *   Sec. III-A  piecewise-linear field on a Freudenthal (Kuhn) triangulation of
 *               the grid; distinct values made concrete by an index tie-break;
 *               extrema; steepest neighbours n_min(i), n_max(i) (Sec. IV-A).
 *   Eq. 1       the edit g <- max(g - delta, f - xi), with the HALVE choice of
 *               delta (the paper leaves delta open), SNAP (delta large
 *               enough to reach the floor, as Fig. "nonextrema"(c) drops 0.1
 *               to 0) or BELOW-REFERENCE (Sec. IV-A: the offending vertex
 *               drops "to 0.3 or slightly below", just under the vertex it
 *               must fall below).
 *   Sec. III-B  C-loop extremum rules (FPmax spelled out, the other three
 *   Sec. IV-A   follow the same non-increasing logic) and the local-ordering
 *               rules for the descending and ascending directions.
 *   Sec. III-B  convergence: edits only decrease g, clamped at f - xi; a
 *   Sec. IV-C   sweep that finds distortions but changes nothing is reported
 *               as STUCK rather than looping forever.
 *   Sec. IV-B   conflicting edits of one point resolve to the minimum
 *               candidate: with one application per distinct target per
 *               sweep (Jacobi) every candidate is the same value.
 *   Sec. III-A  integral lines / segmentation labels by path following, and
 *   Sec. V-C    the verification counts (wrong labels, false extrema).
 *
 * Readings of points the paper leaves open:
 *   - triangulation: Kuhn subdivision along the main diagonal, neighbour
 *     offsets d in +-({0,1}^n \ {0}): 6 in 2D, 14 in 3D;
 *   - order: j above i  <=>  v_j > v_i  or  (v_j == v_i and j > i);
 *   - "steepest" neighbour = extreme neighbour value (n_min/n_max, Sec. IV-A);
 *   - floor L_i = smallest float32 >= f_i - xi (exact real), ceiling U_i =
 *     largest float32 <= f_i + xi;
 *   - HALVE: s = g - L; h = g - 0.5*s; h = max(h, L); if h is not below g
 *     then h = L.  A target already at its floor is left unchanged.
 *   - targets of a distorted vertex i (extremum cases of Sec. III-B and the
 *     ordering cases of Sec. IV-A, one rule per direction):
 *       ascending  mismatch: lower i if g makes i a maximum, else lower the
 *                  neighbour that is n_max(i) in g (the spurious maximum);
 *       descending mismatch: lower i if f makes i a minimum, else lower the
 *                  neighbour that is n_min(i) in f (the original minimum).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_SELF 15

/* Status values.  The numbering matches the public C ABI's msz_status so that
 * tests can compare the two directly; it is restated here, not shared. */
enum {
    ORC_OK = 0,
    ORC_ERR_INVALID_ARG = 1,
    ORC_ERR_INPUT_BOUND = 2,
    ORC_ERR_CAPACITY = 3,
    ORC_ERR_OOM = 4,
    ORC_ERR_MAX_SWEEPS = 6,
    ORC_STUCK = 8
};

enum { ORC_RULE_HALVE = 0, ORC_RULE_SNAP = 1, ORC_RULE_BELOW = 2 };

/* ---------------------------------------------------------------------------
 * Sec. III-A: the grid, its triangulation and the neighbourhood N(i).
 * Linear index i = x + nx*(y + ny*z), x fastest.  Slot s of the
 * neighbourhood is the offset d_s; positive offsets first, then their
 * negatives in the same order.
 * ------------------------------------------------------------------------- */
static const int D3[14][3] = {
    {1, 0, 0},   {0, 1, 0},   {0, 0, 1},   {1, 1, 0},   {1, 0, 1},   {0, 1, 1},   {1, 1, 1},
    {-1, 0, 0},  {0, -1, 0},  {0, 0, -1},  {-1, -1, 0}, {-1, 0, -1}, {0, -1, -1}, {-1, -1, -1}};
static const int D2[6][2] = {{1, 0}, {0, 1}, {1, 1}, {-1, 0}, {0, -1}, {-1, -1}};

int orc_num_slots(int ndim) { return ndim == 2 ? 6 : 14; }

/* Returns 1 and stores the neighbour's linear index in *j when slot s of
 * vertex i lies inside the grid; returns 0 otherwise. */
int orc_neighbour(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t i, int s, int64_t *j)
{
    int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
    int64_t X, Y, Z;
    if (ndim == 2) {
        if (s < 0 || s >= 6) return 0;
        X = x + D2[s][0];
        Y = y + D2[s][1];
        Z = z;
    } else {
        if (s < 0 || s >= 14) return 0;
        X = x + D3[s][0];
        Y = y + D3[s][1];
        Z = z + D3[s][2];
    }
    if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) return 0;
    *j = X + nx * (Y + ny * Z);
    return 1;
}

/* The total order that makes the values "distinct" (Sec. III-A): is j above i? */
static int above(float vj, int64_t j, float vi, int64_t i)
{
    return vj > vi || (vj == vi && j > i);
}

/* Sec. IV-A: n_max(i) = argmax_{j in N(i)} v_j and n_min(i) = argmin, under
 * the order above.  Sec. III-A: i is a maximum (minimum) when it is above
 * (below) every neighbour.  Both facts are packed into one byte:
 *   low nibble  = slot of n_max(i) if n_max(i) is above i, else SELF (maximum);
 *   high nibble = slot of n_min(i) if n_min(i) is below i, else SELF (minimum). */
uint8_t orc_code_at(const float *v, int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t i)
{
    int64_t hi = i, lo = i, j;
    int shi = ORC_SELF, slo = ORC_SELF;
    int ns = orc_num_slots(ndim);
    for (int s = 0; s < ns; ++s) {
        if (!orc_neighbour(ndim, nx, ny, nz, i, s, &j)) continue;
        if (above(v[j], j, v[hi], hi)) { hi = j; shi = s; }
        if (above(v[lo], lo, v[j], j)) { lo = j; slo = s; }
    }
    return (uint8_t)(shi | (slo << 4));
}

void orc_codes(const float *v, int ndim, int64_t nx, int64_t ny, int64_t nz, uint8_t *codes)
{
    int64_t n = nx * ny * nz;
    for (int64_t i = 0; i < n; ++i) codes[i] = orc_code_at(v, ndim, nx, ny, nz, i);
}

/* ---------------------------------------------------------------------------
 * Error bound (Sec. III-B: |f_i - g_i| <= xi) made exact for float32 values.
 * L = smallest float >= f - xi and U = largest float <= f + xi, where f - xi
 * and f + xi are exact real numbers.  The double sum a + b is made exact with
 * Knuth's TwoSum (s + e == a + b exactly) and then rounded by hand in the
 * wanted direction.
 * ------------------------------------------------------------------------- */
static void two_sum(double a, double b, double *s, double *e)
{
    double sum = a + b;
    double bb = sum - a;
    *e = (a - (sum - bb)) + (b - bb);
    *s = sum;
}

float orc_floor(float f, float xi)
{
    double s, e;
    two_sum((double)f, -(double)xi, &s, &e);
    float r = (float)s;
    if (isinf(r)) return r < 0 ? -FLT_MAX : r;
    if ((double)r < s || ((double)r == s && e > 0)) r = nextafterf(r, INFINITY);
    return r;
}

float orc_ceil(float f, float xi)
{
    double s, e;
    two_sum((double)f, (double)xi, &s, &e);
    float r = (float)s;
    if (isinf(r)) return r > 0 ? FLT_MAX : r;
    if ((double)r > s || ((double)r == s && e < 0)) r = nextafterf(r, -INFINITY);
    return r;
}

/* Input check: finite values and L_i <= fhat_i <= U_i for every i. */
int orc_validate(const float *f, const float *fhat, int64_t n, float xi)
{
    if (!(xi >= 0.0f) || isinf(xi)) return ORC_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(f[i]) || !isfinite(fhat[i])) return ORC_ERR_INPUT_BOUND;
        if (fhat[i] < orc_floor(f[i], xi) || fhat[i] > orc_ceil(f[i], xi)) return ORC_ERR_INPUT_BOUND;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Eq. 1: one edit of vertex t.  Returns 1 when g_t decreased, 0 when g_t was
 * already at its floor L.  HALVE moves g halfway to the floor; SNAP moves it
 * to the floor.
 * ------------------------------------------------------------------------- */
int orc_edit(float *g, float L, int rule)
{
    float gt = *g;
    if (!(gt > L)) return 0;
    float h;
    if (rule == ORC_RULE_SNAP) {
        h = L;
    } else {
        float s = gt - L;
        float half = 0.5f * s;
        h = gt - half;
        if (h < L) h = L;
        if (!(h < gt)) h = L;
    }
    *g = h;
    return 1;
}

/* ---------------------------------------------------------------------------
 * Distortion test and edit targets of vertex i (Sec. III-B C-loop extremum
 * rules + Sec. IV-A local-ordering rules).  cf = code of i in f, cg = code of
 * i in the current g.  Returns the number of targets written to t[0..1].
 * ------------------------------------------------------------------------- */
static int targets_of(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t i,
                      uint8_t cf, uint8_t cg, int64_t t[2])
{
    int k = 0;
    int asc_f = cf & 15, asc_g = cg & 15, desc_f = cf >> 4, desc_g = cg >> 4;
    int64_t j;
    if (asc_g != asc_f) {
        /* FPmax (Sec. III-B): g makes i a maximum although f does not -> lower i.
         * Otherwise the largest neighbour in g is not the one of f (FNmax or the
         * ascending-direction case of Sec. IV-A) -> lower that spurious maximum. */
        if (asc_g == ORC_SELF) t[k++] = i;
        else if (orc_neighbour(ndim, nx, ny, nz, i, asc_g, &j)) t[k++] = j;
    }
    if (desc_g != desc_f) {
        /* FNmin: f makes i a minimum, g does not -> lower i below its neighbours.
         * Otherwise (FPmin or the descending case of Sec. IV-A) lower the
         * original smallest neighbour n_min(i) of f. */
        if (desc_f == ORC_SELF) t[k++] = i;
        else if (orc_neighbour(ndim, nx, ny, nz, i, desc_f, &j)) t[k++] = j;
    }
    return k;
}

/* The vertex each target of i must end up below (BELOW-REFERENCE only), in
 * the order targets_of writes the targets.  Ascending mismatch: the target
 * (i itself for FPmax, else g's largest neighbour) must fall below the vertex
 * that f makes i's steepest ascent (i itself for FNmax): in Fig. nonextrema
 * (d)-(f) the spurious 0.4 falls below the 0.3 of n_max(i).  Descending
 * mismatch: the target (i itself for FNmin, else f's smallest neighbour) must
 * fall below the vertex that g makes i's steepest descent (i itself for FPmin):
 * in Fig. nonextrema (a)-(c) the original minimum 0.1 falls below the spurious
 * 0.08. */
static int references_of(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t i,
                         uint8_t cf, uint8_t cg, int64_t r[2])
{
    int k = 0;
    int asc_f = cf & 15, asc_g = cg & 15, desc_f = cf >> 4, desc_g = cg >> 4;
    int64_t j;
    if (asc_g != asc_f) {
        if (asc_f == ORC_SELF) r[k++] = i;
        else if (orc_neighbour(ndim, nx, ny, nz, i, asc_f, &j)) r[k++] = j;
    }
    if (desc_g != desc_f) {
        if (desc_g == ORC_SELF) r[k++] = i;
        else if (orc_neighbour(ndim, nx, ny, nz, i, desc_g, &j)) r[k++] = j;
    }
    return k;
}

/* BELOW-REFERENCE (Sec. IV-A: decrease the offender "to 0.3 or slightly
 * below"): the largest value that puts target t below reference r, whose
 * current value is vr, in the order of Sec. III-A -- vr itself when r has the
 * larger index (the tie is then broken in r's favour), else the next float
 * below vr. */
static float below_value(int64_t t, int64_t r, float vr)
{
    return r > t ? vr : nextafterf(vr, -INFINITY);
}

/* IEEE totalOrder key of a float: unsigned comparison of keys orders the
 * floats, with -0 below +0. */
static uint32_t total_key(float v)
{
    uint32_t b;
    memcpy(&b, &v, 4);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

/* One BELOW-REFERENCE edit: g moves to the candidate c (the smallest, in
 * totalOrder, of the values its requests ask for in this sweep), kept at or
 * above the floor L.  Returns 1 when g decreased, 0 when g was at its floor. */
int orc_edit_below(float *g, float L, float c)
{
    float h = c < L ? L : c;
    if (!(h < *g)) return 0;
    *g = h;
    return 1;
}

/* ---------------------------------------------------------------------------
 * The correction loop (Sec. III-B iterative strategy, redesigned C-loop of
 * Sec. IV-A, synchronous sweeps).  Sweep k:
 *   1. detect: every vertex i of the worklist W_k whose code in g^k differs
 *      from its code in f is distorted; its targets are collected;
 *   2. stop with OK when no vertex is distorted;
 *   3. edit: every distinct target gets one application of Eq. 1, computed
 *      from g^k (Jacobi);
 *   4. stop with STUCK when no target changed.
 * W_0 = all vertices.  In worklist mode W_{k+1} = the closed neighbourhoods
 * of the vertices changed in sweep k, plus the vertices distorted in sweep k.
 * A vertex's code depends only on g over its closed neighbourhood, so every
 * vertex left out had no distortion in sweep k and sees no change: the
 * sequence g^k is identical to dense sweeps (use_worklist = 0).
 *
 * stats (may be NULL), 8 entries:
 *   [0] sweeps that applied edits (0 when fhat is already correct)
 *   [1] total edits applied (value decreases)
 *   [2] distinct edited vertices (g != fhat)
 *   [3] distorted vertices in sweep 0
 *   [4] distorted vertices left at the end (0 on OK)
 *   [5] total worklist entries examined over all sweeps
 *   [6] status
 *   [7] reserved
 * sweep_log (may be NULL): 4 entries per sweep k < log_capacity:
 *   |W_k|, distorted(k), distinct targets(k), changed(k).
 * ------------------------------------------------------------------------- */
int orc_correct(const float *f, const float *fhat, float xi,
                int ndim, int64_t nx, int64_t ny, int64_t nz,
                int use_worklist, int rule, int64_t max_sweeps,
                const float *g_init, float *g,
                uint32_t *edit_idx, float *edit_delta, int64_t edit_capacity, int64_t *edit_count,
                int64_t *stats, int64_t *sweep_log, int64_t log_capacity)
{
    if (!f || !fhat || !g || nx < 1 || ny < 1 || nz < 1 || (ndim != 2 && ndim != 3) ||
        (ndim == 2 && nz != 1) || max_sweeps < 0 ||
        (rule != ORC_RULE_HALVE && rule != ORC_RULE_SNAP && rule != ORC_RULE_BELOW))
        return ORC_ERR_INVALID_ARG;
    int64_t n = nx * ny * nz;
    int st = orc_validate(f, fhat, n, xi);
    if (st != ORC_OK) return st;
    if (g_init) {
        for (int64_t i = 0; i < n; ++i)
            if (!isfinite(g_init[i]) || g_init[i] < orc_floor(f[i], xi) || g_init[i] > orc_ceil(f[i], xi))
                return ORC_ERR_INPUT_BOUND;
    }

    uint8_t *cf = malloc((size_t)n);
    uint8_t *is_target = calloc((size_t)n, 1);
    uint8_t *in_next = calloc((size_t)n, 1);
    int64_t *tlist = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *wl = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *wl_next = malloc(sizeof(int64_t) * (size_t)n);
    float *L = malloc(sizeof(float) * (size_t)n);
    /* BELOW-REFERENCE: per target, the smallest value its requests ask for */
    float *cand = rule == ORC_RULE_BELOW ? malloc(sizeof(float) * (size_t)n) : NULL;
    if (!cf || !is_target || !in_next || !tlist || !wl || !wl_next || !L || (rule == ORC_RULE_BELOW && !cand)) {
        free(cf); free(is_target); free(in_next); free(tlist); free(wl); free(wl_next); free(L); free(cand);
        return ORC_ERR_OOM;
    }

    /* g^(0) = fhat (Sec. III-B), or a proposed start inside the bound. */
    for (int64_t i = 0; i < n; ++i) {
        g[i] = g_init ? g_init[i] : fhat[i];
        L[i] = orc_floor(f[i], xi);
    }
    orc_codes(f, ndim, nx, ny, nz, cf);

    int64_t sweeps = 0, edits = 0, first_distorted = -1, left = 0, examined = 0;
    int64_t nw = n;
    for (int64_t i = 0; i < n; ++i) wl[i] = i;
    int status = ORC_ERR_MAX_SWEEPS;

    for (int64_t k = 0;; ++k) {
        /* 1. detect */
        int64_t distorted = 0, nt = 0;
        examined += nw;
        int64_t nn = 0;
        for (int64_t w = 0; w < nw; ++w) {
            int64_t i = use_worklist ? wl[w] : w;
            uint8_t cg = orc_code_at(g, ndim, nx, ny, nz, i);
            if (cg == cf[i]) continue;
            ++distorted;
            int64_t t[2], r[2];
            int m = targets_of(ndim, nx, ny, nz, i, cf[i], cg, t);
            if (rule == ORC_RULE_BELOW) references_of(ndim, nx, ny, nz, i, cf[i], cg, r);
            for (int q = 0; q < m; ++q) {
                float c = rule == ORC_RULE_BELOW ? below_value(t[q], r[q], g[r[q]]) : 0.0f;
                if (!is_target[t[q]]) {
                    is_target[t[q]] = 1;
                    tlist[nt++] = t[q];
                    if (cand) cand[t[q]] = c;
                } else if (cand && total_key(c) < total_key(cand[t[q]])) {
                    cand[t[q]] = c;  /* conflicting requests: the minimum (Sec. IV-B) */
                }
            }
            if (use_worklist && !in_next[i]) { in_next[i] = 1; wl_next[nn++] = i; }
        }
        if (k == 0) first_distorted = distorted;
        int64_t changed = 0;
        /* 2. stop when nothing is distorted, or at the sweep cap */
        if (distorted == 0) {
            status = ORC_OK;
            if (sweep_log && k < log_capacity) {
                sweep_log[4 * k + 0] = nw; sweep_log[4 * k + 1] = 0;
                sweep_log[4 * k + 2] = 0; sweep_log[4 * k + 3] = 0;
            }
            for (int64_t w = 0; w < nn; ++w) in_next[wl_next[w]] = 0;
            break;
        }
        if (k >= max_sweeps) {
            status = ORC_ERR_MAX_SWEEPS;
            left = distorted;
            if (sweep_log && k < log_capacity) {
                sweep_log[4 * k + 0] = nw; sweep_log[4 * k + 1] = distorted;
                sweep_log[4 * k + 2] = nt; sweep_log[4 * k + 3] = 0;
            }
            for (int64_t w = 0; w < nn; ++w) in_next[wl_next[w]] = 0;
            for (int64_t q = 0; q < nt; ++q) is_target[tlist[q]] = 0;
            break;
        }
        /* 3. edit each distinct target once (Eq. 1) */
        for (int64_t q = 0; q < nt; ++q) {
            int64_t t = tlist[q];
            is_target[t] = 0;
            if (rule == ORC_RULE_BELOW ? !orc_edit_below(&g[t], L[t], cand[t]) : !orc_edit(&g[t], L[t], rule))
                continue;
            ++changed;
            if (use_worklist) {
                if (!in_next[t]) { in_next[t] = 1; wl_next[nn++] = t; }
                int ns = orc_num_slots(ndim);
                for (int s = 0; s < ns; ++s) {
                    int64_t j;
                    if (orc_neighbour(ndim, nx, ny, nz, t, s, &j) && !in_next[j]) {
                        in_next[j] = 1;
                        wl_next[nn++] = j;
                    }
                }
            }
        }
        if (sweep_log && k < log_capacity) {
            sweep_log[4 * k + 0] = nw; sweep_log[4 * k + 1] = distorted;
            sweep_log[4 * k + 2] = nt; sweep_log[4 * k + 3] = changed;
        }
        edits += changed;
        ++sweeps;
        /* 4. a sweep that finds distortions but changes nothing cannot progress */
        if (changed == 0) {
            status = ORC_STUCK;
            left = distorted;
            for (int64_t w = 0; w < nn; ++w) in_next[wl_next[w]] = 0;
            break;
        }
        if (use_worklist) {
            for (int64_t w = 0; w < nn; ++w) { in_next[wl_next[w]] = 0; wl[w] = wl_next[w]; }
            nw = nn;
        }
    }

    /* Edit list (Sec. III-B: g = fhat + delta), sorted by vertex index. */
    int64_t ne = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t a, b;
        memcpy(&a, &g[i], 4);
        memcpy(&b, &fhat[i], 4);
        if (a == b) continue;
        if (ne < edit_capacity && edit_idx && edit_delta) {
            edit_idx[ne] = (uint32_t)i;
            edit_delta[ne] = g[i] - fhat[i];
        }
        ++ne;
    }
    if (edit_count) *edit_count = ne;
    if (stats) {
        stats[0] = sweeps; stats[1] = edits; stats[2] = ne; stats[3] = first_distorted;
        stats[4] = left; stats[5] = examined; stats[6] = status; stats[7] = 0;
    }
    free(cf); free(is_target); free(in_next); free(tlist); free(wl); free(wl_next); free(L); free(cand);
    if (status == ORC_OK && ne > edit_capacity) return ORC_ERR_CAPACITY;
    return status;
}

/* ---------------------------------------------------------------------------
 * Relaxed synchronization (Sec. IV-B), emulated on one device.  The grid is
 * cut into tiles of tx x ty x tz vertices (the paper's per-process blocks);
 * the one-vertex ring around a tile plays the ghost layer.  Iteration k:
 *   1. detect every vertex distorted in g^k; stop with OK when there is none
 *      (or with MAX_SWEEPS after max_iters iterations);
 *   2. every tile that holds a distorted vertex takes a copy of g^k over the
 *      tile and its ring and runs synchronous sweeps on that copy alone: its
 *      own vertices are examined, each distinct target (an own or a ring
 *      vertex) gets one application of Eq. 1 per sweep, until no own vertex is
 *      distorted, a sweep changes nothing, or local_cap sweeps (<= 0: 65536);
 *   3. merge: g^(k+1)_v = the minimum of g^k_v and of every tile's copy at v
 *      (the minimum of the candidates, Sec. IV-B); stop with STUCK when no
 *      value decreased.
 * Tiles read only g^k and the merge is a minimum, so the result does not
 * depend on the order in which tiles run.  Values are compared in IEEE
 * totalOrder (-0 below +0), so even signed zeros merge the same way in any
 * order.  With one tile covering the grid, iteration 0 is the synchronous
 * loop of orc_correct run to its end.
 * stats (may be NULL), 8 entries: [0] iterations that decreased g, [1] local
 * sweeps summed over tile runs, [2] distinct edited vertices (g != fhat),
 * [3] distorted vertices in iteration 0, [4] distorted vertices left, [5] tile
 * runs, [6] status, [7] 0.
 * ------------------------------------------------------------------------- */
int orc_correct_relaxed(const float *f, const float *fhat, float xi, int ndim, int64_t nx, int64_t ny,
                        int64_t nz, int64_t tx, int64_t ty, int64_t tz, int rule, int64_t local_cap,
                        int64_t max_iters, float *g, int64_t *stats)
{
    if (!f || !fhat || !g || nx < 1 || ny < 1 || nz < 1 || (ndim != 2 && ndim != 3) || (ndim == 2 && nz != 1) ||
        tx < 1 || ty < 1 || tz < 1 || max_iters < 0 || (rule != ORC_RULE_HALVE && rule != ORC_RULE_SNAP))
        return ORC_ERR_INVALID_ARG;
    if (local_cap <= 0) local_cap = 65536;
    int64_t n = nx * ny * nz;
    int st = orc_validate(f, fhat, n, xi);
    if (st != ORC_OK) return st;
    int64_t ntx = (nx + tx - 1) / tx, nty = (ny + ty - 1) / ty, ntz = (nz + tz - 1) / tz;
    int64_t ntiles = ntx * nty * ntz;
    uint8_t *cf = malloc((size_t)n);
    uint8_t *active = malloc((size_t)ntiles);
    uint8_t *is_target = calloc((size_t)n, 1);
    int64_t *tlist = malloc(sizeof(int64_t) * (size_t)n);
    float *L = malloc(sizeof(float) * (size_t)n);
    float *snap = malloc(sizeof(float) * (size_t)n);
    float *local = malloc(sizeof(float) * (size_t)n);
    if (!cf || !active || !is_target || !tlist || !L || !snap || !local) {
        free(cf); free(active); free(is_target); free(tlist); free(L); free(snap); free(local);
        return ORC_ERR_OOM;
    }
    for (int64_t i = 0; i < n; ++i) {
        g[i] = fhat[i];
        L[i] = orc_floor(f[i], xi);
    }
    orc_codes(f, ndim, nx, ny, nz, cf);

    int64_t iters = 0, local_sweeps = 0, first_distorted = -1, left = 0, runs = 0;
    int status = ORC_ERR_MAX_SWEEPS;
    for (int64_t k = 0;; ++k) {
        /* 1. detect over the whole grid */
        int64_t distorted = 0;
        memset(active, 0, (size_t)ntiles);
        for (int64_t i = 0; i < n; ++i) {
            if (orc_code_at(g, ndim, nx, ny, nz, i) == cf[i]) continue;
            ++distorted;
            int64_t x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
            active[(x / tx) + ntx * ((y / ty) + nty * (z / tz))] = 1;
        }
        if (k == 0) first_distorted = distorted;
        if (distorted == 0) { status = ORC_OK; break; }
        if (k >= max_iters) { status = ORC_ERR_MAX_SWEEPS; left = distorted; break; }
        /* 2. local sweeps of every active tile on its own copy of g^k */
        memcpy(snap, g, sizeof(float) * (size_t)n);
        memcpy(local, g, sizeof(float) * (size_t)n);
        for (int64_t b = 0; b < ntiles; ++b) {
            if (!active[b]) continue;
            ++runs;
            int64_t bx = b % ntx, by = (b / ntx) % nty, bz = b / (ntx * nty);
            int64_t x0 = bx * tx, y0 = by * ty, z0 = bz * tz;
            int64_t x1 = x0 + tx < nx ? x0 + tx : nx, y1 = y0 + ty < ny ? y0 + ty : ny, z1 = z0 + tz < nz ? z0 + tz : nz;
            /* ring-extended box, clipped to the grid */
            int64_t rx0 = x0 > 0 ? x0 - 1 : 0, ry0 = y0 > 0 ? y0 - 1 : 0, rz0 = z0 > 0 ? z0 - 1 : 0;
            int64_t rx1 = x1 < nx ? x1 + 1 : nx, ry1 = y1 < ny ? y1 + 1 : ny, rz1 = z1 < nz ? z1 + 1 : nz;
            for (int64_t ls = 0; ls < local_cap; ++ls) {
                int64_t nt = 0, dist_here = 0;
                for (int64_t z = z0; z < z1; ++z)
                    for (int64_t y = y0; y < y1; ++y)
                        for (int64_t x = x0; x < x1; ++x) {
                            int64_t i = x + nx * (y + ny * z);
                            uint8_t cg = orc_code_at(local, ndim, nx, ny, nz, i);
                            if (cg == cf[i]) continue;
                            ++dist_here;
                            int64_t t[2];
                            int m = targets_of(ndim, nx, ny, nz, i, cf[i], cg, t);
                            for (int q = 0; q < m; ++q)
                                if (!is_target[t[q]]) { is_target[t[q]] = 1; tlist[nt++] = t[q]; }
                        }
                if (dist_here == 0) break;
                ++local_sweeps;
                int64_t changed = 0;
                for (int64_t q = 0; q < nt; ++q) {
                    is_target[tlist[q]] = 0;
                    changed += orc_edit(&local[tlist[q]], L[tlist[q]], rule);
                }
                if (changed == 0) break;
            }
            /* 3. merge by minimum, then restore the copy for the next tile */
            for (int64_t z = rz0; z < rz1; ++z)
                for (int64_t y = ry0; y < ry1; ++y)
                    for (int64_t x = rx0; x < rx1; ++x) {
                        int64_t i = x + nx * (y + ny * z);
                        if (total_key(local[i]) < total_key(g[i])) g[i] = local[i];
                        local[i] = snap[i];
                    }
        }
        int64_t decreased = 0;
        for (int64_t i = 0; i < n; ++i) decreased += total_key(g[i]) < total_key(snap[i]);
        if (decreased == 0) { status = ORC_STUCK; left = distorted; break; }
        ++iters;
    }
    if (stats) {
        int64_t ne = 0;
        for (int64_t i = 0; i < n; ++i) {
            uint32_t a, c;
            memcpy(&a, &g[i], 4);
            memcpy(&c, &fhat[i], 4);
            ne += a != c;
        }
        stats[0] = iters; stats[1] = local_sweeps; stats[2] = ne; stats[3] = first_distorted;
        stats[4] = left; stats[5] = runs; stats[6] = status; stats[7] = 0;
    }
    free(cf); free(active); free(is_target); free(tlist); free(L); free(snap); free(local);
    return status;
}

/* ---------------------------------------------------------------------------
 * Sec. III-A: integral lines and the ascending/descending segmentations.
 * max_label[i] = the maximum reached from i by repeatedly stepping to n_max
 * (the code's low nibble) until a vertex that is a maximum; min_label[i]
 * likewise through n_min.  Path following, remembering the labels already
 * found so that each vertex is walked once.
 * ------------------------------------------------------------------------- */
static void follow(const uint8_t *codes, int ndim, int64_t nx, int64_t ny, int64_t nz,
                   int shift, int32_t *lab, int64_t *stack)
{
    int64_t n = nx * ny * nz;
    for (int64_t i = 0; i < n; ++i) lab[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        if (lab[i] >= 0) continue;
        int64_t depth = 0, p = i;
        while (lab[p] < 0) {
            int s = (codes[p] >> shift) & 15;
            if (s == ORC_SELF) { lab[p] = (int32_t)p; break; }
            stack[depth++] = p;
            int64_t j = p;
            orc_neighbour(ndim, nx, ny, nz, p, s, &j);
            p = j;
        }
        for (int64_t q = 0; q < depth; ++q) lab[stack[q]] = lab[p];
    }
}

int orc_labels(const uint8_t *codes, int ndim, int64_t nx, int64_t ny, int64_t nz,
               int32_t *min_label, int32_t *max_label)
{
    int64_t n = nx * ny * nz;
    if (n > INT32_MAX) return ORC_ERR_INVALID_ARG;
    int64_t *stack = malloc(sizeof(int64_t) * (size_t)n);
    if (!stack) return ORC_ERR_OOM;
    if (max_label) follow(codes, ndim, nx, ny, nz, 0, max_label, stack);
    if (min_label) follow(codes, ndim, nx, ny, nz, 4, min_label, stack);
    free(stack);
    return ORC_OK;
}

/* Sec. V-C verification counts between the segmentation of f and of g:
 * out[0] wrongly labelled vertices (either label differs), out[1] false
 * positive maxima (maximum in g, not in f), out[2] false negative maxima,
 * out[3] false positive minima, out[4] false negative minima. */
void orc_compare(const uint8_t *codes_f, const uint8_t *codes_g,
                 const int32_t *min_f, const int32_t *max_f,
                 const int32_t *min_g, const int32_t *max_g, int64_t n, int64_t out[5])
{
    for (int q = 0; q < 5; ++q) out[q] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (min_f[i] != min_g[i] || max_f[i] != max_g[i]) ++out[0];
        int maxf = (codes_f[i] & 15) == ORC_SELF, maxg = (codes_g[i] & 15) == ORC_SELF;
        int minf = (codes_f[i] >> 4) == ORC_SELF, ming = (codes_g[i] >> 4) == ORC_SELF;
        if (maxg && !maxf) ++out[1];
        if (maxf && !maxg) ++out[2];
        if (ming && !minf) ++out[3];
        if (minf && !ming) ++out[4];
    }
}
