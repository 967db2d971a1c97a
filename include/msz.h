/*
 * msz.h -- C ABI of the GB300 correction engine for piecewise-linear
 * Morse-Smale segmentations under error-bounded lossy compression
 * (pMSz, arXiv 2601.01787).
 *
 * Problem (Sec. III-B): given the original field f, its decompressed copy
 * fhat and a global error bound xi, find a corrected field g <= fhat (edits
 * only lower values, Eq. 1) with |f_i - g_i| <= xi everywhere such that every
 * vertex has the same extremum status and the same steepest ascending and
 * descending neighbours in g as in f (the relaxed sufficient condition of
 * Sec. IV-A), which preserves the segmentation.
 *
 * Conventions shared by every entry point:
 *   - Grids are regular 2D or 3D, x fastest: linear index i = x + nx*(y + ny*z).
 *     The piecewise-linear interpolant lives on the Kuhn (Freudenthal)
 *     triangulation along the main diagonal (Sec. III-A "constant
 *     triangular/tetrahedral mesh"): neighbour offsets are d and -d for
 *     d in {0,1}^n \ {0}, 6 neighbours in 2D and 14 in 3D.
 *   - Neighbour slots (the numbers stored in direction codes):
 *       3D: 0 (+1,0,0) 1 (0,+1,0) 2 (0,0,+1) 3 (+1,+1,0) 4 (+1,0,+1)
 *           5 (0,+1,+1) 6 (+1,+1,+1), 7..13 the negatives of 0..6 in order;
 *       2D: 0 (+1,0) 1 (0,+1) 2 (+1,+1), 3..5 the negatives of 0..2.
 *   - Order (Sec. III-A assumes distinct values; ties are broken by index):
 *     j is above i  <=>  v_j > v_i  or  (v_j == v_i and j > i).  -0 == +0.
 *   - Error bound: L_i = smallest float32 >= f_i - xi, U_i = largest float32
 *     <= f_i + xi (exact real arithmetic); inputs must satisfy
 *     L_i <= fhat_i <= U_i and be finite.
 *   - Pointers named d_* are DEVICE pointers of the current CUDA device;
 *     pointers named h_* are HOST pointers (pinned memory is fastest).  The
 *     caller owns every buffer; the library allocates no device memory: all
 *     scratch lives in the caller's workspace.
 *   - Every call is ordered on `stream` (NULL = legacy default stream).  Calls
 *     that return results to host memory (counts, stats, status) synchronize
 *     that stream before returning; this is stated per call.
 *   - No call throws or aborts; failures come back as msz_status.  After
 *     MSZ_ERR_CUDA the CUDA context may be unusable (sticky CUDA error).
 *   - At most MSZ_MAX_VERTICES vertices per field (labels are int32, edit
 *     indices uint32).
 */
#ifndef MSZ_H
#define MSZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* = cudaStream_t */
typedef struct CUstream_st *msz_stream_t;

#define MSZ_SELF 15                    /* code nibble of an extremum */
#define MSZ_MAX_VERTICES 2147483647LL  /* 2^31 - 1 */
#define MSZ_MAX_SWEEPS_LIMIT 65536     /* upper limit of msz_options.max_sweeps */
#define MSZ_SMALL_WORKSPACE 65536      /* bytes needed by msz_segment / msz_compare */

typedef enum {
    MSZ_OK = 0,
    MSZ_ERR_INVALID_ARG = 1,  /* null pointer, bad grid, xi < 0 or not finite, bad option */
    MSZ_ERR_INPUT_BOUND = 2,  /* some value not finite, or fhat (or g_init) outside [L_i, U_i] */
    MSZ_ERR_CAPACITY = 3,     /* loop converged but the edit list did not fit; *edit_count = needed */
    MSZ_ERR_WORKSPACE = 4,    /* workspace too small (or NULL) for this grid */
    MSZ_ERR_CUDA = 5,         /* a CUDA runtime call or launch failed */
    MSZ_ERR_MAX_SWEEPS = 6,   /* still distorted after max_sweeps sweeps */
    MSZ_ERR_TIMEOUT = 7,      /* a bounded device-side wait ran out (grid barrier) */
    MSZ_STUCK = 8,            /* a sweep found distortions but every target was at its floor */
    MSZ_ERR_UNSUPPORTED = 9   /* no sm_103a device / not enough co-resident blocks */
} msz_status;

typedef struct {
    int32_t ndim;     /* 2 or 3 */
    int32_t reserved; /* 0 */
    int64_t nx, ny, nz; /* >= 1 each; nz == 1 when ndim == 2 */
} msz_grid;

/* Eq. 1 leaves the edit amount delta open.  HALVE moves g halfway to its floor
 * L (s = g - L; h = g - 0.5*s; h = max(h, L); h = L when h is not below g),
 * SNAP moves it to the floor in one edit (Fig. nonextrema (c): 0.1 -> 0).
 * BELOW_REFERENCE (Sec. IV-A: the spurious maximum is decreased "to 0.3 or
 * slightly below") moves the target to the largest value that puts it below
 * the vertex it must fall under, in the (value, index) order: r's value when
 * the reference r has the larger index, else the float just below it; kept at
 * or above L.  The reference of an ascending mismatch at i is f's steepest
 * ascent of i (i itself when f makes i a maximum); of a descending mismatch,
 * g's steepest descent of i (i itself when g makes i a minimum).  All values
 * come from g of the sweep (Jacobi); a target several vertices ask for takes
 * the smallest candidate in IEEE totalOrder (Sec. IV-B: the minimum of the
 * candidates).  BELOW_REFERENCE is available in msz_correct only (the batch,
 * relaxed and pipelined entry points return MSZ_ERR_INVALID_ARG or
 * MSZ_ERR_WORKSPACE), with the workspace of msz_workspace_size_rule. */
typedef enum { MSZ_RULE_HALVE = 0, MSZ_RULE_SNAP = 1, MSZ_RULE_BELOW_REFERENCE = 2 } msz_rule;

typedef struct {
    int32_t rule;             /* msz_rule; default HALVE */
    int32_t test_fault;       /* 0.  Test hooks of the bounded waits: 1 makes block 0 of the
                                 correction kernel wait at its first grid barrier without
                                 arriving, so every block's wait (shortened to 0.25 s) runs
                                 out; 2 (grids whose planes are staged by TMA) makes block 0
                                 of the code pass withhold its first plane copy, so its
                                 mbarrier wait (shortened to 0.25 s) runs out.  Either way
                                 the call returns MSZ_ERR_TIMEOUT with no output */
    int64_t max_sweeps;       /* <= 0: MSZ_MAX_SWEEPS_LIMIT; else 1..MSZ_MAX_SWEEPS_LIMIT */
    int64_t dense_min_items;  /* > 0: the next sweep scans every uncertified vertex instead of
                                 the worklist when 6 x (vertices distorted in this sweep) >=
                                 this; 0 (default): N on 3D grids, always the worklist on 2D
                                 ones; -1: always the worklist.  The batch entry points decide
                                 for each field by its own distorted count (and its own N).
                                 Affects speed only, never results */
    const float *d_g_init;    /* NULL: start from fhat.  Else N floats, each in [L_i, U_i]: a
                                 proposed start (the learned proposal); edits are still
                                 reported against fhat */
    int64_t *h_sweep_log;     /* NULL, or 4*log_capacity int64 filled per sweep k with
                                 |worklist_k|, distorted_k, distinct targets_k, changed_k */
    int64_t log_capacity;
    int64_t *h_timeline;      /* NULL, or 2*log_capacity int64 (needs h_sweep_log): device
                                 time in ns from the start of the correction (sweep 0's pass)
                                 to the end of sweep k's detection and of its edit phase
                                 (-1: none).  The batch entry points write one timeline for
                                 the whole batch here (filled by msz_batch_collect, or by
                                 msz_correct_batch; they need no h_sweep_log in this struct) */
    int32_t tile_z;           /* z-planes per tile of the code pass (3D); at most 1024; 0: the
                                 deepest of 24, 16, 8 that gives every block of the persistent
                                 grid two tiles (msz_correct; the batch and relaxed entry points
                                 use 24).  Affects speed only (see the autotuner), never results */
    int32_t local_cap;        /* msz_correct_relaxed: local sweeps per tile run; 0: 65536 */
    void *phase_events[3];    /* msz_correct and msz_correct_static only (other entry points
                                 ignore them): each NULL or a cudaEvent_t of the current
                                 device, recorded on the stream [0] before sweep 0's pass
                                 over a 3D grid (its own kernel), [1] between that pass and
                                 the kernel of the later sweeps and the edit list, [2] after
                                 that kernel, so that cudaEventElapsedTime times each kernel
                                 alone.  On 2D grids (one kernel) [0] and [1] are both
                                 recorded before it.  A record that fails returns
                                 MSZ_ERR_CUDA */
} msz_options;

typedef struct {
    int64_t sweeps;           /* sweeps that applied edits (0: fhat already correct) */
    int64_t edits;            /* total value decreases applied */
    int64_t edited;           /* distinct vertices with g != fhat (= edit list length) */
    int64_t first_distorted;  /* distorted vertices found in sweep 0 */
    int64_t left;             /* distorted vertices left (STUCK / MAX_SWEEPS), else 0 */
    int64_t examined;         /* vertices examined over all sweeps (dense sweeps count N) */
    int64_t dense_sweeps;     /* sweeps run as whole-grid scans, sweep 0 included */
    int64_t kernel_ns;        /* device time of the correction kernel (globaltimer) */
    int64_t codes_ns;         /* ... of its first phase: the codes of f and their certification
                                 (3D grids: with sweep 0's detection, done in the same pass) */
    int64_t uncertified;      /* vertices sweep 0 could not certify (only these can ever be
                                 distorted) */
    int64_t local_sweeps;     /* msz_correct_relaxed: local sweeps summed over tile runs */
    int64_t tile_runs;        /* msz_correct_relaxed: tile runs summed over iterations */
} msz_stats;

/* Bytes of device workspace msz_correct needs for this grid (about 13.5 bytes
 * per vertex plus 1.2 MB); 0 for an invalid grid. */
size_t msz_workspace_size(msz_grid grid);

/* Bytes of device workspace msz_correct needs for this grid under edit rule
 * `rule`: msz_workspace_size for HALVE and SNAP, plus 4 bytes per vertex (each
 * target's smallest candidate) for BELOW_REFERENCE; 0 for an invalid grid or
 * rule. */
size_t msz_workspace_size_rule(msz_grid grid, int32_t rule);

/* Sec. IV-A / Sec. III-A: steepest-neighbour codes of one field.
 * codes[i] low nibble = slot of n_max(i) = argmax over N(i) when it is above i,
 * else MSZ_SELF (i is a maximum); high nibble = slot of n_min(i) when below i,
 * else MSZ_SELF (i is a minimum).  d_v: N floats (finite); d_codes: N bytes.
 * Asynchronous (no host sync). */
msz_status msz_directions(const float *d_v, msz_grid grid, uint8_t *d_codes, msz_stream_t stream);

/* The correction loop (Sec. III-B iterative edit strategy with the redesigned
 * C-loop of Sec. IV-A, synchronous Jacobi sweeps):
 *   sweep k detects every vertex whose code in g^k differs from its code in f
 *   and edits, once each (Eq. 1), the distinct targets:
 *     ascending mismatch  -> the vertex itself when g makes it a maximum (FPmax),
 *                            else its largest neighbour in g (FNmax / spurious max);
 *     descending mismatch -> the vertex itself when f makes it a minimum (FNmin),
 *                            else its smallest neighbour in f (FPmin / original min);
 *   it stops when nothing is distorted (MSZ_OK), when a sweep changes nothing
 *   (MSZ_STUCK) or after max_sweeps sweeps (MSZ_ERR_MAX_SWEEPS).
 * Inputs: d_f, d_fhat (N floats each, finite, L_i <= fhat_i <= U_i), xi >= 0.
 * Output: d_out (N floats, must not alias the inputs) = g; the edit list
 *   d_edit_idx / d_edit_delta (edit_capacity entries each, may be NULL when
 *   edit_capacity == 0): every i with g_i != fhat_i (bitwise), ascending i,
 *   delta = float32(g_i - fhat_i); *h_edit_count = the number of such i (may
 *   exceed edit_capacity: then MSZ_ERR_CAPACITY on an otherwise OK run; d_out
 *   is complete either way).
 * Workspace: d_workspace of at least msz_workspace_size_rule(grid, rule) bytes
 *   (msz_workspace_size(grid) for HALVE and SNAP), 256-byte aligned, not used
 *   by any concurrent call.
 * Synchronizes `stream` before returning (status, counts and stats are read back). */
msz_status msz_correct(const float *d_f, const float *d_fhat, float xi, msz_grid grid, float *d_out,
                       uint32_t *d_edit_idx, float *d_edit_delta, int64_t edit_capacity,
                       int64_t *h_edit_count, const msz_options *opt, msz_stats *h_stats,
                       void *d_workspace, size_t workspace_bytes, msz_stream_t stream);

/* Bytes of device workspace msz_correct_host needs: msz_workspace_size plus
 * room for f, fhat, g and an edit list of edit_capacity entries. */
size_t msz_host_workspace_size(msz_grid grid, int64_t edit_capacity);

/* msz_correct with HOST buffers: copies h_f and h_fhat to the device, runs the
 * correction, and copies g and the edit list back into h_out / h_edit_idx /
 * h_edit_delta.  Same semantics and statuses as msz_correct.  Synchronizes
 * `stream`. */
msz_status msz_correct_host(const float *h_f, const float *h_fhat, float xi, msz_grid grid, float *h_out,
                            uint32_t *h_edit_idx, float *h_edit_delta, int64_t edit_capacity,
                            int64_t *h_edit_count, const msz_options *opt, msz_stats *h_stats,
                            void *d_workspace, size_t workspace_bytes, msz_stream_t stream);

/* ---- Pipelined host-buffer correction (no counterpart in the paper: a
 * serving path).  A sequence of fields of one grid -- time steps, say -- is
 * corrected with the copies of consecutive fields overlapped: field k+1's
 * inputs go up while field k is corrected and field k-1's result comes
 * down.  Two slots of device buffers live in the caller's workspace
 * (msz_pipeline_workspace_size bytes, 256-byte aligned); the pipeline owns
 * three CUDA streams, six events and a few hundred bytes of pinned host
 * memory.  Each field's results are those of msz_correct_host. */
typedef struct msz_pipeline msz_pipeline;
size_t msz_pipeline_workspace_size(msz_grid grid, int64_t edit_capacity);
msz_status msz_pipeline_create(msz_grid grid, int64_t edit_capacity, void *d_workspace, size_t workspace_bytes,
                               msz_pipeline **out);
/* Enqueues one field (host buffers of N floats) and returns without waiting.
 * h_out and, when the capacity is > 0, the edit arrays must stay valid until
 * the field is collected.  At most two fields may be submitted and not yet
 * collected (MSZ_ERR_INVALID_ARG otherwise).  opt: as msz_correct, without
 * d_g_init, the sweep log or the test hook.  Pinned host buffers let the
 * copies overlap; pageable ones work but serialize. */
msz_status msz_pipeline_submit(msz_pipeline *pl, const float *h_f, const float *h_fhat, float xi, float *h_out,
                               uint32_t *h_edit_idx, float *h_edit_delta, const msz_options *opt);
/* Waits for the oldest submitted field and returns its status (as
 * msz_correct_host), edit count and stats; its h_out and edit list are
 * filled on return.  MSZ_ERR_INVALID_ARG when nothing is pending. */
msz_status msz_pipeline_collect(msz_pipeline *pl, int64_t *h_edit_count, msz_stats *h_stats);
/* Waits for the pipeline's work, then frees its streams, events and pinned
 * memory (not the workspace). */
void msz_pipeline_destroy(msz_pipeline *pl);

/* The same pipeline returning, per field, the edit list as a stream in the
 * msz_edits_encode format instead of g and the list: what a compressor
 * stores beside its compressed data (g = fhat with the stream applied, see
 * msz_edits_decode).  The stream is encoded on the device behind the
 * correction and only its bytes come down.  Workspace:
 * msz_pipeline_workspace_size_encoded bytes (the two slots plus a stream
 * buffer of msz_edits_encoded_bound(edit_capacity) bytes and its encoder's
 * workspace each).  submit_encoded: h_stream (stream_capacity bytes) must
 * stay valid until the field is collected.  collect_encoded: *h_stream_bytes
 * = the stream's length; MSZ_ERR_CAPACITY when the edits exceed the
 * pipeline's edit capacity or the stream exceeds stream_capacity (then
 * *h_stream_bytes = the length needed, nothing copied).  The field-mode
 * calls reject an encoded pipeline and the other way round. */
size_t msz_pipeline_workspace_size_encoded(msz_grid grid, int64_t edit_capacity);
msz_status msz_pipeline_create_encoded(msz_grid grid, int64_t edit_capacity, void *d_workspace,
                                       size_t workspace_bytes, msz_pipeline **out);
msz_status msz_pipeline_submit_encoded(msz_pipeline *pl, const float *h_f, const float *h_fhat, float xi,
                                       uint8_t *h_stream, size_t stream_capacity, const msz_options *opt);
msz_status msz_pipeline_collect_encoded(msz_pipeline *pl, int64_t *h_edit_count, size_t *h_stream_bytes,
                                        msz_stats *h_stats);

/* Sec. III-A ascending/descending segmentations, for verification:
 * d_max_label[i] = index of the maximum reached by following n_max (the low
 * nibble of d_codes) from i; d_min_label[i] likewise through n_min.  Computed
 * by pointer jumping to a fixed point.  Either label pointer may be NULL.
 * Workspace: at least MSZ_SMALL_WORKSPACE bytes.  Synchronizes `stream`. */
msz_status msz_segment(const uint8_t *d_codes, msz_grid grid, int32_t *d_min_label, int32_t *d_max_label,
                       void *d_workspace, size_t workspace_bytes, msz_stream_t stream);

/* Sec. V-C verification counts between the segmentations of f and g:
 * h_counts[0] wrongly labelled vertices (either label differs), [1] false
 * positive maxima (maximum in g only), [2] false negative maxima, [3] false
 * positive minima, [4] false negative minima, and [5] vertices whose code
 * differs (the loop's stopping condition, Sec. IV-A).  All device arrays hold
 * n entries.  Workspace: at least MSZ_SMALL_WORKSPACE bytes.  Synchronizes
 * `stream`. */
msz_status msz_compare(const uint8_t *d_codes_f, const uint8_t *d_codes_g, const int32_t *d_min_f,
                       const int32_t *d_max_f, const int32_t *d_min_g, const int32_t *d_max_g, int64_t n,
                       int64_t h_counts[6], void *d_workspace, size_t workspace_bytes, msz_stream_t stream);

/* One field of a batch (msz_correct_batch).  Inputs: d_f, d_fhat, xi, grid
 * (ndim 3), d_out and the edit-list arrays as in msz_correct.  Outputs, written
 * by the call: edit_count, status (the msz_correct status this field alone
 * would get) and stats. */
typedef struct {
    const float *d_f;
    const float *d_fhat;
    float xi;
    int32_t status;         /* out */
    msz_grid grid;
    float *d_out;
    uint32_t *d_edit_idx;
    float *d_edit_delta;
    int64_t edit_capacity;
    int64_t edit_count;     /* out */
    msz_stats stats;        /* out */
    int32_t tile_z;         /* 0: msz_options.tile_z */
    int32_t reserved;
} msz_field;

#define MSZ_BATCH_MAX_FIELDS 256
#define MSZ_BATCH_MAX_SWEEPS 4096

/* Bytes of device workspace msz_correct_batch needs for these fields and sweep
 * cap (max_sweeps <= 0: MSZ_BATCH_MAX_SWEEPS); 0 for an invalid batch. */
size_t msz_batch_workspace_size(int32_t n, const msz_field *fields, int64_t max_sweeps);

/* Batched form of msz_correct (an extension: the paper corrects one field per
 * run): n 3D fields of any sizes, each with its own xi, corrected
 * by one cooperative persistent launch.  The fields share one tile queue for
 * the code pass and one set of sweeps; each field stops taking part when it is
 * done, stuck or capped, and every field gets exactly the g, edit list,
 * status and per-sweep counts that a separate msz_correct call would give
 * (with the same options; d_g_init must be NULL).  h_sweep_log (may be NULL):
 * 4*log_capacity int64 per field, field-major, as msz_options.h_sweep_log.
 * Returns MSZ_OK when the launch completed (per-field statuses in fields[k]);
 * MSZ_ERR_INPUT_BOUND when some field's input is out of bound (that field's
 * status says so; no results); otherwise an error for the whole call.
 * Synchronizes `stream`. */
msz_status msz_correct_batch(int32_t n, msz_field *fields, const msz_options *opt, int64_t *h_sweep_log,
                             int64_t log_capacity, void *d_workspace, size_t workspace_bytes, msz_stream_t stream);

/* msz_correct_batch in three steps, so that the launch can be captured in a
 * CUDA graph and replayed (the fields' buffers and the workspace must then
 * stay where they are):
 *   msz_batch_plan_create   checks the batch as msz_correct_batch does,
 *                           uploads the field table into the workspace and
 *                           returns a host-side plan in *plan (synchronizes
 *                           `stream`; not capturable);
 *   msz_batch_launch        one memset of the workspace's control block and
 *                           bitmaps plus the cooperative kernel launch on
 *                           `stream`: asynchronous, no host synchronization,
 *                           capturable (on the plan's device);
 *   msz_batch_collect       synchronizes `stream`, reads the control block,
 *                           the per-field results and the sweep log, and
 *                           fills fields[k] (status, edit_count, stats) and
 *                           h_sweep_log exactly as msz_correct_batch does;
 *                           the fields array must describe the same batch;
 *   msz_batch_plan_destroy  frees the plan (host memory only).
 * The plan owns no device memory. */
typedef struct msz_batch_plan msz_batch_plan;
msz_status msz_batch_plan_create(int32_t n, const msz_field *fields, const msz_options *opt, void *d_workspace,
                                 size_t workspace_bytes, msz_stream_t stream, msz_batch_plan **plan);
msz_status msz_batch_launch(const msz_batch_plan *plan, msz_stream_t stream);
msz_status msz_batch_collect(const msz_batch_plan *plan, msz_field *fields, int64_t *h_sweep_log,
                             int64_t log_capacity, msz_stream_t stream);
void msz_batch_plan_destroy(msz_batch_plan *plan);

/* ---- Learned initial-edit proposal (an extension: the paper has no learned
 * component).  A 4-layer 3D conv net (3x3x3 cross-correlations, zero
 * padding, channels 16 -> 32 -> 32 -> 32 -> 16, ReLU between) classifies each
 * vertex by k = 0..15, the number of HALVE edits the plain loop applies to it
 * (15: fifteen or more).  The start g0 = fhat edited k times by that rule goes
 * to msz_correct as d_g_init and the exact loop finishes from there, so every
 * invariant still holds; a right class reproduces the plain loop's value bit
 * for bit.  Tensors: channels-last BF16 ([z][y][x][C], C = 16 or 32; uint16_t
 * storage), 16-byte aligned; 3D grids only; weights w[o][cout][cin] FP32 with
 * kernel offset o = (dz+1)*9 + (dy+1)*3 + (dx+1) applied to input voxel
 * (x+dx, y+dy, z+dz).  All calls are asynchronous on `stream`. */

/* The 16 input channels (BF16) per vertex: 0 (fhat - f)/xi; 1..3 the forward
 * differences of f along x, y, z divided by 4 xi; 4, 5 f has a maximum / a
 * minimum here; 6, 7 fhat's ascending / descending code differs from f's;
 * 8, 9 the vertex is the target of an ascending / descending mismatch in the
 * first sweep (the msz_correct target rule with g = fhat); 10, 11 fhat has a
 * maximum / a minimum here; 12..14 the forward differences of fhat divided
 * by 4 xi; 15 the fraction of the 14 neighbours whose f equals this vertex's.
 * Differences are clamped to [-1, 1] and read as 0 past the grid's end.
 * d_codes_f / d_codes_fhat: msz_directions of f / fhat; 3D grids only. */
msz_status msz_learned_features(const float *d_f, const float *d_fhat, float xi, msz_grid grid,
                                const uint8_t *d_codes_f, const uint8_t *d_codes_fhat, uint16_t *d_x,
                                msz_stream_t stream);

/* BF16 weight image of a conv with cin input and cout output channels (16 or
 * 32 each) from FP32 weights d_w[27][cout_real][cin_real], zero-padded;
 * mirror != 0: the image of the backward-data conv (input = gradient of the
 * forward output, weights of the mirrored offset, channels swapped).  d_img:
 * msz_learned_weight_image_size(cin, cout) bytes (0 for an unsupported
 * shape): per 16-channel slab pair and (dx, dz) offset, a strip of the five
 * dy = 2 .. -2 weight blocks (the outer two zero), so that one tensor-core
 * operand covers two output rows. */
size_t msz_learned_weight_image_size(int32_t cin, int32_t cout);
msz_status msz_learned_weight_image(const float *d_w, int32_t cout_real, int32_t cin_real, int32_t cin,
                                    int32_t cout, int32_t mirror, uint16_t *d_img, msz_stream_t stream);

/* One 3x3x3 conv layer on tcgen05 tensor cores (BF16 x BF16 -> FP32 in TMEM).
 * mode 0 (ReLU):  d_out_bf16 = max(0, conv(d_x) + d_bias)       cin 16|32, cout 32
 * mode 1 (head):  k = argmax_c (conv(d_x)[c] + d_bias[c]) (lowest c on ties);
 *                 a nonzero k becomes clamp(k + shift, 1, 15); d_out_f32 (may
 *                 be NULL) = k; if d_g0: d_g0 = fhat edited k times by HALVE
 *                 with floor L of d_f, xi                         cin 32, cout 16
 * mode 2 (dgrad): d_out_bf16 = conv(d_x) where d_mask > 0, else 0 (the input
 *                 gradient through a ReLU; d_x = output gradient)  cin 16|32, cout 32
 * mode 3 (raw):   d_out_f32 = conv(d_x) (+ d_bias if not NULL)    any of the above
 * d_err: a device word that gets bit 0 when a bounded wait ran out. */
msz_status msz_learned_conv(const uint16_t *d_x, int32_t cin, int32_t cout, int32_t mode, msz_grid grid,
                            const uint16_t *d_img, const float *d_bias, uint16_t *d_out_bf16, float *d_out_f32,
                            const uint16_t *d_mask, const float *d_f, const float *d_fhat, float xi, int32_t shift,
                            float *d_g0, uint32_t *d_err, msz_stream_t stream);

/* Training loss head: d_z holds the 16 head logits per vertex (the raw head
 * conv with its bias), d_target the class k per vertex (as float).
 * *d_loss_sum += sum of the softmax cross-entropies logsumexp(z) - z_k
 * (double); d_dz16 = scale (softmax(z) - onehot(k)), 16 BF16 per vertex. */
msz_status msz_learned_head_grad(const float *d_z, const float *d_target, int64_t n, float scale,
                                 uint16_t *d_dz16, double *d_loss_sum, msz_stream_t stream);

/* Training classes: d_target[i] = the number of HALVE edits (capped at 15)
 * that take fhat_i to g_i, g the corrected field of msz_correct from fhat. */
msz_status msz_learned_target(const float *d_f, const float *d_fhat, const float *d_g, float xi, int64_t n,
                              float *d_target, msz_stream_t stream);

/* Weight and bias gradients of one layer (FP32, accumulated into d_dw
 * [27][cout_real][cin_real] and d_db[cout_real]): dw[o][co][ci] += sum_v
 * dz[v][co] x[v + d_o][ci].  d_x: the layer's input (cin channels), d_dz: the
 * gradient of its pre-activation output (cout channels).  (cin, cout) is
 * (16, 32), (32, 32) or (32, 16).  The partial sums of a fixed set of thread
 * blocks go to d_workspace (msz_learned_wgrad_workspace_size(cin, cout) bytes,
 * 16-byte aligned; MSZ_ERR_WORKSPACE if smaller) and are added in a fixed
 * order, with no atomics: the same inputs give the same gradient bit for bit
 * on every run. */
size_t msz_learned_wgrad_workspace_size(int32_t cin, int32_t cout);
msz_status msz_learned_wgrad(const uint16_t *d_x, int32_t cin, const uint16_t *d_dz, int32_t cout, msz_grid grid,
                             int32_t cin_real, int32_t cout_real, float *d_dw, float *d_db, void *d_workspace,
                             size_t workspace_bytes, msz_stream_t stream);

/* One Adam step on n FP32 parameters (bias-corrected; step >= 1). */
msz_status msz_learned_adam(float *d_p, const float *d_g, float *d_m, float *d_v, int64_t n, float lr, float beta1,
                            float beta2, float eps, int64_t step, msz_stream_t stream);

/* ---- Relaxed synchronization (Sec. IV-B) emulated on one GPU.  The paper's
 * per-process blocks become tiles of MSZ_RELAXED_TILE_X x _Y x _Z vertices
 * (one thread block each), its ghost layer the one-vertex ring around a tile,
 * its ghost exchange a merge by minimum.  Iteration k: detect every vertex
 * distorted in g^k (none: MSZ_OK); every tile holding one runs synchronous
 * sweeps (the rule of msz_correct) on its own copy of g^k over the tile and
 * its ring -- its own vertices are examined, targets may lie on the ring --
 * until no own vertex is distorted, a sweep changes nothing, or
 * opt->local_cap sweeps; then g^(k+1) = the minimum, in IEEE totalOrder, of
 * g^k and every tile's copy (MSZ_STUCK when nothing decreased).  The result
 * does not depend on the order in which tiles run.  3D grids only; no
 * d_g_init; opt->max_sweeps caps the iterations.  stats: sweeps = iterations
 * that decreased g, local_sweeps, tile_runs, edited, first_distorted, left,
 * kernel_ns, codes_ns, uncertified (other fields 0).  h_sweep_log per
 * iteration: tile runs, distorted vertices, local sweeps, decreased values.
 * Arguments, outputs and statuses otherwise as msz_correct.  Workspace:
 * msz_relaxed_workspace_size(grid) bytes (msz_workspace_size plus 4 bytes and
 * one bit per vertex).  Synchronizes `stream`. */
#define MSZ_RELAXED_TILE_X 32
#define MSZ_RELAXED_TILE_Y 8
#define MSZ_RELAXED_TILE_Z 8
size_t msz_relaxed_workspace_size(msz_grid grid);
msz_status msz_correct_relaxed(const float *d_f, const float *d_fhat, float xi, msz_grid grid, float *d_out,
                               uint32_t *d_edit_idx, float *d_edit_delta, int64_t edit_capacity,
                               int64_t *h_edit_count, const msz_options *opt, msz_stats *h_stats,
                               void *d_workspace, size_t workspace_bytes, msz_stream_t stream);

/* msz_correct for callers that cannot allocate device memory.  (The paper has
 * no counterpart: this entry point exists for how callers use the library.)
 * Some callers cannot call cudaMalloc -- a plugin whose host application owns
 * every device allocation, code where an allocation would block or synchronize
 * the device, a process that must keep its footprint fixed after start-up --
 * so this variant takes no workspace: its scratch memory is a fixed array of
 * about 8.0 MB compiled into the library, held by every GPU that loads it until
 * the process exits.  Grids of more than MSZ_STATIC_MAX_VERTICES vertices are
 * rejected with MSZ_ERR_WORKSPACE.  Arguments, results and synchronization are
 * those of msz_correct.  Each call looks up the array's device address on the
 * current device (the first call on a device loads the library's module there;
 * make that call before any stream capture).  Every call shares the array:
 * calls that overlap on the GPU race, so serialize them. */
#define MSZ_STATIC_MAX_VERTICES 4194304LL
msz_status msz_correct_static(const float *d_f, const float *d_fhat, float xi, msz_grid grid, float *d_out,
                              uint32_t *d_edit_idx, float *d_edit_delta, int64_t edit_capacity,
                              int64_t *h_edit_count, const msz_options *opt, msz_stats *h_stats,
                              msz_stream_t stream);

/* ---- Edit-list encoding.  The paper stores the corrected field as the
 * decompressed field plus its edits and counts their storage as the method's
 * overhead (Sec. V, computation and storage overhead); it fixes no format.
 * This one is exact and decodes block by block in parallel.
 *
 * An edit is (i, m): a vertex i where g and fhat differ bitwise and its ulp
 * distance m = (ord(fhat_i) - ord(g_i)) mod 2^32, where ord maps a float's
 * bits b to an unsigned key in value order (b | 0x80000000 when the sign bit
 * is clear, ~b when it is set); g_i = ord^-1(ord(fhat_i) - m) bit for bit.
 * Stream (little-endian), B = MSZ_EDIT_BLOCK, nb = ceil(count / B):
 *   u32 MSZ_EDIT_MAGIC, u32 B, u64 count;
 *   nb x u32: the first index of each block;
 *   nb x u32: where each block's payload starts, in 32-bit words from the
 *             start of the payload;
 *   nb x u8 wd (bit width of the block's index gaps), nb x u8 wm (bit width
 *   of its ulp distances minus one); zero bytes up to a multiple of 4;
 *   payload, per block of c edits: d_j (d_0 = 0, d_j = i_j - i_{j-1} - 1)
 *   packed wd bits each, LSB first, into 32-bit words (value j at bit j*wd
 *   of the section), padded to a whole word; then (m_j - 1) mod 2^32 packed
 *   wm bits each the same way.
 * A width is the bit length of its section's largest value (0: no words). */
#define MSZ_EDIT_MAGIC 0x45535A4Du
#define MSZ_EDIT_BLOCK 256

/* Largest stream of `count` edits (bytes): the table plus 8 bytes an edit. */
size_t msz_edits_encoded_bound(int64_t count);
/* Device workspace of msz_edits_encode / msz_edits_decode for `count` edits:
 * 256 bytes plus about 10 bytes a block.  0 when count < 0. */
size_t msz_edits_workspace_size(int64_t count);

/* Encodes the edits at d_idx[0 .. count) (strictly ascending vertex indices
 * below n, as msz_correct lists them) of g = d_g against d_fhat (n floats
 * each) into d_stream (capacity bytes, 4-byte aligned); *h_bytes = the
 * stream's length.  Workspace: msz_edits_workspace_size(count) bytes, 256-byte
 * aligned.  MSZ_ERR_INVALID_ARG: a null pointer, n outside [0,
 * MSZ_MAX_VERTICES], count outside [0, n], a misaligned d_stream, or indices
 * not strictly ascending or not below n (nothing is written to d_stream);
 * MSZ_ERR_CAPACITY: the stream needs more than capacity bytes (*h_bytes =
 * needed; nothing is written); MSZ_ERR_WORKSPACE.  Synchronizes `stream`. */
msz_status msz_edits_encode(const float *d_fhat, const float *d_g, int64_t n, const uint32_t *d_idx, int64_t count,
                            uint8_t *d_stream, size_t capacity, size_t *h_bytes, void *d_workspace,
                            size_t workspace_bytes, msz_stream_t stream);

/* Applies the stream d_stream (bytes long, 4-byte aligned) to d_field (n
 * floats: fhat on entry, g on return); *h_count = its number of edits.
 * Workspace: msz_edits_workspace_size(*h_count) bytes (the count is in bytes
 * 8..15 of the stream).  MSZ_ERR_INVALID_ARG: not a stream of this format,
 * shorter than its table or payload, a width above 32, an index not below n
 * or indices not ascending -- the whole stream is checked before d_field is
 * touched.  Synchronizes `stream`. */
msz_status msz_edits_decode(const uint8_t *d_stream, size_t bytes, float *d_field, int64_t n, int64_t *h_count,
                            void *d_workspace, size_t workspace_bytes, msz_stream_t stream);

/* Human-readable name of a status. */
const char *msz_status_str(msz_status status);

#ifdef __cplusplus
}
#endif

#endif /* MSZ_H */
