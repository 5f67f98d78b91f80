/*
 * dose.h -- C ABI of libdose: the dose-deposition SpMV and its optimisation-step
 * forms on one GB300 (sm_103a).
 *
 * The dose in the patient is one sparse matrix-vector product d = A x, where A
 * is the dose-deposition matrix (rows = voxels, columns = beam spots) and x the
 * spot weights; A is built once and only x changes across the optimiser's
 * iterations (Sec. II-A).  A is stored in CSR with reduced-width values
 * (Sec. II-C, Sec. II-D).  Results are bitwise reproducible for the same
 * handle, inputs and GPU: no reduction anywhere depends on the order in which
 * threads happen to run (Sec. II-D, second requirement).
 *
 * Conventions for every call below
 *   - Plain pointers and sizes only.  "device" pointers are CUDA device memory of
 *     the current device; "host" pointers are CPU memory.
 *   - Compute calls (dose_spmv, dose_spmv_batched, dose_adjoint,
 *     dose_fwd_adj_quadratic, dose_pg_step) are asynchronous on the caller's
 *     cudaStream_t (passed as void*; NULL = legacy default stream).  They never
 *     allocate, never synchronise the host, and may be captured in a CUDA graph.
 *   - Output buffers are caller-owned and fully overwritten.  Inputs are never
 *     modified (except x in dose_pg_step, documented there).
 *   - A matrix handle is library-owned from dose_create_matrix to dose_destroy.
 *     Calls that use the same handle must be ordered on one stream (the handle
 *     owns the scratch of the adjoint reduction).
 *   - Errors: every call returns a dose_status; dose_last_error() gives a
 *     thread-local message for the last failure on the calling thread.  Invalid
 *     arguments are rejected on the host before anything is launched.
 */
#ifndef DOSE_H
#define DOSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dose_matrix dose_matrix; /* opaque, library-owned */

typedef enum {
    DOSE_OK = 0,
    DOSE_ERR_INVALID_ARG = 1, /* bad pointer, size, structure or value */
    DOSE_ERR_OOM = 2,         /* host or device allocation failed (for tests: with
                                 DOSE_TEST_ALLOC_LIMIT=<bytes> in the environment,
                                 every device allocation larger than that fails so) */
    DOSE_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    DOSE_ERR_UNSUPPORTED = 4, /* valid request outside what this build implements */
    DOSE_ERR_TIMEOUT = 5,     /* a kernel's bounded wait ran out (dose_device_status) */
    DOSE_ERR_IO = 6,          /* the autotune cache file could not be read, parsed or written */
    DOSE_ERR_BOUNDS = 7       /* debug-checked build (libdose_debug.so, DOSE_DEBUG_CHECKS): a kernel met an
                                 index outside its buffer and skipped that work (dose_device_status) */
} dose_status;

/* Stored value formats.  The paper stores 16-bit values (Sec. II-D), IEEE half
 * precision in its own kernel (Sec. III, Sec. IV "Half/double"):
 *   U16_SCALE        : uint16 code q, one FP32 scale s per matrix, a = s * q
 *   BF16             : bfloat16 bits, a = value (finite codes only)
 *   FP8E4M3_ROWSCALE : OCP FP8 E4M3 code q, one FP32 scale s_r per row, a = s_r * e4m3(q)
 *   F16              : IEEE 754 binary16 bits, a = value (finite codes only)
 *   F32              : IEEE 754 binary32 bits, a = value (finite only; the paper's "Single"
 *                      configuration, Sec. IV, 8 bytes per entry with 32-bit indices) */
typedef enum {
    DOSE_FMT_U16_SCALE = 0,
    DOSE_FMT_BF16 = 1,
    DOSE_FMT_FP8E4M3_ROWSCALE = 2,
    DOSE_FMT_F16 = 3,
    DOSE_FMT_F32 = 4
} dose_format;

/* A CSR matrix (Sec. II-C: values, column indices, row starts).
 *   nrows, ncols : voxels, spots.  nnz must be < 2^32 (row_ptr is uint32).
 *   row_ptr      : nrows+1 entries, row_ptr[0] = 0, non-decreasing, row_ptr[nrows] = nnz.
 *   col_idx      : nnz entries, each < ncols, unique within a row (any order).
 *   fmt          : stored format of `values`.
 *   values       : nnz encoded values (uint16 for U16/BF16/F16, uint8 for FP8, 32-bit
 *                  for F32), or NULL
 *                  to have the library encode `values_f64`.
 *   scales       : U16: 1 float (s); FP8: nrows floats (s_r); BF16, F16, F32: NULL.  Ignored
 *                  when the library encodes.
 *   values_f64   : nnz non-negative FP64 values, used when values == NULL.
 *   on_device    : 0 = all pointers are host memory; 1 = row_ptr, col_idx, values,
 *                  scales are device memory (values_f64 must then be NULL).
 * The library copies everything it needs; the caller's arrays can be freed after
 * dose_create_matrix returns. */
typedef struct {
    uint32_t nrows;
    uint32_t ncols;
    uint64_t nnz;
    const uint32_t* row_ptr;
    const uint32_t* col_idx;
    dose_format fmt;
    const void* values;
    const float* scales;
    const double* values_f64;
    int on_device;
} dose_csr_desc;

/* dose_create_matrix flags */
#define DOSE_CREATE_COMPENSATED 0x1u /* compensated (TwoSum/TwoProduct) accumulation on rows
                                        longer than 128 entries (with DOSE_CREATE_SELL: in the
                                        chunks whose longest row is longer than 128 entries) */
#define DOSE_CREATE_U16_INDEX 0x2u   /* dose_spmv reads 16-bit column indices: 2 + value bytes per
                                        entry instead of 4 + value bytes (the reduced index width the
                                        paper's Sec. V proposes as future work); needs ncols <= 65536.
                                        The handle keeps a 16-bit copy of the indices beside the
                                        32-bit ones (the other kernels use those): +2 B per entry of
                                        device memory. */
#define DOSE_CREATE_SELL 0x4u        /* dose_spmv runs on a SELL-32-sigma copy of the matrix (the
                                        SIMT-oriented format the paper names as future work, Sec. III):
                                        rows ordered by length inside windows of sigma rows
                                        (dose_tuning.sell_sigma), chunks of 32 rows padded to their longest
                                        row, one row per lane.  The other calls keep using the CSR
                                        arrays; the copy costs its padded size in device memory
                                        (dose_info.sell_entries). */

/* Schedule knobs of a matrix (row-length binning and pipeline shape).  All
 * fields 0 = library default.  Changing them never changes which rows an
 * output depends on; it may change the last bits of FP32 results. */
typedef struct {
    /* forward SpMV (dose_spmv, dose_spmv_batched) */
    uint32_t tile_nnz;       /* max entries staged per pipeline stage (256..16384) */
    uint32_t tile_rows;      /* max rows per stage (32..8192) */
    uint32_t coop_nnz;       /* rows longer than this are reduced by the whole CTA (default: the tile;
                                the adjoint schedule uses at most 1024) */
    uint32_t lane_target;    /* lanes per row = power of two nearest mean row length / lane_target */
    uint32_t stages;         /* pipeline depth (2..8) */
    uint32_t consumer_warps; /* 4, 8 or 16 */
    uint32_t l2_prefetch;    /* stages prefetched into L2 ahead of the shared-memory ring (0..31);
                                set 32 to mean "off" */
    /* adjoint and fused objective pass (dose_adjoint, dose_fwd_adj_quadratic, dose_pg_step) */
    uint32_t adj_tile_nnz;      /* (256..16384) */
    uint32_t adj_tile_rows;     /* (32..8192) */
    uint32_t adj_stages;        /* (2..8) */
    uint32_t adj_forward_warps; /* warps computing d, f, r in the fused pass (1..15) */
    uint32_t adj_scatter_warps; /* warps owning gradient accumulators (0..18): at most this many,
                                   fewer if their accumulators do not fit (0 = as many as fit;
                                   never more than 19 - forward warps) */
    uint32_t adj_l2_prefetch;   /* as l2_prefetch, for these passes (32 = off) */
    /* order of a row block's non-empty rows among the consumer groups */
    uint32_t row_order;         /* forward: 1 = matrix order, 2 = rows with the most 4-entry groups first
                                   (default: the rows one warp reduces together then have similar trip
                                   counts) */
    uint32_t adj_row_order;     /* the same for the adjoint schedule */
    uint32_t sell_sigma;        /* DOSE_CREATE_SELL: rows per sorting window (1 = no sorting;
                                   default 2^20); read at create only */
    /* layout of the adjoint and fused objective passes (read at create; later calls may
       switch between the layouts that were built):
         0 = row groups where they apply (and their arrays fit in device memory), else CSR
             (default);
         1 = CSR (per-row scatter; the row-group layout is not built);
         2 = row groups (create fails with DOSE_ERR_UNSUPPORTED if they do not apply).
       Row groups: up to four consecutive non-empty rows share one list of the union of
       their columns, with the four rows' values stored side by side (stored zeros where
       a row has no entry); built when no row has more than 4096 entries.  The union
       order is chosen per group (shared-memory banks), so these passes sum a row's terms
       in another order than dose_spmv.  A non-finite x_j or residual reaches every row
       of a group whose union holds column j (0 * inf), not only the rows that store j. */
    uint32_t adj_layout;
    uint32_t rg_tile_union;     /* row groups: union columns per pipeline stage (512..8192; default
                                   by format, about 24 KB of columns and values) */
    uint32_t rg_tile_rows;      /* row groups: rows per stage (256..8192) */
    uint32_t rg_stages;         /* row groups: pipeline depth (2..8) */
    uint32_t rg_warps;          /* row groups: worker warps (1..15; 0 = as many as fit) */
    uint32_t rg_l2_prefetch;    /* row groups: stages prefetched into L2 ahead of the ring (1..31;
                                   0 = default, off; 32 = off) */
    uint32_t fwd_layout;        /* layout dose_spmv runs on: 0 = row groups where the handle has them
                                   (and not DOSE_CREATE_COMPENSATED, whose long-row sums run on CSR),
                                   else CSR (default); 1 = CSR; 2 = row groups (create and
                                   dose_set_tuning fail if dose_spmv cannot take them).  On row groups
                                   a row's terms are added in its group's union order (see adj_layout),
                                   so the last bits may differ from the CSR form's.  dose_spmv_f64
                                   takes the row-group form only with fwd_layout = 2 (its arithmetic,
                                   not its bytes, bounds it, and CSR is faster for it). */
} dose_tuning;

typedef struct {
    uint32_t nrows, ncols;
    uint64_t nnz;
    uint32_t fmt, flags;
    uint32_t n_stages;          /* pipeline stages (row blocks) of the forward schedule */
    uint32_t n_coop_rows;       /* rows reduced by a whole CTA */
    uint32_t lanes_hist[6];     /* forward stages per lanes-per-row bin 1,2,4,8,16,32 */
    uint32_t grid, block;       /* launch shape of the forward kernel */
    uint32_t adj_n_stages;      /* stages of the adjoint schedule */
    uint32_t adj_block_fused;   /* threads per CTA of the fused pass (0 if it does not fit) */
    uint32_t adj_block_adjoint; /* threads per CTA of the adjoint (0 if it does not fit) */
    uint32_t max_row_len;
    uint32_t adj_window;        /* columns of each CTA's gradient window in the adjoint schedule */
    uint32_t fwd_window;        /* ncols > 16384: columns of each forward CTA's window of x (staged in
                                   shared memory when it fits beside the ring); else 0 */
    uint64_t device_bytes;      /* device memory held by the handle */
    uint64_t spmv_bytes;        /* algorithmic HBM bytes of one dose_spmv */
    uint64_t adjoint_bytes;     /* ... of one dose_adjoint */
    uint64_t fused_bytes;       /* ... of one dose_fwd_adj_quadratic with d == NULL */
    uint64_t spmv_f64_bytes;    /* ... of one dose_spmv_f64 (x read once, d written once) */
    uint64_t sell_entries;      /* DOSE_CREATE_SELL: stored entries of the SELL copy, padding
                                   included (0 without the flag); spmv_bytes then counts the SELL
                                   arrays */
    float scale;                /* U16: the matrix scale s; else 0 */
    dose_tuning tuning;         /* the knobs in effect */
    uint32_t adj_layout_fused;  /* layout the fused pass runs on: 1 = CSR, 2 = row groups, 0 = none fits */
    uint32_t adj_layout_adjoint;/* ... dose_adjoint */
    uint64_t rg_groups;         /* row groups built (0: the layout was not built) */
    uint64_t rg_union_entries;  /* union columns of all groups (values stored: 4 per union column) */
    uint32_t rg_window;         /* columns of each CTA's gradient window on the row-group layout */
    uint32_t rg_warps_fused;    /* worker warps of the row-group fused pass (0 if it does not fit) */
    uint32_t rg_index_bytes;    /* bytes per union column index (2 when ncols <= 65536, else 4) */
    uint32_t rg_pad;
    uint64_t fingerprint;       /* FNV-1a of the structure (dose_fingerprint_host): the autotune cache key */
    uint32_t spmv_layout;       /* layout dose_spmv runs on: 1 = CSR, 2 = row groups, 3 = SELL */
    uint32_t pad2;
    uint64_t rg_spmv_bytes;     /* algorithmic HBM bytes of one dose_spmv on the row-group layout (0 when
                                   it runs on another layout; spmv_bytes stays the CSR byte model) */
} dose_info;

/* Build a matrix handle: validate the CSR on the host (or on the device for
 * on_device=1, with a synchronising check), encode FP64 values if asked, build
 * the row-binned pipeline schedule, copy everything to the device (enqueued on
 * `stream`, synchronised before return).  flags: DOSE_CREATE_*.  `tuning` may be
 * NULL (defaults).  On success *out is a new handle. */
dose_status dose_create_matrix(const dose_csr_desc* desc, unsigned flags, const dose_tuning* tuning,
                               void* stream, dose_matrix** out);

/* d = A x (Sec. II-A; Sec. III: one output per row, the row's dot product).
 * x: device, ncols floats.  d: device, nrows floats, every row written (empty
 * rows get 0).  FP32 accumulation; U16 and FP8 scales applied once per row.
 * Runs on the row-group layout when the handle has it (dose_tuning.fwd_layout;
 * dose_info.spmv_layout says which form runs), else on the CSR (or SELL)
 * arrays; each form is deterministic, and a row is within 1e-5 relative of the
 * FP64 sum of its terms for rows of up to 4096 entries on either. */
dose_status dose_spmv(const dose_matrix* A, const float* x, float* d, void* stream);

/* dose_spmv_f64 flags */
#define DOSE_SPMV_F64_NATIVE 0x1u /* accumulate with FP64 FMAs (the paper's arithmetic) instead of
                                     double-float FP32 pairs */

/* d = A x with double-precision vectors (Sec. II-D: the optimiser needs the spot
 * weights and the dose in double precision; Sec. IV "Half/double": 16-bit matrix
 * values with double vectors -- DOSE_FMT_F16 is the paper's configuration, any
 * stored format is accepted).
 * x: device, ncols doubles, 8-byte aligned, finite with |x_j| < 3.4e38 (the
 * FP32 range of the split below).  d: device, nrows doubles, 8-byte aligned,
 * every row written (empty rows get +0.0).
 * Arithmetic (flags = 0): x_j is split into FP32 hi + lo (2^-48 relative), each
 * product is formed to ~2^-47 relative with FMAs, and sums are double-float pairs
 * (TwoSum); row results are rounded once to FP64.  A row of n entries then has
 * |d_i - sum_k a_ik x_k| <= (2^-45 + g(m)^2) sum_k |a_ik x_k| + 2^-53 |d_i|, where
 * m <= n is the most terms any one accumulator of the row adds (a handful on the
 * default schedule) and g(m) = m 2^-24 / (1 - m 2^-24).  DOSE_SPMV_F64_NATIVE
 * accumulates with FP64 FMAs: |error| <= (n + 2) 2^-53 sum_k |a_ik x_k|.
 * Uses a handle-owned scratch copy of x (ncols + 1 doubles) and two launches on
 * `stream`; the same-stream rule for calls on one handle applies. */
dose_status dose_spmv_f64(const dose_matrix* A, const double* x, double* d, unsigned flags, void* stream);

/* D_m = A_m X_m for m < count, all in one persistent launch (one dose evaluation
 * of many beams and uncertainty scenarios, Sec. I).  X[m]: device, ncols_m x nvec
 * floats row-major (spot j's nvec weights contiguous).  D[m]: device, nrows_m x
 * nvec floats row-major.  1 <= nvec <= 16; count <= 4096.  The handles must be
 * distinct only in the sense that their outputs must not overlap.  Runs on the
 * row-group layout when every matrix has it (one format, index width and grid;
 * dose_spmv_batched_plan), else on the CSR arrays; deterministic either way. */
dose_status dose_spmv_batched(const dose_matrix* const* A, int count, const float* const* X,
                              float* const* D, int nvec, void* stream);

/* The form dose_spmv_batched takes for these matrices, without launching
 * anything: *layout = 2 when every matrix is run on its row-group layout (one
 * launch per 32 matrices), 1 for
 * the CSR forms (one launch per 64 matrices), 0 for count = 0; *launches = the
 * kernels one call launches.  Host only; the same arguments as dose_spmv_batched
 * (layout and launches must not be NULL; nvec in [1, 16]). */
dose_status dose_spmv_batched_plan(const dose_matrix* const* A, int count, int nvec, int* layout, int* launches);

/* g = A^T r, the adjoint (gradient of any dose objective with dD/dd = r).
 * r: device, nrows floats, 16-byte aligned.  g: device, ncols floats.  Deterministic: per-warp
 * private accumulators combined in a fixed order, no atomics on values.  Runs on the
 * row-group layout when the handle has it (dose_tuning.adj_layout), else on the CSR arrays. */
dose_status dose_adjoint(const dose_matrix* A, const float* r, float* g, void* stream);

/* One pass over A of the quadratic dose objective
 *   d = A x,  f = sum_i w_i (d_i - p_i)^2 (FP64),  g = A^T [2 w (d - p)]
 * x: device ncols floats; p, w: device nrows floats, 16-byte aligned; d: device nrows floats or
 * NULL (not written); f: device, one double; g: device ncols floats. */
dose_status dose_fwd_adj_quadratic(const dose_matrix* A, const float* x, const float* p,
                                   const float* w, float* d, double* f, float* g, void* stream);

/* One projected-gradient step of the quadratic objective:
 *   f = f(x), g = grad f(x), then x <- max(0, x - eta g)   (x updated in place)
 * f: device double (f before the step), g: device floats or NULL. */
dose_status dose_pg_step(const dose_matrix* A, float* x, const float* p, const float* w, float eta,
                         double* f, float* g, void* stream);

/* g = A^T r without any device allocation -- for callers that cannot call
 * cudaMalloc (device memory owned by another runtime or a fixed arena,
 * allocation forbidden after start-up, or a frozen capture memory plan); such
 * callers cannot create a handle, so A is passed as device CSR arrays.  The
 * paper has no counterpart: this is a deployment variant of dose_adjoint.
 *   row_ptr (nrows+1), col_idx (nnz), values (nnz, fmt-encoded): device memory,
 *   a valid CSR (rows whose pointers run backwards or past nnz, and columns
 *   >= ncols, are skipped, never read or written out of bounds).  The columns
 *   of a row must be distinct: nothing checks it on the device, and a row that
 *   repeats a column makes two lanes update one accumulator word in the same
 *   instruction, so one of the two updates is lost and g is wrong and may
 *   differ from run to run (dose_create_matrix rejects such rows);
 *   row_scales: FP8 only, device nrows floats; scale: U16 matrix scale;
 *   r: device nrows floats; g: device ncols floats (written).
 * Scratch is a 4 MiB static __device__ array that every GPU loading the
 * library holds until exit; all calls on a device share it, so calls that
 * overlap on the GPU race -- order them.  The first call on a device looks up
 * the array's address; make it before any stream capture.  That address is
 * kept for the life of the process: it assumes the device's primary context
 * lives as long (after cudaDeviceReset, or anything else that tears the context
 * down, this entry point must not be called again in the same process).
 * ncols beyond the scratch (2^20 floats) or beyond one shared-memory
 * accumulator is rejected with DOSE_ERR_INVALID_ARG.  Deterministic,
 * asynchronous on `stream`. */
dose_status dose_adjoint_noalloc(uint32_t nrows, uint32_t ncols, uint64_t nnz, const uint32_t* row_ptr,
                                 const uint32_t* col_idx, dose_format fmt, const void* values,
                                 const float* row_scales, float scale, const float* r, float* g,
                                 void* stream);

/* A plan of several beams on one voxel grid (Sec. I: the dose of a plan comes from
 * multiple beams): one handle whose columns are the beams' spots in beam order, so
 * that with x = [x_1; ...; x_B] every call above computes the plan's total dose
 * d = sum_b A_b x_b (and A^T r gives every beam's gradient).  beams: nbeams (1..64)
 * host CSR descriptors (on_device = 0) with the same nrows and format; either all
 * give values_f64 (encoded once, after merging) or all give codes (BF16, F16,
 * F32; U16 only if every beam has the same scale; not FP8, whose row scales
 * would differ within a merged row).  flags, tuning, stream: as for
 * dose_create_matrix, which validates the merged matrix. */
dose_status dose_create_multibeam(const dose_csr_desc* beams, int nbeams, unsigned flags, const dose_tuning* tuning,
                                  void* stream, dose_matrix** out);

/* Robust optimisation over uncertainty scenarios (Sec. I: doses under several
 * realisations of the uncertainties in every iteration).  A scenario set groups
 * count (1..64) matrices of one shape -- the same plan under different setup
 * shifts -- with probabilities prob (host, count values >= 0 summing to 1; NULL =
 * uniform).  The set owns scratch of count x ncols floats; the matrices must
 * outlive it; calls on one set must be ordered on one stream.  Objective of the
 * quadratic dose term f_s(x) = sum_i w_i ((A_s x)_i - p_i)^2 of each scenario:
 *   DOSE_ROBUST_EXPECTED:   F = sum_s prob_s f_s,  g = sum_s prob_s grad f_s
 *   DOSE_ROBUST_WORST_CASE: F = max_s f_s, g = grad f_s* for the first s* with the
 *                           largest f_s (a subgradient of the maximum); a NaN f_s
 *                           counts as the largest, so a diverged scenario shows in F. */
typedef struct dose_scenarios dose_scenarios; /* opaque, library-owned */
#define DOSE_ROBUST_EXPECTED 0
#define DOSE_ROBUST_WORST_CASE 1
dose_status dose_create_scenarios(const dose_matrix* const* A, int count, const double* prob, dose_scenarios** out);
dose_status dose_destroy_scenarios(dose_scenarios* S); /* synchronises the device; NULL -> DOSE_OK */

/* F and g of the robust objective: one fused pass per scenario (as
 * dose_fwd_adj_quadratic) and one combine kernel, sums in scenario order.
 * x: device ncols floats; p, w: device nrows floats, 16-byte aligned; f: device
 * double; f_scen: device count doubles (each f_s) or NULL; g: device ncols floats. */
dose_status dose_robust_quadratic(const dose_scenarios* S, int mode, const float* x, const float* p, const float* w,
                                  double* f, double* f_scen, float* g, void* stream);

/* One projected-gradient step of the robust objective: F and g at x, then
 * x <- max(0, x - eta g) in place.  g may be NULL. */
dose_status dose_robust_pg_step(const dose_scenarios* S, int mode, float* x, const float* p, const float* w,
                                float eta, double* f, float* g, void* stream);

/* Free the handle and its device memory (synchronises the device first).  NULL -> DOSE_OK. */
dose_status dose_destroy(dose_matrix* A);

/* Describe a handle (sizes, schedule, algorithmic bytes of each call). */
dose_status dose_matrix_info(const dose_matrix* A, dose_info* out);

/* Re-schedule a handle with new knobs (synchronous; not during capture). */
dose_status dose_set_tuning(dose_matrix* A, const dose_tuning* tuning);

/* Autotuner (the execution-configuration sweep of Sec. V-A, Fig. 4, for this
 * library's knobs).  Purposes: which calls the knobs are chosen for. */
#define DOSE_TUNE_FORWARD 1u /* dose_spmv: stage tiles, lanes-per-row target, pipeline depth */
#define DOSE_TUNE_FUSED 2u   /* dose_fwd_adj_quadratic / dose_pg_step with p = w = 1: adjoint layout
                                (row groups or CSR) and its tiles and warps */
#define DOSE_TUNE_BATCHED 4u /* dose_spmv_batched of this matrix with 16 vectors (same knobs as
                                DOSE_TUNE_FUSED; with both, their summed time is minimised) */
enum {
    DOSE_AUTOTUNE_ENV = -1,   /* read $DOSE_AUTOTUNE: off | cached | full (unset: off) */
    DOSE_AUTOTUNE_OFF = 0,    /* change nothing */
    DOSE_AUTOTUNE_CACHED = 1, /* apply the cache's knobs for this matrix and GPU; on a miss, sweep and store */
    DOSE_AUTOTUNE_FULL = 2    /* sweep and store (replacing the entry) */
};
typedef struct {
    int32_t source;       /* 0 = nothing done (off), 1 = knobs from the cache, 2 = swept (and stored) */
    uint32_t purposes;    /* the purposes the knobs were chosen for */
    uint64_t fingerprint; /* the matrix's cache key (dose_info.fingerprint) */
    double ms[3];         /* times of dose_spmv, the fused pass, the 16-vector batched call with
                             the chosen knobs (0 = not a purpose; from the sweep that chose them) */
} dose_autotune_report;

/* Time candidate schedules of dose_spmv and of the fused objective pass on this
 * GPU with x (device, ncols floats; NULL = all ones) and keep the fastest; the
 * chosen knobs are returned in *best (may be NULL).  No cache.  Synchronous;
 * uses `stream`; not during capture. */
dose_status dose_autotune(dose_matrix* A, const float* x, void* stream, dose_tuning* best);

/* The autotuner with its cache.  The cache is a JSON file (format
 * "dose-autotune-1": a list of entries, each the GPU name as dose_gpu_name gives
 * it, the matrix fingerprint in 16 hex digits, the purposes, every dose_tuning
 * field by name and the sweep's times).  path: the file; NULL = $DOSE_AUTOTUNE_CACHE,
 * else $XDG_CACHE_HOME/dose/autotune.json, else $HOME/.cache/dose/autotune.json.
 * mode: DOSE_AUTOTUNE_*.  purposes: DOSE_TUNE_* (0 = FORWARD | FUSED).  A hit
 * applies the entry with dose_set_tuning; a miss (or mode FULL) sweeps, applies
 * the fastest knobs and rewrites the file (a temporary file renamed over it; a
 * concurrent writer's entry may be lost, never half written).  A file that is
 * not such a cache is refused (DOSE_ERR_IO), not overwritten; if the write
 * fails the swept knobs stay applied.  x as for dose_autotune.  Synchronous.
 * With DOSE_AUTOTUNE=cached|full in the environment, dose_create_matrix calls
 * this (x = NULL, purposes 0, path NULL) on handles created with tuning = NULL. */
dose_status dose_autotune_cached(dose_matrix* A, const float* x, int mode, unsigned purposes, const char* path,
                                 void* stream, dose_tuning* best, dose_autotune_report* report);

/* Host only.  The fingerprint dose_create_matrix gives this CSR with these
 * creation flags (host arrays; the values do not enter). */
dose_status dose_fingerprint_host(const dose_csr_desc* desc, unsigned flags, uint64_t* out);

/* Host only.  Read or write one entry of a cache file (key: gpu, fingerprint,
 * purposes).  lookup: *found = 1 and *out, ms[3] (each may be NULL) when the
 * entry exists, *found = 0 otherwise or when the file does not exist.  store:
 * adds or replaces the entry (ms may be NULL). */
dose_status dose_autotune_cache_lookup(const char* path, const char* gpu, uint64_t fingerprint, unsigned purposes,
                                       dose_tuning* out, double* ms, int* found);
dose_status dose_autotune_cache_store(const char* path, const char* gpu, uint64_t fingerprint, unsigned purposes,
                                      const dose_tuning* tuning, const double* ms);

/* The GPU name the cache keys on ("<name> (<SMs> SMs, sm_<cc>)") for a CUDA
 * device, written to buf (len bytes, truncated); returns buf, or NULL if buf is NULL. */
const char* dose_gpu_name(int device, char* buf, int len);

/* Host-only encoder of the library's stored formats (no GPU needed):
 * values_f64 (nnz, non-negative) -> codes (uint16, uint8 or 32-bit, nnz) and scales
 * (U16: 1 float; FP8: nrows floats; BF16, F16, F32: untouched, may be NULL; F16 rounds
 * to nearest, ties to even, and gives infinity above the half range).  Uses
 * row_ptr (host, nrows+1) for FP8 row scales. */
dose_status dose_encode_host(dose_format fmt, uint32_t nrows, const uint32_t* row_ptr,
                             uint64_t nnz, const double* values_f64, void* codes, float* scales);

/* Synchronise `stream` and report a kernel-side failure recorded on the
 * handle since the last call (DOSE_ERR_TIMEOUT if a bounded wait ran out;
 * DOSE_ERR_BOUNDS in the debug-checked build if a row-group kernel met a group
 * record or union column outside its stage, window or matrix and skipped that
 * group), then clear it.  The debug-checked build is libdose_debug.so, compiled
 * with DOSE_DEBUG_CHECKS; its results are bitwise those of the release build
 * when nothing is out of bounds. */
dose_status dose_device_status(const dose_matrix* A, void* stream);

/* Self-test of the bounded waits that guard every pipelined kernel: one GPU
 * thread waits on an mbarrier phase that never completes and gives up after
 * limit_us microseconds (1..1e6), as the kernels' ring waits do after ~4 s.
 * Returns DOSE_ERR_TIMEOUT when the wait ran out as designed (the expected
 * result; the CUDA context stays usable), DOSE_OK if the wait did not run out
 * (the self-test failed), DOSE_ERR_CUDA on a CUDA error.  Synchronises
 * `stream`. */
dose_status dose_selftest_bounded_wait(uint32_t limit_us, void* stream);

/* Message of the last failure on this thread ("" if none). */
const char* dose_last_error(void);

/* Library version string. */
const char* dose_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DOSE_H */
