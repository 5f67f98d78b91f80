// Internal definitions shared by the library's translation units: the matrix
// handle, the pipeline schedule, and sm_100-family device helpers (mbarrier,
// bulk async copies, bounded waits, value decoders).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dose.h"

namespace dose {

// ------------------------------------------------------------ schedule
//
// The matrix rows are cut into pipeline stages ("row blocks"), each staged in
// shared memory by bulk async copies:
//   NORMAL stage: consecutive rows [row0, row1), at most tile_rows rows and
//                 tile_nnz entries, none longer than coop_nnz.  Its non-empty
//                 rows are listed (u16 offsets from row0, ne list) so that every
//                 consumer warp gets an even share of them; they are reduced by
//                 groups of L = 2^lanes_log2 lanes, L chosen per stage from the
//                 stage's mean row length (row-length binning).  Empty rows get 0.
//   COOP stage:   one chunk (<= tile_nnz entries) of one row longer than
//                 coop_nnz; all consumer warps reduce it together.  A row of
//                 several chunks occupies consecutive stages FIRST..LAST.
// Work items (a NORMAL stage, or all chunks of one long row) are assigned to
// CTAs statically, so every reduction order is fixed at create time:
//   forward schedule: dealt round-robin in matrix order, so every CTA gets a
//                     similar mix of empty and dense row blocks;
//   adjoint schedule: sorted by their lowest column, cut into a few groups of
//                     equal estimated cost, each dealt round-robin to its own
//                     share of the CTAs.  Each CTA then touches a narrow column
//                     window [wlo, wlo + wwidth) (a pencil beam's row block sees
//                     only the spots near its voxels), so its per-warp gradient
//                     accumulators and its copy of x hold wwidth columns instead
//                     of ncols, and more warps fit.
enum : uint32_t {
    STAGE_LANES_MASK = 0x7u,  // log2 of lanes per row (0..5)
    STAGE_COOP = 0x8u,
    STAGE_FIRST = 0x10u,
    STAGE_LAST = 0x20u,
};

// One stage, as stored on the device (32 bytes, two 16-byte loads).
struct StageDesc {
    uint32_t row0, row1;  // rows [row0, row1) (COOP: row1 = row0 + 1)
    uint32_t nz0, nz1;    // entries [nz0, nz1) of this stage
    uint32_t ne0, ne1;    // its slice of the non-empty-row list
    uint32_t meta;        // STAGE_* bits
    uint32_t pad;
};

struct Tuning {
    uint32_t tile_nnz = 8192;
    uint32_t tile_rows = 2048;
    uint32_t coop_nnz = 8192;   // rows longer than this (longer than a tile) are reduced by the whole CTA
    uint32_t lane_target = 24;  // entries per lane: 4 per unrolled step, about 6 steps
    uint32_t stages = 3;
    uint32_t consumer_warps = 16;
    uint32_t l2_prefetch = 2;   // stages prefetched into L2 ahead of the shared-memory ring
    uint32_t row_order = 2;     // non-empty rows of a stage: 1 = matrix order, 2 = most 4-entry groups first
    uint32_t layout = 0;        // dose_spmv: 0 = row groups where built, 1 = CSR, 2 = row groups
};

// SELL-32-sigma copy of a matrix for the forward SpMV (DOSE_CREATE_SELL).
struct SellArrays {
    void* val = nullptr;      // stored values in SELL order
    void* col = nullptr;      // column indices (4 or 2 bytes) in SELL order
    uint2* chunk = nullptr;   // per chunk: first entry / 128, groups of four entries
    uint32_t* perm = nullptr; // original row of each chunk slot (~0: none)
    uint32_t nchunks = 0, sigma = 0;
    uint64_t entries = 0;     // stored entries including padding
    uint64_t bytes = 0;       // device bytes of the arrays above
};

struct Schedule {
    std::vector<StageDesc> desc;      // n_stages, stored CTA by CTA
    std::vector<uint16_t> ne;         // non-empty rows of NORMAL stages (offset from row0)
    std::vector<uint32_t> cta_begin;  // grid + 1: CTA c runs desc[cta_begin[c] .. cta_begin[c+1])
    std::vector<uint32_t> wlo;        // grid: first column of each CTA's window (adjoint schedule)
    uint32_t wwidth = 0;              // window width in columns, a multiple of 32
    uint32_t n_coop_rows = 0;
    uint32_t lanes_hist[6] = {0, 0, 0, 0, 0, 0};
};

// Device copy of a schedule.
struct DevSchedule {
    StageDesc* desc = nullptr;
    uint16_t* ne = nullptr;
    uint32_t* cta_begin = nullptr;
    uint32_t* wlo = nullptr;
    uint32_t wwidth = 0;
    uint32_t n_stages = 0;
    uint32_t grid = 0;
    uint32_t n_coop_rows = 0;
    uint32_t lanes_hist[6] = {0, 0, 0, 0, 0, 0};
    Tuning tuning;
};

// Kernel-side view of a schedule, passed by value.
struct ScheduleView {
    const StageDesc* desc;
    const uint16_t* ne;
    const uint32_t* cta_begin;
    const uint32_t* wlo;  // adjoint schedule only (else null)
};

// A work item for dealing stages to CTAs: descriptors [s, e), the columns its
// entries touch [lo, hi] (lo > hi: none) and its estimated cost.
struct DealItem {
    uint32_t s, e;
    uint32_t lo, hi;
    uint64_t cost;
};

// Row-group layout of a matrix, built at create for the adjoint and the fused
// objective pass.  The non-empty rows, in matrix order, are cut into groups of
// up to four consecutive ones whose columns mostly coincide (neighbouring voxels
// see the same spots).  A group stores the union of its rows' columns once and,
// for each union column, the four rows' stored values side by side (the stored
// zero where a row has no entry).  One warp then takes a whole group: per union
// column one gather of x feeds four rows' dot products, and after the four
// residuals are known one read-modify-write of the gradient accumulator adds
// all four rows' contributions.
//   stage (StageDesc reused): rows [row0, row1), union entries [nz0, nz1),
//   groups [ne0, ne1); meta unused.
//   group record (uint4): x = first union entry, y = union size, z / w = the
//   rows' offsets from the stage's row0 as u16 pairs (0xFFFF: no row).
struct RgHostGroup {
    uint32_t row[4];   // absolute rows (~0u: none)
    uint32_t uoff, nu; // union entries [uoff, uoff + nu)
    uint32_t lo, hi;   // lowest / highest union column
};

struct RowGroups {
    bool built = false;
    uint32_t iw = 4;                // bytes per union column index (2 when ncols <= 65536)
    uint64_t n_union = 0;           // union entries of all groups
    void* ucol = nullptr;           // union column indices
    void* uval = nullptr;           // four stored values per union entry
    uint4* grp = nullptr;           // group records (depend on the stage cut)
    uint32_t* mask = nullptr;       // one bit per row: the row has entries
    double* f_rows = nullptr;       // objective sums of the finalize's row blocks
    uint32_t* ticket = nullptr;     // finalize: row blocks done (reset by the last one)
    uint32_t nblk_rows = 0;         // finalize row blocks (256 rows per warp, 8 warps)
    DevSchedule sched;              // stages of groups, dealt to CTAs with column windows
    uint32_t tile_u = 0, tile_g = 0, tile_rows = 0;  // stage limits of the schedule in effect
    uint64_t bytes = 0;             // device bytes of the arrays above
    std::vector<RgHostGroup> host; // kept for re-cutting the stages
};

// Shape of the adjoint / fused kernels (warp specialisation and pipeline).
struct AdjTuning {
    uint32_t tile_nnz = 5120;
    uint32_t tile_rows = 1024;
    uint32_t stages = 3;
    uint32_t forward_warps = 8;   // fused pass: warps computing d, f and r
    uint32_t scatter_warps = 0;   // warps owning gradient accumulators (0 = as many as fit, up to the cap)
    uint32_t l2_prefetch = 8;     // stages prefetched into L2 ahead of the shared-memory ring
    uint32_t row_order = 2;       // as Tuning::row_order, for the adjoint schedule
    // layout of the adjoint / fused passes: 0 = row groups where they apply, else
    // CSR; 1 = CSR; 2 = row groups (create fails if they do not apply)
    uint32_t layout = 0;
    uint32_t rg_tile_u = 0;        // row groups: union entries per stage (0 = by format)
    uint32_t rg_tile_rows = 512;   // row groups: rows a stage may span
    uint32_t rg_stages = 2;        // row groups: pipeline depth
    uint32_t rg_warps = 0;         // row groups: worker warps (0 = as many as fit, up to kRgMaxWarps)
    uint32_t rg_l2_prefetch = 0;   // row groups: stages prefetched into L2 ahead of the ring (0 = off)
};

}  // namespace dose

struct dose_matrix {
    uint32_t nrows = 0, ncols = 0;
    uint64_t nnz = 0;
    dose_format fmt = DOSE_FMT_U16_SCALE;
    unsigned flags = 0;
    int device = 0;
    int sm_count = 0;
    uint32_t max_row_len = 0;
    float scale = 1.0f;  // U16 matrix scale

    // matrix arrays (device, padded so aligned bulk copies stay in bounds)
    uint32_t* row_ptr = nullptr;
    uint32_t* col = nullptr;
    uint16_t* col16 = nullptr;   // DOSE_CREATE_U16_INDEX: 16-bit copy of col for the forward SpMV
    void* val = nullptr;
    float* row_scale = nullptr;  // FP8 only

    dose::DevSchedule fwd;      // schedule of dose_spmv (and the batched SpMM)
    bool fwd_windowed = false;  // ncols too many for all of x in shared memory: the forward schedule
                                // has column windows and the kernels stage each CTA's window
    dose::DevSchedule fwd64;    // dose_spmv_f64's own schedule when its 8-byte window of x would not
    bool fwd64_own = false;     // fit (x then comes from L2 and full tiles pay more than windows)
    dose::DevSchedule adj;      // schedule of the adjoint / fused kernels
    dose::AdjTuning adj_tuning;

    // dose_spmv_f64 scratch: x as the kernel reads it (ncols + 1 elements of 8 bytes)
    uint2* x64 = nullptr;

    dose::SellArrays sell;  // DOSE_CREATE_SELL only

    dose::RowGroups rg;     // row-group layout of the adjoint / fused passes (when it applies)

    // adjoint scratch: per-CTA partial gradients and objective values
    float* g_part = nullptr;     // adj.grid * ncols
    double* f_part = nullptr;    // adj.grid

    int* err = nullptr;  // device error word (0 = ok)
    uint64_t device_bytes = 0;
    uint64_t fingerprint = 0;  // of the structure (autotune cache key; autotune.cu)
    std::vector<uint32_t> host_row_ptr;  // kept for re-scheduling
    std::vector<uint32_t> host_row_cmin;  // lowest / highest column of each row (empty rows:
    std::vector<uint32_t> host_row_cmax;  // cmin > cmax), for the adjoint's column windows
};

namespace dose {

// Host helpers (dose_api.cu)
void set_error(const std::string& msg);
dose_status cuda_fail(cudaError_t e, const char* what);
// Every device allocation of the library goes through here.  A test hook:
// with DOSE_TEST_ALLOC_LIMIT=<bytes> in the environment, a request for more
// than that many bytes fails as out of memory without reaching the driver, so
// the out-of-memory paths run without exhausting the device.
cudaError_t dev_malloc(void** p, size_t bytes);
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void**>(p), bytes);
}

// Launchers (spmv_kernel.cu, spmv_f64_kernel.cu, adjoint_kernel.cu, batched_kernel.cu)
size_t spmv_smem_bytes(const dose_matrix* A, const Tuning& t, bool x_in_smem);
// Columns of x a forward CTA stages (all of x, or the schedule's window width).
uint32_t spmv_x_cols(const dose_matrix* A);
// Whether the forward kernel can stage its x (or window of x) beside the ring of tuning t.
bool spmv_x_in_smem(const dose_matrix* A, const Tuning& t);
cudaError_t launch_spmv(const dose_matrix* A, const float* x, float* d, cudaStream_t s);
size_t spmv_f64_smem_bytes(const dose_matrix* A, bool x_in_smem);
// SELL-32-sigma (sell_kernel.cu): build from host CSR columns and encoded values, free, launch.
cudaError_t build_sell(dose_matrix* A, const std::vector<uint32_t>& col, const unsigned char* vals, uint32_t sigma,
                       std::string* why);
void free_sell(dose_matrix* A);
cudaError_t launch_spmv_sell(const dose_matrix* A, const float* x, float* d, cudaStream_t s);
bool spmv_f64_x_in_smem(const dose_matrix* A);
cudaError_t launch_spmv_f64(const dose_matrix* A, const double* x, double* d, bool native, cudaStream_t s);
// Adjoint shape that fits in shared memory: fills forward/scatter warp counts; false if none.
bool adjoint_shape(const dose_matrix* A, const AdjTuning& in, bool quad, AdjTuning* out, size_t* smem);
cudaError_t launch_adjoint(const dose_matrix* A, int mode, const float* x, const float* p,
                           const float* w, const float* r, float* d, double* f, float* g,
                           float* x_update, float eta, cudaStream_t s);
// Whether the adjoint / fused kernels can run on A (window and accumulators fit;
// per-row vectors 16-byte aligned); sets the error message if not.
dose_status adjoint_supported(const dose_matrix* A, bool quad, const float* const* vecs, int nvec);
// Row-group layout (rg_layout.cu, rg_kernel.cu).  build_row_groups forms the
// groups from the host CSR and the stored values; false (with *why) if some row
// does not fit one stage.  rg_schedule cuts the stages and deals them
// (re-run when the tuning changes).
bool build_row_groups(dose_matrix* A, const uint32_t* rp, const uint32_t* col, const unsigned char* vals,
                      std::string* why, cudaError_t* err);
cudaError_t rg_schedule(dose_matrix* A, const AdjTuning& t);
void free_row_groups(dose_matrix* A);
// Worker warps that fit for tuning t (0: none); *smem the dynamic shared memory.
uint32_t rg_shape(const dose_matrix* A, const AdjTuning& t, bool quad, size_t* smem);
// Whether the adjoint (quad = false) / fused pass of A runs on the row-group layout.
bool rg_active(const dose_matrix* A, bool quad);
cudaError_t launch_rg(const dose_matrix* A, int mode, const float* x, const float* p, const float* w,
                      const float* r, float* d, double* f, float* g, float* x_update, float eta, cudaStream_t s);
uint64_t rg_fused_bytes(const dose_matrix* A, bool with_d);
// Batched SpMM on the row-group layout (rg_spmm.cu): whether it applies to the
// matrices A[0 .. count) (count <= kRgSpmmMaxPerLaunch), and the launches.
constexpr uint32_t kRgSpmmMaxPerLaunch = 32;
bool rg_spmm_applies(const dose_matrix* const* A, int count, size_t* smem, uint32_t* depth);
// d = A x on the row-group layout (rg_spmm.cu): whether it fits, and the launch.
bool rg_spmv_applies(const dose_matrix* A, size_t* smem, uint32_t* depth);
// dose_spmv_f64 on the row-group layout (rg_spmm.cu): x64 is the handle's
// prepared x (ncols + 1 elements of 8 bytes, the last one zero).
bool rg_spmv64_applies(const dose_matrix* A, size_t* smem, uint32_t* depth);
cudaError_t launch_rg_spmv64(const dose_matrix* A, const void* x64, double* d, bool native, cudaStream_t s);
// Whether dose_spmv takes the row-group form for this handle (dose_api.cu).
bool spmv_on_row_groups(const dose_matrix* A);
cudaError_t launch_rg_spmv(const dose_matrix* A, const float* x, float* d, cudaStream_t s);
// Which form dose_spmv_batched takes for these matrices (2 row groups, 1 CSR)
// and how many kernels one call launches.
void spmm_batched_plan(const dose_matrix* const* A, int count, int* layout, int* launches);
cudaError_t launch_rg_spmm(const dose_matrix* const* A, int count, const float* const* X, float* const* D, int nvec,
                           cudaStream_t s);
uint64_t rg_adjoint_bytes(const dose_matrix* A);
uint64_t rg_spmv_bytes(const dose_matrix* A);
// Sum of the per-CTA partials (g, f) in a fixed order; optional projected-gradient step.
cudaError_t launch_adjoint_finalize(const dose_matrix* A, const float* g_part, const uint32_t* wlo, uint32_t wwidth,
                                    uint32_t nparts, bool quad, float* g, double* f, float* x_update, float eta,
                                    cudaStream_t s);
void deal_items(Schedule& S, const std::vector<DealItem>& items, uint32_t grid, uint32_t ncols, bool windowed,
                bool align_wlo);

cudaError_t launch_spmm_batched(const dose_matrix* const* A, int count, const float* const* X,
                                float* const* D, int nvec, cudaStream_t s, std::string* why);

// Knobs and schedules (dose_api.cu): range checks, the merge of a caller's
// dose_tuning into the internal knobs and back, and the re-cut of a schedule.
dose_status check_tuning(const dose_matrix* A, Tuning& t);
dose_status check_adj_tuning(const AdjTuning& t);
void merge_tuning(Tuning& t, AdjTuning& a, const dose_tuning* in);
void export_tuning(const Tuning& t, const AdjTuning& a, dose_tuning* out);
dose_status apply_schedule(dose_matrix* A, DevSchedule& D, const Tuning& t, bool windowed = false);
Tuning adj_schedule_tuning(const Tuning& fwd, const AdjTuning& a);
// FNV-1a of the matrix's shape, format, creation flags, row pointers and the
// column extent of each non-empty row (autotune.cu).
uint64_t matrix_fingerprint(const dose_matrix* A);

constexpr uint32_t kMaxSmemPerBlock = 227 * 1024;

// Stored bytes per value of a format.
__host__ __device__ constexpr uint32_t value_bytes(int fmt) {
    return fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1u : (fmt == DOSE_FMT_F32 ? 4u : 2u);
}
// Worker warps of the row-group kernel (plus one producer): 16 warps in all, so
// that each of the SM's four register files holds four warps of up to 128 registers.
constexpr uint32_t kRgMaxWarps = 15;
constexpr uint32_t kRgMaxUnionReg = 320;  // union columns a group may hold to stay in registers
constexpr uint32_t kMaxAdjWarps = 20;      // producer + forward + scatter warps of the adjoint kernels
constexpr uint32_t kSellDefaultSigma = 1u << 20;  // rows per sorting window of the SELL copy
constexpr uint32_t kAdjMinScatterWarps = 8;
constexpr uint32_t kAdjCoopNnz = 1024;  // the adjoint schedule reduces rows longer than this with the whole CTA  // below this the default adjoint tile shrinks to 4096 entries
constexpr uint32_t kAdjColumnGroups = 16;  // column groups of the adjoint schedule (CTAs per group: grid / 16)
constexpr uint32_t kXSmemMaxCols = 16384;  // x staged in shared memory up to 64 KB
constexpr uint32_t kCompThreshold = 128;   // compensated accumulation above this row length
constexpr int ADJ_MODE_ADJOINT = 0;   // g = A^T r
constexpr int ADJ_MODE_QUADRATIC = 1; // d, f, g of the quadratic objective

// Error codes written into the device error word.
constexpr int kErrTimeoutFull = 1;
constexpr int kErrTimeoutEmpty = 2;
constexpr int kErrBounds = 3;  // debug-checked build: an index outside its buffer (the work was skipped)

}  // namespace dose

// ------------------------------------------------------------------ device
#ifdef __CUDACC__
namespace dose {
namespace dev {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// try_wait with a suspend-time hint: the thread sleeps (issuing nothing) until
// the phase completes or about `ns` nanoseconds pass.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete, giving up after limit_ns of wall
// time.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        for (int i = 0; i < 16; ++i)
            if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// The waits of the pipelined kernels: ~4 s (the kernels run for milliseconds).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    return mbar_wait_limit(bar, parity, 4000000000ull);
}

// The same bound with plain try_wait polls (each poll blocks for a short,
// hardware-chosen time and returns as soon as the phase completes); the
// global timer is read once per 64 polls.
__device__ __forceinline__ bool mbar_wait_poll(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > 4000000000ull) return false;
    }
}

// Bulk async copy global -> shared (no tensor map), completion counted on `bar`.
// dst, src 16-byte aligned; bytes a non-zero multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Explicit shared-memory accesses on 32-bit shared addresses (the staged data
// is written by the async proxy between mbarrier waits, so these are volatile:
// never moved across a wait).
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u8(uint32_t a) {
    uint16_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_f32(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// Predicated forms: access only when k < ke (no branch); loads give 0 otherwise.
__device__ __forceinline__ uint32_t lds_u32_lt(uint32_t k, uint32_t ke, uint32_t a) {
    uint32_t v = 0;
    asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %1, %2;\n\t@q ld.shared.u32 %0, [%3];\n\t}"
                 : "+r"(v) : "r"(k), "r"(ke), "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u16_lt(uint32_t k, uint32_t ke, uint32_t a) {
    uint16_t v = 0;
    asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %1, %2;\n\t@q ld.shared.u16 %0, [%3];\n\t}"
                 : "+h"(v) : "r"(k), "r"(ke), "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u8_lt(uint32_t k, uint32_t ke, uint32_t a) {
    uint16_t v = 0;
    asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %1, %2;\n\t@q ld.shared.u8 %0, [%3];\n\t}"
                 : "+h"(v) : "r"(k), "r"(ke), "r"(a));
    return v;
}
__device__ __forceinline__ float lds_f32_lt(uint32_t k, uint32_t ke, uint32_t a) {
    float v = 0.f;
    asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %1, %2;\n\t@q ld.shared.f32 %0, [%3];\n\t}"
                 : "+f"(v) : "r"(k), "r"(ke), "r"(a));
    return v;
}
// Predicated on a boolean: load only when p (0 otherwise) / store only when p.
__device__ __forceinline__ float lds_f32_if(bool p, uint32_t a) {
    float v = 0.f;
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t@q ld.shared.f32 %0, [%2];\n\t}"
                 : "+f"(v) : "r"((uint32_t)p), "r"(a));
    return v;
}
__device__ __forceinline__ void sts_f32_if(bool p, uint32_t a, float v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.shared.f32 [%1], %2;\n\t}"
                 ::"r"((uint32_t)p), "r"(a), "f"(v) : "memory");
}
// Vector loads (a 16- resp. 8- resp. 4-byte aligned), only when p; zeros otherwise.
// Index check of the debug-checked build (DOSE_DEBUG_CHECKS): records
// kErrBounds in the error word (the first failure wins) and returns whether
// the work may go ahead.  Release builds compile it to `true`.
__device__ __forceinline__ bool in_bounds(bool ok, int* err) {
#ifdef DOSE_DEBUG_CHECKS
    if (!ok) atomicCAS(err, 0, kErrBounds);
    return ok;
#else
    (void)ok;
    (void)err;
    return true;
#endif
}

__device__ __forceinline__ uint4 lds_v4_if(bool p, uint32_t a) {
    uint4 v = make_uint4(0, 0, 0, 0);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t@q ld.shared.v4.u32 {%0, %1, %2, %3}, [%5];\n\t}"
                 : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w) : "r"((uint32_t)p), "r"(a));
    return v;
}
__device__ __forceinline__ uint2 lds_v2_if(bool p, uint32_t a) {
    uint2 v = make_uint2(0, 0);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.shared.v2.u32 {%0, %1}, [%3];\n\t}"
                 : "+r"(v.x), "+r"(v.y) : "r"((uint32_t)p), "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32_if(bool p, uint32_t a) {
    uint32_t v = 0;
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t@q ld.shared.u32 %0, [%2];\n\t}"
                 : "+r"(v) : "r"((uint32_t)p), "r"(a));
    return v;
}

__device__ __forceinline__ void sts_f32_lt(uint32_t k, uint32_t ke, uint32_t a, float v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %0, %1;\n\t@q st.shared.f32 [%2], %3;\n\t}"
                 ::"r"(k), "r"(ke), "r"(a), "f"(v) : "memory");
}

// Bulk prefetch global -> L2 (no shared memory, no completion): addr 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void named_barrier(uint32_t id, uint32_t nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---- value decoders (exact conversions to FP32)
__device__ __forceinline__ float dec_u16(uint16_t q) { return static_cast<float>(q); }

__device__ __forceinline__ float dec_bf16(uint16_t b) {
    return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

__device__ __forceinline__ float f16_to_f32(uint16_t h) {
    float f;
    asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
    return f;
}

// OCP E4M3 -> FP32 through the hardware E4M3x2 -> F16x2 conversion (exact:
// every E4M3 value is representable in F16), then F16 -> F32 (exact).
__device__ __forceinline__ float dec_e4m3(uint8_t q) {
    uint32_t h2;
    const uint16_t in = (uint16_t)(q | (q << 8));  // same code in both bytes: either half is the value
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(in));
    float f;
    asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(static_cast<uint16_t>(h2 & 0xFFFFu)));
    return f;
}

// ---- error-free transformations for compensated dot products (Ogita, Rump,
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005: TwoSum of
// Knuth and TwoProduct by FMA).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Double-float accumulation (hi + lo, |lo| <= ulp(hi)/2 after each step) of the
// objective term w (d - p)^2 from FP32 operands, using only FP32 arithmetic:
// e = d - p exactly (TwoSum), e^2 and w e^2 by TwoProduct with the first-order
// cross terms, then a TwoSum into the accumulator and a renormalisation.  Each
// term and each step carries a relative error of a few u^2 (u = 2^-24), so the
// per-lane sum matches FP64 accumulation without using the FP64 pipe.
__device__ __forceinline__ float df_add_wsq(float& hi, float& lo, float w, float d, float p) {
    float eh, el, qh, ql, th, tl, sh, se;
    two_sum(d, -p, eh, el);
    two_prod(eh, eh, qh, ql);
    ql = __fmaf_rn(__fmul_rn(2.0f, eh), el, ql);
    two_prod(w, qh, th, tl);
    tl = __fmaf_rn(w, ql, tl);
    two_sum(hi, th, sh, se);
    const float l = __fadd_rn(lo, __fadd_rn(se, tl));
    hi = __fadd_rn(sh, l);                  // renormalise (fast TwoSum: |sh| >= |l|)
    lo = __fsub_rn(l, __fsub_rn(hi, sh));
    return eh;                              // e rounded to FP32 (exact difference's leading part)
}

}  // namespace dev
}  // namespace dose
#endif
