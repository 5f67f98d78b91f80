// Batched dose SpMM: D_m = A_m X_m for many matrices (beams x uncertainty
// scenarios) and up to 16 spot-weight vectors per matrix, in one persistent
// launch.  The optimiser evaluates the dose of several beams, possibly under
// several realisations of the uncertainties, in every iteration (Sec. I); each
// beam has its own dose-deposition matrix (Sec. II-B).
//
// Work units are the row blocks of every matrix's own schedule, enumerated
// matrix by matrix; each CTA owns a contiguous range of units (static, so the
// result never depends on timing).  A row is reduced by one half-warp: lane v
// owns output vector v, walks the row's entries in storage order and gathers
// X[col, v] (64 contiguous bytes per entry for 16 vectors, L1/L2-resident).
#include "stage_common.cuh"

#include <string>

namespace dose {
namespace {

constexpr int kMaxBatchPerLaunch = 64;

struct BatchItem {
    const uint32_t* row_ptr;
    const uint32_t* col;
    const void* val;
    const float* row_scale;
    const float* X;
    float* D;
    const StageDesc* desc;
    float scale;
    uint32_t nrows, n_stages;
    uint32_t unit_begin;  // first global unit of this matrix
    int fmt;
};

struct BatchParams {
    BatchItem item[kMaxBatchPerLaunch];
    uint32_t count, total_units, nvec;
};

template <int FMT>
__device__ __forceinline__ void spmm_row(const BatchItem& it, uint32_t row, uint32_t v, uint32_t nvec) {
    using T = typename Fmt<FMT>::T;
    const T* val = static_cast<const T*>(it.val);
    const uint32_t kb = __ldg(it.row_ptr + row), ke = __ldg(it.row_ptr + row + 1);
    const bool act = v < nvec;
    float acc = 0.f;
#pragma unroll 4
    for (uint32_t k = kb; k < ke; ++k) {
        const uint32_t c = __ldg(it.col + k);
        const float a = Fmt<FMT>::dec(val[k]);
        const float xv = act ? __ldg(it.X + (size_t)c * nvec + v) : 0.f;
        acc = __fmaf_rn(a, xv, acc);
    }
    if (act) {
        float s = 1.0f;
        if (FMT == DOSE_FMT_U16_SCALE) s = it.scale;
        if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) s = __ldg(it.row_scale + row);
        it.D[(size_t)row * nvec + v] = FMT == DOSE_FMT_BF16 ? acc : __fmul_rn(s, acc);
    }
}

__global__ void __launch_bounds__(256) spmm_batched_kernel(const __grid_constant__ BatchParams p) {
    const uint32_t G = gridDim.x;
    const uint32_t u_begin = (uint32_t)(((uint64_t)p.total_units * blockIdx.x) / G);
    const uint32_t u_end = (uint32_t)(((uint64_t)p.total_units * (blockIdx.x + 1)) / G);
    const uint32_t hw = threadIdx.x >> 4;         // half-warp index in the CTA
    const uint32_t nhw = blockDim.x >> 4;
    const uint32_t v = threadIdx.x & 15;
    uint32_t m = 0;
    for (uint32_t u = u_begin; u < u_end; ++u) {
        while (m + 1 < p.count && p.item[m + 1].unit_begin <= u) ++m;
        const BatchItem& it = p.item[m];
        const uint32_t s = u - it.unit_begin;
        const StageDesc D = it.desc[s];
        const uint32_t meta = D.meta;
        uint32_t r0 = D.row0, r1 = D.row1;
        if (meta & STAGE_COOP) {
            if (!(meta & STAGE_FIRST)) continue;  // a long row is reduced once, at its first chunk
            r1 = r0 + 1;
        }
        for (uint32_t row = r0 + hw; row < r1; row += nhw) {
            switch (it.fmt) {
                case DOSE_FMT_U16_SCALE: spmm_row<DOSE_FMT_U16_SCALE>(it, row, v, p.nvec); break;
                case DOSE_FMT_BF16: spmm_row<DOSE_FMT_BF16>(it, row, v, p.nvec); break;
                default: spmm_row<DOSE_FMT_FP8E4M3_ROWSCALE>(it, row, v, p.nvec); break;
            }
        }
    }
}

}  // namespace

cudaError_t launch_spmm_batched(const dose_matrix* const* A, int count, const float* const* X, float* const* D,
                                int nvec, cudaStream_t s, std::string* why) {
    int dev = A[0]->device;
    for (int m = 0; m < count; ++m)
        if (A[m]->device != dev) {
            *why = "dose_spmv_batched: all matrices must live on one device";
            return cudaSuccess;
        }
    for (int base = 0; base < count; base += kMaxBatchPerLaunch) {
        const int n = count - base < kMaxBatchPerLaunch ? count - base : kMaxBatchPerLaunch;
        BatchParams p;
        p.count = (uint32_t)n;
        p.nvec = (uint32_t)nvec;
        uint32_t units = 0;
        for (int i = 0; i < n; ++i) {
            const dose_matrix* M = A[base + i];
            BatchItem& it = p.item[i];
            it.row_ptr = M->row_ptr;
            it.col = M->col;
            it.val = M->val;
            it.row_scale = M->row_scale;
            it.X = X[base + i];
            it.D = D[base + i];
            it.desc = M->fwd.desc;
            it.scale = M->scale;
            it.nrows = M->nrows;
            it.n_stages = M->fwd.n_stages;
            it.unit_begin = units;
            it.fmt = M->fmt;
            units += M->fwd.n_stages;
        }
        p.total_units = units;
        if (units == 0) continue;
        const uint32_t grid = (uint32_t)A[0]->sm_count * 4;
        spmm_batched_kernel<<<grid, 256, 0, s>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dose
