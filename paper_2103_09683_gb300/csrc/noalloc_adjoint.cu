// dose_adjoint_noalloc: g = A^T r for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc: a host application that hands this
// library memory it manages itself (a fixed arena, a pool owned by another
// runtime), code running inside a stream capture whose memory plan is frozen,
// or an embedded deployment that forbids allocation after start-up.  Such a
// caller already holds A in CSR on the device and cannot create a handle
// (dose_create_matrix allocates), so this entry point takes the CSR arrays
// directly and keeps its per-CTA partial gradients in a file-scope __device__
// array instead of handle-owned scratch.
//
// The array holds kStaticScratchFloats floats (4 MiB); every GPU that loads the
// library holds it until the process exits.  All calls on a device share it and
// each call overwrites the part it uses, so calls that overlap on the GPU (two
// streams, or two host threads) race on it; order them.  The first call on a
// device looks up the array's device address (cudaGetSymbolAddress) and caches
// it for the rest of the process, which assumes that the device's primary
// context lives as long; make that first call before any stream capture.
//
// The columns of a row must be distinct (dose_create_matrix rejects rows that
// repeat one; this entry point takes the caller's arrays unchecked): the lanes
// of a warp update their accumulator words with plain read-modify-writes, so a
// repeated column loses one of its updates.
//
// The reduction order is fixed (per-warp shared accumulators in row order, warp
// order, then CTA order), so results are bitwise reproducible for the same
// inputs, grid and GPU.  Rows are split evenly across CTAs and warps; this
// variant has no row-block schedule and no bulk-copy pipeline.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "dose_internal.cuh"
#include "nvtx_range.cuh"

namespace dose {
namespace {

constexpr size_t kStaticScratchFloats = 1u << 20;  // 4 MiB
constexpr uint32_t kNoallocMaxCtas = 1024;
constexpr uint32_t kMaxDevices = 64;

// Per-CTA partial gradients: [nparts][ncols].
static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];

float* scratch_addr[kMaxDevices] = {};
std::mutex scratch_mu;

__device__ __forceinline__ float dec_value(int fmt, const void* values, uint32_t k) {
    if (fmt == DOSE_FMT_FP8E4M3_ROWSCALE) return dev::dec_e4m3(static_cast<const uint8_t*>(values)[k]);
    if (fmt == DOSE_FMT_F32) return static_cast<const float*>(values)[k];
    const uint16_t q = static_cast<const uint16_t*>(values)[k];
    if (fmt == DOSE_FMT_F16) return dev::f16_to_f32(q);
    return fmt == DOSE_FMT_BF16 ? dev::dec_bf16(q) : dev::dec_u16(q);
}

// CTA c scatters rows [c*nrows/P, (c+1)*nrows/P); warp w takes every W-th row
// of that range in order into its own shared accumulator (the columns of a row
// are distinct, so the lanes of a warp never update the same word at once).
// Malformed structure is skipped, never followed out of bounds.
__global__ void noalloc_adjoint_partials(uint32_t nrows, uint32_t ncols, uint64_t nnz,
                                         const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                                         int fmt, const void* __restrict__ values,
                                         const float* __restrict__ row_scales, const float* __restrict__ r,
                                         float* __restrict__ partials) {
    extern __shared__ float acc[];  // W x ncols
    const uint32_t W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint32_t j = threadIdx.x; j < W * ncols; j += blockDim.x) acc[j] = 0.f;
    __syncthreads();
    const uint32_t P = gridDim.x;
    const uint32_t r0 = (uint32_t)((uint64_t)nrows * blockIdx.x / P);
    const uint32_t r1 = (uint32_t)((uint64_t)nrows * (blockIdx.x + 1) / P);
    float* gw = acc + warp * ncols;
    for (uint32_t i = r0 + warp; i < r1; i += W) {
        const uint32_t kb = __ldg(row_ptr + i), ke = __ldg(row_ptr + i + 1);
        if (ke < kb || ke > nnz) continue;
        float ri = __ldg(r + i);
        if (fmt == DOSE_FMT_FP8E4M3_ROWSCALE) ri = __fmul_rn(ri, __ldg(row_scales + i));
        for (uint32_t k = kb + lane; k < ke; k += 32) {
            const uint32_t c = __ldg(col + k);
            if (c < ncols) gw[c] = __fmaf_rn(dec_value(fmt, values, k), ri, gw[c]);
        }
        __syncwarp();
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < ncols; j += blockDim.x) {
        float t = acc[j];
        for (uint32_t w2 = 1; w2 < W; ++w2) t = __fadd_rn(t, acc[w2 * ncols + j]);
        partials[(size_t)blockIdx.x * ncols + j] = t;
    }
}

// g_j = scale * sum over the P partials in CTA order.
__global__ void noalloc_adjoint_sum(const float* __restrict__ partials, uint32_t nparts, uint32_t ncols, float scale,
                                    float* __restrict__ g) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    float t = 0.f;
    for (uint32_t c = 0; c < nparts; ++c) t = __fadd_rn(t, partials[(size_t)c * ncols + j]);
    g[j] = __fmul_rn(scale, t);
}

// Device address of the static scratch on the current device (looked up once).
dose_status static_scratch(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "dose_adjoint_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= (int)kMaxDevices) {
        set_error("dose_adjoint_noalloc: device index beyond the supported range");
        return DOSE_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(scratch_mu);
    if (!scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "dose_adjoint_noalloc: cudaGetSymbolAddress");
        scratch_addr[dev] = static_cast<float*>(p);
    }
    *out = scratch_addr[dev];
    return DOSE_OK;
}

}  // namespace
}  // namespace dose

using namespace dose;

extern "C" dose_status dose_adjoint_noalloc(uint32_t nrows, uint32_t ncols, uint64_t nnz, const uint32_t* row_ptr,
                                            const uint32_t* col_idx, dose_format fmt, const void* values,
                                            const float* row_scales, float scale, const float* r, float* g,
                                            void* stream) {
    NvtxRange nvtx_range("dose_adjoint_noalloc");
    if (fmt != DOSE_FMT_U16_SCALE && fmt != DOSE_FMT_BF16 && fmt != DOSE_FMT_FP8E4M3_ROWSCALE &&
        fmt != DOSE_FMT_F16 && fmt != DOSE_FMT_F32) {
        set_error("dose_adjoint_noalloc: unknown format");
        return DOSE_ERR_INVALID_ARG;
    }
    if (ncols == 0) return DOSE_OK;
    if (!g || (nrows && (!row_ptr || !r)) || (nnz && (!col_idx || !values)) ||
        (fmt == DOSE_FMT_FP8E4M3_ROWSCALE && nrows && !row_scales)) {
        set_error("dose_adjoint_noalloc: null pointer argument");
        return DOSE_ERR_INVALID_ARG;
    }
    if (nnz >= (1ull << 32)) {
        set_error("dose_adjoint_noalloc: nnz must be < 2^32");
        return DOSE_ERR_INVALID_ARG;
    }
    if ((size_t)ncols > kStaticScratchFloats) {
        set_error("dose_adjoint_noalloc: ncols = " + std::to_string(ncols) + " exceeds the static scratch (" +
                  std::to_string(kStaticScratchFloats) + " floats)");
        return DOSE_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "dose_adjoint_noalloc: device query");
    // warps per CTA: as many 32-lane accumulators of ncols floats as fit (<= 8)
    uint32_t W = 8;
    while (W > 0 && (size_t)W * ncols * 4 > (size_t)max_smem) --W;
    if (W == 0) {
        set_error("dose_adjoint_noalloc: one accumulator of ncols floats does not fit in shared memory (ncols <= " +
                  std::to_string(max_smem / 4) + ")");
        return DOSE_ERR_INVALID_ARG;
    }
    uint32_t P = (uint32_t)std::max(1, sms);
    P = std::min<uint32_t>(P, kNoallocMaxCtas);
    P = std::min<uint32_t>(P, (uint32_t)(kStaticScratchFloats / ncols));
    float* scratch = nullptr;
    dose_status st = static_scratch(&scratch);
    if (st != DOSE_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t smem = (size_t)W * ncols * 4;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(noalloc_adjoint_partials, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "dose_adjoint_noalloc: shared memory attribute");
    }
    noalloc_adjoint_partials<<<P, 32 * W, smem, s>>>(nrows, ncols, nnz, row_ptr, col_idx, (int)fmt, values,
                                                      row_scales, r, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "dose_adjoint_noalloc: partials launch");
    noalloc_adjoint_sum<<<(ncols + 255) / 256, 256, 0, s>>>(scratch, P, ncols,
                                                            fmt == DOSE_FMT_U16_SCALE ? scale : 1.0f, g);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "dose_adjoint_noalloc: sum launch");
    return DOSE_OK;
}
