// SELL-C-sigma storage for the forward dose SpMV (the SIMT-oriented sparse format
// the paper names as future work beside ELLPACK, Sec. III and Sec. VI; Kreutzer
// et al., SIAM J. Sci. Comput. 2014).
//
// Layout (C = 32, one row per lane of a warp):
//   * the rows are cut into windows of sigma consecutive rows and ordered by
//     length inside each window, longest first (stable); the resulting row
//     order is cut into chunks of 32 consecutive rows; empty rows end up in
//     chunks of length 0;
//   * chunk c holds ng_c = ceil(longest row / 4) groups; group g of lane l
//     (its row's entries 4g .. 4g + 3) sits at entries
//     off_c + 128 g + 4 l .. + 3, so a warp reads each group as 32 consecutive
//     16-byte (columns) and 8-byte (values) pieces; entries past a row's end are
//     padding with value code 0 and column 0, which add exactly 0;
//   * perm[32 c + l] is the original row of chunk c's lane l (~0 for the slots
//     past the matrix's last row).
// sigma = 1 keeps the row order (chunks of 32 consecutive rows, each padded to
// its longest row: ELLPACK per chunk of 32 rows); ELLPACK proper (one chunk for
// the whole matrix) would pad every one of the 10.5 M rows of the clinical beam
// to its longest row and is not offered.
//
// Kernel: every warp takes chunks c = warp id, + number of warps, ...; lane l
// sums its row over the chunk's groups with four accumulators (combined as
// (0 + 1) + (2 + 3)), x in shared memory; the row's dose is written to
// d[perm].  With DOSE_CREATE_COMPENSATED, the lanes of a chunk whose longest
// row has more than 128 entries accumulate compensated sums instead (Dot2 of
// Ogita, Rump and Oishi per accumulator: TwoProduct by FMA, TwoSum; the four
// (sum, error) pairs combined by TwoSum).  A row is summed by one lane in
// storage order, so the result does not depend on the chunk-to-warp
// assignment: bitwise reproducible.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "stage_common.cuh"

namespace dose {
namespace {

constexpr uint32_t kSellC = 32;
constexpr uint32_t kSellWarps = 16;  // warps per CTA
constexpr uint32_t kSellCtasPerSm = 4;

struct SellParams {
    const void* col;       // IW-byte column indices, SELL order
    const void* val;       // stored values, SELL order
    const uint2* chunk;    // {first entry / 128, groups} per chunk
    const uint32_t* perm;  // 32 per chunk
    const float* row_scale;
    float scale;
    const float* x;
    float* d;
    uint32_t ncols, nchunks;
};

template <int FMT, uint32_t IW, bool XSMEM, bool COMP>
__global__ void __launch_bounds__(kSellWarps * 32) sell_spmv_kernel(const SellParams p) {
    using T = typename Fmt<FMT>::T;
    extern __shared__ __align__(16) float xs_smem[];
    if (XSMEM) {
        for (uint32_t j = threadIdx.x; j < p.ncols; j += blockDim.x) xs_smem[j] = __ldg(p.x + j);
        __syncthreads();
    }
    const float* xs = XSMEM ? xs_smem : p.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * kSellWarps;
    for (uint32_t c = blockIdx.x * kSellWarps + (threadIdx.x >> 5); c < p.nchunks; c += nwarps) {
        const uint2 ch = __ldg(p.chunk + c);
        const size_t base = (size_t)ch.x * 128 + 4 * lane;
        const T* vp = static_cast<const T*>(p.val) + base;
        const unsigned char* cp = static_cast<const unsigned char*>(p.col) + base * IW;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        float err[4] = {0.f, 0.f, 0.f, 0.f};  // compensated chunks: the running error terms
        const bool comp = COMP && ch.y * 4 > kCompThreshold;
        // raw words of one group: four column indices (16 or 8 bytes) and four values (16, 8 or 4 bytes)
        struct Raw {
            uint4 c, v;
        };
        auto load = [&](uint32_t g) {
            Raw r;
            if (IW == 4) {
                r.c = __ldg(reinterpret_cast<const uint4*>(cp + (size_t)g * 128 * IW));
            } else {
                const uint2 q = __ldg(reinterpret_cast<const uint2*>(cp + (size_t)g * 128 * IW));
                r.c = make_uint4(q.x, q.y, 0u, 0u);
            }
            if constexpr (sizeof(T) == 4) {
                r.v = __ldg(reinterpret_cast<const uint4*>(vp + (size_t)g * 128));
            } else if constexpr (sizeof(T) == 2) {
                const uint2 q = __ldg(reinterpret_cast<const uint2*>(vp + (size_t)g * 128));
                r.v = make_uint4(q.x, q.y, 0u, 0u);
            } else {
                r.v = make_uint4(__ldg(reinterpret_cast<const uint32_t*>(vp + (size_t)g * 128)), 0u, 0u, 0u);
            }
            return r;
        };
        auto use = [&](const Raw& r) {
            uint32_t cc[4];
            if (IW == 4) {
                cc[0] = r.c.x; cc[1] = r.c.y; cc[2] = r.c.z; cc[3] = r.c.w;
            } else {
                cc[0] = r.c.x & 0xFFFFu; cc[1] = r.c.x >> 16; cc[2] = r.c.y & 0xFFFFu; cc[3] = r.c.y >> 16;
            }
            float a[4];
            if constexpr (sizeof(T) == 4) {
                a[0] = __uint_as_float(r.v.x); a[1] = __uint_as_float(r.v.y);
                a[2] = __uint_as_float(r.v.z); a[3] = __uint_as_float(r.v.w);
            } else {
                Fmt<FMT>::dec4(r.v.x, r.v.y, a);
            }
            if (COMP && comp) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float pr, ep, t, es;
                    dev::two_prod(a[u], XSMEM ? xs[cc[u]] : __ldg(xs + cc[u]), pr, ep);
                    dev::two_sum(acc[u], pr, t, es);
                    acc[u] = t;
                    err[u] = __fadd_rn(err[u], __fadd_rn(es, ep));
                }
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = __fmaf_rn(a[u], XSMEM ? xs[cc[u]] : __ldg(xs + cc[u]), acc[u]);
            }
        };
        // two groups in flight ahead of the one being summed
        Raw r0 = ch.y > 0 ? load(0) : Raw{}, r1 = ch.y > 1 ? load(1) : Raw{};
        for (uint32_t g = 0; g < ch.y; ++g) {
            const Raw cur = r0;
            r0 = r1;
            if (g + 2 < ch.y) r1 = load(g + 2);
            use(cur);
        }
        const uint32_t row = __ldg(p.perm + (size_t)c * kSellC + lane);
        if (row != 0xFFFFFFFFu) {
            float v;
            if (COMP && comp) {
                float sum = acc[0], e = err[0];
                for (int u = 1; u < 4; ++u) {
                    float t, es;
                    dev::two_sum(sum, acc[u], t, es);
                    sum = t;
                    e = __fadd_rn(e, __fadd_rn(err[u], es));
                }
                v = __fadd_rn(sum, e);
            } else {
                v = __fadd_rn(__fadd_rn(acc[0], acc[1]), __fadd_rn(acc[2], acc[3]));
            }
            if (FMT == DOSE_FMT_U16_SCALE) v = __fmul_rn(p.scale, v);
            if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) v = __fmul_rn(__ldg(p.row_scale + row), v);
            p.d[row] = v;
        }
    }
}

template <int FMT, uint32_t IW>
cudaError_t launch_t(const dose_matrix* A, const SellParams& p, cudaStream_t s) {
    const bool xsmem = A->ncols <= kXSmemMaxCols;
    const size_t smem = xsmem ? (size_t)A->ncols * 4 : 0;
    const bool comp = (A->flags & DOSE_CREATE_COMPENSATED) != 0;
    auto k = xsmem ? (comp ? sell_spmv_kernel<FMT, IW, true, true> : sell_spmv_kernel<FMT, IW, true, false>)
                   : (comp ? sell_spmv_kernel<FMT, IW, false, true> : sell_spmv_kernel<FMT, IW, false, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint32_t grid = std::max(1u, std::min<uint32_t>((uint32_t)A->sm_count * kSellCtasPerSm,
                                                          (A->sell.nchunks + kSellWarps - 1) / kSellWarps));
    k<<<grid, kSellWarps * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_fmt(const dose_matrix* A, const SellParams& p, cudaStream_t s) {
    return (A->flags & DOSE_CREATE_U16_INDEX) ? launch_t<FMT, 2>(A, p, s) : launch_t<FMT, 4>(A, p, s);
}

}  // namespace

// Host: SELL-32-sigma arrays of A from its host CSR (values and indices given
// in CSR order; esize / iw bytes each).  Returns the device arrays in A->sell.
cudaError_t build_sell(dose_matrix* A, const std::vector<uint32_t>& col, const unsigned char* vals, uint32_t sigma,
                       std::string* why) {
    const std::vector<uint32_t>& rp = A->host_row_ptr;
    const uint32_t nrows = A->nrows, esize = value_bytes(A->fmt);
    const uint32_t iw = (A->flags & DOSE_CREATE_U16_INDEX) ? 2 : 4;
    std::vector<uint32_t> order(nrows);
    std::iota(order.begin(), order.end(), 0u);
    std::vector<uint2> chunk;
    std::vector<uint32_t> perm;
    uint64_t groups = 0;  // 128-entry blocks
    if (sigma > 1)
        for (uint32_t w0 = 0; w0 < nrows; w0 += sigma) {
            const uint32_t w1 = (uint32_t)std::min<uint64_t>(nrows, (uint64_t)w0 + sigma);
            std::stable_sort(order.begin() + w0, order.begin() + w1, [&](uint32_t a, uint32_t b) {
                return rp[a + 1] - rp[a] > rp[b + 1] - rp[b];
            });
        }
    for (uint32_t c0 = 0; c0 < nrows; c0 += kSellC) {
        const uint32_t c1 = std::min(nrows, c0 + kSellC);
        uint32_t longest = 0;
        for (uint32_t k = c0; k < c1; ++k) longest = std::max(longest, rp[order[k] + 1] - rp[order[k]]);
        const uint32_t ng = (longest + 3) / 4;
        if (groups > 0xFFFFFFFFull) {
            *why = "SELL storage needs more than 2^32 blocks of 128 entries";
            return cudaErrorInvalidValue;
        }
        chunk.push_back(make_uint2((uint32_t)groups, ng));
        groups += ng;
        for (uint32_t k = c0; k < c0 + kSellC; ++k) perm.push_back(k < c1 ? order[k] : 0xFFFFFFFFu);
    }
    const size_t entries = (size_t)groups * 128;
    std::vector<unsigned char> sval(entries * esize + 64, 0), scol(entries * iw + 64, 0);
    for (size_t c = 0; c < chunk.size(); ++c)
        for (uint32_t l = 0; l < kSellC; ++l) {
            const uint32_t r = perm[c * kSellC + l];
            if (r == 0xFFFFFFFFu) continue;
            for (uint32_t k = 0; k < rp[r + 1] - rp[r]; ++k) {
                const size_t pos = (size_t)chunk[c].x * 128 + (size_t)(k / 4) * 128 + 4 * l + (k % 4);
                const size_t src = (size_t)rp[r] + k;
                std::memcpy(sval.data() + pos * esize, vals + src * esize, esize);
                if (iw == 4) {
                    std::memcpy(scol.data() + pos * 4, &col[src], 4);
                } else {
                    const uint16_t c16 = (uint16_t)col[src];
                    std::memcpy(scol.data() + pos * 2, &c16, 2);
                }
            }
        }
    SellArrays& S = A->sell;
    cudaError_t e;
    if ((e = dev_malloc(&S.val, sval.size())) != cudaSuccess) return e;
    if ((e = dev_malloc(&S.col, scol.size())) != cudaSuccess) return e;
    if ((e = dev_malloc(&S.chunk, std::max<size_t>(chunk.size(), 1) * sizeof(uint2))) != cudaSuccess) return e;
    if ((e = dev_malloc(&S.perm, std::max<size_t>(perm.size(), 1) * 4)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(S.val, sval.data(), sval.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(S.col, scol.data(), scol.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if (!chunk.empty() &&
        (e = cudaMemcpy(S.chunk, chunk.data(), chunk.size() * sizeof(uint2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    if (!perm.empty() && (e = cudaMemcpy(S.perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    S.nchunks = (uint32_t)chunk.size();
    S.entries = entries;
    S.sigma = sigma;
    S.bytes = sval.size() + scol.size() + chunk.size() * sizeof(uint2) + perm.size() * 4;
    return cudaSuccess;
}

void free_sell(dose_matrix* A) {
    cudaFree(A->sell.val);
    cudaFree(A->sell.col);
    cudaFree(A->sell.chunk);
    cudaFree(A->sell.perm);
    A->sell = SellArrays();
}

cudaError_t launch_spmv_sell(const dose_matrix* A, const float* x, float* d, cudaStream_t s) {
    if (A->nrows == 0 || A->sell.nchunks == 0) return cudaSuccess;
    SellParams p;
    p.col = A->sell.col;
    p.val = A->sell.val;
    p.chunk = A->sell.chunk;
    p.perm = A->sell.perm;
    p.row_scale = A->row_scale;
    p.scale = A->scale;
    p.x = x;
    p.d = d;
    p.ncols = A->ncols;
    p.nchunks = A->sell.nchunks;
    switch (A->fmt) {
        case DOSE_FMT_U16_SCALE: return launch_fmt<DOSE_FMT_U16_SCALE>(A, p, s);
        case DOSE_FMT_BF16: return launch_fmt<DOSE_FMT_BF16>(A, p, s);
        case DOSE_FMT_F16: return launch_fmt<DOSE_FMT_F16>(A, p, s);
        case DOSE_FMT_F32: return launch_fmt<DOSE_FMT_F32>(A, p, s);
        case DOSE_FMT_FP8E4M3_ROWSCALE: return launch_fmt<DOSE_FMT_FP8E4M3_ROWSCALE>(A, p, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dose
