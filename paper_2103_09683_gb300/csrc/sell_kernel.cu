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
// Kernel: the forward kernel's pipeline.  Consecutive chunks form stages (at
// most tile_nnz entries and tile_rows / 32 chunks), dealt round-robin to
// persistent CTAs; a producer warp bulk-copies each stage's perm slots (in the
// row-pointer slice of the ring slot), chunk offsets (in the row-list slice),
// values and columns -- one contiguous range each -- into a shared-memory ring.
// Consumer warps take the stage's chunks round-robin; lane l sums its row over
// the chunk's groups with four accumulators, x in shared memory, and writes
// d[perm].  A chunk longer than a tile spans several stages of its own, summed
// by the first consumer warp.  A row is summed by one lane in storage order:
// bitwise reproducible.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "stage_common.cuh"

namespace dose {
namespace {

constexpr uint32_t kSellC = 32;
constexpr uint32_t kSellPart = STAGE_COOP;  // a stage holding part of one long chunk

struct SellParams {
    const uint32_t* perm;  // 32 per chunk (+ padding), the ring's "row pointer" slice
    const void* col;       // IW-byte column indices, SELL order
    const void* val;       // stored values, SELL order
    float scale;
    const float* x;
    float* d;
    uint32_t ncols;
    ScheduleView sched;    // stages; sched.ne = chunk offsets (groups from the stage's first entry)
    VecSet vecs;           // FP8: row scales in slot order
    uint32_t tile_nnz, tile_rows, depth, cwarps, l2pf;
    int* err;
};

constexpr uint32_t kHeaderBytes = 3072;

template <int FMT, uint32_t IW, bool XSMEM>
__device__ __forceinline__ void sum_groups(const SlotPtrs<FMT, IW>& sp, const float* __restrict__ xs, uint32_t base,
                                           uint32_t ng, float (&acc)[4]) {
    for (uint32_t g = 0; g < ng; ++g) {
        const uint32_t k = base + 128 * g;
        uint32_t cc[4];
        if (IW == 4) {
            const uint4 q = *reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(sp.col) + k);
            cc[0] = q.x; cc[1] = q.y; cc[2] = q.z; cc[3] = q.w;
        } else {
            const uint2 q = *reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(sp.col) + k);
            cc[0] = q.x & 0xFFFFu; cc[1] = q.x >> 16; cc[2] = q.y & 0xFFFFu; cc[3] = q.y >> 16;
        }
        float a[4];
        load_vals4<FMT>(sp.val + k, a);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = __fmaf_rn(a[u], XSMEM ? xs[cc[u]] : __ldg(xs + cc[u]), acc[u]);
    }
}

template <int FMT>
__device__ __forceinline__ float row_out(const SellParams& p, uint32_t slot, const SlotLayout& SL, uint32_t s_row0,
                                         uint32_t slot_idx, const float (&acc)[4]) {
    float v = __fadd_rn(__fadd_rn(acc[0], acc[1]), __fadd_rn(acc[2], acc[3]));
    if (FMT == DOSE_FMT_U16_SCALE) v = __fmul_rn(p.scale, v);
    if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) v = __fmul_rn(slot_vec(slot, SL, p.vecs, 0, s_row0, slot_idx), v);
    return v;
}

template <int FMT, uint32_t IW, bool XSMEM>
__global__ void __launch_bounds__(544, 1) sell_spmv_kernel(const SellParams p) {
    using T = typename Fmt<FMT>::T;
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth, W = p.cwarps;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + S;
    uint64_t* dbar = full + 16;
    StageDesc* dwin = reinterpret_cast<StageDesc*>(smem + 1024);
    float* xs = reinterpret_cast<float*>(smem + kHeaderBytes);
    const uint32_t x_bytes = XSMEM ? round_up(p.ncols * 4, 128) : 0;
    unsigned char* slot_base = smem + kHeaderBytes + x_bytes;
    const SlotLayout SL = slot_layout(p.tile_nnz, p.tile_rows, sizeof(T), p.vecs.n, false, IW);
    const uint32_t s_begin = p.sched.cta_begin[blockIdx.x], s_end = p.sched.cta_begin[blockIdx.x + 1];

    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < S; ++i) {
            dev::mbar_init(&full[i], 1);
            dev::mbar_init(&empty[i], W);
        }
        dev::mbar_init(&dbar[0], 1);
        dev::mbar_init(&dbar[1], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (s_begin >= s_end) return;
    if (warp == 0) {
        if (lane == 0)
            run_producer<FMT, IW>(p.sched, s_begin, s_end, p.perm, p.col, p.val, p.vecs, slot_base, SL, full, empty, S,
                                  dwin, dbar, p.l2pf, p.err);
        return;
    }
    const uint32_t cw = warp - 1, ctid = threadIdx.x - 32, nct = W * 32;
    if (XSMEM) {
        for (uint32_t j = ctid; j < p.ncols; j += nct) xs[j] = __ldg(p.x + j);
        dev::named_barrier(1, nct);
    }
    const float* xsrc = XSMEM ? xs : p.x;
    const uint32_t slot0 = dev::smem_u32(slot_base);
    float part[4] = {0.f, 0.f, 0.f, 0.f};  // a long chunk's sums across its stages (first consumer warp)
    uint32_t st = 0, ph = 0;
    for (uint32_t s = s_begin; s < s_end; ++s) {
        if (!dev::mbar_wait_bounded(&full[st], ph)) {
            atomicExch(p.err, kErrTimeoutFull);
            return;
        }
        const uint32_t slot = slot0 + st * SL.bytes;
        const StageDesc D = slot_desc(slot);
        const SlotView v = slot_view<FMT, IW>(slot, SL, D);
        const SlotPtrs<FMT, IW> sp = slot_ptrs<FMT, IW>(slot_base + st * SL.bytes, SL, D);
        if (!(D.meta & kSellPart)) {
            const uint32_t nch = D.ne1 - D.ne0, total = (D.nz1 - D.nz0) / 128;
            for (uint32_t k = cw; k < nch; k += W) {
                const uint32_t g0 = dev::lds_u16(v.ne + 2 * k);
                const uint32_t g1 = k + 1 < nch ? dev::lds_u16(v.ne + 2 * (k + 1)) : total;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                sum_groups<FMT, IW, XSMEM>(sp, xsrc, D.nz0 + 128 * g0 + 4 * lane, g1 - g0, acc);
                const uint32_t si = D.row0 + 32 * k + lane;  // this lane's slot
                const uint32_t row = dev::lds_u32(v.rp + 4 * si);
                if (row != 0xFFFFFFFFu) p.d[row] = row_out<FMT>(p, slot, SL, D.row0, si, acc);
            }
        } else if (cw == 0) {
            if (D.meta & STAGE_FIRST) part[0] = part[1] = part[2] = part[3] = 0.f;
            sum_groups<FMT, IW, XSMEM>(sp, xsrc, D.nz0 + 4 * lane, (D.nz1 - D.nz0) / 128, part);
            if (D.meta & STAGE_LAST) {
                // (the ring stages no perm slice for these stages: read it from global memory)
                const uint32_t si = D.row0 + lane;
                const uint32_t row = __ldg(p.perm + si);
                if (row != 0xFFFFFFFFu) p.d[row] = row_out<FMT>(p, slot, SL, D.row0, si, part);
            }
        }
        __syncwarp();
        if (lane == 0) dev::mbar_arrive(&empty[st]);
        if (++st == S) {
            st = 0;
            ph ^= 1;
        }
    }
}

uint32_t sell_tile_rows(const Tuning& t) { return std::max(32u, t.tile_rows / 32 * 32); }

size_t sell_smem(const dose_matrix* A, const Tuning& t, bool xsmem) {
    const uint32_t esize = value_bytes(A->fmt), iw = (A->flags & DOSE_CREATE_U16_INDEX) ? 2 : 4;
    const uint32_t nvec = A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0;
    const SlotLayout SL = slot_layout(t.tile_nnz, sell_tile_rows(t), esize, nvec, false, iw);
    return kHeaderBytes + (xsmem ? round_up(A->ncols * 4, 128) : 0) + (size_t)t.stages * SL.bytes;
}

template <int FMT, uint32_t IW, bool XSMEM>
cudaError_t launch_t(const dose_matrix* A, const SellParams& p, size_t smem, cudaStream_t s) {
    auto k = sell_spmv_kernel<FMT, IW, XSMEM>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<A->sell.grid, 32 * (p.cwarps + 1), smem, s>>>(p);
    return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_fmt(const dose_matrix* A, const SellParams& p, size_t smem, bool xsmem, cudaStream_t s) {
    if (A->flags & DOSE_CREATE_U16_INDEX)
        return xsmem ? launch_t<FMT, 2, true>(A, p, smem, s) : launch_t<FMT, 2, false>(A, p, smem, s);
    return xsmem ? launch_t<FMT, 4, true>(A, p, smem, s) : launch_t<FMT, 4, false>(A, p, smem, s);
}

template <class V>
cudaError_t upload_vec(V** dst, const std::vector<V>& src, size_t pad) {
    cudaError_t e = cudaMalloc(dst, (src.size() + pad) * sizeof(V));
    if (e == cudaSuccess) e = cudaMemset(*dst, 0, (src.size() + pad) * sizeof(V));
    if (e == cudaSuccess && !src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

// Host: SELL-32-sigma arrays of A from its host CSR (values and indices given
// in CSR order; esize / iw bytes each) and their stage schedule.
cudaError_t build_sell(dose_matrix* A, const std::vector<uint32_t>& col, const unsigned char* vals,
                       const float* row_scale, uint32_t sigma, std::string* why) {
    const std::vector<uint32_t>& rp = A->host_row_ptr;
    const uint32_t nrows = A->nrows, esize = value_bytes(A->fmt);
    const uint32_t iw = (A->flags & DOSE_CREATE_U16_INDEX) ? 2 : 4;
    std::vector<uint32_t> order(nrows);
    std::iota(order.begin(), order.end(), 0u);
    std::vector<uint2> chunk;  // first group, groups
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
        chunk.push_back(make_uint2((uint32_t)groups, ng));
        groups += ng;
        for (uint32_t k = c0; k < c0 + kSellC; ++k) perm.push_back(k < c1 ? order[k] : 0xFFFFFFFFu);
    }
    if (groups * 128 >= (1ull << 32)) {
        *why = "SELL storage needs 2^32 or more entries (padding included)";
        return cudaErrorInvalidValue;
    }
    const size_t entries = (size_t)groups * 128;
    std::vector<unsigned char> sval(entries * esize, 0), scol(entries * iw, 0);
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
    // Stages: consecutive chunks with at most tile_nnz entries and tile_rows / 32
    // chunks; a chunk longer than a tile gets stages of its own (FIRST .. LAST).
    const Tuning& t = A->fwd.tuning;
    const uint32_t gmax = std::max(1u, t.tile_nnz / 128), cmax = sell_tile_rows(t) / kSellC;
    std::vector<StageDesc> desc;
    std::vector<uint16_t> choff(chunk.size(), 0);
    std::vector<std::pair<uint32_t, uint32_t>> items;  // stage ranges, dealt whole
    for (uint32_t c = 0; c < chunk.size();) {
        if (chunk[c].y > gmax) {
            const uint32_t s0 = (uint32_t)desc.size();
            for (uint32_t g = 0; g < chunk[c].y; g += gmax) {
                StageDesc D{};
                D.row0 = kSellC * c;
                D.row1 = kSellC * (c + 1);
                D.nz0 = (chunk[c].x + g) * 128;
                D.nz1 = (chunk[c].x + std::min(chunk[c].y, g + gmax)) * 128;
                D.ne0 = c;
                D.ne1 = c + 1;
                D.meta = kSellPart | (g == 0 ? STAGE_FIRST : 0u) | (g + gmax >= chunk[c].y ? STAGE_LAST : 0u);
                desc.push_back(D);
            }
            items.push_back({s0, (uint32_t)desc.size()});
            ++c;
            continue;
        }
        StageDesc D{};
        D.row0 = kSellC * c;
        D.ne0 = c;
        D.nz0 = chunk[c].x * 128;
        uint32_t g = 0, c1 = c;
        while (c1 < chunk.size() && c1 - c < cmax && chunk[c1].y <= gmax && g + chunk[c1].y <= gmax) {
            choff[c1] = (uint16_t)g;
            g += chunk[c1].y;
            ++c1;
        }
        D.row1 = kSellC * c1;
        D.ne1 = c1;
        D.nz1 = D.nz0 + g * 128;
        items.push_back({(uint32_t)desc.size(), (uint32_t)desc.size() + 1});
        desc.push_back(D);
        c = c1;
    }
    const uint32_t grid = (uint32_t)std::max(1, A->sm_count);
    std::vector<std::vector<uint32_t>> per(grid);
    for (size_t i = 0; i < items.size(); ++i)
        for (uint32_t k = items[i].first; k < items[i].second; ++k) per[i % grid].push_back(k);
    std::vector<StageDesc> sorted;
    std::vector<uint32_t> cta_begin(grid + 1, 0);
    for (uint32_t b = 0; b < grid; ++b) {
        cta_begin[b] = (uint32_t)sorted.size();
        for (uint32_t k : per[b]) sorted.push_back(desc[k]);
    }
    cta_begin[grid] = (uint32_t)sorted.size();
    // FP8 row scales in slot order (the ring stages them like the perm slots)
    std::vector<float> sscale;
    if (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE) {
        sscale.assign(perm.size(), 1.0f);
        for (size_t i = 0; i < perm.size(); ++i)
            if (perm[i] != 0xFFFFFFFFu) sscale[i] = row_scale[perm[i]];
    }
    SellArrays& S = A->sell;
    cudaError_t e;
    if ((e = upload_vec(reinterpret_cast<unsigned char**>(&S.val), sval, 64)) != cudaSuccess) return e;
    if ((e = upload_vec(reinterpret_cast<unsigned char**>(&S.col), scol, 64)) != cudaSuccess) return e;
    if ((e = upload_vec(&S.perm, perm, 32)) != cudaSuccess) return e;
    if ((e = upload_vec(&S.choff, choff, 32)) != cudaSuccess) return e;
    if ((e = upload_vec(&S.desc, sorted, 1)) != cudaSuccess) return e;
    if ((e = upload_vec(&S.cta_begin, cta_begin, 0)) != cudaSuccess) return e;
    if (!sscale.empty() && (e = upload_vec(&S.scale_perm, sscale, 32)) != cudaSuccess) return e;
    S.nchunks = (uint32_t)chunk.size();
    S.nslots = (uint32_t)perm.size();
    S.n_stages = (uint32_t)sorted.size();
    S.grid = grid;
    S.entries = entries;
    S.sigma = sigma;
    S.bytes = sval.size() + scol.size() + (perm.size() + 32) * 4 + (choff.size() + 32) * 2 +
              (sorted.size() + 1) * sizeof(StageDesc) + cta_begin.size() * 4 + (sscale.size() + 32) * 4;
    return cudaSuccess;
}

void free_sell(dose_matrix* A) {
    cudaFree(A->sell.val);
    cudaFree(A->sell.col);
    cudaFree(A->sell.perm);
    cudaFree(A->sell.choff);
    cudaFree(A->sell.desc);
    cudaFree(A->sell.cta_begin);
    cudaFree(A->sell.scale_perm);
    A->sell = SellArrays();
}

bool sell_fits(const dose_matrix* A) { return sell_smem(A, A->fwd.tuning, false) <= kMaxSmemPerBlock; }

cudaError_t launch_spmv_sell(const dose_matrix* A, const float* x, float* d, cudaStream_t s) {
    if (A->nrows == 0 || A->sell.n_stages == 0) return cudaSuccess;
    const Tuning& t = A->fwd.tuning;
    SellParams p;
    p.perm = A->sell.perm;
    p.col = A->sell.col;
    p.val = A->sell.val;
    p.scale = A->scale;
    p.x = x;
    p.d = d;
    p.ncols = A->ncols;
    p.sched = ScheduleView{A->sell.desc, A->sell.choff, A->sell.cta_begin, nullptr};
    p.vecs.n = 0;
    if (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE) {
        p.vecs.n = 1;
        p.vecs.ptr[0] = A->sell.scale_perm;
        p.vecs.lim[0] = A->sell.nslots;
    }
    p.tile_nnz = t.tile_nnz;
    p.tile_rows = sell_tile_rows(t);
    p.depth = t.stages;
    p.cwarps = t.consumer_warps;
    p.l2pf = t.l2_prefetch;
    p.err = A->err;
    const bool xsmem = A->ncols <= kXSmemMaxCols && sell_smem(A, t, true) <= kMaxSmemPerBlock;
    const size_t smem = sell_smem(A, t, xsmem);
    switch (A->fmt) {
        case DOSE_FMT_U16_SCALE: return launch_fmt<DOSE_FMT_U16_SCALE>(A, p, smem, xsmem, s);
        case DOSE_FMT_BF16: return launch_fmt<DOSE_FMT_BF16>(A, p, smem, xsmem, s);
        case DOSE_FMT_F16: return launch_fmt<DOSE_FMT_F16>(A, p, smem, xsmem, s);
        case DOSE_FMT_F32: return launch_fmt<DOSE_FMT_F32>(A, p, smem, xsmem, s);
        case DOSE_FMT_FP8E4M3_ROWSCALE: return launch_fmt<DOSE_FMT_FP8E4M3_ROWSCALE>(A, p, smem, xsmem, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dose
