// Forward dose SpMV d = A x on sm_103a (Sec. II-A: the dose is one matrix-vector
// product; Sec. III, Listing 1: one output per row, the row's dot product,
// lanes of a warp read consecutive entries and reduce with warp shuffles).
//
// GB300 design (not the paper's one-warp-per-row grid):
//   * persistent CTAs, one per SM, each owning a contiguous range of row blocks
//     ("stages") fixed at create time;
//   * one producer warp streams each stage's row_ptr / non-empty-row list /
//     value / column slices into a shared-memory ring with bulk async copies
//     (cp.async.bulk + mbarrier transaction counts), so HBM sees a few large
//     contiguous reads per stage and consumers never wait on global memory;
//   * consumer warps write 0 for the stage's empty rows (coalesced) and share
//     its non-empty rows evenly: groups of L lanes per row, L chosen per stage
//     from its mean row length (row-length binning); rows longer than coop_nnz
//     are reduced by the whole CTA;
//   * values are decoded in registers (u16, bf16, f16, e4m3 -> f32; f32 as is),
//     x sits in shared memory, accumulation is FP32 (optionally compensated),
//     and the U16/FP8 scale is applied once per row.
// Every reduction has a fixed shape, so results are bitwise reproducible.
#include "stage_common.cuh"

namespace dose {
namespace {

struct SpmvParams {
    const uint32_t* row_ptr;
    const void* col;  // column indices of IW bytes
    const void* val;
    float scale;
    const float* x;
    float* d;
    uint32_t nrows, ncols;
    uint32_t xcols;  // columns of x staged per CTA (ncols, or the window width)
    ScheduleView sched;
    VecSet vecs;  // FP8: the row scales
    uint32_t tile_nnz, tile_rows, depth, cwarps, l2pf;
    int* err;
};

constexpr uint32_t kHeaderBytes = 3072;  // mbarriers, CTA reduction scratch, 2 KB of stage descriptors

// Combine the (sum, compensation) pairs of the `width` lanes of a group.
template <bool COMP>
__device__ __forceinline__ void group_reduce(float& sum, float& comp, uint32_t width) {
    for (uint32_t off = width >> 1; off > 0; off >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, sum, off);
        if (COMP) {
            const float oc = __shfl_xor_sync(0xffffffffu, comp, off);
            float t, e;
            dev::two_sum(sum, os, t, e);
            sum = t;
            comp = __fadd_rn(__fadd_rn(comp, oc), e);
        } else {
            sum = __fadd_rn(sum, os);
        }
    }
}

template <int FMT>
__device__ __forceinline__ float row_result(const SpmvParams& p, uint32_t slot, const SlotLayout& SL, uint32_t row0,
                                            uint32_t row, float v) {
    if (FMT == DOSE_FMT_U16_SCALE) return __fmul_rn(p.scale, v);
    if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) return __fmul_rn(slot_vec(slot, SL, p.vecs, 0, row0, row), v);
    return v;
}

// Sum over the entries kb, kb + step, ... < ke (plain or compensated).
template <int FMT, bool COMP, bool XSMEM, uint32_t IW>
__device__ __forceinline__ void row_dot(const SlotView& v, uint32_t xs, const float* __restrict__ xg, uint32_t kb,
                                        uint32_t ke, uint32_t step, bool comp_row, float& sum, float& comp) {
    if (COMP && comp_row) {
        dot_strided_comp<FMT, IW>(v, xs, xg, XSMEM, kb, ke, step, sum, comp);
    } else {
        const float t = XSMEM ? dot_strided<FMT, IW>(v, xs, kb, ke, step) : dot_strided_gx<FMT, IW>(v, xg, kb, ke, step);
        if (COMP) {
            float u, e;
            dev::two_sum(sum, t, u, e);
            sum = u;
            comp = __fadd_rn(comp, e);
        } else {
            sum = __fadd_rn(sum, t);
        }
    }
}

// The non-empty rows of a NORMAL stage, 2^LG lanes per row.  The stage's list
// is dealt round-robin to the CTA's G groups, starting `rotw` warps further on.
template <int FMT, bool COMP, bool XSMEM, uint32_t IW, uint32_t LG>
__device__ __forceinline__ void normal_rows(const SpmvParams& p, const StageDesc& D, const SlotView& v,
                                            uint32_t slot, const SlotLayout& SL, uint32_t xs_a,
                                            const SlotPtrs<FMT, IW>& sp, const float* xsp, uint32_t zc,
                                            uint32_t ctid, uint32_t lane, uint32_t nct, uint32_t rotw) {
    constexpr uint32_t L = 1u << LG;
    const uint32_t gid = ctid >> LG, li = lane & (L - 1), G = nct >> LG;
    const uint32_t j0 = (gid + G - ((rotw << (5 - LG)) & (G - 1))) & (G - 1);
    const uint32_t n_ne = D.ne1 - D.ne0;
    for (uint32_t base = 0; base < n_ne; base += G) {
        const uint32_t i = base + j0;
        const bool has = i < n_ne;
        float sum = 0.f, comp = 0.f;
        // groups without a row read the stage's first entries (masked) and write nothing
        uint32_t row = 0, rs = D.nz0, re = D.nz0;
        if (has) {
            row = D.row0 + dev::lds_u16(v.ne + 2 * i);
            rs = dev::lds_u32(v.rp + 4 * row);
            re = dev::lds_u32(v.rp + 4 * row + 4);
        }
        if (XSMEM && !COMP) {
            // one trip count for the whole warp: no divergent loop tails
            const uint32_t span = re > rs ? re - (rs & ~3u) : 0;
            const uint32_t iters = __reduce_max_sync(0xffffffffu, (span + 4 * L - 1) / (4 * L));
            sum = dot_vec_p<FMT, L, IW>(sp, xsp, zc, rs, re, li, iters);
        } else if (has) {
            if (COMP && re - rs > kCompThreshold)
                dot_strided_comp<FMT, IW>(v, xs_a, p.x, XSMEM, rs + li, re, L, sum, comp);
            else
                sum = XSMEM ? dot_fixed<FMT, L, IW>(v, xs_a, rs + li, re) : dot_strided_gx<FMT, IW>(v, p.x, rs + li, re, L);
        }
        group_reduce<COMP>(sum, comp, L);
        if (has && li == 0) p.d[row] = row_result<FMT>(p, slot, SL, D.row0, row, COMP ? __fadd_rn(sum, comp) : sum);
    }
}

template <int FMT, bool COMP, bool XSMEM, uint32_t IW>
__global__ void __launch_bounds__(544, 1) spmv_kernel(const SpmvParams p) {
    using T = typename Fmt<FMT>::T;
    extern __shared__ __align__(128) unsigned char smem[];

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth, W = p.cwarps;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + S;
    uint64_t* dbar = full + 16;                         // 2 descriptor-window barriers
    float* red = reinterpret_cast<float*>(smem + 256);  // 64 floats: CTA reduction
    StageDesc* dwin = reinterpret_cast<StageDesc*>(smem + 1024);  // 2 x kDescWin descriptors
    float* xs = reinterpret_cast<float*>(smem + kHeaderBytes);
    const uint32_t x_bytes = XSMEM ? round_up((p.xcols + 1) * 4, 128) : 0;  // x (window) and one zero element
    unsigned char* slot_base = smem + kHeaderBytes + x_bytes;
    const SlotLayout SL = slot_layout(p.tile_nnz, p.tile_rows, sizeof(T), p.vecs.n, false, IW);

    const uint32_t s_begin = p.sched.cta_begin[blockIdx.x];
    const uint32_t s_end = p.sched.cta_begin[blockIdx.x + 1];

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
            run_producer<FMT, IW>(p.sched, s_begin, s_end, p.row_ptr, p.col, p.val, p.vecs, slot_base, SL, full,
                              empty, S, dwin, dbar, p.l2pf, p.err);
        return;
    }

    // -------------------- consumers
    const uint32_t cw = warp - 1;
    const uint32_t ctid = threadIdx.x - 32;
    const uint32_t nct = W * 32;
    // x, or this CTA's window [wlo, wlo + xcols) of it, then a zero element; the
    // base is moved down by wlo words, so shifted_base + column lands in place
    // (shared addresses wrap mod 2^32; the generic pointer is only offset)
    const uint32_t wlo = p.sched.wlo ? p.sched.wlo[blockIdx.x] : 0u;
    if (XSMEM) {
        for (uint32_t j = ctid; j <= p.xcols; j += nct)
            xs[j] = (j < p.xcols && wlo + j < p.ncols) ? __ldg(p.x + wlo + j) : 0.f;
        dev::named_barrier(1, nct);
    }
    const uint32_t xs_a = dev::smem_u32(xs) - 4u * wlo;
    const float* xsw = xs - wlo;
    const uint32_t zc = wlo + p.xcols;  // the zero element's column
    const uint32_t slot0 = dev::smem_u32(slot_base);
    float coop_s = 0.f, coop_c = 0.f;

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

        if (!(D.meta & STAGE_COOP)) {
            // empty rows: write 0 (coalesced)
            for (uint32_t r = D.row0 + ctid; r < D.row1; r += nct)
                if (dev::lds_u32(v.rp + 4 * r) == dev::lds_u32(v.rp + 4 * r + 4)) p.d[r] = 0.0f;
            // non-empty rows: groups of L lanes (L chosen per stage)
            const uint32_t rotw = s & (W - 1);
            switch (D.meta & STAGE_LANES_MASK) {
                case 0: normal_rows<FMT, COMP, XSMEM, IW, 0>(p, D, v, slot, SL, xs_a, sp, xsw, zc, ctid, lane, nct, rotw); break;
                case 1: normal_rows<FMT, COMP, XSMEM, IW, 1>(p, D, v, slot, SL, xs_a, sp, xsw, zc, ctid, lane, nct, rotw); break;
                case 2: normal_rows<FMT, COMP, XSMEM, IW, 2>(p, D, v, slot, SL, xs_a, sp, xsw, zc, ctid, lane, nct, rotw); break;
                case 3: normal_rows<FMT, COMP, XSMEM, IW, 3>(p, D, v, slot, SL, xs_a, sp, xsw, zc, ctid, lane, nct, rotw); break;
                case 4: normal_rows<FMT, COMP, XSMEM, IW, 4>(p, D, v, slot, SL, xs_a, sp, xsw, zc, ctid, lane, nct, rotw); break;
                default: normal_rows<FMT, COMP, XSMEM, IW, 5>(p, D, v, slot, SL, xs_a, sp, xsw, zc, ctid, lane, nct, rotw); break;
            }
        } else {
            // one chunk of a long row, reduced by every consumer thread
            if (D.meta & STAGE_FIRST) {
                coop_s = 0.f;
                coop_c = 0.f;
            }
            row_dot<FMT, COMP, XSMEM, IW>(v, xs_a, p.x, D.nz0 + ctid, D.nz1, nct, true, coop_s, coop_c);
            if (D.meta & STAGE_LAST) {
                float sum = coop_s, comp = coop_c;
                group_reduce<COMP>(sum, comp, 32);
                if (lane == 0) {
                    red[cw] = sum;
                    red[32 + cw] = comp;
                }
                dev::named_barrier(1, nct);
                if (ctid == 0) {
                    float tot = red[0], tc = red[32];
                    for (uint32_t w2 = 1; w2 < W; ++w2) {
                        if (COMP) {
                            float t, e;
                            dev::two_sum(tot, red[w2], t, e);
                            tot = t;
                            tc = __fadd_rn(__fadd_rn(tc, red[32 + w2]), e);
                        } else {
                            tot = __fadd_rn(tot, red[w2]);
                        }
                    }
                    p.d[D.row0] = row_result<FMT>(p, slot, SL, D.row0, D.row0, COMP ? __fadd_rn(tot, tc) : tot);
                }
                dev::named_barrier(1, nct);
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

template <int FMT, bool COMP, bool XSMEM, uint32_t IW>
cudaError_t launch_t(const dose_matrix* A, const SpmvParams& p, size_t smem, cudaStream_t s) {
    auto k = spmv_kernel<FMT, COMP, XSMEM, IW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<A->fwd.grid, 32 * (p.cwarps + 1), smem, s>>>(p);
    return cudaGetLastError();
}

template <int FMT, uint32_t IW>
cudaError_t launch_iw(const dose_matrix* A, const SpmvParams& p, size_t smem, bool comp, bool xsmem,
                      cudaStream_t s) {
    if (comp)
        return xsmem ? launch_t<FMT, true, true, IW>(A, p, smem, s) : launch_t<FMT, true, false, IW>(A, p, smem, s);
    return xsmem ? launch_t<FMT, false, true, IW>(A, p, smem, s) : launch_t<FMT, false, false, IW>(A, p, smem, s);
}

template <int FMT>
cudaError_t launch_fmt(const dose_matrix* A, const SpmvParams& p, size_t smem, bool comp, bool xsmem, bool idx16,
                       cudaStream_t s) {
    return idx16 ? launch_iw<FMT, 2>(A, p, smem, comp, xsmem, s) : launch_iw<FMT, 4>(A, p, smem, comp, xsmem, s);
}

}  // namespace

uint32_t spmv_x_cols(const dose_matrix* A) { return A->fwd_windowed ? A->fwd.wwidth : A->ncols; }

bool spmv_x_in_smem(const dose_matrix* A, const Tuning& t) {
    if (!A->fwd_windowed) return A->ncols <= kXSmemMaxCols;
    return A->fwd.wwidth > 0 && spmv_smem_bytes(A, t, true) <= kMaxSmemPerBlock;
}

size_t spmv_smem_bytes(const dose_matrix* A, const Tuning& t, bool x_in_smem) {
    const uint32_t esize = value_bytes(A->fmt);
    const uint32_t nvec = A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0;
    const uint32_t iw = (A->flags & DOSE_CREATE_U16_INDEX) ? 2 : 4;
    const SlotLayout SL = slot_layout(t.tile_nnz, t.tile_rows, esize, nvec, false, iw);
    return kHeaderBytes + (x_in_smem ? round_up((spmv_x_cols(A) + 1) * 4, 128) : 0) + (size_t)t.stages * SL.bytes;
}

cudaError_t launch_spmv(const dose_matrix* A, const float* x, float* d, cudaStream_t s) {
    if (A->nrows == 0) return cudaSuccess;
    SpmvParams p;
    const bool idx16 = (A->flags & DOSE_CREATE_U16_INDEX) != 0;
    p.row_ptr = A->row_ptr;
    p.col = idx16 ? static_cast<const void*>(A->col16) : static_cast<const void*>(A->col);
    p.val = A->val;
    p.scale = A->scale;
    p.x = x;
    p.d = d;
    p.nrows = A->nrows;
    p.ncols = A->ncols;
    p.xcols = spmv_x_cols(A);
    p.sched = ScheduleView{A->fwd.desc, A->fwd.ne, A->fwd.cta_begin, A->fwd_windowed ? A->fwd.wlo : nullptr};
    p.vecs.n = 0;
    if (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE) {  // library-owned, padded: every row can be copied
        p.vecs.n = 1;
        p.vecs.ptr[0] = A->row_scale;
        p.vecs.lim[0] = round_up(A->nrows, 4);
    }
    p.tile_nnz = A->fwd.tuning.tile_nnz;
    p.tile_rows = A->fwd.tuning.tile_rows;
    p.depth = A->fwd.tuning.stages;
    p.cwarps = A->fwd.tuning.consumer_warps;
    p.l2pf = A->fwd.tuning.l2_prefetch;
    p.err = A->err;
    const bool xsmem = spmv_x_in_smem(A, A->fwd.tuning);
    const size_t smem = spmv_smem_bytes(A, A->fwd.tuning, xsmem);
    const bool comp = (A->flags & DOSE_CREATE_COMPENSATED) != 0;
    switch (A->fmt) {
        case DOSE_FMT_U16_SCALE: return launch_fmt<DOSE_FMT_U16_SCALE>(A, p, smem, comp, xsmem, idx16, s);
        case DOSE_FMT_BF16: return launch_fmt<DOSE_FMT_BF16>(A, p, smem, comp, xsmem, idx16, s);
        case DOSE_FMT_F16: return launch_fmt<DOSE_FMT_F16>(A, p, smem, comp, xsmem, idx16, s);
        case DOSE_FMT_F32: return launch_fmt<DOSE_FMT_F32>(A, p, smem, comp, xsmem, idx16, s);
        case DOSE_FMT_FP8E4M3_ROWSCALE:
            return launch_fmt<DOSE_FMT_FP8E4M3_ROWSCALE>(A, p, smem, comp, xsmem, idx16, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dose
