// Dose SpMV with double-precision vectors, d = A x with x and d in FP64
// (Sec. II-D: the optimiser needs the spot weights and the dose in double
// precision while the matrix is stored in 16 bits; Sec. IV: the "Half/double"
// kernel, half-precision values with double vectors).
//
// GB300 design.  The pipeline is the FP32 forward kernel's: persistent CTAs on
// the forward schedule, a producer warp streaming each row block's row_ptr /
// non-empty-row list / value / column slices into a shared-memory ring with
// bulk async copies, consumer groups of L lanes per row, and a whole-CTA
// reduction of long rows.  What changes is the arithmetic.  GB300 executes FP64
// at a small fraction of its FP32 rate, so an FP64 FMA per entry (the paper's
// arithmetic) would make this memory-bound kernel compute-bound.  The default
// therefore accumulates in double-float, on FP32 instructions only:
//   * x is split once per call into FP32 pairs (hi, lo), hi = fl32(x_j),
//     lo = fl32(x_j - hi), so hi + lo equals x_j to 2^-48 relative;
//   * a decoded value a (at most 24 significant bits, exactly an FP32 number)
//     times x_j is p + e with p = fl(a*hi) and e = fma(a, lo, fma(a, hi, -p)):
//     the inner FMA is the exact error of the product, so p + e equals a*x_j to
//     about 2^-47 relative;
//   * each accumulator is a pair (s, c): s takes p through TwoSum (Knuth), whose
//     exact rounding error goes into c together with e (Dot2 of Ogita, Rump and
//     Oishi); pairs are combined the same way;
//   * the row result is one FP64 addition, d_i = s + c (after the U16 / FP8
//     scale is applied to the pair exactly in the same manner).
// DOSE_SPMV_F64_NATIVE instead converts each decoded value to FP64 and
// accumulates with FP64 FMAs (the paper's arithmetic), to compare the two.
// Every reduction has a fixed shape, so results are bitwise reproducible.
#include "dfloat.cuh"

namespace dose {
namespace {

struct Spmv64Params {
    const uint32_t* row_ptr;
    const void* col;  // column indices of IW bytes
    const void* val;
    float scale;
    const uint2* x;   // ncols + 1 elements of 8 bytes, the last one zero: DF (hi, lo) pairs, DP doubles
    double* d;
    uint32_t nrows, ncols;
    uint32_t xcols;  // columns of x staged per CTA (ncols, or the window width)
    ScheduleView sched;
    VecSet vecs;  // FP8: the row scales
    uint32_t tile_nnz, tile_rows, depth, cwarps, l2pf;
    int* err;
};

constexpr uint32_t kHeaderBytes = 3072;  // mbarriers, CTA reduction scratch, 2 KB of stage descriptors

// x as the kernels read it: ncols pairs (or doubles) and a zero element at
// index ncols, which masked entries of a group read.
template <int MODE>
__global__ void prepare_x_kernel(const double* __restrict__ x, uint2* __restrict__ out, uint32_t n) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n) return;
    const double v = j < n ? x[j] : 0.0;
    if (MODE == F64_DF) {
        const float hi = __double2float_rn(v);
        const float lo = __double2float_rn(v - (double)hi);  // v - hi is exact in FP64
        out[j] = make_uint2(__float_as_uint(hi), __float_as_uint(lo));
    } else {
        out[j] = make_uint2((uint32_t)__double2loint(v), (uint32_t)__double2hiint(v));
    }
}

// Lane li of an L-lane group takes the groups of four consecutive entries at
// (kb & ~3) + 4 li + 4 L s for `iters` steps (the same for the whole warp),
// exactly as the FP32 kernel does: a group past the row's end reloads the row's
// first group, and every entry outside [kb, ke) gets weight 0 and reads x at the
// zero element zc.  Four accumulators, combined as (0 + 1) + (2 + 3).
template <int FMT, int MODE, uint32_t L, uint32_t IW>
__device__ __forceinline__ Acc<MODE> dot_vec64(const SlotPtrs<FMT, IW>& sp, const uint2* __restrict__ xsp, uint32_t zc,
                                               uint32_t kb, uint32_t ke, uint32_t li, uint32_t iters) {
    Acc<MODE> acc[4];
    const int len = (int)(ke - kb);
    const uint32_t kb4 = kb & ~3u;
    int off = (int)(4 * li) - (int)(kb & 3u);
    uint32_t k4 = kb4 + 4 * li;
    for (uint32_t it = 0; it < iters; ++it, off += 4 * L, k4 += 4 * L) {
        const uint32_t kg = off < len ? k4 : kb4;
        uint32_t c[4];
        if (IW == 4) {
            const uint4 cc = *reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(sp.col) + kg);
            c[0] = cc.x; c[1] = cc.y; c[2] = cc.z; c[3] = cc.w;
        } else {
            const uint2 cc = *reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(sp.col) + kg);
            c[0] = cc.x & 0xFFFFu; c[1] = cc.x >> 16; c[2] = cc.y & 0xFFFFu; c[3] = cc.y >> 16;
        }
        float a[4];
        load_vals4<FMT>(sp.val + kg, a);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool m = (uint32_t)(off + u) < (uint32_t)len;
            acc[u].mac(m ? a[u] : 0.f, xsp, m ? c[u] : zc);
        }
    }
    acc[0].add(acc[1]);
    acc[2].add(acc[3]);
    acc[0].add(acc[2]);
    return acc[0];
}

template <int FMT>
__device__ __forceinline__ float row_scale(const Spmv64Params& p, uint32_t slot, const SlotLayout& SL, uint32_t row0,
                                           uint32_t row) {
    if (FMT == DOSE_FMT_U16_SCALE) return p.scale;
    if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) return slot_vec(slot, SL, p.vecs, 0, row0, row);
    return 1.0f;
}

constexpr bool fmt_scaled(int fmt) { return fmt == DOSE_FMT_U16_SCALE || fmt == DOSE_FMT_FP8E4M3_ROWSCALE; }

// The non-empty rows of a NORMAL stage, 2^LG lanes per row (dealt as in the
// FP32 kernel).
template <int FMT, int MODE, uint32_t IW, uint32_t LG>
__device__ __forceinline__ void normal_rows64(const Spmv64Params& p, const StageDesc& D, const SlotView& v,
                                              uint32_t slot, const SlotLayout& SL, const SlotPtrs<FMT, IW>& sp,
                                              const uint2* xsp, uint32_t zc, uint32_t ctid, uint32_t lane,
                                              uint32_t nct, uint32_t rotw) {
    constexpr uint32_t L = 1u << LG;
    const uint32_t gid = ctid >> LG, li = lane & (L - 1), G = nct >> LG;
    const uint32_t j0 = (gid + G - ((rotw << (5 - LG)) & (G - 1))) & (G - 1);
    const uint32_t n_ne = D.ne1 - D.ne0;
    for (uint32_t base = 0; base < n_ne; base += G) {
        const uint32_t i = base + j0;
        const bool has = i < n_ne;
        uint32_t row = 0, rs = D.nz0, re = D.nz0;  // groups without a row read masked entries
        if (has) {
            row = D.row0 + dev::lds_u16(v.ne + 2 * i);
            rs = dev::lds_u32(v.rp + 4 * row);
            re = dev::lds_u32(v.rp + 4 * row + 4);
        }
        const uint32_t span = re > rs ? re - (rs & ~3u) : 0;
        const uint32_t iters = __reduce_max_sync(0xffffffffu, (span + 4 * L - 1) / (4 * L));
        Acc<MODE> a = dot_vec64<FMT, MODE, L, IW>(sp, xsp, zc, rs, re, li, iters);
        for (uint32_t o = L >> 1; o > 0; o >>= 1) a.add(a.shfl_xor(o));
        if (has && li == 0) p.d[row] = a.result(fmt_scaled(FMT), row_scale<FMT>(p, slot, SL, D.row0, row));
    }
}

template <int FMT, int MODE, bool XSMEM, uint32_t IW>
__global__ void __launch_bounds__(544, 1) spmv_f64_kernel(const Spmv64Params p) {
    using T = typename Fmt<FMT>::T;
    constexpr uint32_t ES = (uint32_t)sizeof(T);
    extern __shared__ __align__(128) unsigned char smem[];

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth, W = p.cwarps;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + S;
    uint64_t* dbar = full + 16;                        // 2 descriptor-window barriers
    uint2* red = reinterpret_cast<uint2*>(smem + 256);  // 32 x 8 bytes: CTA reduction
    StageDesc* dwin = reinterpret_cast<StageDesc*>(smem + 1024);
    uint2* xs = reinterpret_cast<uint2*>(smem + kHeaderBytes);
    const uint32_t x_bytes = XSMEM ? round_up((p.xcols + 1) * 8, 128) : 0;
    unsigned char* slot_base = smem + kHeaderBytes + x_bytes;
    const SlotLayout SL = slot_layout(p.tile_nnz, p.tile_rows, ES, p.vecs.n, false, IW);

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
    // x, or this CTA's window [wlo, wlo + xcols) of it, then a zero element,
    // addressed by column through a pointer moved down by wlo elements
    const uint32_t wlo = p.sched.wlo ? p.sched.wlo[blockIdx.x] : 0u;
    if (XSMEM) {
        for (uint32_t j = ctid; j <= p.xcols; j += nct)
            xs[j] = (j < p.xcols && wlo + j < p.ncols) ? __ldg(p.x + wlo + j) : make_uint2(0u, 0u);
        dev::named_barrier(1, nct);
    }
    const uint2* xsp = XSMEM ? xs - wlo : p.x;
    const uint32_t zc = XSMEM ? wlo + p.xcols : p.ncols;  // the zero element's column
    const uint32_t slot0 = dev::smem_u32(slot_base);
    Acc<MODE> coop;

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
            for (uint32_t r = D.row0 + ctid; r < D.row1; r += nct)
                if (dev::lds_u32(v.rp + 4 * r) == dev::lds_u32(v.rp + 4 * r + 4)) p.d[r] = 0.0;
            const uint32_t rotw = s & (W - 1);
            switch (D.meta & STAGE_LANES_MASK) {
                case 0: normal_rows64<FMT, MODE, IW, 0>(p, D, v, slot, SL, sp, xsp, zc, ctid, lane, nct, rotw); break;
                case 1: normal_rows64<FMT, MODE, IW, 1>(p, D, v, slot, SL, sp, xsp, zc, ctid, lane, nct, rotw); break;
                case 2: normal_rows64<FMT, MODE, IW, 2>(p, D, v, slot, SL, sp, xsp, zc, ctid, lane, nct, rotw); break;
                case 3: normal_rows64<FMT, MODE, IW, 3>(p, D, v, slot, SL, sp, xsp, zc, ctid, lane, nct, rotw); break;
                case 4: normal_rows64<FMT, MODE, IW, 4>(p, D, v, slot, SL, sp, xsp, zc, ctid, lane, nct, rotw); break;
                default: normal_rows64<FMT, MODE, IW, 5>(p, D, v, slot, SL, sp, xsp, zc, ctid, lane, nct, rotw); break;
            }
        } else {
            // one chunk of a long row: every consumer thread takes entries
            // nz0 + ctid, + nct, ...; the partials are combined at its last chunk
            if (D.meta & STAGE_FIRST) coop = Acc<MODE>();
            for (uint32_t k = D.nz0 + ctid; k < D.nz1; k += nct)
                coop.mac(Fmt<FMT>::lds(v.val + ES * k), xsp, col_at<IW>(v, k));
            if (D.meta & STAGE_LAST) {
                Acc<MODE> a = coop;
                for (uint32_t o = 16; o > 0; o >>= 1) a.add(a.shfl_xor(o));
                if (lane == 0) red[cw] = a.pack();
                dev::named_barrier(1, nct);
                if (ctid == 0) {
                    Acc<MODE> tot = Acc<MODE>::unpack(red[0]);
                    for (uint32_t w2 = 1; w2 < W; ++w2) tot.add(Acc<MODE>::unpack(red[w2]));
                    p.d[D.row0] = tot.result(fmt_scaled(FMT), row_scale<FMT>(p, slot, SL, D.row0, D.row0));
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

template <int FMT, int MODE, bool XSMEM, uint32_t IW>
cudaError_t launch_t(const dose_matrix* A, const Spmv64Params& p, size_t smem, cudaStream_t s) {
    auto k = spmv_f64_kernel<FMT, MODE, XSMEM, IW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(A->fwd64_own ? A->fwd64 : A->fwd).grid, 32 * (p.cwarps + 1), smem, s>>>(p);
    return cudaGetLastError();
}

template <int FMT, int MODE>
cudaError_t launch_mode(const dose_matrix* A, const Spmv64Params& p, size_t smem, bool xsmem, bool idx16,
                        cudaStream_t s) {
    if (idx16) return xsmem ? launch_t<FMT, MODE, true, 2>(A, p, smem, s) : launch_t<FMT, MODE, false, 2>(A, p, smem, s);
    return xsmem ? launch_t<FMT, MODE, true, 4>(A, p, smem, s) : launch_t<FMT, MODE, false, 4>(A, p, smem, s);
}

template <int FMT>
cudaError_t launch_fmt(const dose_matrix* A, const Spmv64Params& p, size_t smem, bool native, bool xsmem, bool idx16,
                       cudaStream_t s) {
    return native ? launch_mode<FMT, F64_DP>(A, p, smem, xsmem, idx16, s)
                  : launch_mode<FMT, F64_DF>(A, p, smem, xsmem, idx16, s);
}

}  // namespace

// The schedule dose_spmv_f64 runs on.
static const DevSchedule& f64_schedule(const dose_matrix* A) { return A->fwd64_own ? A->fwd64 : A->fwd; }

size_t spmv_f64_smem_bytes(const dose_matrix* A, bool x_in_smem) {
    const Tuning& t = f64_schedule(A).tuning;
    const uint32_t esize = value_bytes(A->fmt);
    const uint32_t nvec = A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0;
    const uint32_t iw = (A->flags & DOSE_CREATE_U16_INDEX) ? 2 : 4;
    const SlotLayout SL = slot_layout(t.tile_nnz, t.tile_rows, esize, nvec, false, iw);
    const uint32_t xcols = A->fwd64_own ? A->ncols : spmv_x_cols(A);
    return kHeaderBytes + (x_in_smem ? round_up((xcols + 1) * 8, 128) : 0) + (size_t)t.stages * SL.bytes;
}

bool spmv_f64_x_in_smem(const dose_matrix* A) {
    if (A->fwd64_own) return false;
    return spmv_x_cols(A) > 0 && spmv_f64_smem_bytes(A, true) <= kMaxSmemPerBlock;
}

cudaError_t launch_spmv_f64(const dose_matrix* A, const double* x, double* d, bool native, cudaStream_t s) {
    if (A->nrows == 0) return cudaSuccess;
    const uint32_t nx = A->ncols + 1;
    if (native)
        prepare_x_kernel<F64_DP><<<(nx + 255) / 256, 256, 0, s>>>(x, A->x64, A->ncols);
    else
        prepare_x_kernel<F64_DF><<<(nx + 255) / 256, 256, 0, s>>>(x, A->x64, A->ncols);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the row-group form only when the caller asks for it (fwd_layout = 2): this
    // kernel is bound by its arithmetic, not its bytes, and the layout's 1.17
    // stored values per entry cost more than its fewer bytes save (clinical
    // beam, F16: 0.228 ms on row groups against 0.221 ms on CSR)
    if (A->fwd.tuning.layout == 2 && spmv_on_row_groups(A) && rg_spmv64_applies(A, nullptr, nullptr))
        return launch_rg_spmv64(A, A->x64, d, native, s);
    Spmv64Params p;
    const bool idx16 = (A->flags & DOSE_CREATE_U16_INDEX) != 0;
    p.row_ptr = A->row_ptr;
    p.col = idx16 ? static_cast<const void*>(A->col16) : static_cast<const void*>(A->col);
    p.val = A->val;
    p.scale = A->scale;
    p.x = A->x64;
    p.d = d;
    p.nrows = A->nrows;
    p.ncols = A->ncols;
    const DevSchedule& F = f64_schedule(A);
    const bool win = A->fwd_windowed && !A->fwd64_own;
    p.xcols = win ? A->fwd.wwidth : A->ncols;
    p.sched = ScheduleView{F.desc, F.ne, F.cta_begin, win ? F.wlo : nullptr};
    p.vecs.n = 0;
    if (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE) {
        p.vecs.n = 1;
        p.vecs.ptr[0] = A->row_scale;
        p.vecs.lim[0] = round_up(A->nrows, 4);
    }
    p.tile_nnz = F.tuning.tile_nnz;
    p.tile_rows = F.tuning.tile_rows;
    p.depth = F.tuning.stages;
    p.cwarps = F.tuning.consumer_warps;
    p.l2pf = F.tuning.l2_prefetch;
    p.err = A->err;
    const bool xsmem = spmv_f64_x_in_smem(A);
    const size_t smem = spmv_f64_smem_bytes(A, xsmem);
    switch (A->fmt) {
        case DOSE_FMT_U16_SCALE: return launch_fmt<DOSE_FMT_U16_SCALE>(A, p, smem, native, xsmem, idx16, s);
        case DOSE_FMT_BF16: return launch_fmt<DOSE_FMT_BF16>(A, p, smem, native, xsmem, idx16, s);
        case DOSE_FMT_F16: return launch_fmt<DOSE_FMT_F16>(A, p, smem, native, xsmem, idx16, s);
        case DOSE_FMT_F32: return launch_fmt<DOSE_FMT_F32>(A, p, smem, native, xsmem, idx16, s);
        case DOSE_FMT_FP8E4M3_ROWSCALE:
            return launch_fmt<DOSE_FMT_FP8E4M3_ROWSCALE>(A, p, smem, native, xsmem, idx16, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dose
