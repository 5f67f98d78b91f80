// Batched dose SpMM: D_m = A_m X_m for many matrices (beams x uncertainty
// scenarios) and up to 16 spot-weight vectors per matrix, in one persistent
// launch.  The optimiser evaluates the dose of several beams, possibly under
// several realisations of the uncertainties, in every iteration (Sec. I); each
// beam has its own dose-deposition matrix (Sec. II-B).
//
// Staged form (the default): one persistent CTA per SM walks the matrices in
// order, and for each one its own share of that matrix's row blocks, using the
// matrix's column-windowed schedule (the one the adjoint uses).  A producer
// warp streams the row blocks through one shared-memory ring that runs on from
// matrix to matrix.  The consumer warps hold the CTA's window of X_m (window x
// 4 NQ floats, NQ = ceil(nvec / 4)), so each entry's 16 weights are one
// 64-byte shared-memory gather.  Lanes form (slot, quad) pairs: a row is
// reduced by `slots` entry slots x NQ quads of vectors; slot e takes the
// entries kb + e, kb + e + slots, ... (consecutive slots read consecutive
// columns, so the 64-byte gathers of one instruction spread over both halves of
// the banks), and the slots are combined by a fixed shuffle tree.
//
// Global form (fallback, when a CTA's window of X does not fit in shared
// memory): a half-warp per row, X gathered from global memory (L1/L2).
//
// Both forms are deterministic: static work assignment, fixed reduction trees.
#include "stage_common.cuh"

#include <algorithm>
#include <string>

namespace dose {
namespace {

constexpr int kMaxBatchPerLaunch = 64;
constexpr uint32_t kSpmmConsumerWarps = 16;
constexpr uint32_t kSpmmHeader = 3072;  // mbarriers, 2 KB of stage descriptors

// ------------------------------------------------------------ staged form

struct StagedItem {
    const uint32_t* row_ptr;
    const uint32_t* col;
    const void* val;
    const float* row_scale;  // FP8 only (padded: every row can be copied)
    const float* X;          // ncols x nvec, row-major
    float* D;                // nrows x nvec, row-major
    ScheduleView sched;      // column-windowed schedule
    float scale;
    uint32_t nrows, ncols, wwidth, tile_nnz, tile_rows;
    int fmt;
};

struct StagedParams {
    StagedItem item[kMaxBatchPerLaunch];
    uint32_t count, nvec, depth, slot_stride, l2pf;
    uint32_t vec4;  // nvec % 4 == 0 and every D 16-byte aligned: rows of D stored as float4
    int* err;
};

__device__ __forceinline__ uint32_t esize_of(int fmt) { return value_bytes(fmt); }

__device__ __forceinline__ VecSet item_vecs(const StagedItem& it) {
    VecSet v;
    v.n = 0;
    if (it.fmt == DOSE_FMT_FP8E4M3_ROWSCALE) {
        v.n = 1;
        v.ptr[0] = it.row_scale;
        v.lim[0] = round_up(it.nrows, 4);
    }
    return v;
}

// Bytes between the rows of the X window: NQ quads of 16 bytes.  (A padded
// 80-byte row for NQ = 4 puts the rows of columns c and c + 4 in opposite bank
// halves, but the wider window left room for fewer ring slots and measured
// slower on pencil beams.)
template <uint32_t NQ>
__host__ __device__ constexpr uint32_t xrow_bytes() { return NQ * 16u; }

// Window row of X that holds column c (window-relative): rows are swapped in
// pairs when bit 2 of c is set, so the rows of columns c and c + 4 (read by
// neighbouring entry slots in one instruction) lie in opposite halves of the
// banks.  An involution that maps every multiple of 8 to itself, so the
// window (a multiple of 32 columns) and its zero row keep their places.
__device__ __forceinline__ uint32_t xrow_swz(uint32_t c) { return c ^ ((c >> 2) & 1u); }

// D rows of one group of L = SLOTS * NQ lanes; lanes (e, q): e = entry slot,
// q = quad of vectors.  Slot e takes the groups of four consecutive entries at
// (kb & ~3) + 4 e + 4 SLOTS s (one 16-byte column load, one value load);
// `iters` (warp-uniform) steps.  Plain typed shared-memory loads (the slot's
// data were released by the mbarrier wait, a compiler barrier).
template <int FMT, uint32_t NQ, uint32_t SLOTS>
__device__ __forceinline__ void spmm_rows(const StagedItem& it, const StageDesc& D, const uint32_t* __restrict__ colp,
                                          const typename Fmt<FMT>::T* __restrict__ valp,
                                          const uint32_t* __restrict__ rpp, const uint16_t* __restrict__ nep,
                                          const float4* __restrict__ xw4, uint32_t wlo, uint32_t nvec, bool vec4,
                                          float rs_row0, const float* __restrict__ rsp, uint32_t ctid, uint32_t lane,
                                          uint32_t rot) {
    using T = typename Fmt<FMT>::T;
    constexpr uint32_t L = SLOTS * NQ;  // lanes per row
    constexpr uint32_t G = kSpmmConsumerWarps * 32 / L;
    const uint32_t li = lane & (L - 1), e = li / NQ, q = li % NQ;
    const uint32_t j0 = (ctid / L + rot) % G;
    const uint32_t n_ne = D.ne1 - D.ne0;
    const uint32_t zrow = it.wwidth;  // the window's all-zero row, read by masked entries
    (void)rs_row0;
    for (uint32_t base = 0; base < n_ne; base += G) {
        const uint32_t i = base + j0;
        const bool has = i < n_ne;
        // lanes without a row read the stage's first aligned group (masked) and write nothing
        uint32_t row = 0, kb = D.nz0, ke = D.nz0;
        if (has) {
            row = D.row0 + nep[i];
            kb = rpp[row];
            ke = rpp[row + 1];
        }
        const int len = (int)(ke - kb);
        const uint32_t kb4 = kb & ~3u;
        const uint32_t span = ke > kb ? ke - kb4 : 0;
        const uint32_t iters = __reduce_max_sync(0xffffffffu, (span + 4 * SLOTS - 1) / (4 * SLOTS));
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        int off = (int)(4 * e) - (int)(kb & 3u);
        uint32_t k4 = kb4 + 4 * e;
        for (uint32_t s2 = 0; s2 < iters; ++s2, off += 4 * SLOTS, k4 += 4 * SLOTS) {
            // a group outside the row reads the row's first group instead (always in the slot)
            const uint32_t kg = off < len ? k4 : kb4;
            const uint4 cc = *reinterpret_cast<const uint4*>(colp + kg);
            float av[4];
            load_vals4<FMT>(valp + kg, av);
            const uint32_t cu[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool m = (uint32_t)(off + u) < (uint32_t)len;
                const uint32_t c = m ? xrow_swz(cu[u] - wlo) : zrow;
                const float a = m ? av[u] : 0.f;
                const float4 x = xw4[c * NQ + q];
                acc.x = __fmaf_rn(a, x.x, acc.x);
                acc.y = __fmaf_rn(a, x.y, acc.y);
                acc.z = __fmaf_rn(a, x.z, acc.z);
                acc.w = __fmaf_rn(a, x.w, acc.w);
            }
        }
#pragma unroll
        for (uint32_t o = NQ; o < L; o <<= 1) {
            acc.x = __fadd_rn(acc.x, __shfl_xor_sync(0xffffffffu, acc.x, o));
            acc.y = __fadd_rn(acc.y, __shfl_xor_sync(0xffffffffu, acc.y, o));
            acc.z = __fadd_rn(acc.z, __shfl_xor_sync(0xffffffffu, acc.z, o));
            acc.w = __fadd_rn(acc.w, __shfl_xor_sync(0xffffffffu, acc.w, o));
        }
        if (has && e == 0) {
            float sc = 1.0f;
            if (FMT == DOSE_FMT_U16_SCALE) sc = it.scale;
            if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) sc = rsp[row];
            const float r4[4] = {__fmul_rn(sc, acc.x), __fmul_rn(sc, acc.y), __fmul_rn(sc, acc.z),
                                 __fmul_rn(sc, acc.w)};
            float* dst = it.D + (size_t)row * nvec;
            if (vec4) {
                // nvec = 12 runs four quads: the fourth lies past the row
                if (4 * q < nvec) *reinterpret_cast<float4*>(dst + 4 * q) = make_float4(r4[0], r4[1], r4[2], r4[3]);
            } else {
#pragma unroll
                for (uint32_t u = 0; u < 4; ++u)
                    if (4 * q + u < nvec) dst[4 * q + u] = r4[u];
            }
        }
    }
}

// One stage of matrix `it` by all consumer threads.
template <int FMT, uint32_t NQ>
__device__ __forceinline__ void spmm_stage(const StagedItem& it, const SlotLayout& SL, unsigned char* slotp,
                                           uint32_t slot, const float4* xw4, uint32_t xw, uint32_t wlo,
                                           uint32_t nvec, bool vec4, uint32_t ctid, uint32_t lane, uint32_t cw,
                                           uint32_t nct, uint32_t rot) {
    using T = typename Fmt<FMT>::T;
    constexpr uint32_t VA = Fmt<FMT>::kAlign;
    const StageDesc D = slot_desc(slot);
    // typed views of the slot, indexed by global entry / row / list position
    const uint32_t* colp = reinterpret_cast<const uint32_t*>(slotp + SL.col_off) - (D.nz0 & ~3u);
    const T* valp = reinterpret_cast<const T*>(slotp + SL.val_off) - (D.nz0 & ~(VA - 1));
    const uint32_t* rpp = reinterpret_cast<const uint32_t*>(slotp + SL.rp_off) - (D.row0 & ~3u);
    const uint16_t* nep = reinterpret_cast<const uint16_t*>(slotp + SL.ne_off) + (D.ne0 & 7u);  // [i], i in the stage's list
    const float* rsp = reinterpret_cast<const float*>(slotp + SL.vec_off) - (D.row0 & ~3u);
    if (!(D.meta & STAGE_COOP)) {
        // empty rows: zero rows of D
        for (uint32_t r = D.row0 + ctid; r < D.row1; r += nct)
            if (rpp[r] == rpp[r + 1]) {
                float* dst = it.D + (size_t)r * nvec;
                if (vec4)
                    for (uint32_t u = 0; u < nvec; u += 4) *reinterpret_cast<float4*>(dst + u) = make_float4(0.f, 0.f, 0.f, 0.f);
                else
                    for (uint32_t u = 0; u < nvec; ++u) dst[u] = 0.f;
            }
        // entry slots per row from the stage's mean row length (about 16 entries per slot)
        const uint32_t n_ne = D.ne1 - D.ne0;
        const uint32_t mean = n_ne ? (D.nz1 - D.nz0) / n_ne : 0;
        constexpr uint32_t kMaxLg = NQ == 1 ? 5 : NQ == 2 ? 4 : 3;  // up to 32 lanes per row
        uint32_t lg = 0;
        while (lg < kMaxLg && (16u << lg) < mean) ++lg;
        switch (lg) {
            case 0: spmm_rows<FMT, NQ, 1>(it, D, colp, valp, rpp, nep, xw4, wlo, nvec, vec4, 0.f, rsp, ctid, lane, rot); break;
            case 1: spmm_rows<FMT, NQ, 2>(it, D, colp, valp, rpp, nep, xw4, wlo, nvec, vec4, 0.f, rsp, ctid, lane, rot); break;
            case 2: spmm_rows<FMT, NQ, 4>(it, D, colp, valp, rpp, nep, xw4, wlo, nvec, vec4, 0.f, rsp, ctid, lane, rot); break;
            case 3: spmm_rows<FMT, NQ, 8>(it, D, colp, valp, rpp, nep, xw4, wlo, nvec, vec4, 0.f, rsp, ctid, lane, rot); break;
            case 4: spmm_rows<FMT, NQ, (16 <= 32 / NQ ? 16 : 32 / NQ)>(it, D, colp, valp, rpp, nep, xw4, wlo, nvec, vec4, 0.f, rsp, ctid, lane, rot); break;
            default: spmm_rows<FMT, NQ, 32 / NQ>(it, D, colp, valp, rpp, nep, xw4, wlo, nvec, vec4, 0.f, rsp, ctid, lane, rot); break;
        }
    } else if ((D.meta & STAGE_FIRST) && cw == 0) {
        // a row longer than the stage limit: consumer warp 0 reduces all of it
        // from global memory once, at its first chunk (lanes (e, q) as above)
        using T = typename Fmt<FMT>::T;
        const T* val = static_cast<const T*>(it.val);
        constexpr uint32_t SL32 = 32 / NQ;
        const uint32_t e = lane / NQ, q = lane % NQ;
        const uint32_t row = D.row0;
        const uint32_t kb = __ldg(it.row_ptr + row), ke = __ldg(it.row_ptr + row + 1);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (uint32_t k = kb + e; k < ke; k += SL32) {
            const uint32_t c = xrow_swz(__ldg(it.col + k) - wlo);
            const float a = Fmt<FMT>::dec(val[k]);
            float4 x;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w)
                         : "r"(xw + c * xrow_bytes<NQ>() + q * 16));
            acc.x = __fmaf_rn(a, x.x, acc.x);
            acc.y = __fmaf_rn(a, x.y, acc.y);
            acc.z = __fmaf_rn(a, x.z, acc.z);
            acc.w = __fmaf_rn(a, x.w, acc.w);
        }
#pragma unroll
        for (uint32_t o = NQ; o < 32; o <<= 1) {
            acc.x = __fadd_rn(acc.x, __shfl_xor_sync(0xffffffffu, acc.x, o));
            acc.y = __fadd_rn(acc.y, __shfl_xor_sync(0xffffffffu, acc.y, o));
            acc.z = __fadd_rn(acc.z, __shfl_xor_sync(0xffffffffu, acc.z, o));
            acc.w = __fadd_rn(acc.w, __shfl_xor_sync(0xffffffffu, acc.w, o));
        }
        if (e == 0) {
            float s = 1.0f;
            if (FMT == DOSE_FMT_U16_SCALE) s = it.scale;
            if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) s = __ldg(it.row_scale + row);
            const float r4[4] = {__fmul_rn(s, acc.x), __fmul_rn(s, acc.y), __fmul_rn(s, acc.z), __fmul_rn(s, acc.w)};
            float* dst = it.D + (size_t)row * nvec;
#pragma unroll
            for (uint32_t u = 0; u < 4; ++u)
                if (4 * q + u < nvec) dst[4 * q + u] = r4[u];
        }
    }
}

template <uint32_t NQ>
__global__ void __launch_bounds__(32 * (kSpmmConsumerWarps + 1), 1) spmm_staged_kernel(const __grid_constant__ StagedParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + 8;
    uint64_t* dbar = full + 16;
    StageDesc* dwin = reinterpret_cast<StageDesc*>(smem + 1024);
    float* xwin = reinterpret_cast<float*>(smem + kSpmmHeader);
    uint32_t xw_bytes = 0;
    for (uint32_t m = 0; m < p.count; ++m)
        xw_bytes = max(xw_bytes, round_up((p.item[m].wwidth + 1) * xrow_bytes<NQ>(), 128));  // + the zero row
    unsigned char* slot_base = smem + kSpmmHeader + xw_bytes;

    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < S; ++i) {
            dev::mbar_init(&full[i], 1);
            dev::mbar_init(&empty[i], kSpmmConsumerWarps);
        }
        dev::mbar_init(&dbar[0], 1);
        dev::mbar_init(&dbar[1], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0) {
            ProducerRing R;
            for (uint32_t m = 0; m < p.count; ++m) {
                const StagedItem& it = p.item[m];
                const uint32_t sb = it.sched.cta_begin[blockIdx.x], se = it.sched.cta_begin[blockIdx.x + 1];
                const VecSet vecs = item_vecs(it);
                const SlotLayout SL = slot_layout(it.tile_nnz, it.tile_rows, esize_of(it.fmt), vecs.n, false);
                switch (it.fmt) {
                    case DOSE_FMT_U16_SCALE:
                        produce_stages<DOSE_FMT_U16_SCALE>(R, it.sched, sb, se, it.row_ptr, it.col, it.val, vecs,
                                                           slot_base, SL, p.slot_stride, full, empty, S, dwin, dbar,
                                                           p.l2pf, p.err);
                        break;
                    case DOSE_FMT_BF16:
                        produce_stages<DOSE_FMT_BF16>(R, it.sched, sb, se, it.row_ptr, it.col, it.val, vecs, slot_base,
                                                      SL, p.slot_stride, full, empty, S, dwin, dbar, p.l2pf, p.err);
                        break;
                    case DOSE_FMT_F16:  // same bytes as BF16: only the decode differs
                        produce_stages<DOSE_FMT_BF16>(R, it.sched, sb, se, it.row_ptr, it.col, it.val, vecs, slot_base,
                                                      SL, p.slot_stride, full, empty, S, dwin, dbar, p.l2pf, p.err);
                        break;
                    case DOSE_FMT_F32:
                        produce_stages<DOSE_FMT_F32>(R, it.sched, sb, se, it.row_ptr, it.col, it.val, vecs, slot_base,
                                                     SL, p.slot_stride, full, empty, S, dwin, dbar, p.l2pf, p.err);
                        break;
                    default:
                        produce_stages<DOSE_FMT_FP8E4M3_ROWSCALE>(R, it.sched, sb, se, it.row_ptr, it.col, it.val,
                                                                  vecs, slot_base, SL, p.slot_stride, full, empty, S,
                                                                  dwin, dbar, p.l2pf, p.err);
                        break;
                }
            }
            producer_drain(R, full, S);
        }
        return;
    }

    const uint32_t cw = warp - 1, ctid = threadIdx.x - 32, nct = kSpmmConsumerWarps * 32;
    const uint32_t xw0 = dev::smem_u32(xwin), slot0 = dev::smem_u32(slot_base);
    const float4* xw4 = reinterpret_cast<const float4*>(xwin);
    uint32_t st = 0, ph = 0, rot = 0;
    for (uint32_t m = 0; m < p.count; ++m) {
        const StagedItem& it = p.item[m];
        const uint32_t sb = it.sched.cta_begin[blockIdx.x], se = it.sched.cta_begin[blockIdx.x + 1];
        if (sb >= se) continue;  // the same for every consumer thread
        const uint32_t wlo = it.sched.wlo[blockIdx.x];
        const SlotLayout SL = slot_layout(it.tile_nnz, it.tile_rows, esize_of(it.fmt),
                                          it.fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1u : 0u, false);
        // this matrix's window of X (quads padded with zeros); the previous
        // matrix's rows are all done before it is overwritten
        dev::named_barrier(1, nct);
        constexpr uint32_t XF = xrow_bytes<NQ>() / 4;  // floats per window row
        for (uint32_t j = ctid; j < (it.wwidth + 1) * XF; j += nct) {  // row wwidth: all zeros
            const uint32_t jc = xrow_swz(j / XF), c = wlo + jc, u = j % XF;  // window row j holds column jc
            xwin[j] = (jc < it.wwidth && c < it.ncols && u < p.nvec) ? __ldg(it.X + (size_t)c * p.nvec + u) : 0.f;
        }
        dev::named_barrier(1, nct);
        for (uint32_t s = sb; s < se; ++s, ++rot) {
            if (!dev::mbar_wait_bounded(&full[st], ph)) {
                atomicExch(p.err, kErrTimeoutFull);
                return;
            }
            const uint32_t slot = slot0 + st * p.slot_stride;
            unsigned char* slotp = slot_base + st * p.slot_stride;
            const uint32_t r = rot & (kSpmmConsumerWarps - 1);
            switch (it.fmt) {
                case DOSE_FMT_U16_SCALE:
                    spmm_stage<DOSE_FMT_U16_SCALE, NQ>(it, SL, slotp, slot, xw4, xw0, wlo, p.nvec, p.vec4 != 0, ctid,
                                                       lane, cw, nct, r);
                    break;
                case DOSE_FMT_BF16:
                    spmm_stage<DOSE_FMT_BF16, NQ>(it, SL, slotp, slot, xw4, xw0, wlo, p.nvec, p.vec4 != 0, ctid, lane,
                                                  cw, nct, r);
                    break;
                case DOSE_FMT_F16:
                    spmm_stage<DOSE_FMT_F16, NQ>(it, SL, slotp, slot, xw4, xw0, wlo, p.nvec, p.vec4 != 0, ctid, lane,
                                                 cw, nct, r);
                    break;
                case DOSE_FMT_F32:
                    spmm_stage<DOSE_FMT_F32, NQ>(it, SL, slotp, slot, xw4, xw0, wlo, p.nvec, p.vec4 != 0, ctid, lane,
                                                 cw, nct, r);
                    break;
                default:
                    spmm_stage<DOSE_FMT_FP8E4M3_ROWSCALE, NQ>(it, SL, slotp, slot, xw4, xw0, wlo, p.nvec,
                                                              p.vec4 != 0, ctid, lane, cw, nct, r);
                    break;
            }
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&empty[st]);
            if (++st == S) {
                st = 0;
                ph ^= 1;
            }
        }
    }
}

// ------------------------------------------------------------ global form

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
        it.D[(size_t)row * nvec + v] =
            (FMT == DOSE_FMT_U16_SCALE || FMT == DOSE_FMT_FP8E4M3_ROWSCALE) ? __fmul_rn(s, acc) : acc;
    }
}

// Work units are the row blocks of every matrix's forward schedule, enumerated
// matrix by matrix; each CTA owns a contiguous range of units.  A row is
// reduced by one half-warp: lane v owns output vector v.
__global__ void __launch_bounds__(256) spmm_global_kernel(const __grid_constant__ BatchParams p) {
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
                case DOSE_FMT_F16: spmm_row<DOSE_FMT_F16>(it, row, v, p.nvec); break;
                case DOSE_FMT_F32: spmm_row<DOSE_FMT_F32>(it, row, v, p.nvec); break;
                default: spmm_row<DOSE_FMT_FP8E4M3_ROWSCALE>(it, row, v, p.nvec); break;
            }
        }
    }
}

uint32_t staged_slot_bytes(const dose_matrix* M) {
    const uint32_t es = value_bytes(M->fmt);
    const uint32_t nv = M->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0;
    return slot_layout(M->adj.tuning.tile_nnz, M->adj.tuning.tile_rows, es, nv, false).bytes;
}

template <uint32_t NQ>
cudaError_t launch_staged(const dose_matrix* const* A, const float* const* X, float* const* D, int n, int nvec,
                          uint32_t depth, uint32_t stride, size_t smem, cudaStream_t s) {
    StagedParams p;
    p.count = (uint32_t)n;
    p.nvec = (uint32_t)nvec;
    p.depth = depth;
    p.slot_stride = stride;
    p.l2pf = 0;
    p.err = A[0]->err;
    p.vec4 = nvec % 4 == 0;
    for (int i = 0; i < n; ++i)
        if (reinterpret_cast<uintptr_t>(D[i]) & 15u) p.vec4 = 0;
    for (int i = 0; i < n; ++i) {
        const dose_matrix* M = A[i];
        StagedItem& it = p.item[i];
        it.row_ptr = M->row_ptr;
        it.col = M->col;
        it.val = M->val;
        it.row_scale = M->row_scale;
        it.X = X[i];
        it.D = D[i];
        it.sched = ScheduleView{M->adj.desc, M->adj.ne, M->adj.cta_begin, M->adj.wlo};
        it.scale = M->scale;
        it.nrows = M->nrows;
        it.ncols = M->ncols;
        it.wwidth = M->adj.wwidth;
        it.tile_nnz = M->adj.tuning.tile_nnz;
        it.tile_rows = M->adj.tuning.tile_rows;
        it.fmt = M->fmt;
        p.l2pf = std::max(p.l2pf, M->adj_tuning.l2_prefetch);
    }
    auto k = spmm_staged_kernel<NQ>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<A[0]->adj.grid, 32 * (kSpmmConsumerWarps + 1), smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

void spmm_batched_plan(const dose_matrix* const* A, int count, int* layout, int* launches) {
    bool rg = count > 0;
    for (int base = 0; base < count && rg; base += (int)kRgSpmmMaxPerLaunch)
        rg = rg_spmm_applies(A + base, std::min<int>(count - base, (int)kRgSpmmMaxPerLaunch), nullptr, nullptr);
    const int per = rg ? (int)kRgSpmmMaxPerLaunch : kMaxBatchPerLaunch;
    int n = 0;
    for (int base = 0; base < count; base += per) {
        uint64_t rows = 0;
        for (int i = base; i < std::min(count, base + per); ++i) rows += A[i]->nrows;
        if (rows) ++n;
    }
    *layout = rg ? 2 : 1;
    *launches = n;
}

cudaError_t launch_spmm_batched(const dose_matrix* const* A, int count, const float* const* X, float* const* D,
                                int nvec, cudaStream_t s, std::string* why) {
    int dev = A[0]->device;
    for (int m = 0; m < count; ++m)
        if (A[m]->device != dev || A[m]->adj.grid != A[0]->adj.grid) {
            *why = "dose_spmv_batched: all matrices must live on one device";
            return cudaSuccess;
        }
    // the row-group form where every matrix has that layout (rg_spmm.cu)
    bool rg = true;
    for (int base = 0; base < count && rg; base += (int)kRgSpmmMaxPerLaunch)
        rg = rg_spmm_applies(A + base, std::min<int>(count - base, (int)kRgSpmmMaxPerLaunch), nullptr, nullptr);
    if (rg) return launch_rg_spmm(A, count, X, D, nvec, s);
    const uint32_t nq = nvec <= 4 ? 1 : nvec <= 8 ? 2 : 4;
    for (int base = 0; base < count; base += kMaxBatchPerLaunch) {
        const int n = count - base < kMaxBatchPerLaunch ? count - base : kMaxBatchPerLaunch;
        // staged form if the widest window of X and a ring of two or more slots fit
        uint32_t xw = 0, stride = 0, depth = 8;
        uint64_t rows = 0;
        for (int i = 0; i < n; ++i) {
            const dose_matrix* M = A[base + i];
            xw = std::max(xw, round_up((M->adj.wwidth + 1) * nq * 16u, 128));  // + the zero row
            stride = std::max(stride, staged_slot_bytes(M));
            depth = std::min(depth, M->adj_tuning.stages);
            rows += M->nrows;
        }
        if (rows == 0) continue;
        const size_t room = kMaxSmemPerBlock > kSpmmHeader + xw ? kMaxSmemPerBlock - kSpmmHeader - xw : 0;
        depth = std::min<uint32_t>(depth, (uint32_t)std::min<size_t>(8, room / std::max<uint32_t>(stride, 1)));
        cudaError_t e;
        if (depth >= 2) {
            const size_t smem = kSpmmHeader + xw + (size_t)depth * stride;
            e = nq == 1 ? launch_staged<1>(A + base, X + base, D + base, n, nvec, depth, stride, smem, s)
                : nq == 2 ? launch_staged<2>(A + base, X + base, D + base, n, nvec, depth, stride, smem, s)
                          : launch_staged<4>(A + base, X + base, D + base, n, nvec, depth, stride, smem, s);
        } else {
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
            spmm_global_kernel<<<(uint32_t)A[0]->sm_count * 4, 256, 0, s>>>(p);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dose
