// Adjoint g = A^T r and the fused quadratic-objective pass
//   d = A x,  f = sum_i w_i (d_i - p_i)^2,  g = A^T [2 w (d - p)]
// in one pass over A.  The gradient of the dose objective is what the
// optimiser the paper motivates needs every iteration (Sec. I: function values
// and gradients of the beam variables; Sec. II-A: A fixed, x changing).
//
// Warp specialisation (one persistent CTA per SM, shared-memory ring filled by
// bulk async copies as in the forward kernel):
//   warp 0            producer: row_ptr / non-empty list / values / columns /
//                     per-row vectors (p, w or r) of each stage;
//   forward warps     (fused pass only) d for the stage's rows, the FP64
//                     objective terms, and r_i = 2 w_i (d_i - p_i) per non-empty
//                     row into the slot; then signal `fwd_done`;
//   scatter warps     each owns a private shared-memory accumulator of the
//                     CTA's column window of the gradient and scatters a_ij r_i
//                     for its share of the stage's non-empty rows, one row at a
//                     time.
// Determinism (Sec. II-D: no reductions whose order is not fixed, so no float
// atomics): the entries of a row have distinct columns, so the lanes of a
// scatter warp never update the same word in one instruction; each warp's rows
// follow a fixed order; at the end each CTA sums its warps' accumulators in
// warp order into a per-CTA partial, and a second kernel sums the partials in
// CTA order (and applies an optional projected-gradient step x <- max(0, x - eta g)).
#include "stage_common.cuh"

namespace dose {
namespace {

struct AdjParams {
    const uint32_t* row_ptr;
    const uint32_t* col;
    const void* val;
    float scale;
    const float* x;   // QUADRATIC
    float* d;         // QUADRATIC, may be null
    float* g_part;    // grid x wwidth: CTA c's window of the gradient
    double* f_part;   // grid
    uint32_t nrows, ncols;
    uint32_t wwidth;  // columns of each CTA's window [wlo, wlo + wwidth), wlo = sched.wlo[cta]
    ScheduleView sched;
    VecSet vecs;      // QUADRATIC: p, w [, row scale]; ADJOINT: r [, row scale]
    uint32_t tile_nnz, tile_rows, depth, fwarps, swarps, l2pf;
    int* err;
};

constexpr uint32_t kAdjHeader = 3072;  // mbarriers, CTA reduction scratch, 2 KB of stage descriptors

template <int FMT>
__device__ __forceinline__ float finish_dot(const AdjParams& p, float rs, float acc) {
    if (FMT == DOSE_FMT_U16_SCALE) return __fmul_rn(p.scale, acc);
    if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) return __fmul_rn(rs, acc);
    return acc;
}

// gw[col_k] += a_k * rj for the entries k = kb, kb + step, ... < ke of one row
// (gw: shared address of a warp's accumulator).  The columns of a row are
// distinct, so the four loads may precede the four stores.
template <int FMT>
__device__ __forceinline__ void scatter_entries(uint32_t gw, const SlotView& v, uint32_t kb, uint32_t ke,
                                                uint32_t step, float rj) {
    constexpr uint32_t ES = (uint32_t)sizeof(typename Fmt<FMT>::T);
    for (uint32_t k0 = kb; k0 < ke; k0 += 4 * step) {
        uint32_t ga[4];
        float a[4], gv[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t k = k0 + step * u;
            ok[u] = k < ke;
            ga[u] = gw + 4 * (ok[u] ? dev::lds_u32(v.col + 4 * k) : 0u);
            a[u] = ok[u] ? Fmt<FMT>::lds(v.val + ES * k) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) gv[u] = ok[u] ? dev::lds_f32(ga[u]) : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (ok[u]) dev::sts_f32(ga[u], __fmaf_rn(a[u], rj, gv[u]));
    }
}

// Scatter of a NORMAL stage's non-empty rows i = first, first + Ws, ... by one
// warp, software-pipelined: the next row's list entry, row pointers and r are
// loaded while the current row's accumulator updates are in flight.  Rows are
// still applied strictly in order (the LSU keeps each warp's shared-memory
// accesses in program order), so the result does not change.
template <int FMT, bool QUAD, uint32_t kRowScaleVec>
__device__ __forceinline__ void scatter_rows(uint32_t gw, const SlotView& v, uint32_t slot, const SlotLayout& SL,
                                             const VecSet& vecs, const StageDesc& D, uint32_t first, uint32_t Ws,
                                             uint32_t lane) {
    constexpr uint32_t ES = (uint32_t)sizeof(typename Fmt<FMT>::T);
    const uint32_t n_ne = D.ne1 - D.ne0;
    const uint32_t rl = slot + SL.rl_off;
    auto meta = [&](uint32_t i, uint32_t& kb, uint32_t& ke, float& rj) {
        const uint32_t row = D.row0 + dev::lds_u16(v.ne + 2 * i);
        kb = dev::lds_u32(v.rp + 4 * row);
        ke = dev::lds_u32(v.rp + 4 * row + 4);
        if (QUAD) {
            rj = dev::lds_f32(rl + 4 * i);
        } else {
            rj = slot_vec(slot, SL, vecs, 0, D.row0, row);
            if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) rj = __fmul_rn(rj, slot_vec(slot, SL, vecs, kRowScaleVec, D.row0, row));
        }
    };
    uint32_t i = first;
    if (i >= n_ne) return;
    uint32_t kb, ke;
    float rj;
    meta(i, kb, ke, rj);
    bool more;
    do {
        // this row: lane l takes the groups at (kb & ~3) + 4 l + 128 s
        const int len = (int)(ke - kb);
        int off = (int)(4 * lane) - (int)(kb & 3u);
        const uint32_t k0 = (kb & ~3u) + 4 * lane;
        uint32_t ca = v.col + 4 * k0, va = v.val + ES * k0;
        const uint32_t steps = (uint32_t)(len + (int)(kb & 3u) + 127) >> 7;  // the same for every lane
        const float r = rj;
        uint32_t c[4];
        float a[4];
        load_group<FMT>(off, len, ca, va, c, a);
        // the next row's metadata is fetched while this row's first step is in flight
        i += Ws;
        more = i < n_ne;
        if (more) meta(i, kb, ke, rj);
        scatter_group(off, len, gw, c, a, r);
#pragma unroll 1
        for (uint32_t s = 1; s < steps; ++s) {
            off += 128;
            ca += 512;
            va += 128 * ES;
            load_group<FMT>(off, len, ca, va, c, a);
            scatter_group(off, len, gw, c, a, r);
        }
        __syncwarp();  // all lanes' updates of this row precede the next row's loads
    } while (more);
}

// Forward part of the fused pass for the non-empty rows of a NORMAL stage,
// 2^LG lanes per row: d, the objective terms, and r_i = 2 w_i (d_i - p_i) (FP8:
// times the row scale) into the slot's r list.
template <int FMT, uint32_t LG, uint32_t kRowScaleVec>
__device__ __forceinline__ void fwd_rows(const AdjParams& p, const StageDesc& D, const SlotView& v, uint32_t slot,
                                         const SlotLayout& SL, const SlotPtrs<FMT, 4>& sp, const float* xsp,
                                         uint32_t zc, uint32_t ftid, uint32_t lane, uint32_t nft, uint32_t rotw,
                                         float& f_hi, float& f_lo) {
    constexpr uint32_t L = 1u << LG;
    const uint32_t gid = ftid >> LG, li = lane & (L - 1), G = nft >> LG;
    const uint32_t j0 = (gid + G - ((rotw << (5 - LG)) & (G - 1))) & (G - 1);
    const uint32_t n_ne = D.ne1 - D.ne0;
    const uint32_t rl = slot + SL.rl_off;
    for (uint32_t base = 0; base < n_ne; base += G) {
        const uint32_t i = base + j0;
        const bool has = i < n_ne;
        // groups without a row read the stage's first entries (masked) and write nothing
        uint32_t row = 0, rs = D.nz0, re = D.nz0;
        if (has) {
            row = D.row0 + dev::lds_u16(v.ne + 2 * i);
            rs = dev::lds_u32(v.rp + 4 * row);
            re = dev::lds_u32(v.rp + 4 * row + 4);
        }
        const uint32_t span = re > rs ? re - (rs & ~3u) : 0;
        const uint32_t iters = __reduce_max_sync(0xffffffffu, (span + 4 * L - 1) / (4 * L));
        float sum = dot_vec_p<FMT, L, 4>(sp, xsp, zc, rs, re, li, iters);
#pragma unroll
        for (uint32_t off = L >> 1; off > 0; off >>= 1) sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, off));
        if (has && li == 0) {
            const float rsc =
                FMT == DOSE_FMT_FP8E4M3_ROWSCALE ? slot_vec(slot, SL, p.vecs, kRowScaleVec, D.row0, row) : 1.f;
            const float dv = finish_dot<FMT>(p, rsc, sum);
            if (p.d) p.d[row] = dv;
            const float wv = slot_vec(slot, SL, p.vecs, 1, D.row0, row);
            const float e = dev::df_add_wsq(f_hi, f_lo, wv, dv, slot_vec(slot, SL, p.vecs, 0, D.row0, row));
            dev::sts_f32(rl + 4 * i, __fmul_rn(__fmul_rn(__fmul_rn(2.0f, wv), e), rsc));
        }
    }
}

template <int FMT, int MODE>
__global__ void __launch_bounds__(kMaxAdjWarps * 32, 1) adjoint_kernel(const AdjParams p) {
    using T = typename Fmt<FMT>::T;
    constexpr bool QUAD = MODE == ADJ_MODE_QUADRATIC;
    constexpr uint32_t kRowScaleVec = QUAD ? 2 : 1;  // index of the FP8 row scales in vecs
    extern __shared__ __align__(128) unsigned char smem[];

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth, Wf = QUAD ? p.fwarps : 0, Ws = p.swarps;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + 8;
    uint64_t* fwd_done = full + 16;
    uint64_t* dbar = full + 24;                              // 2 descriptor-window barriers
    StageDesc* dwin = reinterpret_cast<StageDesc*>(smem + 1024);  // 2 x kDescWin descriptors
    float* red = reinterpret_cast<float*>(smem + 256);      // 32 floats: long-row partials
    double* fred = reinterpret_cast<double*>(smem + 512);   // 32 doubles: per-warp objective
    // This CTA's entries have columns in [wlo, wlo + wwidth): the accumulators
    // and x hold that window, addressed by column through a base moved down by
    // wlo words (shared addresses wrap mod 2^32, so base + 4 c lands in place).
    const uint32_t wlo = p.sched.wlo[blockIdx.x];
    const uint32_t gw_floats = round_up(p.wwidth * 4, 128) / 4;
    float* gacc = reinterpret_cast<float*>(smem + kAdjHeader);  // Ws x gw_floats
    float* xs = gacc + Ws * gw_floats;
    const uint32_t x_bytes = QUAD ? round_up((p.wwidth + 1) * 4, 128) : 0;  // the window of x and a zero
    unsigned char* slot_base = reinterpret_cast<unsigned char*>(xs) + x_bytes;
    const SlotLayout SL = slot_layout(p.tile_nnz, p.tile_rows, sizeof(T), p.vecs.n, QUAD);

    const uint32_t s_begin = p.sched.cta_begin[blockIdx.x];
    const uint32_t s_end = p.sched.cta_begin[blockIdx.x + 1];
    const uint32_t ncons = (Wf + Ws) * 32;

    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < S; ++i) {
            dev::mbar_init(&full[i], 1);
            dev::mbar_init(&empty[i], Ws);
            if (QUAD) dev::mbar_init(&fwd_done[i], Wf);
        }
        dev::mbar_init(&dbar[0], 1);
        dev::mbar_init(&dbar[1], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0)
            run_producer<FMT>(p.sched, s_begin, s_end, p.row_ptr, p.col, p.val, p.vecs, slot_base, SL, full,
                              empty, S, dwin, dbar, p.l2pf, p.err);
        return;
    }

    const uint32_t ctid = threadIdx.x - 32;
    for (uint32_t j = ctid; j < Ws * gw_floats; j += ncons) gacc[j] = 0.f;
    if (QUAD)
        for (uint32_t j = ctid; j <= p.wwidth; j += ncons)
            xs[j] = j < p.wwidth && wlo + j < p.ncols ? __ldg(p.x + wlo + j) : 0.f;
    dev::named_barrier(1, ncons);

    const uint32_t xs_a = dev::smem_u32(xs) - 4 * wlo;
    const uint32_t slot0 = dev::smem_u32(slot_base);
    const bool is_fwd = QUAD && warp <= Wf;
    bool failed = false;
    float f_hi = 0.f, f_lo = 0.f;  // this lane's objective terms, double-float

    if (is_fwd) {
        // ------------------------------------------------ forward warps
        const uint32_t fw = warp - 1, ftid = fw * 32 + lane, nft = Wf * 32;  // Wf is a power of two
        const float* xsp = xs - wlo;         // x of column c at xsp[c] (c in this CTA's window)
        const uint32_t zc = wlo + p.wwidth;  // the zero element after the window
        float coop_s = 0.f;
        uint32_t st = 0, ph = 0;
        for (uint32_t s = s_begin; s < s_end; ++s) {
            const uint32_t rotw = s & (Wf - 1);
            if (!dev::mbar_wait_bounded(&full[st], ph)) {
                atomicExch(p.err, kErrTimeoutFull);
                failed = true;
                break;
            }
            const uint32_t slot = slot0 + st * SL.bytes;
            const StageDesc D = slot_desc(slot);
            const SlotView v = slot_view<FMT>(slot, SL, D);
            const SlotPtrs<FMT, 4> sp = slot_ptrs<FMT, 4>(slot_base + st * SL.bytes, SL, D);
            if (!(D.meta & STAGE_COOP)) {
                for (uint32_t r = D.row0 + ftid; r < D.row1; r += nft) {
                    if (dev::lds_u32(v.rp + 4 * r) == dev::lds_u32(v.rp + 4 * r + 4)) {
                        if (p.d) p.d[r] = 0.0f;
                        // an empty row with p = 0 adds exactly nothing (d = 0), unless w is not finite
                        const float pv = slot_vec(slot, SL, p.vecs, 0, D.row0, r);
                        const float wv = slot_vec(slot, SL, p.vecs, 1, D.row0, r);
                        if (pv != 0.0f || !(fabsf(wv) < INFINITY)) dev::df_add_wsq(f_hi, f_lo, wv, 0.0f, pv);
                    }
                }
                switch (D.meta & STAGE_LANES_MASK) {
                    case 0: fwd_rows<FMT, 0, kRowScaleVec>(p, D, v, slot, SL, sp, xsp, zc, ftid, lane, nft, rotw, f_hi, f_lo); break;
                    case 1: fwd_rows<FMT, 1, kRowScaleVec>(p, D, v, slot, SL, sp, xsp, zc, ftid, lane, nft, rotw, f_hi, f_lo); break;
                    case 2: fwd_rows<FMT, 2, kRowScaleVec>(p, D, v, slot, SL, sp, xsp, zc, ftid, lane, nft, rotw, f_hi, f_lo); break;
                    case 3: fwd_rows<FMT, 3, kRowScaleVec>(p, D, v, slot, SL, sp, xsp, zc, ftid, lane, nft, rotw, f_hi, f_lo); break;
                    case 4: fwd_rows<FMT, 4, kRowScaleVec>(p, D, v, slot, SL, sp, xsp, zc, ftid, lane, nft, rotw, f_hi, f_lo); break;
                    default: fwd_rows<FMT, 5, kRowScaleVec>(p, D, v, slot, SL, sp, xsp, zc, ftid, lane, nft, rotw, f_hi, f_lo); break;
                }
            } else {
                // one chunk of a long row: every forward thread takes part
                if (D.meta & STAGE_FIRST) coop_s = 0.f;
                coop_s = __fadd_rn(coop_s, dot_strided<FMT>(v, xs_a, D.nz0 + ftid, D.nz1, nft));
                if (D.meta & STAGE_LAST) {
                    float sum = coop_s;
                    for (uint32_t off = 16; off > 0; off >>= 1)
                        sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, off));
                    if (lane == 0) red[fw] = sum;
                    dev::named_barrier(2, nft);
                    if (ftid == 0) {
                        float tot = red[0];
                        for (uint32_t w2 = 1; w2 < Wf; ++w2) tot = __fadd_rn(tot, red[w2]);
                        const float rsc = FMT == DOSE_FMT_FP8E4M3_ROWSCALE
                                              ? slot_vec(slot, SL, p.vecs, kRowScaleVec, D.row0, D.row0)
                                              : 1.f;
                        const float dv = finish_dot<FMT>(p, rsc, tot);
                        if (p.d) p.d[D.row0] = dv;
                        const float wv = slot_vec(slot, SL, p.vecs, 1, D.row0, D.row0);
                        const float e =
                            dev::df_add_wsq(f_hi, f_lo, wv, dv, slot_vec(slot, SL, p.vecs, 0, D.row0, D.row0));
                        dev::sts_f32(slot + SL.hdr_off + 32, __fmul_rn(__fmul_rn(__fmul_rn(2.0f, wv), e), rsc));
                    }
                    dev::named_barrier(2, nft);
                }
            }
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&fwd_done[st]);
            if (++st == S) {
                st = 0;
                ph ^= 1;
            }
        }
    } else {
        // ------------------------------------------------ scatter warps
        const uint32_t sw = warp - 1 - Wf;
        const uint32_t gw = dev::smem_u32(gacc + sw * gw_floats) - 4 * wlo;
        uint32_t st = 0, ph = 0, first = sw;  // first list entry of this warp, rotating per stage
        for (uint32_t s = s_begin; s < s_end; ++s, first = first + 1 == Ws ? 0 : first + 1) {
            if (!dev::mbar_wait_bounded(&full[st], ph) || (QUAD && !dev::mbar_wait_bounded(&fwd_done[st], ph))) {
                atomicExch(p.err, kErrTimeoutFull);
                failed = true;
                break;
            }
            const uint32_t slot = slot0 + st * SL.bytes;
            const StageDesc D = slot_desc(slot);
            const SlotView v = slot_view<FMT>(slot, SL, D);
            if (!(D.meta & STAGE_COOP)) {
                scatter_rows<FMT, QUAD, kRowScaleVec>(gw, v, slot, SL, p.vecs, D, first, Ws, lane);
            } else if (QUAD) {
                if (D.meta & STAGE_LAST) {
                    // the whole long row, from global memory (its earlier chunks left the ring)
                    const float rj = dev::lds_f32(slot + SL.hdr_off + 32);
                    const uint32_t kb = __ldg(p.row_ptr + D.row0), ke = __ldg(p.row_ptr + D.row0 + 1);
                    const T* vg = static_cast<const T*>(p.val);
                    for (uint32_t k = kb + sw * 32 + lane; k < ke; k += Ws * 32) {
                        const uint32_t ga = gw + 4 * __ldg(p.col + k);
                        dev::sts_f32(ga, __fmaf_rn(Fmt<FMT>::dec(vg[k]), rj, dev::lds_f32(ga)));
                    }
                }
            } else {
                float rj = slot_vec(slot, SL, p.vecs, 0, D.row0, D.row0);
                if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE)
                    rj = __fmul_rn(rj, slot_vec(slot, SL, p.vecs, kRowScaleVec, D.row0, D.row0));
                scatter_entries<FMT>(gw, v, D.nz0 + sw * 32 + lane, D.nz1, Ws * 32, rj);
            }
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&empty[st]);
            if (++st == S) {
                st = 0;
                ph ^= 1;
            }
        }
    }
    // Timeouts are consistent across warps (all wait on the same phases), so a
    // failed warp leaves no one waiting at the barriers below.
    if (failed) return;

    // CTA partials: accumulators summed in warp order; f in a fixed tree.
    if (is_fwd) {
        double f_lane = (double)f_hi + (double)f_lo;
        for (uint32_t off = 16; off > 0; off >>= 1) f_lane += __shfl_xor_sync(0xffffffffu, f_lane, off);
        if (lane == 0) fred[warp - 1] = f_lane;
    }
    dev::named_barrier(1, ncons);
    for (uint32_t j = ctid; j < p.wwidth; j += ncons) {
        float t = gacc[j];
        for (uint32_t w2 = 1; w2 < Ws; ++w2) t = __fadd_rn(t, gacc[w2 * gw_floats + j]);
        p.g_part[(size_t)blockIdx.x * p.wwidth + j] = t;
    }
    if (ctid == 0) {
        double t = 0.0;
        for (uint32_t w2 = 0; w2 < Wf; ++w2) t += fred[w2];
        p.f_part[blockIdx.x] = t;
    }
}

// g_j = s * sum_c g_part[c][j - wlo_c] over the CTAs c whose window holds j,
// and f = sum_c f_part[c], both in a fixed order; optional projected-gradient
// step on x.  Block: 256 threads = 8 warps x 32 columns; warp w sums the
// partials c = w, w + 8, ...; warp 0 adds the eight.
__global__ void __launch_bounds__(256) adjoint_finalize(const float* __restrict__ g_part,
                                                        const uint32_t* __restrict__ wlo, uint32_t wwidth,
                                                        const double* __restrict__ f_part, uint32_t nparts,
                                                        uint32_t ncols, float scale, float* g, double* f,
                                                        float* x_update, float eta) {
    __shared__ float part[8][33];
    __shared__ double fpart[256];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t j = blockIdx.x * 32 + lane;
    float t = 0.f;
    if (j < ncols)
        for (uint32_t c = w; c < nparts; c += 8) {
            const uint32_t off = j - __ldg(wlo + c);
            if (off < wwidth) t = __fadd_rn(t, g_part[(size_t)c * wwidth + off]);
        }
    part[w][lane] = t;
    if (f && blockIdx.x == 0) {
        double ft = 0.0;
        for (uint32_t c = threadIdx.x; c < nparts; c += 256) ft += f_part[c];
        fpart[threadIdx.x] = ft;
    }
    __syncthreads();
    if (w == 0 && j < ncols) {
        float tot = part[0][lane];
        for (uint32_t k = 1; k < 8; ++k) tot = __fadd_rn(tot, part[k][lane]);
        tot = __fmul_rn(scale, tot);
        if (g) g[j] = tot;
        if (x_update) {
            const float xn = __fsub_rn(x_update[j], __fmul_rn(eta, tot));
            x_update[j] = xn > 0.f ? xn : 0.f;
        }
    }
    if (f && blockIdx.x == 0 && threadIdx.x == 0) {
        double ft = 0.0;
        for (uint32_t k = 0; k < 256; ++k) ft += fpart[k];
        *f = ft;
    }
}

template <int FMT, int MODE>
cudaError_t launch_adj_t(const dose_matrix* A, const AdjParams& p, size_t smem, cudaStream_t s) {
    auto k = adjoint_kernel<FMT, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint32_t warps = 1 + (MODE == ADJ_MODE_QUADRATIC ? p.fwarps : 0) + p.swarps;
    k<<<A->adj.grid, 32 * warps, smem, s>>>(p);
    return cudaGetLastError();
}

size_t adj_smem(const dose_matrix* A, const AdjTuning& t, bool quad, uint32_t ws) {
    const uint32_t esize = value_bytes(A->fmt);
    const uint32_t nvec = (quad ? 2 : 1) + (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0);
    const SlotLayout SL = slot_layout(t.tile_nnz, t.tile_rows, esize, nvec, quad);
    const size_t col_bytes = round_up(A->adj.wwidth * 4, 128);
    const size_t x_bytes = quad ? round_up((A->adj.wwidth + 1) * 4, 128) : 0;  // the window of x and a zero
    return kAdjHeader + ws * col_bytes + x_bytes + (size_t)t.stages * SL.bytes;
}

}  // namespace

bool adjoint_shape(const dose_matrix* A, const AdjTuning& in, bool quad, AdjTuning* out, size_t* smem) {
    AdjTuning t = in;
    uint32_t fwq = in.forward_warps ? in.forward_warps : 8;
    if (fwq > 8) fwq = 8;
    while (fwq & (fwq - 1)) fwq &= fwq - 1;  // a power of two: 1, 2, 4 or 8
    t.forward_warps = quad ? fwq : 0;
    if (t.stages < 2 || t.stages > 8) return false;
    // scatter warps: as many as fit (at most the requested number, if any)
    uint32_t max_ws = kMaxAdjWarps - 1 - t.forward_warps;
    if (in.scatter_warps && in.scatter_warps < max_ws) max_ws = in.scatter_warps;
    uint32_t ws = 0;
    for (uint32_t w = max_ws; w >= 1; --w)
        if (adj_smem(A, t, quad, w) <= kMaxSmemPerBlock) {
            ws = w;
            break;
        }
    if (ws == 0) return false;
    t.scatter_warps = ws;
    if (out) *out = t;
    if (smem) *smem = adj_smem(A, t, quad, ws);
    return true;
}

cudaError_t launch_adjoint(const dose_matrix* A, int mode, const float* x, const float* p, const float* w,
                           const float* r, float* d, double* f, float* g, float* x_update, float eta,
                           cudaStream_t s) {
    const bool quad = mode == ADJ_MODE_QUADRATIC;
    if (rg_active(A, quad)) return launch_rg(A, mode, x, p, w, r, d, f, g, x_update, eta, s);
    AdjTuning t;
    size_t smem = 0;
    if (!adjoint_shape(A, A->adj_tuning, quad, &t, &smem)) return cudaErrorInvalidConfiguration;
    if (A->nrows > 0) {
        AdjParams prm;
        prm.row_ptr = A->row_ptr;
        prm.col = A->col;
        prm.val = A->val;
        prm.scale = A->scale;
        prm.x = x;
        prm.d = d;
        prm.g_part = A->g_part;
        prm.f_part = A->f_part;
        prm.nrows = A->nrows;
        prm.ncols = A->ncols;
        prm.wwidth = A->adj.wwidth;
        prm.sched = ScheduleView{A->adj.desc, A->adj.ne, A->adj.cta_begin, A->adj.wlo};
        const uint32_t user_lim = A->nrows & ~3u;  // caller arrays: whole 16-byte pieces only
        prm.vecs.n = 0;
        if (quad) {
            prm.vecs.ptr[0] = p;
            prm.vecs.lim[0] = user_lim;
            prm.vecs.ptr[1] = w;
            prm.vecs.lim[1] = user_lim;
            prm.vecs.n = 2;
        } else {
            prm.vecs.ptr[0] = r;
            prm.vecs.lim[0] = user_lim;
            prm.vecs.n = 1;
        }
        if (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE) {
            prm.vecs.ptr[prm.vecs.n] = A->row_scale;
            prm.vecs.lim[prm.vecs.n] = round_up(A->nrows, 4);
            prm.vecs.n++;
        }
        prm.tile_nnz = t.tile_nnz;
        prm.tile_rows = t.tile_rows;
        prm.depth = t.stages;
        prm.fwarps = t.forward_warps;
        prm.swarps = t.scatter_warps;
        prm.l2pf = t.l2_prefetch;
        prm.err = A->err;
        cudaError_t e = cudaSuccess;
        switch (A->fmt) {
            case DOSE_FMT_U16_SCALE:
                e = quad ? launch_adj_t<DOSE_FMT_U16_SCALE, ADJ_MODE_QUADRATIC>(A, prm, smem, s)
                         : launch_adj_t<DOSE_FMT_U16_SCALE, ADJ_MODE_ADJOINT>(A, prm, smem, s);
                break;
            case DOSE_FMT_BF16:
                e = quad ? launch_adj_t<DOSE_FMT_BF16, ADJ_MODE_QUADRATIC>(A, prm, smem, s)
                         : launch_adj_t<DOSE_FMT_BF16, ADJ_MODE_ADJOINT>(A, prm, smem, s);
                break;
            case DOSE_FMT_F16:
                e = quad ? launch_adj_t<DOSE_FMT_F16, ADJ_MODE_QUADRATIC>(A, prm, smem, s)
                         : launch_adj_t<DOSE_FMT_F16, ADJ_MODE_ADJOINT>(A, prm, smem, s);
                break;
            case DOSE_FMT_F32:
                e = quad ? launch_adj_t<DOSE_FMT_F32, ADJ_MODE_QUADRATIC>(A, prm, smem, s)
                         : launch_adj_t<DOSE_FMT_F32, ADJ_MODE_ADJOINT>(A, prm, smem, s);
                break;
            case DOSE_FMT_FP8E4M3_ROWSCALE:
                e = quad ? launch_adj_t<DOSE_FMT_FP8E4M3_ROWSCALE, ADJ_MODE_QUADRATIC>(A, prm, smem, s)
                         : launch_adj_t<DOSE_FMT_FP8E4M3_ROWSCALE, ADJ_MODE_ADJOINT>(A, prm, smem, s);
                break;
        }
        if (e != cudaSuccess) return e;
    }
    return launch_adjoint_finalize(A, A->g_part, A->adj.wlo, A->adj.wwidth, A->nrows > 0 ? A->adj.grid : 0, quad, g,
                                   f, x_update, eta, s);
}

cudaError_t launch_adjoint_finalize(const dose_matrix* A, const float* g_part, const uint32_t* wlo, uint32_t wwidth,
                                    uint32_t nparts, bool quad, float* g, double* f, float* x_update, float eta,
                                    cudaStream_t s) {
    const float scale = A->fmt == DOSE_FMT_U16_SCALE ? A->scale : 1.0f;
    const uint32_t blocks = A->ncols ? (A->ncols + 31) / 32 : 1;
    adjoint_finalize<<<blocks, 256, 0, s>>>(g_part, wlo, wwidth, A->f_part, nparts, A->ncols, scale, g,
                                            quad ? f : nullptr, x_update, eta);
    return cudaGetLastError();
}

}  // namespace dose
