// Adjoint g = A^T r and the fused quadratic-objective pass
//   d = A x,  f = sum_i w_i (d_i - p_i)^2,  g = A^T [2 w (d - p)]
// on the row-group layout (rg_layout.cu): the gradient of the dose objective
// that the optimiser needs every iteration (Sec. I; Sec. II-A).
//
// One persistent CTA per SM.  Warp 0's lane 0 streams stages (a run of row
// groups, their union columns and values, the rows' non-empty bits and the
// per-row vectors) into a shared-memory ring with bulk async copies.  Every
// other warp is a worker that owns a private shared-memory accumulator of the
// CTA's column window of the gradient and takes whole groups, one at a time:
//   1. lane l reads union positions l, l + 32, ... : column index and the four
//      rows' values (decoded to FP32 and kept in registers), gathers x[c] once
//      and adds it into four row sums;
//   2. a transposed butterfly reduces the four sums over the warp (lane l ends
//      with row l / 8's dose);
//   3. one lane per row writes d, adds w (d - p)^2 to its double-float objective
//      and forms r = 2 w (d - p); four shuffles give every lane the four r;
//   4. for each of its union columns a lane adds sum_g a_gc r_g into the
//      accumulator with one read-modify-write.
// Rows without entries get d = 0 and their objective term from the finalize
// kernel (rg_finalize), which runs them while the main kernel drains.
// Determinism (Sec. II-D: no float atomics, fixed reduction order): the union
// columns of a group are distinct, so no two lanes of a warp update one word
// in one instruction; each warp takes its groups in a fixed order; the CTA sums
// its warps' accumulators in warp order and a second kernel sums the CTAs'
// partials in CTA order.
#include "rg_common.cuh"

namespace dose {
namespace {

constexpr uint32_t kRgHeader = 3072;  // mbarriers, objective partials, 2 KB of stage descriptors

struct RgParams {
    const uint4* grp;
    const void* ucol;
    const void* uval;
    float scale;
    const float* x;   // QUADRATIC
    float* d;         // QUADRATIC, may be null
    float* g_part;    // grid x wwidth
    double* f_part;   // grid
    uint32_t nrows, ncols, wwidth;
    ScheduleView sched;
    VecSet vecs;      // QUADRATIC: p, w [, row scale]; ADJOINT: r [, row scale]
    RgSlot SL;
    uint32_t depth, nw, l2pf;
    int* err;
};


// Producer (one thread): descriptors in double-buffered windows of kDescWin as
// in the CSR pipeline, then per stage the group records, union columns, union
// values, non-empty bits (fused pass) and per-row vectors.  Bounded waits.
template <int FMT, uint32_t IW, bool QUAD>
__device__ void rg_produce(const RgParams& p, uint32_t s_begin, uint32_t s_end, unsigned char* slot_base,
                           uint64_t* full, uint64_t* empty, StageDesc* dwin, uint64_t* dbar) {
    constexpr uint32_t ES = (uint32_t)sizeof(typename Fmt<FMT>::T);
    constexpr uint32_t RV = 4 * ES;                  // bytes of one union entry's values
    constexpr uint32_t VA = RV >= 16 ? 1 : 16 / RV;  // union entries per 16 bytes of values
    constexpr uint32_t CA = 16 / IW;                 // column indices per 16 bytes
    const RgSlot& SL = p.SL;
    const uint32_t S = p.depth;
    const unsigned char* ucol = static_cast<const unsigned char*>(p.ucol);
    const unsigned char* uval = static_cast<const unsigned char*>(p.uval);
    if (s_begin >= s_end) return;
    const uint32_t nst = s_end - s_begin, nwin = (nst + kDescWin - 1) / kDescWin;
    auto load_window = [&](uint32_t w) {
        const uint32_t first = s_begin + w * kDescWin;
        if (first >= s_end) return;
        const uint32_t n = min(kDescWin, s_end - first);
        dev::mbar_arrive_expect_tx(&dbar[w & 1], n * (uint32_t)sizeof(StageDesc));
        dev::bulk_g2s(dwin + (w & 1) * kDescWin, p.sched.desc + first, n * (uint32_t)sizeof(StageDesc), &dbar[w & 1]);
    };
    load_window(0);
    load_window(1);
    uint32_t w_issued = min(nwin, 2u), w_waited = 0;
    auto have_window = [&](uint32_t w) -> bool {
        while (w_waited <= w) {
            if (!dev::mbar_wait_poll(&dbar[w_waited & 1], (w_waited >> 1) & 1)) return false;
            ++w_waited;
        }
        return true;
    };
    auto prefetch = [&](uint32_t j) {
        const uint32_t w = j / kDescWin;
        if (w >= w_issued || !have_window(w)) return;
        const StageDesc P = dwin[(w & 1) * kDescWin + j % kDescWin];
        if (P.nz1 > P.nz0) {
            const uint32_t c_a = P.nz0 & ~(CA - 1), v_a = P.nz0 & ~(VA - 1);
            dev::bulk_prefetch_l2(ucol + (size_t)c_a * IW, (round_up(P.nz1, CA) - c_a) * IW);
            dev::bulk_prefetch_l2(uval + (size_t)v_a * RV, (round_up(P.nz1, VA) - v_a) * RV);
        }
    };
    for (uint32_t j = 0; j < p.l2pf && j < nst; ++j) prefetch(j);
    uint32_t st = 0, ph = 0, issued = 0;
    bool ok = true;
    for (uint32_t s = s_begin; s < s_end; ++s) {
        const uint32_t j = s - s_begin, w = j / kDescWin, jw = j % kDescWin;
        if (p.l2pf && j + p.l2pf < nst) prefetch(j + p.l2pf);
        if (!have_window(w)) {
            atomicExch(p.err, kErrTimeoutEmpty);
            ok = false;
            break;
        }
        const StageDesc D = dwin[(w & 1) * kDescWin + jw];
        if (jw == kDescWin - 1 && w + 2 < nwin) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            load_window(w + 2);
            w_issued = w + 3;
        }
        if (!dev::mbar_wait_poll(&empty[st], ph ^ 1)) {
            atomicExch(p.err, kErrTimeoutEmpty);
            ok = false;
            break;
        }
        unsigned char* buf = slot_base + st * SL.bytes;
        *reinterpret_cast<StageDesc*>(buf) = D;
        const uint32_t ng = D.ne1 - D.ne0;
        const bool work = ng > 0;
        uint32_t bytes = 0;
        const uint32_t c_a = D.nz0 & ~(CA - 1), c_n = D.nz1 > D.nz0 ? round_up(D.nz1, CA) - c_a : 0;
        const uint32_t v_a = D.nz0 & ~(VA - 1), v_n = D.nz1 > D.nz0 ? round_up(D.nz1, VA) - v_a : 0;
        const uint32_t r_a = D.row0 & ~3u;
        uint32_t vn[kMaxVec] = {0, 0, 0};
        bytes += ng * 16 + c_n * IW + v_n * RV;
        if (work)
            for (uint32_t k = 0; k < p.vecs.n; ++k) {
                const uint32_t e = min(round_up(D.row1, 4), p.vecs.lim[k]);
                vn[k] = e > r_a ? e - r_a : 0;
                bytes += vn[k] * 4;
                float* dst = reinterpret_cast<float*>(buf + SL.vec_off + k * SL.vec_stride);
                bool tail = false;
                for (uint32_t r = max(p.vecs.lim[k], r_a + vn[k]); r < D.row1; ++r) {
                    dst[r - r_a] = __ldg(p.vecs.ptr[k] + r);
                    tail = true;
                }
                if (tail) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
        dev::mbar_arrive_expect_tx(&full[st], bytes);
        if (ng) dev::bulk_g2s(buf + SL.grp_off, p.grp + D.ne0, ng * 16, &full[st]);
        if (c_n) dev::bulk_g2s(buf + SL.col_off, ucol + (size_t)c_a * IW, c_n * IW, &full[st]);
        if (v_n) dev::bulk_g2s(buf + SL.val_off, uval + (size_t)v_a * RV, v_n * RV, &full[st]);
        for (uint32_t k = 0; k < p.vecs.n; ++k)
            if (vn[k]) dev::bulk_g2s(buf + SL.vec_off + k * SL.vec_stride, p.vecs.ptr[k] + r_a, vn[k] * 4, &full[st]);
        ++issued;
        if (++st == S) {
            st = 0;
            ph ^= 1;
        }
    }
    for (uint32_t w = w_waited; w < w_issued; ++w) dev::mbar_wait_poll(&dbar[w & 1], (w >> 1) & 1);
    // never leave copies in flight into the CTA's shared memory
    const uint32_t n = issued < S ? issued : S;
    for (uint32_t i = 0; i < n; ++i) {
        if (st == 0) {
            st = S - 1;
            ph ^= 1;
        } else {
            --st;
        }
        dev::mbar_wait_poll(&full[st], ph);
    }
    (void)ok;
}

// Per-stage shared addresses of a worker (32-bit shared addresses, rebased so
// that global indices can be used directly: 32-bit wrap-around arithmetic,
// only the sums are addresses).
struct RgStage {
    uint32_t col;   // + IW * (union entry)
    uint32_t val;   // + RV * (union entry)
    uint32_t vec0;  // + 4 * (row - r_a): p (fused) or r (adjoint)
    uint32_t vec1;  // w (fused)
    uint32_t vrs;   // FP8 row scales
    uint32_t row0, r_a;
};

// One group whose union takes more than KF and at most K steps of 32 columns
// (K = 0: any number of steps, union re-read for the scatter).  Steps
// 0 .. KF-1 are full; only the lanes of the later steps are masked (a fully
// masked step reads x at the zero element and adds nothing).  Fused pass: row sums, d, objective terms,
// residuals and the accumulator updates; adjoint: the updates with the staged
// residuals.
template <int FMT, int MODE, uint32_t IW, int K, int KF>
__device__ __forceinline__ void rg_group(const RgParams& p, const RgStage& C, const uint4 G, uint32_t xs_a,
                                         uint32_t gw_a, uint32_t zc, uint32_t lane, float& f_hi, float& f_lo) {
    constexpr bool QUAD = MODE == ADJ_MODE_QUADRATIC;
    constexpr bool FP8 = FMT == DOSE_FMT_FP8E4M3_ROWSCALE;
    constexpr uint32_t RV = 4 * (uint32_t)sizeof(typename Fmt<FMT>::T);
    const uint32_t nU = G.y, u0 = G.x;
    // this lane's row of the group (lane l: row l / 8) and its per-row values,
    // fetched first so that their latency hides behind the union loads
    const uint32_t off = rg_row_off(G, lane >> 3);
    const bool has = off != 0xFFFFu;
    const uint32_t ra = has ? 4 * (C.row0 + off) : 4 * C.r_a;  // byte offset of the row in the staged vectors
    float r0, r1, r2, r3;
    float pv = 0.f, wv = 0.f, rsc = 1.f;
    if (QUAD) {
        pv = dev::lds_f32(C.vec0 + ra);
        wv = dev::lds_f32(C.vec1 + ra);
        if (FP8) rsc = dev::lds_f32(C.vrs + ra);
    } else {
        float rv = dev::lds_f32(C.vec0 + ra);
        if (FP8) rv = __fmul_rn(rv, dev::lds_f32(C.vrs + ra));
        rv = has ? rv : 0.f;
        r0 = __shfl_sync(0xffffffffu, rv, 0);
        r1 = __shfl_sync(0xffffffffu, rv, 8);
        r2 = __shfl_sync(0xffffffffu, rv, 16);
        r3 = __shfl_sync(0xffffffffu, rv, 24);
    }
    // this lane's union positions lane, lane + 32, ...: column index and value addresses
    const uint32_t ca = C.col + IW * (u0 + lane), va = C.val + RV * (u0 + lane);
    constexpr int KR = K ? K : 1;  // steps held in registers
    // the longest register-held groups keep the stored bits (two registers per
    // step for 16-bit values) and decode them again for the scatter
    constexpr bool KEEP_RAW = K >= 9;
    constexpr int KV = KEEP_RAW ? 1 : KR;
    uint32_t c[KR];
    uint4 raw[KR];
    float v[KV][4];
    if (K) {
#pragma unroll
        for (int it = 0; it < KR; ++it) {
            if (it < KF) {
                c[it] = rg_ldcol<IW>(ca + IW * 32 * it);
                raw[it] = rg_ldval<FMT>(va + RV * 32 * it);
            } else {
                // masked lanes read x at the zero element and values 0
                c[it] = rg_ldcol_lt<IW>(32 * it + lane, nU, ca + IW * 32 * it, zc);
                raw[it] = rg_ldval_lt<FMT>(32 * it + lane, nU, va + RV * 32 * it);
            }
        }
    }
    if (QUAD) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (K) {
#pragma unroll
            for (int it = 0; it < KR; ++it) {
                const float xv = dev::lds_f32(xs_a + 4 * c[it]);
                float q[4];
                rg_dec4<FMT>(raw[it], q);
                if (!KEEP_RAW)
                    for (int u = 0; u < 4; ++u) v[KEEP_RAW ? 0 : it][u] = q[u];
                a0 = __fmaf_rn(q[0], xv, a0);
                a1 = __fmaf_rn(q[1], xv, a1);
                a2 = __fmaf_rn(q[2], xv, a2);
                a3 = __fmaf_rn(q[3], xv, a3);
            }
        } else {
            const uint32_t nit = (nU + 31) >> 5;
            for (uint32_t it = 0; it < nit; ++it) {
                const uint32_t k = 32 * it + lane;
                const uint32_t cc = rg_ldcol_lt<IW>(k, nU, ca + IW * 32 * it, zc);
                float q[4];
                rg_dec4<FMT>(rg_ldval_lt<FMT>(k, nU, va + RV * 32 * it), q);
                const float xv = dev::lds_f32(xs_a + 4 * cc);
                a0 = __fmaf_rn(q[0], xv, a0);
                a1 = __fmaf_rn(q[1], xv, a1);
                a2 = __fmaf_rn(q[2], xv, a2);
                a3 = __fmaf_rn(q[3], xv, a3);
            }
        }
        const float sum = rg_reduce4(a0, a1, a2, a3, lane);
        const float dv = FMT == DOSE_FMT_U16_SCALE ? __fmul_rn(p.scale, sum) : (FP8 ? __fmul_rn(rsc, sum) : sum);
        const float rr = has ? __fmul_rn(__fmul_rn(__fmul_rn(2.0f, wv), __fsub_rn(dv, pv)), rsc) : 0.f;
        r0 = __shfl_sync(0xffffffffu, rr, 0);
        r1 = __shfl_sync(0xffffffffu, rr, 8);
        r2 = __shfl_sync(0xffffffffu, rr, 16);
        r3 = __shfl_sync(0xffffffffu, rr, 24);
        // objective term and d: one lane per row (no branch, so the scheduler can
        // interleave it with the accumulator updates below)
        const bool lead = has && (lane & 7u) == 0;
        float nh = f_hi, nl = f_lo;
        dev::df_add_wsq(nh, nl, wv, dv, pv);
        f_hi = lead ? nh : f_hi;
        f_lo = lead ? nl : f_lo;
        if (lead && p.d) p.d[C.row0 + off] = dv;
    } else if (K && !KEEP_RAW) {
#pragma unroll
        for (int it = 0; it < KR; ++it) rg_dec4<FMT>(raw[it], v[KEEP_RAW ? 0 : it]);
    }
    if (K) {
        // all loads of the accumulator before its stores (the union columns are distinct)
        float gv[KR];
#pragma unroll
        for (int it = 0; it < KR; ++it)
            gv[it] = it < KF ? dev::lds_f32(gw_a + 4 * c[it]) : dev::lds_f32_lt(32 * it + lane, nU, gw_a + 4 * c[it]);
#pragma unroll
        for (int it = 0; it < KR; ++it) {
            float q[4];
            if (KEEP_RAW) {
                rg_dec4<FMT>(raw[it], q);
            } else {
                for (int u = 0; u < 4; ++u) q[u] = v[KEEP_RAW ? 0 : it][u];
            }
            float t = __fmul_rn(q[0], r0);
            t = __fmaf_rn(q[1], r1, t);
            t = __fmaf_rn(q[2], r2, t);
            t = __fmaf_rn(q[3], r3, t);
            if (it < KF)
                dev::sts_f32(gw_a + 4 * c[it], __fadd_rn(gv[it], t));
            else
                dev::sts_f32_lt(32 * it + lane, nU, gw_a + 4 * c[it], __fadd_rn(gv[it], t));
        }
    } else {
        const uint32_t nit = (nU + 31) >> 5;
        for (uint32_t it = 0; it < nit; ++it) {
            const uint32_t k = 32 * it + lane;
            if (k < nU) {
                const uint32_t cc = rg_ldcol<IW>(ca + IW * 32 * it);
                float q[4];
                rg_dec4<FMT>(rg_ldval<FMT>(va + RV * 32 * it), q);
                float t = __fmul_rn(q[0], r0);
                t = __fmaf_rn(q[1], r1, t);
                t = __fmaf_rn(q[2], r2, t);
                t = __fmaf_rn(q[3], r3, t);
                const uint32_t ga = gw_a + 4 * cc;
                dev::sts_f32(ga, __fadd_rn(dev::lds_f32(ga), t));
            }
        }
    }
}

template <int FMT, int MODE, uint32_t IW>
__global__ void __maxnreg__(104) rg_kernel(const RgParams p) {
    constexpr bool QUAD = MODE == ADJ_MODE_QUADRATIC;
    constexpr uint32_t RV = 4 * (uint32_t)sizeof(typename Fmt<FMT>::T);
    constexpr uint32_t VA = RV >= 16 ? 1 : 16 / RV;
    constexpr uint32_t CA = 16 / IW;
    constexpr uint32_t kRsVec = QUAD ? 2 : 1;  // index of the FP8 row scales among the vectors
    extern __shared__ __align__(128) unsigned char smem[];

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth, NW = p.nw;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + 8;
    uint64_t* dbar = full + 16;
    double* fred = reinterpret_cast<double*>(smem + 256);        // 32 doubles: per-warp objective
    StageDesc* dwin = reinterpret_cast<StageDesc*>(smem + 1024);  // 2 x kDescWin descriptors
    const uint32_t W = p.wwidth, wlo = p.sched.wlo[blockIdx.x];
    const uint32_t gw_floats = round_up(W * 4, 128) / 4;
    float* gacc = reinterpret_cast<float*>(smem + kRgHeader);  // NW x gw_floats
    float* xs = gacc + NW * gw_floats;                          // QUAD: window of x and a zero
    const uint32_t x_bytes = QUAD ? round_up((W + 1) * 4, 128) : 0;
    unsigned char* slot_base = reinterpret_cast<unsigned char*>(xs) + x_bytes;
    const RgSlot SL = p.SL;
    const uint32_t s_begin = p.sched.cta_begin[blockIdx.x], s_end = p.sched.cta_begin[blockIdx.x + 1];
    const uint32_t nct = NW * 32;

    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < S; ++i) {
            dev::mbar_init(&full[i], 1);
            dev::mbar_init(&empty[i], NW);
        }
        dev::mbar_init(&dbar[0], 1);
        dev::mbar_init(&dbar[1], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();

    // every CTA is resident: the finalize kernel may be scheduled onto SMs as
    // their CTAs finish (it waits for this grid before reading its results)
    asm volatile("griddepcontrol.launch_dependents;");
    if (warp == 0) {
        if (lane == 0) rg_produce<FMT, IW, QUAD>(p, s_begin, s_end, slot_base, full, empty, dwin, dbar);
        return;
    }

    const uint32_t wi = warp - 1, ctid = threadIdx.x - 32;
    for (uint32_t j = ctid; j < NW * gw_floats; j += nct) gacc[j] = 0.f;
    if (QUAD)
        for (uint32_t j = ctid; j <= W; j += nct) xs[j] = j < W && wlo + j < p.ncols ? __ldg(p.x + wlo + j) : 0.f;
    dev::named_barrier(1, nct);

    // x of column c at xs_a + 4 c and this warp's accumulator of c at gw_a + 4 c
    // (c in the window); zc: the zero element after the window
    const uint32_t xs_a = dev::smem_u32(xs) - 4 * wlo;
    const uint32_t gw_a = dev::smem_u32(gacc + wi * gw_floats) - 4 * wlo;
    const uint32_t zc = wlo + W;
    const uint32_t slot0 = dev::smem_u32(slot_base);
    bool failed = false;
    float f_hi = 0.f, f_lo = 0.f;  // this lane's objective terms, double-float
    uint32_t st = 0, ph = 0, rot = 0;
    for (uint32_t s = s_begin; s < s_end; ++s) {
        if (!dev::mbar_wait_poll(&full[st], ph)) {
            atomicExch(p.err, kErrTimeoutFull);
            failed = true;
            break;
        }
        const uint32_t slot = slot0 + st * SL.bytes;
        const StageDesc D = slot_desc(slot);
        RgStage C;
        C.row0 = D.row0;
        C.r_a = D.row0 & ~3u;
        C.vec0 = slot + SL.vec_off - 4 * C.r_a;  // + 4 * row
        C.vec1 = C.vec0 + SL.vec_stride;
        C.vrs = C.vec0 + kRsVec * SL.vec_stride;
        C.col = slot + SL.col_off - IW * (D.nz0 & ~(CA - 1));
        C.val = slot + SL.val_off - RV * (D.nz0 & ~(VA - 1));
        const uint32_t grp_a = slot + SL.grp_off - 16 * D.ne0;
        for (uint32_t j = D.ne0 + (wi >= rot ? wi - rot : wi + NW - rot); j < D.ne1; j += NW) {
            const uint4 G = dev::lds_v4_if(true, grp_a + 16 * j);
            if (!rg_group_ok<IW>(G, D, C.col, p.nrows, zc, W, lane, p.err)) continue;
            // four code paths (each unrolled for its step count) keep the
            // kernel's instructions within the instruction cache
            const uint32_t nit = (G.y + 31) >> 5;
            if (nit <= 2)
                rg_group<FMT, MODE, IW, 2, 0>(p, C, G, xs_a, gw_a, zc, lane, f_hi, f_lo);
            else if (nit <= 4)
                rg_group<FMT, MODE, IW, 4, 2>(p, C, G, xs_a, gw_a, zc, lane, f_hi, f_lo);
            else if (nit <= 6)
                rg_group<FMT, MODE, IW, 6, 4>(p, C, G, xs_a, gw_a, zc, lane, f_hi, f_lo);
            else if (nit <= 9)
                rg_group<FMT, MODE, IW, 9, 6>(p, C, G, xs_a, gw_a, zc, lane, f_hi, f_lo);
            else
                rg_group<FMT, MODE, IW, 0, 0>(p, C, G, xs_a, gw_a, zc, lane, f_hi, f_lo);
            __syncwarp();  // this group's updates precede the next group's loads in every lane
        }
        rot = rot + 1 == NW ? 0 : rot + 1;
        __syncwarp();
        if (lane == 0) dev::mbar_arrive(&empty[st]);
        if (++st == S) {
            st = 0;
            ph ^= 1;
        }
    }
    // every worker waits on the same phases, so a timeout is seen by all of them
    if (failed) return;
    if (QUAD) {
        double f_lane = (double)f_hi + (double)f_lo;
        for (uint32_t o = 16; o > 0; o >>= 1) f_lane += __shfl_xor_sync(0xffffffffu, f_lane, o);
        if (lane == 0) fred[wi] = f_lane;
    }
    dev::named_barrier(1, nct);
    for (uint32_t j = ctid; j < W; j += nct) {
        float t = gacc[j];
        for (uint32_t w2 = 1; w2 < NW; ++w2) t = __fadd_rn(t, gacc[w2 * gw_floats + j]);
        p.g_part[(size_t)blockIdx.x * W + j] = t;
    }
    if (QUAD && ctid == 0) {
        double t = 0.0;
        for (uint32_t w2 = 0; w2 < NW; ++w2) t += fred[w2];
        p.f_part[blockIdx.x] = t;
    }
}

// Second kernel of the row-group passes, one wave of blocks, launched as a
// programmatic dependent of the main kernel so that it starts on SMs whose
// main CTA has finished:
//   fused pass only, first: the rows without entries (they do not depend on
//     the main kernel), four consecutive rows per thread and step (16-byte
//     loads of p and w, grid-stride): d = 0 and the objective term w p^2;
//   then, after the main kernel has completed: column blocks cb = block,
//     block + grid, ... : g_j = s * (sum of the partials of the CTAs whose
//     window holds j, in CTA order), and the optional projected-gradient step
//     on x; each block's objective sum goes to f_rows, and the last block to
//     finish (integer ticket) writes f = the CTAs' objective partials and the
//     blocks' sums, added in one fixed order, then resets the ticket.
struct RgFin {
    const float* g_part;
    const uint32_t* wlo;
    uint32_t W, nparts, ncols;
    float scale;
    float* g;
    float* x_update;
    float eta;
    const double* f_part;
    double* f;
    const uint32_t* mask;
    const float* p;
    const float* w;
    float* d;
    uint32_t nrows;
    double* f_rows;
    uint32_t* ticket;
    uint32_t nblk_g;
};

__global__ void __launch_bounds__(256, 8) rg_finalize(const RgFin q) {
    __shared__ float part[8][33];
    __shared__ double red[256];
    __shared__ uint32_t last;
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float hi = 0.f, lo = 0.f;
    if (q.f) {
        // rows without entries: thread takes rows 4i .. 4i+3 for i = tid, tid + T, ...
        // (two such steps' loads issued together)
        constexpr uint32_t U = 2;
        const uint32_t nq = (q.nrows + 3) / 4, T = gridDim.x * 256;
        const uint32_t full_q = q.nrows / 4;  // quads inside p and w (16-byte loads)
        const float4* __restrict__ p4 = reinterpret_cast<const float4*>(q.p);
        const float4* __restrict__ w4 = reinterpret_cast<const float4*>(q.w);
        for (uint32_t i0 = blockIdx.x * 256 + threadIdx.x; i0 < nq; i0 += U * T) {
            uint32_t m[U];
            float4 a[U], b[U];
#pragma unroll
            for (uint32_t k = 0; k < U; ++k) {
                const uint32_t i = i0 + k * T, r = 4 * i;
                m[k] = i < nq ? (__ldg(q.mask + (r >> 5)) >> (r & 31)) & 0xFu : 0xFu;
                if (i < nq && r + 4 > q.nrows) m[k] |= (0xFu << (q.nrows - r)) & 0xFu;  // rows past the end
                if (i < full_q) {
                    a[k] = __ldg(p4 + i);
                    b[k] = __ldg(w4 + i);
                } else {
                    float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    for (uint32_t u = 0; u < 4; ++u)
                        if (i < nq && r + u < q.nrows) {
                            t[u] = __ldg(q.p + r + u);
                            t[4 + u] = __ldg(q.w + r + u);
                        }
                    a[k] = make_float4(t[0], t[1], t[2], t[3]);
                    b[k] = make_float4(t[4], t[5], t[6], t[7]);
                }
            }
#pragma unroll
            for (uint32_t k = 0; k < U; ++k) {
                const uint32_t r = 4 * (i0 + k * T);
                const float pv[4] = {a[k].x, a[k].y, a[k].z, a[k].w}, wv[4] = {b[k].x, b[k].y, b[k].z, b[k].w};
#pragma unroll
                for (uint32_t u = 0; u < 4; ++u) {
                    if ((m[k] >> u) & 1u) continue;  // a row with entries, or past the end
                    if (q.d) q.d[r + u] = 0.0f;
                    if (pv[u] != 0.0f || !(fabsf(wv[u]) < INFINITY)) dev::df_add_wsq(hi, lo, wv[u], 0.0f, pv[u]);
                }
            }
        }
    }
    // the rest reads the main kernel's partials (and may update x, which it reads)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (uint32_t cb = blockIdx.x; cb < q.nblk_g; cb += gridDim.x) {
        const uint32_t j = cb * 32 + lane;
        float t = 0.f;
        if (j < q.ncols) {
            // warp w adds the partials c = w, w + 8, ... in order; eight loads in flight
            uint32_t c = w;
            for (; c + 56 < q.nparts; c += 64) {
                float v[8];
#pragma unroll
                for (uint32_t u = 0; u < 8; ++u) {
                    const uint32_t cc = c + 8 * u;
                    const uint32_t off = j - __ldg(q.wlo + cc);
                    v[u] = off < q.W ? __ldg(q.g_part + (size_t)cc * q.W + off) : 0.f;
                }
#pragma unroll
                for (uint32_t u = 0; u < 8; ++u) t = __fadd_rn(t, v[u]);
            }
            for (; c < q.nparts; c += 8) {
                const uint32_t off = j - __ldg(q.wlo + c);
                if (off < q.W) t = __fadd_rn(t, __ldg(q.g_part + (size_t)c * q.W + off));
            }
        }
        part[w][lane] = t;
        __syncthreads();
        if (w == 0 && j < q.ncols) {
            float tot = part[0][lane];
            for (uint32_t k = 1; k < 8; ++k) tot = __fadd_rn(tot, part[k][lane]);
            tot = __fmul_rn(q.scale, tot);
            if (q.g) q.g[j] = tot;
            if (q.x_update) {
                const float xn = __fsub_rn(q.x_update[j], __fmul_rn(q.eta, tot));
                q.x_update[j] = xn > 0.f ? xn : 0.f;
            }
        }
        __syncthreads();
    }
    if (!q.f) return;
    double fl = (double)hi + (double)lo;
    for (uint32_t o = 16; o > 0; o >>= 1) fl += __shfl_xor_sync(0xffffffffu, fl, o);
    if (lane == 0) red[w] = fl;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (uint32_t k = 0; k < 8; ++k) b += red[k];
        q.f_rows[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(q.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc = 0.0;
    const uint32_t n = q.nparts + gridDim.x;
    for (uint32_t i = threadIdx.x; i < n; i += 256)
        acc += i < q.nparts ? __ldcg(q.f_part + i) : __ldcg(q.f_rows + (i - q.nparts));
    red[threadIdx.x] = acc;
    __syncthreads();
    for (uint32_t st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *q.f = red[0];
        *q.ticket = 0;
    }
}

size_t rg_smem(const dose_matrix* A, const AdjTuning& t, bool quad, uint32_t nw) {
    const RowGroups& R = A->rg;
    const uint32_t es = value_bytes(A->fmt);
    const uint32_t nvec = 1 + (quad ? 1 : 0) + (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0);
    const RgSlot SL = rg_slot(R.tile_u, R.tile_g, R.tile_rows, es, R.iw, nvec);
    const size_t acc = round_up(R.sched.wwidth * 4, 128);
    const size_t x_bytes = quad ? round_up((R.sched.wwidth + 1) * 4, 128) : 0;
    return kRgHeader + nw * acc + x_bytes + (size_t)t.rg_stages * SL.bytes;
}

template <int FMT, int MODE, uint32_t IW>
cudaError_t launch_rg_t(const dose_matrix* A, const RgParams& p, size_t smem, cudaStream_t s) {
    auto k = rg_kernel<FMT, MODE, IW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<A->rg.sched.grid, 32 * (1 + p.nw), smem, s>>>(p);
    return cudaGetLastError();
}

template <int MODE, uint32_t IW>
cudaError_t launch_rg_fmt(const dose_matrix* A, const RgParams& p, size_t smem, cudaStream_t s) {
    switch (A->fmt) {
        case DOSE_FMT_U16_SCALE: return launch_rg_t<DOSE_FMT_U16_SCALE, MODE, IW>(A, p, smem, s);
        case DOSE_FMT_BF16: return launch_rg_t<DOSE_FMT_BF16, MODE, IW>(A, p, smem, s);
        case DOSE_FMT_F16: return launch_rg_t<DOSE_FMT_F16, MODE, IW>(A, p, smem, s);
        case DOSE_FMT_F32: return launch_rg_t<DOSE_FMT_F32, MODE, IW>(A, p, smem, s);
        case DOSE_FMT_FP8E4M3_ROWSCALE: return launch_rg_t<DOSE_FMT_FP8E4M3_ROWSCALE, MODE, IW>(A, p, smem, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

uint32_t rg_shape(const dose_matrix* A, const AdjTuning& t, bool quad, size_t* smem) {
    if (!A->rg.built || !A->rg.sched.desc) return 0;
    if (quad && A->rg.sched.wwidth > kXSmemMaxCols) return 0;
    uint32_t hi = t.rg_warps ? std::min<uint32_t>(t.rg_warps, kRgMaxWarps) : kRgMaxWarps;
    for (uint32_t nw = hi; nw >= 1; --nw)
        if (rg_smem(A, t, quad, nw) <= kMaxSmemPerBlock) {
            if (smem) *smem = rg_smem(A, t, quad, nw);
            return nw;
        }
    return 0;
}

bool rg_active(const dose_matrix* A, bool quad) {
    return A->adj_tuning.layout != 1 && rg_shape(A, A->adj_tuning, quad, nullptr) > 0;
}

uint64_t rg_matrix_bytes(const dose_matrix* A) {
    const RowGroups& R = A->rg;
    return R.n_union * (R.iw + 4ull * value_bytes(A->fmt)) + 16ull * R.host.size();
}

// Bytes of one fused pass: the layout once, the non-empty bits, p and w of every
// row (the kernel stages the grouped rows', the finalize reads the others'),
// FP8 row scales of the grouped rows, d if written, x in, g out, and the CTA
// partials written and read once.
uint64_t rg_fused_bytes(const dose_matrix* A, bool with_d) {
    const uint64_t nr = A->nrows, nc = A->ncols, P = A->rg.sched.grid, W = A->rg.sched.wwidth;
    return rg_matrix_bytes(A) + (nr + 7) / 8 + 8 * nr + (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 4 * nr : 0) +
           (with_d ? 4 * nr : 0) + 8 * nc + 8ull * P * W + 8 * P + 8;
}

// Bytes of one dose_spmv on the layout: the layout once, the non-empty bits,
// FP8 row scales, x in (once), d out (every row).
uint64_t rg_spmv_bytes(const dose_matrix* A) {
    const uint64_t nr = A->nrows, nc = A->ncols;
    return rg_matrix_bytes(A) + (nr + 7) / 8 + (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 4 * nr : 0) + 4 * nc + 4 * nr;
}

uint64_t rg_adjoint_bytes(const dose_matrix* A) {
    const uint64_t nr = A->nrows, nc = A->ncols, P = A->rg.sched.grid, W = A->rg.sched.wwidth;
    return rg_matrix_bytes(A) + 4 * nr + (A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 4 * nr : 0) + 4 * nc +
           8ull * P * W;
}

cudaError_t launch_rg(const dose_matrix* A, int mode, const float* x, const float* p, const float* w, const float* r,
                      float* d, double* f, float* g, float* x_update, float eta, cudaStream_t s) {
    const bool quad = mode == ADJ_MODE_QUADRATIC;
    size_t smem = 0;
    const uint32_t nw = rg_shape(A, A->adj_tuning, quad, &smem);
    if (!nw) return cudaErrorInvalidConfiguration;
    const RowGroups& R = A->rg;
    if (A->nrows > 0) {
        RgParams prm;
        prm.grp = R.grp;
        prm.ucol = R.ucol;
        prm.uval = R.uval;
        prm.scale = A->scale;
        prm.x = x;
        prm.d = d;
        prm.g_part = A->g_part;
        prm.f_part = A->f_part;
        prm.nrows = A->nrows;
        prm.ncols = A->ncols;
        prm.wwidth = R.sched.wwidth;
        prm.sched = ScheduleView{R.sched.desc, nullptr, R.sched.cta_begin, R.sched.wlo};
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
        const uint32_t es = value_bytes(A->fmt);
        prm.SL = rg_slot(R.tile_u, R.tile_g, R.tile_rows, es, R.iw, prm.vecs.n);
        prm.depth = A->adj_tuning.rg_stages;
        prm.nw = nw;
        prm.l2pf = A->adj_tuning.rg_l2_prefetch;
        prm.err = A->err;
        cudaError_t e;
        if (R.iw == 2)
            e = quad ? launch_rg_fmt<ADJ_MODE_QUADRATIC, 2>(A, prm, smem, s) : launch_rg_fmt<ADJ_MODE_ADJOINT, 2>(A, prm, smem, s);
        else
            e = quad ? launch_rg_fmt<ADJ_MODE_QUADRATIC, 4>(A, prm, smem, s) : launch_rg_fmt<ADJ_MODE_ADJOINT, 4>(A, prm, smem, s);
        if (e != cudaSuccess) return e;
    }
    RgFin q;
    q.g_part = A->g_part;
    q.wlo = R.sched.wlo;
    q.W = R.sched.wwidth;
    q.nparts = A->nrows > 0 ? R.sched.grid : 0;
    q.ncols = A->ncols;
    q.scale = A->fmt == DOSE_FMT_U16_SCALE ? A->scale : 1.0f;
    q.g = g;
    q.x_update = x_update;
    q.eta = eta;
    q.f_part = A->f_part;
    q.f = quad ? f : nullptr;
    q.mask = R.mask;
    q.p = p;
    q.w = w;
    q.d = d;
    q.nrows = A->nrows;
    q.f_rows = R.f_rows;
    q.ticket = R.ticket;
    q.nblk_g = A->ncols ? (A->ncols + 31) / 32 : 1;
    // one wave: the blocks that fit on every SM at once take the columns, then
    // (fused pass) the rows without entries
    const uint32_t nblk = quad ? R.nblk_rows : q.nblk_g;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblk);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = A->nrows > 0 ? 1 : 0;  // without a main kernel, an ordinary launch
    return cudaLaunchKernelEx(&cfg, rg_finalize, q);
}

}  // namespace dose
