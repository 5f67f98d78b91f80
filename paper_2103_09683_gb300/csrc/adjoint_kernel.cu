// Adjoint g = A^T r and the fused quadratic-objective pass
//   d = A x,  f = sum_i w_i (d_i - p_i)^2,  g = A^T [2 w (d - p)]
// in one pass over A.  The gradient of the dose objective is what the
// optimiser the paper motivates needs every iteration (Sec. I: function values
// and gradients of the beam variables; Sec. II-A: A fixed, x changing).
//
// Determinism (Sec. II-D: no reductions whose order is not fixed, so no float
// atomics): every consumer warp owns a private shared-memory accumulator of all
// ncols gradient entries.  A warp scatters one row at a time; the entries of a
// row have distinct columns, so the 32 lanes never update the same word in one
// instruction, and rows follow a fixed order per warp.  At the end each CTA
// sums its warps' accumulators in warp order into a per-CTA partial, and a
// second kernel sums the partials in CTA order (and applies an optional
// projected-gradient update x <- max(0, x - eta g)).  The stage pipeline is the
// one of the forward kernel (bulk async copies into a shared-memory ring).
#include "stage_common.cuh"

namespace dose {
namespace {

struct AdjParams {
    const uint32_t* row_ptr;
    const uint32_t* col;
    const void* val;
    const float* row_scale;
    float scale;
    const float* x;   // QUADRATIC
    const float* p;   // QUADRATIC
    const float* w;   // QUADRATIC
    const float* r;   // ADJOINT
    float* d;         // QUADRATIC, may be null
    float* g_part;    // grid x ncols
    double* f_part;   // grid
    uint32_t nrows, ncols;
    ScheduleView sched;
    uint32_t tile_nnz, tile_rows, depth, cwarps;
    int* err;
};

constexpr uint32_t kAdjHeader = 4096;  // barriers, warp reduction scratch, row lists (512 B), row results (2 KB)

template <int FMT>
__device__ __forceinline__ float row_factor(const AdjParams& p, uint32_t row) {
    // Per-row factor folded into r for the scatter (FP8 row scale); the U16
    // matrix scale is applied once per column in the finalize kernel.
    if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) return __ldg(p.row_scale + row);
    return 1.0f;
}

template <int FMT>
__device__ __forceinline__ float finish_dot(const AdjParams& p, uint32_t row, float acc) {
    if (FMT == DOSE_FMT_U16_SCALE) return __fmul_rn(p.scale, acc);
    if (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) return __fmul_rn(__ldg(p.row_scale + row), acc);
    return acc;
}

// gw[col_k] += a_k * rj for the entries k in [kb, ke) of one row, lanes strided
// by 32 (columns in a row are distinct: the four loads precede the four stores).
template <int FMT>
__device__ __forceinline__ void scatter_row(float* __restrict__ gw, const typename Fmt<FMT>::T* __restrict__ vs,
                                            uint32_t vb, const uint32_t* __restrict__ cs, uint32_t cb,
                                            uint32_t kb, uint32_t ke, uint32_t lane, float rj) {
    for (uint32_t k0 = kb + lane; k0 < ke; k0 += 128) {
        uint32_t c[4];
        float a[4], gv[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t k = k0 + 32u * u;
            ok[u] = k < ke;
            c[u] = ok[u] ? cs[k - cb] : 0;
            a[u] = ok[u] ? Fmt<FMT>::dec(vs[k - vb]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) gv[u] = ok[u] ? gw[c[u]] : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (ok[u]) gw[c[u]] = __fmaf_rn(a[u], rj, gv[u]);
    }
}

template <int FMT, int MODE>
__global__ void __launch_bounds__(544, 1) adjoint_kernel(const AdjParams p) {
    using T = typename Fmt<FMT>::T;
    constexpr uint32_t VA = Fmt<FMT>::kAlign;
    constexpr bool QUAD = MODE == ADJ_MODE_QUADRATIC;
    extern __shared__ __align__(128) unsigned char smem[];

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth, W = p.cwarps;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + S;
    float* red = reinterpret_cast<float*>(smem + 256);          // 32 floats
    double* fred = reinterpret_cast<double*>(smem + 384);       // 16 doubles
    uint8_t* rowlist = smem + 512;                               // 16 x 32 bytes
    float* dres = reinterpret_cast<float*>(smem + 1024);        // 16 x 32 floats
    const uint32_t gw_bytes = round_up(p.ncols * 4, 128);
    float* gacc = reinterpret_cast<float*>(smem + kAdjHeader);   // W x ncols
    float* xs = reinterpret_cast<float*>(smem + kAdjHeader + W * gw_bytes);
    const uint32_t x_bytes = QUAD ? round_up(p.ncols * 4, 128) : 0;
    unsigned char* stage_base = smem + kAdjHeader + W * gw_bytes + x_bytes;
    const StageLayout SL = stage_layout(p.tile_nnz, p.tile_rows, sizeof(T));

    const uint32_t s_begin = p.sched.cta_begin[blockIdx.x];
    const uint32_t s_end = p.sched.cta_begin[blockIdx.x + 1];

    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < S; ++i) {
            dev::mbar_init(&full[i], 1);
            dev::mbar_init(&empty[i], W);
        }
        dev::fence_mbar_init();
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0)
            run_producer<FMT>(p.sched, s_begin, s_end, p.row_ptr, p.col, p.val, stage_base, SL, full, empty, S,
                              p.err);
        return;
    }

    const uint32_t cw = warp - 1;
    const uint32_t ctid = threadIdx.x - 32;
    const uint32_t nct = W * 32;
    for (uint32_t j = ctid; j < W * (gw_bytes / 4); j += nct) gacc[j] = 0.f;
    if (QUAD)
        for (uint32_t j = ctid; j < p.ncols; j += nct) xs[j] = __ldg(p.x + j);
    dev::named_barrier(1, nct);

    float* gw = gacc + cw * (gw_bytes / 4);
    uint8_t* my_rows = rowlist + cw * 32;
    float* my_d = dres + cw * 32;
    double f_lane = 0.0;
    float coop_s = 0.f;
    bool failed = false;

    uint32_t st = 0, ph = 0;
    for (uint32_t s = s_begin; s < s_end; ++s) {
        if (!dev::mbar_wait_bounded(&full[st], ph)) {
            atomicExch(p.err, kErrTimeoutFull);
            failed = true;
            break;
        }
        const unsigned char* buf = stage_base + st * SL.bytes;
        const uint8_t meta = p.sched.meta[s];
        const uint32_t nz0 = p.sched.nz0[s], nz1 = p.sched.nz0[s + 1];
        const T* vs = reinterpret_cast<const T*>(buf + SL.val_off);
        const uint32_t* cs = reinterpret_cast<const uint32_t*>(buf + SL.col_off);
        const uint32_t vb = nz0 & ~(VA - 1), cb = nz0 & ~3u;

        if (!(meta & STAGE_COOP)) {
            const uint32_t r0 = p.sched.row0[s], r1 = p.sched.row0[s + 1];
            const uint32_t* rps = reinterpret_cast<const uint32_t*>(buf + SL.rp_off);
            const uint32_t rb0 = r0 & ~3u;
            const uint32_t lg = meta & STAGE_LANES_MASK;
            const uint32_t L = 1u << lg, NG = 32u >> lg;
            const uint32_t g = lane >> lg, li = lane & (L - 1);
            const uint32_t nchunks = (r1 - r0 + 31) / 32;
            for (uint32_t c = (cw + W - (s % W)) % W; c < nchunks; c += W) {
                const uint32_t rb = r0 + c * 32;
                const uint32_t r = rb + lane;
                const bool valid = r < r1;
                const uint32_t beg = valid ? rps[r - rb0] : 0, end = valid ? rps[r + 1 - rb0] : 0;
                const unsigned nonempty = __ballot_sync(0xffffffffu, end > beg);
                const uint32_t cnt = __popc(nonempty);
                float rv = 0.f;
                if (QUAD) {
                    const float pv = valid ? __ldg(p.p + r) : 0.f;
                    const float wv = valid ? __ldg(p.w + r) : 0.f;
                    if (end > beg) my_rows[__popc(nonempty & ((1u << lane) - 1))] = (uint8_t)lane;
                    __syncwarp();
                    // forward: d for the non-empty rows, L lanes per row
                    for (uint32_t base = 0; base < cnt; base += NG) {
                        const uint32_t idx = base + g;
                        const bool has = idx < cnt;
                        const uint32_t j = has ? my_rows[idx] : 0;
                        const uint32_t rs = __shfl_sync(0xffffffffu, beg, j);
                        const uint32_t re = __shfl_sync(0xffffffffu, end, j);
                        float sum = 0.f;
                        if (has) {
#pragma unroll 4
                            for (uint32_t k = rs + li; k < re; k += L)
                                sum = __fmaf_rn(Fmt<FMT>::dec(vs[k - vb]), xs[cs[k - cb]], sum);
                        }
                        for (uint32_t off = L >> 1; off > 0; off >>= 1)
                            sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, off));
                        if (has && li == 0) my_d[j] = finish_dot<FMT>(p, rb + j, sum);
                    }
                    __syncwarp();
                    const float dv = end > beg ? my_d[lane] : 0.f;
                    if (valid) {
                        if (p.d) p.d[r] = dv;
                        const double ed = (double)dv - (double)pv;  // residual in FP64
                        f_lane += (double)wv * ed * ed;
                        rv = (float)(2.0 * (double)wv * ed);
                    }
                } else {
                    rv = valid ? __ldg(p.r + r) : 0.f;
                }
                if (valid && end > beg) rv = __fmul_rn(rv, row_factor<FMT>(p, r));
                // scatter the non-empty rows one at a time, in row order
                unsigned m = nonempty;
                while (m) {
                    const uint32_t j = __ffs(m) - 1;
                    m &= m - 1;
                    const uint32_t rs = __shfl_sync(0xffffffffu, beg, j);
                    const uint32_t re = __shfl_sync(0xffffffffu, end, j);
                    const float rj = __shfl_sync(0xffffffffu, rv, j);
                    scatter_row<FMT>(gw, vs, vb, cs, cb, rs, re, lane, rj);
                    __syncwarp();
                }
            }
        } else {
            // one chunk of a long row: every consumer thread takes part
            const uint32_t row = p.sched.row0[s];
            if (QUAD) {
                if (meta & STAGE_FIRST) coop_s = 0.f;
                for (uint32_t k = nz0 + ctid; k < nz1; k += nct)
                    coop_s = __fmaf_rn(Fmt<FMT>::dec(vs[k - vb]), xs[cs[k - cb]], coop_s);
                if (meta & STAGE_LAST) {
                    float sum = coop_s;
                    for (uint32_t off = 16; off > 0; off >>= 1)
                        sum = __fadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, off));
                    if (lane == 0) red[cw] = sum;
                    dev::named_barrier(1, nct);
                    float tot = red[0];
                    for (uint32_t w2 = 1; w2 < W; ++w2) tot = __fadd_rn(tot, red[w2]);
                    const float dv = finish_dot<FMT>(p, row, tot);
                    const float pv = __ldg(p.p + row), wv = __ldg(p.w + row);
                    const double ed = (double)dv - (double)pv;
                    if (ctid == 0) {
                        if (p.d) p.d[row] = dv;
                        f_lane += (double)wv * ed * ed;
                    }
                    const float rj = __fmul_rn((float)(2.0 * (double)wv * ed), row_factor<FMT>(p, row));
                    const uint32_t kb = p.row_ptr[row], ke = p.row_ptr[row + 1];
                    // warp cw scatters entries kb + 32*(cw + W*t) + lane into its own accumulator
                    for (uint32_t k0 = kb + cw * 32; k0 < ke; k0 += nct) {
                        const uint32_t k = k0 + lane;
                        if (k < ke) {
                            const uint32_t cc = __ldg(p.col + k);
                            gw[cc] = __fmaf_rn(Fmt<FMT>::dec(static_cast<const T*>(p.val)[k]), rj, gw[cc]);
                        }
                    }
                    dev::named_barrier(1, nct);
                }
            } else {
                const float rj = __fmul_rn(__ldg(p.r + row), row_factor<FMT>(p, row));
                for (uint32_t k0 = nz0 + cw * 32; k0 < nz1; k0 += nct) {
                    const uint32_t k = k0 + lane;
                    if (k < nz1) {
                        const uint32_t cc = cs[k - cb];
                        gw[cc] = __fmaf_rn(Fmt<FMT>::dec(vs[k - vb]), rj, gw[cc]);
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) dev::mbar_arrive(&empty[st]);
        if (++st == S) {
            st = 0;
            ph ^= 1;
        }
    }
    if (failed) return;  // every consumer times out on the same phase: no one is left at a barrier

    // CTA partials: warp accumulators summed in warp order; f in a fixed tree.
    if (QUAD) {
        for (uint32_t off = 16; off > 0; off >>= 1) f_lane += __shfl_xor_sync(0xffffffffu, f_lane, off);
        if (lane == 0) fred[cw] = f_lane;
    }
    dev::named_barrier(1, nct);
    const uint32_t gstride = gw_bytes / 4;
    for (uint32_t j = ctid; j < p.ncols; j += nct) {
        float t = gacc[j];
        for (uint32_t w2 = 1; w2 < W; ++w2) t = __fadd_rn(t, gacc[w2 * gstride + j]);
        p.g_part[(size_t)blockIdx.x * p.ncols + j] = t;
    }
    if (ctid == 0) {
        double t = 0.0;
        if (QUAD)
            for (uint32_t w2 = 0; w2 < W; ++w2) t += fred[w2];
        p.f_part[blockIdx.x] = t;
    }
}

// g_j = s * sum_c g_part[c][j] (CTA order), f = sum_c f_part[c]; optional
// projected-gradient update of x.
__global__ void adjoint_finalize(const float* __restrict__ g_part, const double* __restrict__ f_part,
                                 uint32_t nparts, uint32_t ncols, float scale, float* g, double* f,
                                 float* x_update, float eta) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < ncols) {
        float t = 0.f;
        for (uint32_t c = 0; c < nparts; ++c) t = __fadd_rn(t, g_part[(size_t)c * ncols + j]);
        t = __fmul_rn(scale, t);
        if (g) g[j] = t;
        if (x_update) {
            const float xn = __fsub_rn(x_update[j], __fmul_rn(eta, t));
            x_update[j] = xn > 0.f ? xn : 0.f;
        }
    }
    if (f && blockIdx.x == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (uint32_t c = 0; c < nparts; ++c) t += f_part[c];
        *f = t;
    }
}

template <int FMT, int MODE>
cudaError_t launch_adj_t(const dose_matrix* A, const AdjParams& p, size_t smem, cudaStream_t s) {
    auto k = adjoint_kernel<FMT, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<A->grid, 32 * (p.cwarps + 1), smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

size_t adjoint_smem_bytes(const dose_matrix* A, const Tuning& t, uint32_t warps, bool need_x) {
    const uint32_t esize = A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 2;
    const StageLayout SL = stage_layout(t.tile_nnz, t.tile_rows, esize);
    const size_t col_bytes = round_up(A->ncols * 4, 128);
    return kAdjHeader + warps * col_bytes + (need_x ? col_bytes : 0) + (size_t)t.stages * SL.bytes;
}

// Consumer warps that fit in shared memory next to the stage ring (0 = none).
uint32_t adjoint_warps(const dose_matrix* A, const Tuning& t, bool need_x, int max_smem) {
    for (uint32_t w = 16; w >= 1; --w)
        if (adjoint_smem_bytes(A, t, w, need_x) <= (size_t)max_smem) return w;
    return 0;
}

// Pipeline shape of the adjoint kernels: the forward schedule with at most 3
// ring slots, leaving shared memory for the per-warp accumulators.
static Tuning adjoint_tuning(const dose_matrix* A) {
    Tuning t = A->tuning;
    if (t.stages > 3) t.stages = 3;
    return t;
}

cudaError_t launch_adjoint(const dose_matrix* A, int mode, const float* x, const float* p, const float* w,
                           const float* r, float* d, double* f, float* g, float* x_update, float eta,
                           cudaStream_t s) {
    const bool quad = mode == ADJ_MODE_QUADRATIC;
    const Tuning t = adjoint_tuning(A);
    const uint32_t W = adjoint_warps(A, t, quad, kMaxSmemPerBlock);
    if (W == 0) return cudaErrorInvalidConfiguration;
    if (A->nrows > 0) {
        AdjParams prm;
        prm.row_ptr = A->row_ptr;
        prm.col = A->col;
        prm.val = A->val;
        prm.row_scale = A->row_scale;
        prm.scale = A->scale;
        prm.x = x;
        prm.p = p;
        prm.w = w;
        prm.r = r;
        prm.d = d;
        prm.g_part = A->g_part;
        prm.f_part = A->f_part;
        prm.nrows = A->nrows;
        prm.ncols = A->ncols;
        prm.sched = ScheduleView{A->st_row0, A->st_nz0, A->st_meta, A->st_cta_begin};
        prm.tile_nnz = t.tile_nnz;
        prm.tile_rows = t.tile_rows;
        prm.depth = t.stages;
        prm.cwarps = W;
        prm.err = A->err;
        const size_t smem = adjoint_smem_bytes(A, t, W, quad);
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
            case DOSE_FMT_FP8E4M3_ROWSCALE:
                e = quad ? launch_adj_t<DOSE_FMT_FP8E4M3_ROWSCALE, ADJ_MODE_QUADRATIC>(A, prm, smem, s)
                         : launch_adj_t<DOSE_FMT_FP8E4M3_ROWSCALE, ADJ_MODE_ADJOINT>(A, prm, smem, s);
                break;
        }
        if (e != cudaSuccess) return e;
    }
    const uint32_t nparts = A->nrows > 0 ? A->grid : 0;
    const float scale = A->fmt == DOSE_FMT_U16_SCALE ? A->scale : 1.0f;
    const uint32_t blocks = A->ncols ? (A->ncols + 255) / 256 : 1;
    adjoint_finalize<<<blocks, 256, 0, s>>>(A->g_part, A->f_part, nparts, A->ncols, scale, g, quad ? f : nullptr,
                                            x_update, eta);
    return cudaGetLastError();
}

}  // namespace dose
