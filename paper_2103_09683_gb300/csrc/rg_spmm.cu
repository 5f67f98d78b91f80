// Batched dose SpMM on the row-group layout: D_m = A_m X_m for several
// matrices (beams x uncertainty scenarios, Sec. I) and up to 16 spot-weight
// vectors each, in one persistent launch.
//
// One CTA per SM walks the matrices in order and, for each, its share of that
// matrix's row-group stages (the column-windowed schedule of rg_layout.cu),
// streamed by a producer thread through a shared-memory ring that runs on from
// matrix to matrix.  The workers hold the CTA's window of X_m in shared memory
// (16 floats per column, zero past nvec, and a zero column after the window).
// A warp takes a whole group: lane l = 8 q + t computes row t / 2 of the group
// for vectors 8 (t % 2) .. 8 (t % 2) + 7 over the union positions u = q, q + 4,
// ... (one X-row gather serves the four rows of the group), then the four
// lane slices q are added by a fixed butterfly and every lane stores two of its
// row's results.  Rows without entries get D = 0 from a separate pass that
// runs beside it (the SpMM kernel is its programmatic dependent).
// Deterministic: static assignment of groups to warps, fixed per-lane order,
// fixed butterfly.
#include "rg_common.cuh"

#include <algorithm>
#include <string>

namespace dose {
namespace {

constexpr uint32_t kMmMaxPerLaunch = kRgSpmmMaxPerLaunch;
constexpr uint32_t kMmWorkers = 16;      // worker warps (plus one producer)
constexpr uint32_t kMmHeader = 1024;     // mbarriers
constexpr uint32_t kMmXStride = 16;      // floats per column of the staged window of X

struct MmItem {
    const uint4* grp;
    const void* ucol;
    const void* uval;
    const StageDesc* desc;
    const uint32_t* cta_begin;
    const uint32_t* wlo;
    const float* row_scale;  // FP8 (padded to whole 16-byte pieces)
    const float* X;          // ncols x nvec, row-major
    float* D;                // nrows x nvec, row-major
    float scale;             // U16
    uint32_t nrows, ncols, W;
};

struct MmParams {
    MmItem item[kMmMaxPerLaunch];
    uint32_t count, nvec, depth, nw;
    RgSlot SL;
    int* err;
};

// Rows without entries: D = 0 (every matrix of the launch, grid-stride over
// 16-byte pieces of D when nvec is a multiple of 4, else over floats).
struct MmZero {
    const uint32_t* mask[kMmMaxPerLaunch];
    float* D[kMmMaxPerLaunch];
    uint32_t nrows[kMmMaxPerLaunch];
    uint32_t count, nvec;
};

__global__ void __launch_bounds__(256) rg_spmm_zero(const __grid_constant__ MmZero z) {
    // the SpMM kernel (launched next, as a programmatic dependent) writes the
    // other rows and may run beside this one
    asm volatile("griddepcontrol.launch_dependents;");
    const uint32_t T = gridDim.x * blockDim.x;
    for (uint32_t m = 0; m < z.count; ++m) {
        float* D = z.D[m];
        const uint32_t* mask = z.mask[m];
        if ((z.nvec & 3u) == 0 && (reinterpret_cast<uintptr_t>(D) & 15u) == 0) {
            // 16-byte pieces, consecutive threads on consecutive pieces
            const uint32_t per = z.nvec / 4;  // 1 .. 4
            const uint64_t n = (uint64_t)z.nrows[m] * per;
            for (uint64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += T) {
                const uint32_t r = per == 4 ? (uint32_t)(i >> 2) : (uint32_t)(i / per);
                if (!((__ldg(mask + (r >> 5)) >> (r & 31)) & 1u))
                    reinterpret_cast<float4*>(D)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            const uint64_t n = (uint64_t)z.nrows[m] * z.nvec;
            for (uint64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += T) {
                const uint32_t r = (uint32_t)(i / z.nvec);
                if (!((__ldg(mask + (r >> 5)) >> (r & 31)) & 1u)) D[i] = 0.0f;
            }
        }
    }
}

// One stored value (row g's, of a union entry) at a, decoded; 0 unless k < n.
template <int FMT>
__device__ __forceinline__ float mm_val_lt(uint32_t k, uint32_t n, uint32_t a) {
    if constexpr (FMT == DOSE_FMT_F32) return dev::lds_f32_lt(k, n, a);
    if constexpr (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) return dev::dec_e4m3((uint8_t)dev::lds_u8_lt(k, n, a));
    const uint32_t q = dev::lds_u16_lt(k, n, a);
    if constexpr (FMT == DOSE_FMT_BF16) return __uint_as_float(q << 16);
    if constexpr (FMT == DOSE_FMT_F16) return dev::f16_to_f32((uint16_t)q);
    return __fsub_rn(__uint_as_float(0x4B000000u | q), 8388608.0f);  // u16 code, exactly
}

__device__ __forceinline__ float4 mm_ld4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ StageDesc mm_desc(const StageDesc* d) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(d)), b = __ldg(reinterpret_cast<const uint4*>(d) + 1);
    StageDesc D;
    D.row0 = a.x;
    D.row1 = a.y;
    D.nz0 = a.z;
    D.nz1 = a.w;
    D.ne0 = b.x;
    D.ne1 = b.y;
    D.meta = b.z;
    D.pad = 0;
    return D;
}

// Producer (one thread): the CTA's stages of every matrix in order through one
// ring: group records, union columns, union values and (FP8) the rows' scales.
// The next stage's descriptor is read while the current one's slot is awaited.
// Bounded waits; the copies in flight are drained before returning.
template <int FMT, uint32_t IW>
__device__ void mm_produce(const MmParams& p, unsigned char* slot_base, uint64_t* full, uint64_t* empty) {
    constexpr uint32_t RV = 4 * (uint32_t)sizeof(typename Fmt<FMT>::T);
    constexpr uint32_t VA = RV >= 16 ? 1 : 16 / RV;
    constexpr uint32_t CA = 16 / IW;
    constexpr bool FP8 = FMT == DOSE_FMT_FP8E4M3_ROWSCALE;
    const RgSlot& SL = p.SL;
    const uint32_t S = p.depth;
    uint32_t st = 0, ph = 0, issued = 0;
    bool ok = true;
    for (uint32_t m = 0; m < p.count && ok; ++m) {
        const MmItem& it = p.item[m];
        const uint32_t sb = it.cta_begin[blockIdx.x], se = it.cta_begin[blockIdx.x + 1];
        const unsigned char* ucol = static_cast<const unsigned char*>(it.ucol);
        const unsigned char* uval = static_cast<const unsigned char*>(it.uval);
        StageDesc next{};
        if (sb < se) next = mm_desc(it.desc + sb);
        for (uint32_t s = sb; s < se; ++s) {
            const StageDesc D = next;
            if (s + 1 < se) next = mm_desc(it.desc + s + 1);
            if (!dev::mbar_wait_poll(&empty[st], ph ^ 1)) {
                atomicExch(p.err, kErrTimeoutEmpty);
                ok = false;
                break;
            }
            unsigned char* buf = slot_base + st * SL.bytes;
            *reinterpret_cast<StageDesc*>(buf) = D;
            const uint32_t ng = D.ne1 - D.ne0;
            const uint32_t c_a = D.nz0 & ~(CA - 1), c_n = D.nz1 > D.nz0 ? round_up(D.nz1, CA) - c_a : 0;
            const uint32_t v_a = D.nz0 & ~(VA - 1), v_n = D.nz1 > D.nz0 ? round_up(D.nz1, VA) - v_a : 0;
            const uint32_t r_a = D.row0 & ~3u;
            uint32_t vn = 0;
            if (FP8) {
                const uint32_t e = min(round_up(D.row1, 4), round_up(it.nrows, 4));
                vn = e > r_a ? e - r_a : 0;
            }
            dev::mbar_arrive_expect_tx(&full[st], ng * 16 + c_n * IW + v_n * RV + vn * 4);
            if (ng) dev::bulk_g2s(buf + SL.grp_off, it.grp + D.ne0, ng * 16, &full[st]);
            if (c_n) dev::bulk_g2s(buf + SL.col_off, ucol + (size_t)c_a * IW, c_n * IW, &full[st]);
            if (v_n) dev::bulk_g2s(buf + SL.val_off, uval + (size_t)v_a * RV, v_n * RV, &full[st]);
            if (vn) dev::bulk_g2s(buf + SL.vec_off, it.row_scale + r_a, vn * 4, &full[st]);
            ++issued;
            if (++st == S) {
                st = 0;
                ph ^= 1;
            }
        }
    }
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
}

template <int FMT, uint32_t IW>
__global__ void __launch_bounds__((kMmWorkers + 1) * 32, 1) rg_spmm_kernel(const __grid_constant__ MmParams p) {
    constexpr uint32_t RV = 4 * (uint32_t)sizeof(typename Fmt<FMT>::T);
    constexpr uint32_t ES = (uint32_t)sizeof(typename Fmt<FMT>::T);
    constexpr uint32_t VA = RV >= 16 ? 1 : 16 / RV;
    constexpr uint32_t CA = 16 / IW;
    constexpr bool FP8 = FMT == DOSE_FMT_FP8E4M3_ROWSCALE;
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth, NW = p.nw;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + 8;
    float* xs = reinterpret_cast<float*>(smem + kMmHeader);  // (W + 1) x 16 floats: the window of X and a zero column
    uint32_t wmax = 0;
    for (uint32_t m = 0; m < p.count; ++m) wmax = max(wmax, p.item[m].W);
    unsigned char* slot_base = smem + kMmHeader + round_up((wmax + 1) * kMmXStride * 4, 128);
    const RgSlot SL = p.SL;
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < S; ++i) {
            dev::mbar_init(&full[i], 1);
            dev::mbar_init(&empty[i], NW);
        }
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (warp == 0) {
        if (lane == 0) mm_produce<FMT, IW>(p, slot_base, full, empty);
        return;
    }
    const uint32_t wi = warp - 1, ctid = threadIdx.x - 32, nct = NW * 32;
    // lane = 8 q + t: union positions u = q (mod 4), row g = t / 2, vectors 8 h .. 8 h + 7
    const uint32_t q = lane >> 3, g = (lane >> 1) & 3u, h = lane & 1u;
    const uint32_t slot0 = dev::smem_u32(slot_base);
    uint32_t st = 0, ph = 0, rot = 0;
    for (uint32_t m = 0; m < p.count; ++m) {
        const MmItem& it = p.item[m];
        const uint32_t W = it.W, wlo = it.wlo[blockIdx.x];
        dev::named_barrier(1, nct);  // every worker is done with the previous window of X
        for (uint32_t j = ctid; j < (W + 1) * kMmXStride; j += nct) {
            const uint32_t c = j / kMmXStride, v = j % kMmXStride;
            xs[j] = c < W && wlo + c < it.ncols && v < p.nvec ? __ldg(it.X + (size_t)(wlo + c) * p.nvec + v) : 0.f;
        }
        dev::named_barrier(1, nct);
        const uint32_t xs_a = dev::smem_u32(xs) - 4 * kMmXStride * wlo + 32 * h;  // + 64 c: x[c][8h ..]
        const uint32_t zc = wlo + W;                                             // the zero column
        const uint32_t sb = it.cta_begin[blockIdx.x], se = it.cta_begin[blockIdx.x + 1];
        for (uint32_t s = sb; s < se; ++s) {
            if (!dev::mbar_wait_poll(&full[st], ph)) {
                atomicExch(p.err, kErrTimeoutFull);
                return;  // every worker waits on the same phases, so all of them leave here
            }
            const uint32_t slot = slot0 + st * SL.bytes;
            const StageDesc D = slot_desc(slot);
            const uint32_t col_a = slot + SL.col_off - IW * (D.nz0 & ~(CA - 1));
            const uint32_t val_a = slot + SL.val_off - RV * (D.nz0 & ~(VA - 1)) + ES * g;
            const uint32_t vrs = slot + SL.vec_off - 4 * (D.row0 & ~3u);
            const uint32_t grp_a = slot + SL.grp_off - 16 * D.ne0;
            for (uint32_t j = D.ne0 + (wi + NW - rot) % NW; j < D.ne1; j += NW) {
                const uint4 G = dev::lds_v4_if(true, grp_a + 16 * j);
                const uint32_t nU = G.y, u0 = G.x, nfull = nU >> 2;
                float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                auto mac = [&](float a, uint32_t c) {
                    const float4 x0 = mm_ld4(xs_a + 64 * c), x1 = mm_ld4(xs_a + 64 * c + 16);
                    acc[0] = __fmaf_rn(a, x0.x, acc[0]);
                    acc[1] = __fmaf_rn(a, x0.y, acc[1]);
                    acc[2] = __fmaf_rn(a, x0.z, acc[2]);
                    acc[3] = __fmaf_rn(a, x0.w, acc[3]);
                    acc[4] = __fmaf_rn(a, x1.x, acc[4]);
                    acc[5] = __fmaf_rn(a, x1.y, acc[5]);
                    acc[6] = __fmaf_rn(a, x1.z, acc[6]);
                    acc[7] = __fmaf_rn(a, x1.w, acc[7]);
                };
                // this lane's union positions u = q, q + 4, ...: steps where all four
                // slices have a position need no mask
                const uint32_t ca = col_a + IW * (u0 + q), va = val_a + RV * (u0 + q);
#pragma unroll 4
                for (uint32_t k = 0; k < nfull; ++k) {
                    const uint32_t c = rg_ldcol<IW>(ca + 4 * IW * k);
                    mac(mm_val_lt<FMT>(0u, 1u, va + 4 * RV * k), c);
                }
                if (nU & 3u) {
                    const uint32_t u = 4 * nfull + q;
                    const uint32_t c = rg_ldcol_lt<IW>(u, nU, ca + 4 * IW * nfull, zc);
                    mac(mm_val_lt<FMT>(u, nU, va + 4 * RV * nfull), c);
                }
                // the four slices of the union: a fixed butterfly over q
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    acc[i] = __fadd_rn(acc[i], __shfl_xor_sync(0xffffffffu, acc[i], 8));
                    acc[i] = __fadd_rn(acc[i], __shfl_xor_sync(0xffffffffu, acc[i], 16));
                }
                const uint32_t off = rg_row_off(G, g);
                if (off != 0xFFFFu) {
                    const uint32_t row = D.row0 + off;
                    const float sc = FP8 ? dev::lds_f32(vrs + 4 * row) : (FMT == DOSE_FMT_U16_SCALE ? it.scale : 1.f);
                    // lane slice q stores vectors 8 h + 2 q and 8 h + 2 q + 1
                    const float r0 = q == 0 ? acc[0] : q == 1 ? acc[2] : q == 2 ? acc[4] : acc[6];
                    const float r1 = q == 0 ? acc[1] : q == 1 ? acc[3] : q == 2 ? acc[5] : acc[7];
                    const uint32_t v = 8 * h + 2 * q;
                    const bool scaled = FP8 || FMT == DOSE_FMT_U16_SCALE;
                    float* dr = it.D + (size_t)row * p.nvec;
                    if (v < p.nvec) dr[v] = scaled ? __fmul_rn(sc, r0) : r0;
                    if (v + 1 < p.nvec) dr[v + 1] = scaled ? __fmul_rn(sc, r1) : r1;
                }
            }
            rot = rot + 1 == NW ? 0 : rot + 1;
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&empty[st]);
            if (++st == S) {
                st = 0;
                ph ^= 1;
            }
        }
    }
    // the zero pass this launch depends on has finished before this grid does
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int FMT, uint32_t IW>
cudaError_t mm_launch_t(const MmParams& p, uint32_t grid, size_t smem, cudaStream_t s) {
    auto k = rg_spmm_kernel<FMT, IW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * (1 + p.nw));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, p);
}

template <uint32_t IW>
cudaError_t mm_launch_iw(int fmt, const MmParams& p, uint32_t grid, size_t smem, cudaStream_t s) {
    switch (fmt) {
        case DOSE_FMT_U16_SCALE: return mm_launch_t<DOSE_FMT_U16_SCALE, IW>(p, grid, smem, s);
        case DOSE_FMT_BF16: return mm_launch_t<DOSE_FMT_BF16, IW>(p, grid, smem, s);
        case DOSE_FMT_F16: return mm_launch_t<DOSE_FMT_F16, IW>(p, grid, smem, s);
        case DOSE_FMT_F32: return mm_launch_t<DOSE_FMT_F32, IW>(p, grid, smem, s);
        case DOSE_FMT_FP8E4M3_ROWSCALE: return mm_launch_t<DOSE_FMT_FP8E4M3_ROWSCALE, IW>(p, grid, smem, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// The row-group form of dose_spmv_batched applies when every matrix has its
// row-group layout (not switched off with adj_layout = 1), all share one stored
// format, index width and grid, and the widest window of X plus a ring of two
// slots fits in shared memory.
bool rg_spmm_applies(const dose_matrix* const* A, int count, size_t* smem_out, uint32_t* depth_out) {
    if (count < 1) return false;
    uint32_t wmax = 0, tu = 0, tg = 0, tr = 0;
    for (int m = 0; m < count; ++m) {
        const dose_matrix* M = A[m];
        if (!M->rg.built || !M->rg.sched.desc || M->adj_tuning.layout == 1) return false;
        if (M->fmt != A[0]->fmt || M->rg.iw != A[0]->rg.iw || M->rg.sched.grid != A[0]->rg.sched.grid) return false;
        wmax = std::max(wmax, M->rg.sched.wwidth);
        tu = std::max(tu, M->rg.tile_u);
        tg = std::max(tg, M->rg.tile_g);
        tr = std::max(tr, M->rg.tile_rows);
    }
    const RgSlot SL = rg_slot(tu, tg, tr, value_bytes(A[0]->fmt), A[0]->rg.iw,
                              A[0]->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0);
    const size_t fixed = kMmHeader + round_up((wmax + 1) * kMmXStride * 4, 128);
    if (fixed + 2ull * SL.bytes > kMaxSmemPerBlock) return false;
    const uint32_t depth = (uint32_t)std::min<size_t>(4, (kMaxSmemPerBlock - fixed) / SL.bytes);
    if (smem_out) *smem_out = fixed + (size_t)depth * SL.bytes;
    if (depth_out) *depth_out = depth;
    return true;
}

cudaError_t launch_rg_spmm(const dose_matrix* const* A, int count, const float* const* X, float* const* D, int nvec,
                           cudaStream_t s) {
    for (int base = 0; base < count; base += (int)kMmMaxPerLaunch) {
        const int n = std::min<int>(count - base, (int)kMmMaxPerLaunch);
        size_t smem = 0;
        uint32_t depth = 0;
        if (!rg_spmm_applies(A + base, n, &smem, &depth)) return cudaErrorInvalidConfiguration;
        MmZero z;
        MmParams p;
        p.count = z.count = (uint32_t)n;
        p.nvec = z.nvec = (uint32_t)nvec;
        p.depth = depth;
        p.nw = kMmWorkers;
        p.err = A[base]->err;
        uint32_t tu = 0, tg = 0, tr = 0;
        uint64_t rows = 0;
        for (int i = 0; i < n; ++i) {
            const dose_matrix* M = A[base + i];
            const RowGroups& R = M->rg;
            MmItem& it = p.item[i];
            it.grp = R.grp;
            it.ucol = R.ucol;
            it.uval = R.uval;
            it.desc = R.sched.desc;
            it.cta_begin = R.sched.cta_begin;
            it.wlo = R.sched.wlo;
            it.row_scale = M->row_scale;
            it.X = X[base + i];
            it.D = D[base + i];
            it.scale = M->scale;
            it.nrows = M->nrows;
            it.ncols = M->ncols;
            it.W = R.sched.wwidth;
            z.mask[i] = R.mask;
            z.D[i] = D[base + i];
            z.nrows[i] = M->nrows;
            tu = std::max(tu, R.tile_u);
            tg = std::max(tg, R.tile_g);
            tr = std::max(tr, R.tile_rows);
            rows += M->nrows;
        }
        if (rows == 0) continue;
        p.SL = rg_slot(tu, tg, tr, value_bytes(A[base]->fmt), A[base]->rg.iw,
                       A[base]->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0);
        const uint32_t sms = (uint32_t)std::max(1, A[base]->sm_count);
        // the zero pass keeps the shared-memory carveout of the SpMM kernel so
        // that both can share an SM while they overlap
        cudaFuncSetAttribute(rg_spmm_zero, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        rg_spmm_zero<<<4 * sms, 256, 0, s>>>(z);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const uint32_t grid = A[base]->rg.sched.grid;
        e = A[base]->rg.iw == 2 ? mm_launch_iw<2>(A[base]->fmt, p, grid, smem, s)
                                : mm_launch_iw<4>(A[base]->fmt, p, grid, smem, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dose
