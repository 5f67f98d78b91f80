// Batched dose SpMM on the row-group layout: D_m = A_m X_m for several
// matrices (beams x uncertainty scenarios, Sec. I) and up to 16 spot-weight
// vectors each, in one persistent launch.
//
// One CTA per SM walks the matrices in order and, for each, its share of that
// matrix's row-group stages (the column-windowed schedule of rg_layout.cu),
// streamed by a producer thread through a shared-memory ring that runs on from
// matrix to matrix.  The workers hold the CTA's window of X_m in shared memory
// (16 floats per column, zero past nvec, and a zero column after the window)
// in blocks of 8 columns whose 16-byte pieces j of 8 columns fill one 128-byte
// row.  A warp takes a whole group: lane l = 2 s + r computes rows 2 r and
// 2 r + 1 of the group for all 16 vectors over the union positions u = s,
// s + 16, ...: per position one column load, the two rows' values in one
// load, four 16-byte X loads (16 positions per warp-step; each X load serves
// two rows) and 16 packed FP32 FMAs (f32x2: two IEEE FMAs each).  The sixteen
// lane slices s are added by a fixed transposed butterfly that leaves every
// lane two of one row's results to store.  Two more warps write D = 0 for the
// CTA's share of the rows without entries while the workers compute.
// Deterministic: static assignment of groups to warps, fixed per-lane order,
// fixed butterfly.
#include "dfloat.cuh"
#include "rg_common.cuh"

#include <algorithm>
#include <string>

namespace dose {
namespace {

constexpr uint32_t kMmMaxPerLaunch = kRgSpmmMaxPerLaunch;
constexpr uint32_t kMmWorkers = 16;      // worker warps (plus one producer and the zero warps)
constexpr uint32_t kMmZeroWarps = 2;     // warps writing the rows without entries
constexpr uint32_t kMvWorkers = 28;      // worker warps of the single-vector form (about 50 registers each)
constexpr uint32_t kMmHeader = 1024;     // mbarriers
constexpr uint32_t kMmSmemBudget = kMaxSmemPerBlock;
constexpr uint32_t kMmXStride = 16;      // floats per column of the staged window of X (vectors <= 16)

// Shared bytes of a window of W columns of X and the zero column after it
// (whole blocks of 8 columns x 16 floats).
__host__ __device__ constexpr uint32_t mm_xs_bytes(uint32_t W) { return ((W + 1 + 7) / 8 * 8 * 64 + 127) / 128 * 128; }

// ... of a window of W columns of x and the zero element after it (one float each).
__host__ __device__ constexpr uint32_t mm_x1_bytes(uint32_t W) { return ((W + 1) * 4 + 127) / 128 * 128; }

struct MmItem {
    const uint4* grp;
    const void* ucol;
    const void* uval;
    const StageDesc* desc;
    const uint32_t* cta_begin;
    const uint32_t* wlo;
    const float* row_scale;  // FP8 (padded to whole 16-byte pieces)
    const uint32_t* mask;    // rows with entries, one bit each
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

// Rows without entries: D = 0.  Zero warp z of NZ takes the CTA's share of the
// matrix's row-mask words (32 rows each) 32 words at a time and writes the
// rows without entries, consecutive lanes on consecutive 16-byte pieces
// (4-byte pieces unless nvec is a multiple of 4 and D 16-byte aligned).
__device__ void mm_zero_rows(const uint32_t* mask, float* D, uint32_t nrows, uint32_t nv, uint32_t z, uint32_t NZ,
                             uint32_t lane) {
    const uint32_t nword = (nrows + 31) / 32;
    const uint32_t wb = (uint32_t)((uint64_t)nword * blockIdx.x / gridDim.x);
    const uint32_t we = (uint32_t)((uint64_t)nword * (blockIdx.x + 1) / gridDim.x);
    const bool vec = (nv & 3u) == 0 && (reinterpret_cast<uintptr_t>(D) & 15u) == 0;
    const uint32_t per = vec ? nv / 4 : nv;  // pieces per row
    for (uint32_t w0 = wb + 32 * z; w0 < we; w0 += 32 * NZ) {
        const uint32_t mine = w0 + lane < we ? __ldg(mask + w0 + lane) : 0xFFFFFFFFu;
        for (uint32_t i = 0; i < 32 && w0 + i < we; ++i) {
            uint32_t word = __shfl_sync(0xffffffffu, mine, i);
            const uint32_t r0 = 32 * (w0 + i);
            if (r0 + 32 > nrows) word |= ~0u << (nrows - r0);  // rows past the end: nothing to write
            if (word == 0xFFFFFFFFu) continue;
            if (vec) {
                float4* d4 = reinterpret_cast<float4*>(D + (size_t)r0 * nv);
                for (uint32_t k = lane; k < 32 * per; k += 32) {
                    const uint32_t r = per == 4 ? k >> 2 : k / per;
                    if (!((word >> r) & 1u)) d4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            } else {
                float* d = D + (size_t)r0 * nv;
                if (per == 1) {  // one vector: lane l writes row r0 + l
                    if (!((word >> lane) & 1u)) d[lane] = 0.f;
                } else {
                    for (uint32_t k = lane; k < 32 * per; k += 32)
                        if (!((word >> (k / per)) & 1u)) d[k] = 0.f;
                }
            }
        }
    }
}

// Packed FP32 pairs (Blackwell f32x2): {lo, hi} in one 64-bit register; the
// fused multiply-add of a pair is two IEEE FMAs, rounded as __fmaf_rn rounds.
__device__ __forceinline__ uint64_t f2_splat(float a) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ void f2_fma(uint64_t& acc, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ void f2_split(uint64_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_pack(uint32_t lo, uint32_t hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// 16 bytes of shared memory at a as two packed pairs.
__device__ __forceinline__ void f2_ld4(uint32_t a, uint64_t& p0, uint64_t& p1) {
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(p0), "=l"(p1) : "r"(a));
}

// The stored values of two rows of one union entry at a (2 x the element
// size), as raw bits in the low bytes; zeros unless k < n.
template <int FMT>
__device__ __forceinline__ uint2 mm_ldval2_lt(uint32_t k, uint32_t n, uint32_t a) {
    uint2 v = make_uint2(0u, 0u);
    if constexpr (FMT == DOSE_FMT_F32)
        asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %2, %3;\n\t@q ld.shared.v2.u32 {%0, %1}, [%4];\n\t}"
                     : "+r"(v.x), "+r"(v.y) : "r"(k), "r"(n), "r"(a));
    else if constexpr (FMT == DOSE_FMT_FP8E4M3_ROWSCALE)
        v.x = dev::lds_u16_lt(k, n, a);
    else
        asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %1, %2;\n\t@q ld.shared.u32 %0, [%3];\n\t}"
                     : "+r"(v.x) : "r"(k), "r"(n), "r"(a));
    return v;
}
template <int FMT>
__device__ __forceinline__ uint2 mm_ldval2(uint32_t a) {
    if constexpr (FMT == DOSE_FMT_F32) {
        uint2 v;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
        return v;
    } else if constexpr (FMT == DOSE_FMT_FP8E4M3_ROWSCALE) {
        return make_uint2(dev::lds_u16(a), 0u);
    } else {
        return make_uint2(dev::lds_u32(a), 0u);
    }
}
// Two stored values decoded to FP32 (exact).
template <int FMT>
__device__ __forceinline__ void mm_dec2(const uint2& q, float& a0, float& a1) {
    if constexpr (FMT == DOSE_FMT_U16_SCALE) {
        a0 = __fsub_rn(__uint_as_float(__byte_perm(q.x, 0x4B00u, 0x5410u)), 8388608.0f);
        a1 = __fsub_rn(__uint_as_float(__byte_perm(q.x, 0x4B00u, 0x5432u)), 8388608.0f);
    } else if constexpr (FMT == DOSE_FMT_F32) {
        a0 = __uint_as_float(q.x);
        a1 = __uint_as_float(q.y);
    } else if constexpr (FMT == DOSE_FMT_BF16) {
        a0 = __uint_as_float(q.x << 16);
        a1 = __uint_as_float(q.x & 0xFFFF0000u);
    } else if constexpr (FMT == DOSE_FMT_F16) {
        a0 = dev::f16_to_f32((uint16_t)(q.x & 0xFFFFu));
        a1 = dev::f16_to_f32((uint16_t)(q.x >> 16));
    } else {
        a0 = dev::dec_e4m3((uint8_t)(q.x & 0xFFu));
        a1 = dev::dec_e4m3((uint8_t)((q.x >> 8) & 0xFFu));
    }
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
__global__ void __launch_bounds__((kMmWorkers + 1 + kMmZeroWarps) * 32, 1) rg_spmm_kernel(const __grid_constant__ MmParams p) {
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
    // the window of X: blocks of 8 columns, each 4 rows of 128 bytes (4 floats of
    // all 8 columns per row), so that 8 lanes reading the same 4 floats of 8
    // columns that differ mod 8 touch 8 distinct bank quads
    float* xs = reinterpret_cast<float*>(smem + kMmHeader);
    uint32_t wmax = 0;
    for (uint32_t m = 0; m < p.count; ++m) wmax = max(wmax, p.item[m].W);
    unsigned char* slot_base = smem + kMmHeader + mm_xs_bytes(wmax);
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
    if (warp > NW) {
        for (uint32_t m = 0; m < p.count; ++m)
            mm_zero_rows(p.item[m].mask, p.item[m].D, p.item[m].nrows, p.nvec, warp - NW - 1, kMmZeroWarps, lane);
        return;
    }
    const uint32_t wi = warp - 1, ctid = threadIdx.x - 32, nct = NW * 32;
    // lane = 2 s + r: union positions u = s (mod 16), rows 2 r and 2 r + 1 of the
    // group, all 16 vectors
    const uint32_t sl = lane >> 1, rp = lane & 1u;
    const uint32_t slot0 = dev::smem_u32(slot_base);
    uint32_t st = 0, ph = 0, rot = 0;
    for (uint32_t m = 0; m < p.count; ++m) {
        const MmItem& it = p.item[m];
        const uint32_t W = it.W, wlo = it.wlo[blockIdx.x];
        dev::named_barrier(1, nct);  // every worker is done with the previous window of X
        const uint32_t nx = round_up(W + 1, 8) * kMmXStride;
        for (uint32_t j = ctid; j < nx; j += nct) {
            const uint32_t c = 8 * (j >> 7) + ((j >> 2) & 7u), v = 4 * ((j >> 5) & 3u) + (j & 3u);
            xs[j] = c < W && wlo + c < it.ncols && v < p.nvec ? __ldg(it.X + (size_t)(wlo + c) * p.nvec + v) : 0.f;
        }
        dev::named_barrier(1, nct);
        const uint32_t xs_a = dev::smem_u32(xs) - 64 * wlo;  // + 64 (c & ~7) + 16 (c & 7) + 128 j: x[c][4 j ..]
        const uint32_t zc = wlo + W;                        // the zero column
        const uint32_t sb = it.cta_begin[blockIdx.x], se = it.cta_begin[blockIdx.x + 1];
        for (uint32_t s = sb; s < se; ++s) {
            if (!dev::mbar_wait_poll(&full[st], ph)) {
                atomicExch(p.err, kErrTimeoutFull);
                return;  // every worker waits on the same phases, so all of them leave here
            }
            const uint32_t slot = slot0 + st * SL.bytes;
            const StageDesc D = slot_desc(slot);
            const uint32_t col_a = slot + SL.col_off - IW * (D.nz0 & ~(CA - 1));
            const uint32_t val_a = slot + SL.val_off - RV * (D.nz0 & ~(VA - 1)) + 2 * ES * rp;
            const uint32_t vrs = slot + SL.vec_off - 4 * (D.row0 & ~3u);
            const uint32_t grp_a = slot + SL.grp_off - 16 * D.ne0;
            for (uint32_t j = D.ne0 + (wi >= rot ? wi - rot : wi + NW - rot); j < D.ne1; j += NW) {
                const uint4 G = dev::lds_v4_if(true, grp_a + 16 * j);
                if (!rg_group_ok<IW>(G, D, col_a, it.nrows, zc, W, lane, p.err)) continue;
                const uint32_t nU = G.y, u0 = G.x, nfull = nU >> 4;
                // acc2[8 e + i]: row 2 rp + e, vectors 2 i and 2 i + 1 as a packed pair
                uint64_t acc2[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) acc2[i] = 0ull;
                auto mac = [&](const uint2& raw, uint32_t c) {
                    float v0, v1;
                    mm_dec2<FMT>(raw, v0, v1);
                    const uint64_t w0 = f2_splat(v0), w1 = f2_splat(v1);
                    const uint32_t xa = xs_a + 64 * (c & ~7u) + 16 * (c & 7u);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        uint64_t x01, x23;
                        f2_ld4(xa + 128 * jj, x01, x23);
                        f2_fma(acc2[2 * jj], w0, x01);
                        f2_fma(acc2[2 * jj + 1], w0, x23);
                        f2_fma(acc2[8 + 2 * jj], w1, x01);
                        f2_fma(acc2[8 + 2 * jj + 1], w1, x23);
                    }
                };
                // this lane's union positions u = s, s + 16, ...: steps where all
                // sixteen slices have a position need no mask
                const uint32_t ca = col_a + IW * (u0 + sl), va = val_a + RV * (u0 + sl);
#pragma unroll 2
                for (uint32_t k = 0; k < nfull; ++k) mac(mm_ldval2<FMT>(va + 16 * RV * k), rg_ldcol<IW>(ca + 16 * IW * k));
                if (nU & 15u) {
                    const uint32_t u = 16 * nfull + sl;
                    mac(mm_ldval2_lt<FMT>(u, nU, va + 16 * RV * nfull), rg_ldcol_lt<IW>(u, nU, ca + 16 * IW * nfull, zc));
                }
                // acc[16 e + v]: row 2 rp + e, vector v
                float acc[32];
#pragma unroll
                for (int i = 0; i < 16; ++i) f2_split(acc2[i], acc[2 * i], acc[2 * i + 1]);
                // the sixteen slices: a transposed butterfly over s (lane bits 4, 3,
                // 2, 1); each level keeps the half that the lane's bit selects and adds
                // the partner's copy of it, so that lane 2 s + rp ends with row
                // g = 2 rp + b4, vectors v0 = 8 b3 + 4 b2 + 2 b1 and v0 + 1
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const bool b = lane & 16u;
                    const float snd = b ? acc[i] : acc[i + 16], kp = b ? acc[i + 16] : acc[i];
                    acc[i] = __fadd_rn(kp, __shfl_xor_sync(0xffffffffu, snd, 16));
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const bool b = lane & 8u;
                    const float snd = b ? acc[i] : acc[i + 8], kp = b ? acc[i + 8] : acc[i];
                    acc[i] = __fadd_rn(kp, __shfl_xor_sync(0xffffffffu, snd, 8));
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool b = lane & 4u;
                    const float snd = b ? acc[i] : acc[i + 4], kp = b ? acc[i + 4] : acc[i];
                    acc[i] = __fadd_rn(kp, __shfl_xor_sync(0xffffffffu, snd, 4));
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const bool b = lane & 2u;
                    const float snd = b ? acc[i] : acc[i + 2], kp = b ? acc[i + 2] : acc[i];
                    acc[i] = __fadd_rn(kp, __shfl_xor_sync(0xffffffffu, snd, 2));
                }
                const uint32_t g = 2 * rp + ((lane >> 4) & 1u);
                const uint32_t off = rg_row_off(G, g);
                if (off != 0xFFFFu) {
                    const uint32_t row = D.row0 + off;
                    const float sc = FP8 ? dev::lds_f32(vrs + 4 * row) : (FMT == DOSE_FMT_U16_SCALE ? it.scale : 1.f);
                    const bool scaled = FP8 || FMT == DOSE_FMT_U16_SCALE;
                    const uint32_t v = 8 * ((lane >> 3) & 1u) + 4 * ((lane >> 2) & 1u) + 2 * ((lane >> 1) & 1u);
                    float* dr = it.D + (size_t)row * p.nvec;
                    if (v < p.nvec) dr[v] = scaled ? __fmul_rn(sc, acc[0]) : acc[0];
                    if (v + 1 < p.nvec) dr[v + 1] = scaled ? __fmul_rn(sc, acc[1]) : acc[1];
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
}

// K steps of 32 union positions of one group for lane `lane` (K = 0: any
// number, in a loop): the four rows' values times x_c, added to a0..a3 in
// step order.  Positions past nU read nothing and add 0 * x of the zero element.
template <int FMT, uint32_t IW, int K>
__device__ __forceinline__ void mv_steps(uint32_t ca, uint32_t va, uint32_t nU, uint32_t lane, uint32_t zc,
                                         uint32_t xs_a, float& a0, float& a1, float& a2, float& a3) {
    constexpr uint32_t RV = 4 * (uint32_t)sizeof(typename Fmt<FMT>::T);
    // U16 and BF16: rows (0, 1) and (2, 3) as packed FP32 pairs: two codes decoded
    // by one packed add (U16: 2^23 + q - 2^23, exact) and two rows' FMAs in one
    // f32x2 instruction; the same IEEE operations, so the same bits as the
    // scalar form (a0..a3 are zero on entry)
    constexpr bool PACKED = FMT == DOSE_FMT_U16_SCALE || FMT == DOSE_FMT_BF16;
    uint64_t a01 = 0ull, a23 = 0ull;
    const uint64_t bias = f2_splat(-8388608.0f);
    auto mac = [&](const uint4& q, uint32_t c) {
        const float x = dev::lds_f32(xs_a + 4 * c);
        if constexpr (PACKED) {
            uint64_t v01, v23;
            if constexpr (FMT == DOSE_FMT_U16_SCALE) {
                v01 = f2_add(f2_pack(__byte_perm(q.x, 0x4B00u, 0x5410u), __byte_perm(q.x, 0x4B00u, 0x5432u)), bias);
                v23 = f2_add(f2_pack(__byte_perm(q.y, 0x4B00u, 0x5410u), __byte_perm(q.y, 0x4B00u, 0x5432u)), bias);
            } else {
                v01 = f2_pack(q.x << 16, q.x & 0xFFFF0000u);
                v23 = f2_pack(q.y << 16, q.y & 0xFFFF0000u);
            }
            const uint64_t xx = f2_splat(x);
            f2_fma(a01, v01, xx);
            f2_fma(a23, v23, xx);
        } else {
            float v[4];
            rg_dec4<FMT>(q, v);
            a0 = __fmaf_rn(v[0], x, a0);
            a1 = __fmaf_rn(v[1], x, a1);
            a2 = __fmaf_rn(v[2], x, a2);
            a3 = __fmaf_rn(v[3], x, a3);
        }
    };
    if constexpr (K == 0) {
        const uint32_t nfull = nU >> 5;
#pragma unroll 2
        for (uint32_t k = 0; k < nfull; ++k) mac(rg_ldval<FMT>(va + 32 * RV * k), rg_ldcol<IW>(ca + 32 * IW * k));
        if (nU & 31u) {
            const uint32_t u = 32 * nfull + lane;
            mac(rg_ldval_lt<FMT>(u, nU, va + 32 * RV * nfull), rg_ldcol_lt<IW>(u, nU, ca + 32 * IW * nfull, zc));
        }
    } else {
        uint4 q[K];
        uint32_t c[K];
#pragma unroll
        for (int k = 0; k < K - 1; ++k) {
            q[k] = rg_ldval<FMT>(va + 32 * RV * k);
            c[k] = rg_ldcol<IW>(ca + 32 * IW * k);
        }
        const uint32_t u = 32 * (K - 1) + lane;
        q[K - 1] = rg_ldval_lt<FMT>(u, nU, va + 32 * RV * (K - 1));
        c[K - 1] = rg_ldcol_lt<IW>(u, nU, ca + 32 * IW * (K - 1), zc);
#pragma unroll
        for (int k = 0; k < K; ++k) mac(q[k], c[k]);
    }
    if constexpr (PACKED) {
        f2_split(a01, a0, a1);
        f2_split(a23, a2, a3);
    }
}

// Single-vector form (d = A x on the row-group layout, dose_spmv): the same
// producer, ring and zero warps; the window of x is one float per column.  A
// warp takes a group: lane l handles the union positions u = l, l + 32, ...
// (one column load, the four rows' values in one load, one x gather: the 32
// positions of a step have columns that differ mod 32, so the gather is one
// wavefront), keeps the four rows' partial sums and reduces them with the
// transposed butterfly of rg_reduce4; lane 8 g stores row g's dose.
template <int FMT, uint32_t IW>
__global__ void __launch_bounds__((kMvWorkers + 1 + kMmZeroWarps) * 32, 1) rg_spmv_kernel(const __grid_constant__ MmParams p) {
    constexpr uint32_t RV = 4 * (uint32_t)sizeof(typename Fmt<FMT>::T);
    constexpr uint32_t VA = RV >= 16 ? 1 : 16 / RV;
    constexpr uint32_t CA = 16 / IW;
    constexpr bool FP8 = FMT == DOSE_FMT_FP8E4M3_ROWSCALE;
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth, NW = p.nw;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + 8;
    float* xs = reinterpret_cast<float*>(smem + kMmHeader);  // W + 1 floats: the window of x and a zero
    uint32_t wmax = 0;
    for (uint32_t m = 0; m < p.count; ++m) wmax = max(wmax, p.item[m].W);
    unsigned char* slot_base = smem + kMmHeader + mm_x1_bytes(wmax);
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
    if (warp > NW) {
        for (uint32_t m = 0; m < p.count; ++m)
            mm_zero_rows(p.item[m].mask, p.item[m].D, p.item[m].nrows, 1, warp - NW - 1, kMmZeroWarps, lane);
        return;
    }
    const uint32_t wi = warp - 1, ctid = threadIdx.x - 32, nct = NW * 32;
    const uint32_t slot0 = dev::smem_u32(slot_base);
    uint32_t st = 0, ph = 0, rot = 0;
    for (uint32_t m = 0; m < p.count; ++m) {
        const MmItem& it = p.item[m];
        const uint32_t W = it.W, wlo = it.wlo[blockIdx.x];
        dev::named_barrier(1, nct);  // every worker is done with the previous window of x
        for (uint32_t c = ctid; c <= W; c += nct)
            xs[c] = c < W && wlo + c < it.ncols ? __ldg(it.X + wlo + c) : 0.f;
        dev::named_barrier(1, nct);
        const uint32_t xs_a = dev::smem_u32(xs) - 4 * wlo;  // x_c at xs_a + 4 c
        const uint32_t zc = wlo + W;                        // the zero element
        const uint32_t sb = it.cta_begin[blockIdx.x], se = it.cta_begin[blockIdx.x + 1];
        for (uint32_t s = sb; s < se; ++s) {
            if (!dev::mbar_wait_poll(&full[st], ph)) {
                atomicExch(p.err, kErrTimeoutFull);
                return;  // every worker waits on the same phases, so all of them leave here
            }
            const uint32_t slot = slot0 + st * SL.bytes;
            const StageDesc D = slot_desc(slot);
            const uint32_t col_a = slot + SL.col_off - IW * (D.nz0 & ~(CA - 1));
            const uint32_t val_a = slot + SL.val_off - RV * (D.nz0 & ~(VA - 1));
            const uint32_t vrs = slot + SL.vec_off - 4 * (D.row0 & ~3u);
            const uint32_t grp_a = slot + SL.grp_off - 16 * D.ne0;
            for (uint32_t j = D.ne0 + (wi >= rot ? wi - rot : wi + NW - rot); j < D.ne1; j += NW) {
                const uint4 G = dev::lds_v4_if(true, grp_a + 16 * j);
                if (!rg_group_ok<IW>(G, D, col_a, it.nrows, zc, W, lane, p.err)) continue;
                const uint32_t nU = G.y, u0 = G.x;
                const uint32_t ca = col_a + IW * (u0 + lane), va = val_a + RV * (u0 + lane);
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
                // groups of up to 320 union columns: every step's loads issued up
                // front, only the last step masked; longer single rows: a loop
                switch ((nU + 31) >> 5) {
                    case 1: mv_steps<FMT, IW, 1>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    case 2: mv_steps<FMT, IW, 2>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    case 3: mv_steps<FMT, IW, 3>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    case 4: mv_steps<FMT, IW, 4>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    case 5: mv_steps<FMT, IW, 5>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    case 6: mv_steps<FMT, IW, 6>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    case 7: mv_steps<FMT, IW, 7>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    case 8: mv_steps<FMT, IW, 8>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    case 9: mv_steps<FMT, IW, 9>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    case 10: mv_steps<FMT, IW, 10>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                    default: mv_steps<FMT, IW, 0>(ca, va, nU, lane, zc, xs_a, a0, a1, a2, a3); break;
                }
                const float sum = rg_reduce4(a0, a1, a2, a3, lane);
                const uint32_t off = rg_row_off(G, lane >> 3);
                if ((lane & 7u) == 0 && off != 0xFFFFu) {
                    const uint32_t row = D.row0 + off;
                    const float sc = FP8 ? dev::lds_f32(vrs + 4 * row) : it.scale;
                    it.D[row] = FP8 || FMT == DOSE_FMT_U16_SCALE ? __fmul_rn(sc, sum) : sum;
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
}

// FP64-vector form (dose_spmv_f64 on the row-group layout): x as the 8-byte
// elements prepare_x wrote (double-float pairs or doubles), one per column of
// the window and a zero element; per lane four row accumulators Acc<MODE>,
// combined by the transposed butterfly (pairs added as dfloat.cuh adds them);
// lane 8 g stores row g's FP64 dose.  Rows without entries: the zero warps
// write the two zero words of each double.
__host__ __device__ constexpr uint32_t mm_x2_bytes(uint32_t W) { return ((W + 1) * 8 + 127) / 128 * 128; }

template <int FMT, uint32_t IW, int MODE>
__global__ void __launch_bounds__((kMvWorkers + 1 + kMmZeroWarps) * 32, 1) rg_spmv64_kernel(const __grid_constant__ MmParams p) {
    constexpr uint32_t RV = 4 * (uint32_t)sizeof(typename Fmt<FMT>::T);
    constexpr uint32_t VA = RV >= 16 ? 1 : 16 / RV;
    constexpr uint32_t CA = 16 / IW;
    constexpr bool FP8 = FMT == DOSE_FMT_FP8E4M3_ROWSCALE;
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t S = p.depth, NW = p.nw;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + 8;
    uint2* xs = reinterpret_cast<uint2*>(smem + kMmHeader);  // W + 1 elements: the window of x and a zero
    uint32_t wmax = 0;
    for (uint32_t m = 0; m < p.count; ++m) wmax = max(wmax, p.item[m].W);
    unsigned char* slot_base = smem + kMmHeader + mm_x2_bytes(wmax);
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
    if (warp > NW) {
        for (uint32_t m = 0; m < p.count; ++m)  // a double row is two zero floats
            mm_zero_rows(p.item[m].mask, p.item[m].D, p.item[m].nrows, 2, warp - NW - 1, kMmZeroWarps, lane);
        return;
    }
    const uint32_t wi = warp - 1, ctid = threadIdx.x - 32, nct = NW * 32;
    const uint32_t slot0 = dev::smem_u32(slot_base);
    uint32_t st = 0, ph = 0, rot = 0;
    for (uint32_t m = 0; m < p.count; ++m) {
        const MmItem& it = p.item[m];
        const uint2* x64 = reinterpret_cast<const uint2*>(it.X);  // ncols + 1 elements, the last one zero
        double* d64 = reinterpret_cast<double*>(it.D);
        const uint32_t W = it.W, wlo = it.wlo[blockIdx.x];
        dev::named_barrier(1, nct);  // every worker is done with the previous window of x
        for (uint32_t c = ctid; c <= W; c += nct)
            xs[c] = c < W && wlo + c < it.ncols ? x64[wlo + c] : make_uint2(0u, 0u);
        dev::named_barrier(1, nct);
        const uint32_t xs_a = dev::smem_u32(xs) - 8 * wlo;  // x_c at xs_a + 8 c
        const uint32_t zc = wlo + W;                        // the zero element
        const uint32_t sb = it.cta_begin[blockIdx.x], se = it.cta_begin[blockIdx.x + 1];
        for (uint32_t s = sb; s < se; ++s) {
            if (!dev::mbar_wait_poll(&full[st], ph)) {
                atomicExch(p.err, kErrTimeoutFull);
                return;  // every worker waits on the same phases, so all of them leave here
            }
            const uint32_t slot = slot0 + st * SL.bytes;
            const StageDesc D = slot_desc(slot);
            const uint32_t col_a = slot + SL.col_off - IW * (D.nz0 & ~(CA - 1));
            const uint32_t val_a = slot + SL.val_off - RV * (D.nz0 & ~(VA - 1));
            const uint32_t vrs = slot + SL.vec_off - 4 * (D.row0 & ~3u);
            const uint32_t grp_a = slot + SL.grp_off - 16 * D.ne0;
            for (uint32_t j = D.ne0 + (wi >= rot ? wi - rot : wi + NW - rot); j < D.ne1; j += NW) {
                const uint4 G = dev::lds_v4_if(true, grp_a + 16 * j);
                if (!rg_group_ok<IW>(G, D, col_a, it.nrows, zc, W, lane, p.err)) continue;
                const uint32_t nU = G.y, u0 = G.x, nfull = nU >> 5;
                Acc<MODE> a[4];
                auto mac = [&](const uint4& q, uint32_t c) {
                    float v[4];
                    rg_dec4<FMT>(q, v);
                    uint2 xq;
                    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(xq.x), "=r"(xq.y) : "r"(xs_a + 8 * c));
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        if constexpr (MODE == F64_DF)
                            df_mac(v[g], make_float2(__uint_as_float(xq.x), __uint_as_float(xq.y)), a[g].s, a[g].c);
                        else
                            a[g].v = __fma_rn((double)v[g], __hiloint2double((int)xq.y, (int)xq.x), a[g].v);
                    }
                };
                const uint32_t ca = col_a + IW * (u0 + lane), va = val_a + RV * (u0 + lane);
#pragma unroll 2
                for (uint32_t k = 0; k < nfull; ++k) mac(rg_ldval<FMT>(va + 32 * RV * k), rg_ldcol<IW>(ca + 32 * IW * k));
                if (nU & 31u) {
                    const uint32_t u = 32 * nfull + lane;
                    mac(rg_ldval_lt<FMT>(u, nU, va + 32 * RV * nfull), rg_ldcol_lt<IW>(u, nU, ca + 32 * IW * nfull, zc));
                }
                // the four row sums over the warp (the butterfly of rg_reduce4 on accumulator pairs):
                // lane l ends with row l / 8's total
                const bool b16 = lane & 16u, b8 = lane & 8u;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    Acc<MODE> k = b16 ? a[i + 2] : a[i];
                    const Acc<MODE> snd = b16 ? a[i] : a[i + 2];
                    k.add(snd.shfl_xor(16));
                    a[i] = k;
                }
                {
                    Acc<MODE> k = b8 ? a[1] : a[0];
                    const Acc<MODE> snd = b8 ? a[0] : a[1];
                    k.add(snd.shfl_xor(8));
                    a[0] = k;
                }
                a[0].add(a[0].shfl_xor(4));
                a[0].add(a[0].shfl_xor(2));
                a[0].add(a[0].shfl_xor(1));
                const uint32_t off = rg_row_off(G, lane >> 3);
                if ((lane & 7u) == 0 && off != 0xFFFFu) {
                    const uint32_t row = D.row0 + off;
                    const float sc = FP8 ? dev::lds_f32(vrs + 4 * row) : it.scale;
                    d64[row] = a[0].result(FP8 || FMT == DOSE_FMT_U16_SCALE, sc);
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
}

template <int FMT, uint32_t IW, int MODE>
cudaError_t mv64_launch_t(const MmParams& p, uint32_t grid, size_t smem, cudaStream_t s) {
    auto k = rg_spmv64_kernel<FMT, IW, MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 32 * (1 + p.nw + kMmZeroWarps), smem, s>>>(p);
    return cudaGetLastError();
}

template <uint32_t IW, int MODE>
cudaError_t mv64_launch_iw(int fmt, const MmParams& p, uint32_t grid, size_t smem, cudaStream_t s) {
    switch (fmt) {
        case DOSE_FMT_U16_SCALE: return mv64_launch_t<DOSE_FMT_U16_SCALE, IW, MODE>(p, grid, smem, s);
        case DOSE_FMT_BF16: return mv64_launch_t<DOSE_FMT_BF16, IW, MODE>(p, grid, smem, s);
        case DOSE_FMT_F16: return mv64_launch_t<DOSE_FMT_F16, IW, MODE>(p, grid, smem, s);
        case DOSE_FMT_F32: return mv64_launch_t<DOSE_FMT_F32, IW, MODE>(p, grid, smem, s);
        case DOSE_FMT_FP8E4M3_ROWSCALE: return mv64_launch_t<DOSE_FMT_FP8E4M3_ROWSCALE, IW, MODE>(p, grid, smem, s);
    }
    return cudaErrorInvalidValue;
}

template <int FMT, uint32_t IW>
cudaError_t mv_launch_t(const MmParams& p, uint32_t grid, size_t smem, cudaStream_t s) {
    auto k = rg_spmv_kernel<FMT, IW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 32 * (1 + p.nw + kMmZeroWarps), smem, s>>>(p);
    return cudaGetLastError();
}

template <uint32_t IW>
cudaError_t mv_launch_iw(int fmt, const MmParams& p, uint32_t grid, size_t smem, cudaStream_t s) {
    switch (fmt) {
        case DOSE_FMT_U16_SCALE: return mv_launch_t<DOSE_FMT_U16_SCALE, IW>(p, grid, smem, s);
        case DOSE_FMT_BF16: return mv_launch_t<DOSE_FMT_BF16, IW>(p, grid, smem, s);
        case DOSE_FMT_F16: return mv_launch_t<DOSE_FMT_F16, IW>(p, grid, smem, s);
        case DOSE_FMT_F32: return mv_launch_t<DOSE_FMT_F32, IW>(p, grid, smem, s);
        case DOSE_FMT_FP8E4M3_ROWSCALE: return mv_launch_t<DOSE_FMT_FP8E4M3_ROWSCALE, IW>(p, grid, smem, s);
    }
    return cudaErrorInvalidValue;
}

template <int FMT, uint32_t IW>
cudaError_t mm_launch_t(const MmParams& p, uint32_t grid, size_t smem, cudaStream_t s) {
    auto k = rg_spmm_kernel<FMT, IW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 32 * (1 + p.nw + kMmZeroWarps), smem, s>>>(p);
    return cudaGetLastError();
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
    const size_t fixed = kMmHeader + mm_xs_bytes(wmax);
    if (fixed + 2ull * SL.bytes > kMmSmemBudget) return false;
    const uint32_t depth = (uint32_t)std::min<size_t>(4, (kMmSmemBudget - fixed) / SL.bytes);
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
        MmParams p;
        p.count = (uint32_t)n;
        p.nvec = (uint32_t)nvec;
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
            it.mask = R.mask;
            tu = std::max(tu, R.tile_u);
            tg = std::max(tg, R.tile_g);
            tr = std::max(tr, R.tile_rows);
            rows += M->nrows;
        }
        if (rows == 0) continue;
        p.SL = rg_slot(tu, tg, tr, value_bytes(A[base]->fmt), A[base]->rg.iw,
                       A[base]->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0);
        const uint32_t grid = A[base]->rg.sched.grid;
        const cudaError_t e = A[base]->rg.iw == 2 ? mm_launch_iw<2>(A[base]->fmt, p, grid, smem, s)
                                : mm_launch_iw<4>(A[base]->fmt, p, grid, smem, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace dose

namespace dose {

// The row-group form of dose_spmv applies when the handle has the layout and
// the window of x plus a ring of two slots fits in shared memory.
bool rg_spmv_applies(const dose_matrix* A, size_t* smem_out, uint32_t* depth_out) {
    const RowGroups& R = A->rg;
    if (!R.built || !R.sched.desc) return false;
    const RgSlot SL = rg_slot(R.tile_u, R.tile_g, R.tile_rows, value_bytes(A->fmt), R.iw,
                              A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0);
    const size_t fixed = kMmHeader + mm_x1_bytes(R.sched.wwidth);
    if (fixed + 2ull * SL.bytes > kMmSmemBudget) return false;
    const uint32_t depth = (uint32_t)std::min<size_t>(8, (kMmSmemBudget - fixed) / SL.bytes);
    if (smem_out) *smem_out = fixed + (size_t)depth * SL.bytes;
    if (depth_out) *depth_out = depth;
    return true;
}

// The one-matrix launch parameters of the single-vector forms.
static MmParams mv_params(const dose_matrix* A, const void* x, void* d, uint32_t depth) {
    const RowGroups& R = A->rg;
    MmParams p;
    p.count = 1;
    p.nvec = 1;
    p.depth = depth;
    p.nw = kMvWorkers;
    p.err = A->err;
    MmItem& it = p.item[0];
    it.grp = R.grp;
    it.ucol = R.ucol;
    it.uval = R.uval;
    it.desc = R.sched.desc;
    it.cta_begin = R.sched.cta_begin;
    it.wlo = R.sched.wlo;
    it.row_scale = A->row_scale;
    it.mask = R.mask;
    it.X = static_cast<const float*>(x);
    it.D = static_cast<float*>(d);
    it.scale = A->scale;
    it.nrows = A->nrows;
    it.ncols = A->ncols;
    it.W = R.sched.wwidth;
    p.SL = rg_slot(R.tile_u, R.tile_g, R.tile_rows, value_bytes(A->fmt), R.iw,
                   A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0);
    return p;
}

// The FP64-vector form: the window of x takes 8 bytes per column.
bool rg_spmv64_applies(const dose_matrix* A, size_t* smem_out, uint32_t* depth_out) {
    const RowGroups& R = A->rg;
    if (!R.built || !R.sched.desc) return false;
    const RgSlot SL = rg_slot(R.tile_u, R.tile_g, R.tile_rows, value_bytes(A->fmt), R.iw,
                              A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0);
    const size_t fixed = kMmHeader + mm_x2_bytes(R.sched.wwidth);
    if (fixed + 2ull * SL.bytes > kMmSmemBudget) return false;
    const uint32_t depth = (uint32_t)std::min<size_t>(8, (kMmSmemBudget - fixed) / SL.bytes);
    if (smem_out) *smem_out = fixed + (size_t)depth * SL.bytes;
    if (depth_out) *depth_out = depth;
    return true;
}

cudaError_t launch_rg_spmv64(const dose_matrix* A, const void* x64, double* d, bool native, cudaStream_t s) {
    size_t smem = 0;
    uint32_t depth = 0;
    if (!rg_spmv64_applies(A, &smem, &depth)) return cudaErrorInvalidConfiguration;
    if (A->nrows == 0) return cudaSuccess;
    const MmParams p = mv_params(A, x64, d, depth);
    const uint32_t grid = A->rg.sched.grid;
    if (native)
        return A->rg.iw == 2 ? mv64_launch_iw<2, F64_DP>(A->fmt, p, grid, smem, s)
                             : mv64_launch_iw<4, F64_DP>(A->fmt, p, grid, smem, s);
    return A->rg.iw == 2 ? mv64_launch_iw<2, F64_DF>(A->fmt, p, grid, smem, s)
                         : mv64_launch_iw<4, F64_DF>(A->fmt, p, grid, smem, s);
}

cudaError_t launch_rg_spmv(const dose_matrix* A, const float* x, float* d, cudaStream_t s) {
    size_t smem = 0;
    uint32_t depth = 0;
    if (!rg_spmv_applies(A, &smem, &depth)) return cudaErrorInvalidConfiguration;
    if (A->nrows == 0) return cudaSuccess;
    const RowGroups& R = A->rg;
    MmParams p;
    p.count = 1;
    p.nvec = 1;
    p.depth = depth;
    p.nw = kMvWorkers;
    p.err = A->err;
    MmItem& it = p.item[0];
    it.grp = R.grp;
    it.ucol = R.ucol;
    it.uval = R.uval;
    it.desc = R.sched.desc;
    it.cta_begin = R.sched.cta_begin;
    it.wlo = R.sched.wlo;
    it.row_scale = A->row_scale;
    it.mask = R.mask;
    it.X = x;
    it.D = d;
    it.scale = A->scale;
    it.nrows = A->nrows;
    it.ncols = A->ncols;
    it.W = R.sched.wwidth;
    p.SL = rg_slot(R.tile_u, R.tile_g, R.tile_rows, value_bytes(A->fmt), R.iw,
                   A->fmt == DOSE_FMT_FP8E4M3_ROWSCALE ? 1 : 0);
    return R.iw == 2 ? mv_launch_iw<2>(A->fmt, p, R.sched.grid, smem, s)
                     : mv_launch_iw<4>(A->fmt, p, R.sched.grid, smem, s);
}

}  // namespace dose
