// Pieces shared by the row-group kernels (rg_kernel.cu: adjoint and fused
// pass; rg_spmm.cu: batched SpMM): the shared-memory layout of a stage slot,
// explicit shared-memory loads of union columns and values, the decoders of
// four stored values, and the group record's row offsets.  The layout itself
// is described in dose_internal.cuh (RowGroups) and rg_layout.cu.
#pragma once

#include "stage_common.cuh"

namespace dose {

// Shared-memory layout of one stage slot.
struct RgSlot {
    uint32_t grp_off, col_off, val_off, vec_off, vec_stride, bytes;
};

__host__ __device__ inline RgSlot rg_slot(uint32_t tile_u, uint32_t tile_g, uint32_t tile_rows, uint32_t es,
                                          uint32_t iw, uint32_t nvec) {
    RgSlot L;
    L.grp_off = 128;  // the StageDesc copy sits in the first 32 bytes
    L.col_off = L.grp_off + round_up(tile_g * 16, 128);
    L.val_off = L.col_off + round_up((tile_u + 16) * iw, 128);         // + slack of 16-byte copy windows
    L.vec_off = L.val_off + round_up((tile_u + 8) * 4 * es, 128);
    L.vec_stride = round_up((tile_rows + 8) * 4, 128);
    L.bytes = L.vec_off + nvec * L.vec_stride;
    return L;
}

// ---- shared-memory accesses on 32-bit shared addresses: explicit ld/st.shared
// (volatile, so they keep their order relative to the ring's mbarrier
// operations); the "_if" forms access only when p.

// Column index (IW bytes) at a.
template <uint32_t IW>
__device__ __forceinline__ uint32_t rg_ldcol(uint32_t a) {
    return IW == 2 ? dev::lds_u16(a) : dev::lds_u32(a);
}
// ... only if k < n (dflt otherwise).
template <uint32_t IW>
__device__ __forceinline__ uint32_t rg_ldcol_lt(uint32_t k, uint32_t n, uint32_t a, uint32_t dflt) {
    uint32_t v = dflt;
    if constexpr (IW == 2)
        asm volatile(
            "{\n\t.reg .pred q;\n\t.reg .b16 h;\n\tsetp.lt.u32 q, %1, %2;\n\t@q ld.shared.u16 h, [%3];\n\t"
            "@q cvt.u32.u16 %0, h;\n\t}"
            : "+r"(v) : "r"(k), "r"(n), "r"(a));
    else
        asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %1, %2;\n\t@q ld.shared.u32 %0, [%3];\n\t}"
                     : "+r"(v) : "r"(k), "r"(n), "r"(a));
    return v;
}

// The four stored values of one union entry at a, as raw bits.
template <int FMT>
__device__ __forceinline__ uint4 rg_ldval(uint32_t a) {
    uint4 v = make_uint4(0, 0, 0, 0);
    if constexpr (FMT == DOSE_FMT_F32)
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    else if constexpr (FMT == DOSE_FMT_FP8E4M3_ROWSCALE)
        v.x = dev::lds_u32(a);
    else
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
// ... only if k < n (zeros otherwise).
template <int FMT>
__device__ __forceinline__ uint4 rg_ldval_lt(uint32_t k, uint32_t n, uint32_t a) {
    uint4 v = make_uint4(0, 0, 0, 0);
    if constexpr (FMT == DOSE_FMT_F32)
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %4, %5;\n\t@q ld.shared.v4.u32 {%0, %1, %2, %3}, [%6];\n\t}"
            : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w) : "r"(k), "r"(n), "r"(a));
    else if constexpr (FMT == DOSE_FMT_FP8E4M3_ROWSCALE)
        asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %1, %2;\n\t@q ld.shared.u32 %0, [%3];\n\t}"
                     : "+r"(v.x) : "r"(k), "r"(n), "r"(a));
    else
        asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %2, %3;\n\t@q ld.shared.v2.u32 {%0, %1}, [%4];\n\t}"
                     : "+r"(v.x), "+r"(v.y) : "r"(k), "r"(n), "r"(a));
    return v;
}

// Raw bits of four stored values decoded to FP32 (exact).  U16: the code's
// 16 bits placed under the exponent of 2^23 (a byte permutation), minus 2^23.
template <int FMT>
__device__ __forceinline__ void rg_dec4(const uint4& q, float (&a)[4]) {
    if constexpr (FMT == DOSE_FMT_U16_SCALE) {
        a[0] = __fsub_rn(__uint_as_float(__byte_perm(q.x, 0x4B00u, 0x5410u)), 8388608.0f);
        a[1] = __fsub_rn(__uint_as_float(__byte_perm(q.x, 0x4B00u, 0x5432u)), 8388608.0f);
        a[2] = __fsub_rn(__uint_as_float(__byte_perm(q.y, 0x4B00u, 0x5410u)), 8388608.0f);
        a[3] = __fsub_rn(__uint_as_float(__byte_perm(q.y, 0x4B00u, 0x5432u)), 8388608.0f);
    } else if constexpr (FMT == DOSE_FMT_F32) {
        a[0] = __uint_as_float(q.x);
        a[1] = __uint_as_float(q.y);
        a[2] = __uint_as_float(q.z);
        a[3] = __uint_as_float(q.w);
    } else {
        Fmt<FMT>::dec4(q.x, q.y, a);
    }
}

// Sum of the four row sums over the warp; lane l returns row (l >> 3)'s total
// (every lane of an octet the same value, in one fixed order).
__device__ __forceinline__ float rg_reduce4(float a0, float a1, float a2, float a3, uint32_t lane) {
    const bool hi = lane & 16;
    float k0 = hi ? a2 : a0, k1 = hi ? a3 : a1;
    const float s0 = hi ? a0 : a2, s1 = hi ? a1 : a3;
    k0 = __fadd_rn(k0, __shfl_xor_sync(0xffffffffu, s0, 16));
    k1 = __fadd_rn(k1, __shfl_xor_sync(0xffffffffu, s1, 16));
    const bool b3 = lane & 8;
    float k = b3 ? k1 : k0;
    const float s = b3 ? k0 : k1;
    k = __fadd_rn(k, __shfl_xor_sync(0xffffffffu, s, 8));
    k = __fadd_rn(k, __shfl_xor_sync(0xffffffffu, k, 4));
    k = __fadd_rn(k, __shfl_xor_sync(0xffffffffu, k, 2));
    k = __fadd_rn(k, __shfl_xor_sync(0xffffffffu, k, 1));
    return k;
}

// Debug-checked builds (DOSE_DEBUG_CHECKS): whether group record G fits its
// stage (its union inside the stage's staged union, its rows inside the
// stage's rows and the matrix) and every union column of it inside the CTA's
// window [zc - W, zc] (zc: the zero element); a group that does not is
// recorded (kErrBounds) and skipped by the whole warp.  Release builds: true.
template <uint32_t IW>
__device__ __forceinline__ bool rg_group_ok(const uint4& G, const StageDesc& D, uint32_t col_a, uint32_t nrows,
                                            uint32_t zc, uint32_t W, uint32_t lane, int* err) {
#ifdef DOSE_DEBUG_CHECKS
    bool ok = G.x >= D.nz0 && G.x + G.y <= D.nz1 && G.x + G.y >= G.x;
    for (uint32_t g = 0; g < 4; ++g) {
        const uint32_t w = g < 2 ? G.z : G.w, off = (g & 1) ? (w >> 16) : (w & 0xFFFFu);
        ok = ok && (off == 0xFFFFu || (D.row0 + off < D.row1 && D.row0 + off < nrows));
    }
    if (ok)
        for (uint32_t k = lane; k < G.y; k += 32) {
            const uint32_t c = IW == 2 ? dev::lds_u16(col_a + IW * (G.x + k)) : dev::lds_u32(col_a + IW * (G.x + k));
            ok = ok && c - (zc - W) <= W;
        }
    return dev::in_bounds(__all_sync(0xffffffffu, ok), err);
#else
    (void)G, (void)D, (void)col_a, (void)nrows, (void)zc, (void)W, (void)lane, (void)err;
    return true;
#endif
}

// Offset of group row g (0..3) from the stage's first row; 0xFFFF: no row.
__device__ __forceinline__ uint32_t rg_row_off(const uint4& G, uint32_t g) {
    const uint32_t w = g < 2 ? G.z : G.w;
    return (g & 1) ? (w >> 16) : (w & 0xFFFFu);
}

}  // namespace dose
