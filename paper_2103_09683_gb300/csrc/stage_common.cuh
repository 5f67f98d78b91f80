// Pieces shared by the staged kernels: stored-format traits, the shared-memory
// layout of one pipeline slot, and the producer loop that fills slots with
// bulk async copies (cp.async.bulk, completion counted by an mbarrier).
#pragma once

#include "dose_internal.cuh"

namespace dose {

template <int FMT>
struct Fmt;
template <>
struct Fmt<DOSE_FMT_U16_SCALE> {
    using T = uint16_t;
    static constexpr uint32_t kAlign = 8;  // elements per 16 bytes
#ifdef __CUDACC__
    __device__ static float dec(T v) { return dev::dec_u16(v); }
#endif
};
template <>
struct Fmt<DOSE_FMT_BF16> {
    using T = uint16_t;
    static constexpr uint32_t kAlign = 8;
#ifdef __CUDACC__
    __device__ static float dec(T v) { return dev::dec_bf16(v); }
#endif
};
template <>
struct Fmt<DOSE_FMT_FP8E4M3_ROWSCALE> {
    using T = uint8_t;
    static constexpr uint32_t kAlign = 16;
#ifdef __CUDACC__
    __device__ static float dec(T v) { return dev::dec_e4m3(v); }
#endif
};

__host__ __device__ constexpr uint32_t round_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

constexpr uint32_t kMaxVec = 3;  // per-row float vectors staged with a slot

// Shared-memory layout of one pipeline slot.  Every region starts on a
// 128-byte boundary; each is sized for the largest stage plus the slack that
// 16-byte-aligned copy windows need.
struct SlotLayout {
    uint32_t hdr_off, rp_off, ne_off, val_off, col_off, vec_off, vec_stride, rl_off, bytes;
};

__host__ __device__ inline SlotLayout slot_layout(uint32_t tile_nnz, uint32_t tile_rows, uint32_t esize,
                                                  uint32_t nvec, bool with_rl) {
    SlotLayout L;
    L.hdr_off = 0;  // StageDesc copy (32 B) + 32 B of per-stage scalars
    L.rp_off = 128;
    L.ne_off = L.rp_off + round_up((tile_rows + 8) * 4, 128);
    L.val_off = L.ne_off + round_up((tile_rows + 16) * 2, 128);
    L.col_off = L.val_off + round_up((tile_nnz + 32) * esize, 128);
    L.vec_off = L.col_off + round_up((tile_nnz + 8) * 4, 128);
    L.vec_stride = round_up((tile_rows + 8) * 4, 128);
    L.rl_off = L.vec_off + nvec * L.vec_stride;
    L.bytes = L.rl_off + (with_rl ? round_up(tile_rows * 4, 128) : 0);
    return L;
}

// Per-row float vectors staged next to the matrix slices.  Rows below `lim`
// are copied with the slot; rows at or above it (the ragged tail of a caller's
// array, which cannot be read in whole 16-byte pieces) are read from global
// memory by whoever needs them.
struct VecSet {
    const float* ptr[kMaxVec];
    uint32_t lim[kMaxVec];
    uint32_t n;
};

#ifdef __CUDACC__

// Producer loop (one thread): for each stage of [s_begin, s_end) wait until its
// ring slot is free, copy the stage descriptor into the slot header, then
// bulk-copy the row_ptr / non-empty-list / value / column / vector slices and
// let the slot's `full` barrier count the bytes.  Before returning, wait until
// every copy it issued has landed, so the CTA never exits with copies into its
// shared memory in flight.  All waits are bounded.
template <int FMT>
__device__ void run_producer(const ScheduleView& sched, uint32_t s_begin, uint32_t s_end,
                             const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                             const void* __restrict__ val, const VecSet& vecs, unsigned char* slot_base,
                             const SlotLayout& SL, uint64_t* full, uint64_t* empty, uint32_t S, int* err) {
    using T = typename Fmt<FMT>::T;
    constexpr uint32_t VA = Fmt<FMT>::kAlign;
    uint32_t st = 0, ph = 0, issued = 0;
    StageDesc nxt;
    if (s_begin < s_end) nxt = sched.desc[s_begin];
    for (uint32_t s = s_begin; s < s_end; ++s) {
        const StageDesc D = nxt;
        if (s + 1 < s_end) nxt = sched.desc[s + 1];  // in flight while this stage is issued
        if (!dev::mbar_wait_bounded(&empty[st], ph ^ 1)) {
            atomicExch(err, kErrTimeoutEmpty);
            break;
        }
        unsigned char* buf = slot_base + st * SL.bytes;
        *reinterpret_cast<StageDesc*>(buf + SL.hdr_off) = D;
        const bool coop = (D.meta & STAGE_COOP) != 0;
        const uint32_t rp_a = D.row0 & ~3u, rp_n = coop ? 0 : round_up(D.row1 + 1, 4) - rp_a;
        const uint32_t ne_a = D.ne0 & ~7u, ne_n = D.ne1 > D.ne0 ? round_up(D.ne1, 8) - ne_a : 0;
        const uint32_t v_a = D.nz0 & ~(VA - 1), v_n = round_up(D.nz1, VA) - v_a;
        const uint32_t c_a = D.nz0 & ~3u, c_n = round_up(D.nz1, 4) - c_a;
        const uint32_t r_a = D.row0 & ~3u;
        uint32_t vn[kMaxVec];
        uint32_t bytes = rp_n * 4 + ne_n * 2 + v_n * (uint32_t)sizeof(T) + c_n * 4;
        for (uint32_t k = 0; k < vecs.n; ++k) {
            const uint32_t e = min(round_up(D.row1, 4), vecs.lim[k]);
            vn[k] = e > r_a ? e - r_a : 0;
            bytes += vn[k] * 4;
        }
        dev::mbar_arrive_expect_tx(&full[st], bytes);
        if (rp_n) dev::bulk_g2s(buf + SL.rp_off, row_ptr + rp_a, rp_n * 4, &full[st]);
        if (ne_n) dev::bulk_g2s(buf + SL.ne_off, sched.ne + ne_a, ne_n * 2, &full[st]);
        if (v_n)
            dev::bulk_g2s(buf + SL.val_off, static_cast<const T*>(val) + v_a, v_n * (uint32_t)sizeof(T),
                          &full[st]);
        if (c_n) dev::bulk_g2s(buf + SL.col_off, col + c_a, c_n * 4, &full[st]);
        for (uint32_t k = 0; k < vecs.n; ++k)
            if (vn[k]) dev::bulk_g2s(buf + SL.vec_off + k * SL.vec_stride, vecs.ptr[k] + r_a, vn[k] * 4, &full[st]);
        ++issued;
        if (++st == S) {
            st = 0;
            ph ^= 1;
        }
    }
    uint32_t n = issued < S ? issued : S;
    for (uint32_t i = 0; i < n; ++i) {
        if (st == 0) {
            st = S - 1;
            ph ^= 1;
        } else {
            --st;
        }
        dev::mbar_wait_bounded(&full[st], ph);
    }
}

// Value of staged vector k for row r of the slot whose stage starts at row0.
__device__ __forceinline__ float slot_vec(const unsigned char* buf, const SlotLayout& SL, const VecSet& vecs,
                                          uint32_t k, uint32_t row0, uint32_t r) {
    if (r < vecs.lim[k])
        return reinterpret_cast<const float*>(buf + SL.vec_off + k * SL.vec_stride)[r - (row0 & ~3u)];
    return __ldg(vecs.ptr[k] + r);
}

#endif

}  // namespace dose
