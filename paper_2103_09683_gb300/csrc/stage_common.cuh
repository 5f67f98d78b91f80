// Pieces shared by the staged kernels: stored-format traits and the
// shared-memory layout of one pipeline stage (row_ptr, value and column slices
// of a row block, each padded for 16-byte-aligned bulk copies).
#pragma once

#include "dose_internal.cuh"

namespace dose {

template <int FMT>
struct Fmt;
template <>
struct Fmt<DOSE_FMT_U16_SCALE> {
    using T = uint16_t;
    static constexpr uint32_t kAlign = 8;  // elements per 16 bytes
    __device__ static float dec(T v) { return dev::dec_u16(v); }
};
template <>
struct Fmt<DOSE_FMT_BF16> {
    using T = uint16_t;
    static constexpr uint32_t kAlign = 8;
    __device__ static float dec(T v) { return dev::dec_bf16(v); }
};
template <>
struct Fmt<DOSE_FMT_FP8E4M3_ROWSCALE> {
    using T = uint8_t;
    static constexpr uint32_t kAlign = 16;
    __device__ static float dec(T v) { return dev::dec_e4m3(v); }
};

__host__ __device__ constexpr uint32_t round_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

// Shared-memory layout of one pipeline stage.
struct StageLayout {
    uint32_t rp_off, val_off, col_off, bytes;
};

__host__ __device__ inline StageLayout stage_layout(uint32_t tile_nnz, uint32_t tile_rows, uint32_t esize) {
    StageLayout L;
    L.rp_off = 0;
    L.val_off = round_up((tile_rows + 8) * 4, 128);
    L.col_off = L.val_off + round_up((tile_nnz + 32) * esize, 128);
    L.bytes = L.col_off + round_up((tile_nnz + 8) * 4, 128);
    return L;
}

// Stage slices are copied from 16-byte-aligned starts: the first needed entry
// of a slice sits at (global index - aligned start).
struct StageSlices {
    uint32_t rp_a, rp_n, v_a, v_n, c_a, c_n;
};

template <int FMT>
__host__ __device__ inline StageSlices stage_slices(bool coop, uint32_t r0, uint32_t r1, uint32_t nz0, uint32_t nz1) {
    constexpr uint32_t VA = Fmt<FMT>::kAlign;
    StageSlices q;
    q.rp_a = r0 & ~3u;
    q.rp_n = coop ? 0 : round_up(r1 + 1, 4) - q.rp_a;
    q.v_a = nz0 & ~(VA - 1);
    q.v_n = round_up(nz1, VA) - q.v_a;
    q.c_a = nz0 & ~3u;
    q.c_n = round_up(nz1, 4) - q.c_a;
    return q;
}

#ifdef __CUDACC__
// Producer loop (one thread): for each stage of [s_begin, s_end) wait until
// its ring slot is free, then bulk-copy the row_ptr / value / column slices
// into the slot and let the slot's `full` barrier count the bytes.  Before
// returning, wait until every copy it issued has landed, so the CTA never
// exits with copies into its shared memory in flight.  All waits are bounded.
template <int FMT>
__device__ void run_producer(const ScheduleView& sched, uint32_t s_begin, uint32_t s_end,
                             const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                             const void* __restrict__ val, unsigned char* stage_base, const StageLayout& SL,
                             uint64_t* full, uint64_t* empty, uint32_t S, int* err) {
    using T = typename Fmt<FMT>::T;
    uint32_t st = 0, ph = 0, issued = 0;
    for (uint32_t s = s_begin; s < s_end; ++s) {
        if (!dev::mbar_wait_bounded(&empty[st], ph ^ 1)) {
            atomicExch(err, kErrTimeoutEmpty);
            break;
        }
        unsigned char* buf = stage_base + st * SL.bytes;
        const bool coop = (sched.meta[s] & STAGE_COOP) != 0;
        const StageSlices q =
            stage_slices<FMT>(coop, sched.row0[s], sched.row0[s + 1], sched.nz0[s], sched.nz0[s + 1]);
        const uint32_t bytes = q.rp_n * 4 + q.v_n * (uint32_t)sizeof(T) + q.c_n * 4;
        dev::mbar_arrive_expect_tx(&full[st], bytes);
        if (q.rp_n) dev::bulk_g2s(buf + SL.rp_off, row_ptr + q.rp_a, q.rp_n * 4, &full[st]);
        if (q.v_n)
            dev::bulk_g2s(buf + SL.val_off, static_cast<const T*>(val) + q.v_a, q.v_n * (uint32_t)sizeof(T),
                          &full[st]);
        if (q.c_n) dev::bulk_g2s(buf + SL.col_off, col + q.c_a, q.c_n * 4, &full[st]);
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
#endif

}  // namespace dose
