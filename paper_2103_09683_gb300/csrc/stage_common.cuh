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
    // decoded value of the stored entry at shared address a (0 unless k < ke)
    __device__ static float lds(uint32_t a) { return (float)dev::lds_u16(a); }
    __device__ static float lds_lt(uint32_t k, uint32_t ke, uint32_t a) { return (float)dev::lds_u16_lt(k, ke, a); }
    // four consecutive entries (index a multiple of 4) decoded, loaded only when p
    __device__ static void lds4(bool p, uint32_t a, float* w) {
        const uint2 q = dev::lds_v2_if(p, a);
        w[0] = (float)(q.x & 0xFFFFu);
        w[1] = (float)(q.x >> 16);
        w[2] = (float)(q.y & 0xFFFFu);
        w[3] = (float)(q.y >> 16);
    }
    // four stored entries packed in q0 (entries 0, 1) and q1 (2, 3), decoded
    __device__ static void dec4(uint32_t q0, uint32_t q1, float (&w)[4]) {
        w[0] = (float)(q0 & 0xFFFFu);
        w[1] = (float)(q0 >> 16);
        w[2] = (float)(q1 & 0xFFFFu);
        w[3] = (float)(q1 >> 16);
    }
#endif
};
template <>
struct Fmt<DOSE_FMT_BF16> {
    using T = uint16_t;
    static constexpr uint32_t kAlign = 8;
#ifdef __CUDACC__
    __device__ static float dec(T v) { return dev::dec_bf16(v); }
    __device__ static float lds(uint32_t a) { return __uint_as_float(dev::lds_u16(a) << 16); }
    __device__ static float lds_lt(uint32_t k, uint32_t ke, uint32_t a) {
        return __uint_as_float(dev::lds_u16_lt(k, ke, a) << 16);
    }
    __device__ static void lds4(bool p, uint32_t a, float* w) {
        const uint2 q = dev::lds_v2_if(p, a);
        w[0] = __uint_as_float(q.x << 16);
        w[1] = __uint_as_float(q.x & 0xFFFF0000u);
        w[2] = __uint_as_float(q.y << 16);
        w[3] = __uint_as_float(q.y & 0xFFFF0000u);
    }
    __device__ static void dec4(uint32_t q0, uint32_t q1, float (&w)[4]) {
        w[0] = __uint_as_float(q0 << 16);
        w[1] = __uint_as_float(q0 & 0xFFFF0000u);
        w[2] = __uint_as_float(q1 << 16);
        w[3] = __uint_as_float(q1 & 0xFFFF0000u);
    }
#endif
};
template <>
struct Fmt<DOSE_FMT_FP8E4M3_ROWSCALE> {
    using T = uint8_t;
    static constexpr uint32_t kAlign = 16;
#ifdef __CUDACC__
    __device__ static float dec(T v) { return dev::dec_e4m3(v); }
    __device__ static float lds(uint32_t a) { return dev::dec_e4m3((uint8_t)dev::lds_u8(a)); }
    __device__ static float lds_lt(uint32_t k, uint32_t ke, uint32_t a) {
        return dev::dec_e4m3((uint8_t)dev::lds_u8_lt(k, ke, a));
    }
    __device__ static void lds4(bool p, uint32_t a, float* w) {
        float v[4];
        dec4(dev::lds_u32_if(p, a), 0u, v);
        w[0] = v[0];
        w[1] = v[1];
        w[2] = v[2];
        w[3] = v[3];
    }
    // four codes in the bytes of q0 (q1 unused): two E4M3x2 -> F16x2 conversions
    __device__ static void dec4(uint32_t q0, uint32_t, float (&w)[4]) {
        uint32_t h01, h23;
        asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h01) : "h"(static_cast<uint16_t>(q0 & 0xFFFFu)));
        asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h23) : "h"(static_cast<uint16_t>(q0 >> 16)));
        w[0] = dev::f16_to_f32(static_cast<uint16_t>(h01 & 0xFFFFu));
        w[1] = dev::f16_to_f32(static_cast<uint16_t>(h01 >> 16));
        w[2] = dev::f16_to_f32(static_cast<uint16_t>(h23 & 0xFFFFu));
        w[3] = dev::f16_to_f32(static_cast<uint16_t>(h23 >> 16));
    }
#endif
};

template <>
struct Fmt<DOSE_FMT_F16> {
    using T = uint16_t;
    static constexpr uint32_t kAlign = 8;
#ifdef __CUDACC__
    __device__ static float dec(T v) { return dev::f16_to_f32(v); }
    __device__ static float lds(uint32_t a) { return dev::f16_to_f32((uint16_t)dev::lds_u16(a)); }
    __device__ static float lds_lt(uint32_t k, uint32_t ke, uint32_t a) {
        return dev::f16_to_f32((uint16_t)dev::lds_u16_lt(k, ke, a));
    }
    __device__ static void lds4(bool p, uint32_t a, float* w) {
        const uint2 q = dev::lds_v2_if(p, a);
        float v[4];
        dec4(q.x, q.y, v);
        w[0] = v[0];
        w[1] = v[1];
        w[2] = v[2];
        w[3] = v[3];
    }
    __device__ static void dec4(uint32_t q0, uint32_t q1, float (&w)[4]) {
        w[0] = dev::f16_to_f32(static_cast<uint16_t>(q0 & 0xFFFFu));
        w[1] = dev::f16_to_f32(static_cast<uint16_t>(q0 >> 16));
        w[2] = dev::f16_to_f32(static_cast<uint16_t>(q1 & 0xFFFFu));
        w[3] = dev::f16_to_f32(static_cast<uint16_t>(q1 >> 16));
    }
#endif
};

template <>
struct Fmt<DOSE_FMT_F32> {
    using T = uint32_t;
    static constexpr uint32_t kAlign = 4;
#ifdef __CUDACC__
    __device__ static float dec(T v) { return __uint_as_float(v); }
    __device__ static float lds(uint32_t a) { return dev::lds_f32(a); }
    __device__ static float lds_lt(uint32_t k, uint32_t ke, uint32_t a) { return dev::lds_f32_lt(k, ke, a); }
    __device__ static void lds4(bool p, uint32_t a, float* w) {
        const uint4 q = dev::lds_v4_if(p, a);
        w[0] = __uint_as_float(q.x);
        w[1] = __uint_as_float(q.y);
        w[2] = __uint_as_float(q.z);
        w[3] = __uint_as_float(q.w);
    }
#endif
};

#ifdef __CUDACC__
// The four stored values at p (a group of four consecutive entries, 4-aligned),
// decoded to FP32: one 16-, 8- or 4-byte load.
template <int FMT>
__device__ __forceinline__ void load_vals4(const typename Fmt<FMT>::T* p, float (&a)[4]) {
    using T = typename Fmt<FMT>::T;
    if constexpr (sizeof(T) == 4) {
        const uint4 q = *reinterpret_cast<const uint4*>(p);
        a[0] = __uint_as_float(q.x);
        a[1] = __uint_as_float(q.y);
        a[2] = __uint_as_float(q.z);
        a[3] = __uint_as_float(q.w);
    } else if constexpr (sizeof(T) == 2) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        Fmt<FMT>::dec4(q.x, q.y, a);
    } else {
        Fmt<FMT>::dec4(*reinterpret_cast<const uint32_t*>(p), 0u, a);
    }
}
#endif

__host__ __device__ constexpr uint32_t round_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

constexpr uint32_t kMaxVec = 3;  // per-row float vectors staged with a slot

// Shared-memory layout of one pipeline slot.  Every region starts on a
// 128-byte boundary; each is sized for the largest stage plus the slack that
// 16-byte-aligned copy windows need.
struct SlotLayout {
    uint32_t hdr_off, rp_off, ne_off, val_off, col_off, vec_off, vec_stride, rl_off, bytes;
};

__host__ __device__ inline SlotLayout slot_layout(uint32_t tile_nnz, uint32_t tile_rows, uint32_t esize,
                                                  uint32_t nvec, bool with_rl, uint32_t iw = 4) {
    SlotLayout L;
    L.hdr_off = 0;  // StageDesc copy (32 B) + 32 B of per-stage scalars
    L.rp_off = 128;
    L.ne_off = L.rp_off + round_up((tile_rows + 8) * 4, 128);
    L.val_off = L.ne_off + round_up((tile_rows + 16) * 2, 128);
    L.col_off = L.val_off + round_up((tile_nnz + 32) * esize, 128);
    L.vec_off = L.col_off + round_up((tile_nnz + 32 / iw) * iw, 128);  // column indices of iw bytes
    L.vec_stride = round_up((tile_rows + 8) * 4, 128);
    L.rl_off = L.vec_off + nvec * L.vec_stride;
    L.bytes = L.rl_off + (with_rl ? round_up(tile_rows * 4, 128) : 0);
    return L;
}

// Per-row float vectors staged next to the matrix slices.  Rows below `lim`
// are bulk-copied with the slot; rows at or above it (the ragged tail of a
// caller's array, which cannot be read in whole 16-byte pieces) are copied by
// the producer thread with plain loads.
struct VecSet {
    const float* ptr[kMaxVec];
    uint32_t lim[kMaxVec];
    uint32_t n;
};

#ifdef __CUDACC__

constexpr uint32_t kDescWin = 32;  // stage descriptors per shared-memory window (1 KB)

// State of a producer thread's ring, carried across the matrices of a batch:
// the next slot and its phase, the stages issued so far, and the descriptor
// windows completed on dbar[0..1] (window g of the whole run uses buffer and
// barrier g & 1, phase (g >> 1) & 1).
struct ProducerRing {
    uint32_t st = 0, ph = 0, issued = 0, wbase = 0;
    bool ok = true;
};

// Producer loop (one thread): for each stage of [s_begin, s_end) wait until its
// ring slot is free, copy the stage descriptor into the slot header, then
// bulk-copy the row_ptr / non-empty-list / value / column / vector slices and
// let the slot's `full` barrier count the bytes.  The CTA's descriptors are
// contiguous in global memory and arrive in double-buffered windows of 32
// (`dwin`, completion on `dbar[2]`), so the loop never waits on a global load.
// Slots are `slot_stride` bytes apart (at least SL.bytes).  All waits are
// bounded; a timeout sets the error word and clears R.ok.
template <int FMT, uint32_t IW = 4>
__device__ void produce_stages(ProducerRing& R, const ScheduleView& sched, uint32_t s_begin, uint32_t s_end,
                               const uint32_t* __restrict__ row_ptr, const void* __restrict__ col_v,
                               const void* __restrict__ val, const VecSet& vecs, unsigned char* slot_base,
                               const SlotLayout& SL, uint32_t slot_stride, uint64_t* full, uint64_t* empty,
                               uint32_t S, StageDesc* dwin, uint64_t* dbar, uint32_t pf, int* err) {
    using T = typename Fmt<FMT>::T;
    constexpr uint32_t VA = Fmt<FMT>::kAlign;
    constexpr uint32_t CA = 16 / IW;  // column indices per 16 bytes
    const unsigned char* col = static_cast<const unsigned char*>(col_v);  // + IW * k
    if (!R.ok || s_begin >= s_end) return;
    uint32_t st = R.st, ph = R.ph, issued = R.issued;
    const uint32_t wb = R.wbase;
    auto load_window = [&](uint32_t w) {
        const uint32_t first = s_begin + w * kDescWin;
        if (first >= s_end) return;
        const uint32_t n = min(kDescWin, s_end - first), g = wb + w;
        dev::mbar_arrive_expect_tx(&dbar[g & 1], n * (uint32_t)sizeof(StageDesc));
        dev::bulk_g2s(dwin + (g & 1) * kDescWin, sched.desc + first, n * (uint32_t)sizeof(StageDesc), &dbar[g & 1]);
    };
    const uint32_t nst = s_end - s_begin;
    const uint32_t nwin = (nst + kDescWin - 1) / kDescWin;
    uint32_t w_issued = 0, w_waited = 0;  // descriptor windows issued / waited for
    // descriptors of earlier calls were read through the generic proxy before
    // their buffers are refilled by bulk copies
    if (wb) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    load_window(0);
    load_window(1);
    w_issued = min(nwin, 2u);
    // Make window w readable (windows are waited for in order).
    auto have_window = [&](uint32_t w) -> bool {
        while (w_waited <= w) {
            const uint32_t g = wb + w_waited;
            if (!dev::mbar_wait_bounded(&dbar[g & 1], (g >> 1) & 1)) return false;
            ++w_waited;
        }
        return true;
    };
    // Ask L2 for stage j's slices (the HBM latency is then paid into L2,
    // not into the shared-memory ring).
    auto prefetch = [&](uint32_t j) {
        const uint32_t w = j / kDescWin;
        if (w >= w_issued || !have_window(w)) return;
        const StageDesc P = dwin[((wb + w) & 1) * kDescWin + j % kDescWin];
        const uint32_t v_a = P.nz0 & ~(VA - 1), v_n = round_up(P.nz1, VA) - v_a;
        const uint32_t c_a = P.nz0 & ~(CA - 1), c_n = round_up(P.nz1, CA) - c_a;
        if (v_n) dev::bulk_prefetch_l2(static_cast<const T*>(val) + v_a, v_n * (uint32_t)sizeof(T));
        if (c_n) dev::bulk_prefetch_l2(col + (size_t)c_a * IW, c_n * IW);
        if (!(P.meta & STAGE_COOP)) {
            const uint32_t rp_a = P.row0 & ~3u;
            dev::bulk_prefetch_l2(row_ptr + rp_a, (round_up(P.row1 + 1, 4) - rp_a) * 4);
        }
    };
    for (uint32_t j = 0; j < pf && j < nst; ++j) prefetch(j);
    for (uint32_t s = s_begin; s < s_end; ++s) {
        const uint32_t j = s - s_begin, w = j / kDescWin, jw = j % kDescWin;
        if (pf && j + pf < nst) prefetch(j + pf);
        if (!have_window(w)) {
            atomicExch(err, kErrTimeoutEmpty);
            R.ok = false;
            break;
        }
        const StageDesc D = dwin[((wb + w) & 1) * kDescWin + jw];
        if (jw == kDescWin - 1 && w + 2 < nwin) {
            // the window's last descriptor is in registers (and the prefetch
            // look-ahead, < kDescWin, reads window w + 1): refill its buffer
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            load_window(w + 2);
            w_issued = w + 3;
        }
        if (!dev::mbar_wait_bounded(&empty[st], ph ^ 1)) {
            atomicExch(err, kErrTimeoutEmpty);
            R.ok = false;
            break;
        }
        unsigned char* buf = slot_base + st * slot_stride;
        *reinterpret_cast<StageDesc*>(buf + SL.hdr_off) = D;
        const bool coop = (D.meta & STAGE_COOP) != 0;
        const uint32_t rp_a = D.row0 & ~3u, rp_n = coop ? 0 : round_up(D.row1 + 1, 4) - rp_a;
        const uint32_t ne_a = D.ne0 & ~7u, ne_n = D.ne1 > D.ne0 ? round_up(D.ne1, 8) - ne_a : 0;
        const uint32_t v_a = D.nz0 & ~(VA - 1), v_n = round_up(D.nz1, VA) - v_a;
        const uint32_t c_a = D.nz0 & ~(CA - 1), c_n = round_up(D.nz1, CA) - c_a;
        const uint32_t r_a = D.row0 & ~3u;
        uint32_t vn[kMaxVec];
        uint32_t bytes = rp_n * 4 + ne_n * 2 + v_n * (uint32_t)sizeof(T) + c_n * IW;
        for (uint32_t k = 0; k < vecs.n; ++k) {
            const uint32_t e = min(round_up(D.row1, 4), vecs.lim[k]);
            vn[k] = e > r_a ? e - r_a : 0;
            bytes += vn[k] * 4;
            // The ragged tail of a caller's array (< 4 rows) is read with plain
            // loads and stored before the arrive below, which releases it.
            float* dst = reinterpret_cast<float*>(buf + SL.vec_off + k * SL.vec_stride);
            bool tail = false;
            for (uint32_t r = max(vecs.lim[k], r_a + vn[k]); r < D.row1; ++r) {
                dst[r - r_a] = __ldg(vecs.ptr[k] + r);
                tail = true;
            }
            // later fills of this slot write the same words through the async proxy
            if (tail) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        dev::mbar_arrive_expect_tx(&full[st], bytes);
        if (rp_n) dev::bulk_g2s(buf + SL.rp_off, row_ptr + rp_a, rp_n * 4, &full[st]);
        if (ne_n) dev::bulk_g2s(buf + SL.ne_off, sched.ne + ne_a, ne_n * 2, &full[st]);
        if (v_n)
            dev::bulk_g2s(buf + SL.val_off, static_cast<const T*>(val) + v_a, v_n * (uint32_t)sizeof(T),
                          &full[st]);
        if (c_n) dev::bulk_g2s(buf + SL.col_off, col + (size_t)c_a * IW, c_n * IW, &full[st]);
        for (uint32_t k = 0; k < vecs.n; ++k)
            if (vn[k])
                dev::bulk_g2s(buf + SL.vec_off + k * SL.vec_stride, vecs.ptr[k] + r_a, vn[k] * 4, &full[st]);
        ++issued;
        if (++st == S) {
            st = 0;
            ph ^= 1;
        }
    }
    // Descriptor windows issued but not waited for (only after a timeout).
    for (uint32_t w = w_waited; w < w_issued; ++w) dev::mbar_wait_bounded(&dbar[(wb + w) & 1], ((wb + w) >> 1) & 1);
    R.st = st;
    R.ph = ph;
    R.issued = issued;
    R.wbase = wb + w_issued;
}

// Wait until every copy the ring issued has landed, so the CTA never exits with
// copies into its shared memory in flight (bounded waits).
__device__ __forceinline__ void producer_drain(const ProducerRing& R, uint64_t* full, uint32_t S) {
    uint32_t st = R.st, ph = R.ph;
    const uint32_t n = R.issued < S ? R.issued : S;
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

// The producer of a single-matrix kernel: all of the CTA's stages, then drain.
template <int FMT, uint32_t IW = 4>
__device__ void run_producer(const ScheduleView& sched, uint32_t s_begin, uint32_t s_end,
                             const uint32_t* __restrict__ row_ptr, const void* __restrict__ col,
                             const void* __restrict__ val, const VecSet& vecs, unsigned char* slot_base,
                             const SlotLayout& SL, uint64_t* full, uint64_t* empty, uint32_t S, StageDesc* dwin,
                             uint64_t* dbar, uint32_t pf, int* err) {
    ProducerRing R;
    produce_stages<FMT, IW>(R, sched, s_begin, s_end, row_ptr, col, val, vecs, slot_base, SL, SL.bytes, full, empty,
                            S, dwin, dbar, pf, err);
    producer_drain(R, full, S);
}

// Value of staged vector k for row r; `slot` is the slot's shared address and
// row0 the stage's first row.
__device__ __forceinline__ float slot_vec(uint32_t slot, const SlotLayout& SL, const VecSet& vecs, uint32_t k,
                                          uint32_t row0, uint32_t r) {
    (void)vecs;
    return dev::lds_f32(slot + SL.vec_off + k * SL.vec_stride + (r - (row0 & ~3u)) * 4);
}

// Read the stage descriptor from a slot header.
__device__ __forceinline__ StageDesc slot_desc(uint32_t slot) {
    StageDesc D;
    D.row0 = dev::lds_u32(slot + 0);
    D.row1 = dev::lds_u32(slot + 4);
    D.nz0 = dev::lds_u32(slot + 8);
    D.nz1 = dev::lds_u32(slot + 12);
    D.ne0 = dev::lds_u32(slot + 16);
    D.ne1 = dev::lds_u32(slot + 20);
    D.meta = dev::lds_u32(slot + 24);
    D.pad = 0;
    return D;
}

// Shared addresses of a slot's slices, rebased so that global indices can be
// used directly (32-bit wrap-around arithmetic: only the sums are addresses).
struct SlotView {
    uint32_t rp;   // + 4 * row
    uint32_t col;  // + IW * k (IW: bytes per column index, 4 or 2)
    uint32_t val;  // + esize * k
    uint32_t ne;   // + 2 * i, i = position in the stage's list
};

template <int FMT, uint32_t IW = 4>
__device__ __forceinline__ SlotView slot_view(uint32_t slot, const SlotLayout& SL, const StageDesc& D) {
    constexpr uint32_t VA = Fmt<FMT>::kAlign;
    constexpr uint32_t ES = (uint32_t)sizeof(typename Fmt<FMT>::T);
    constexpr uint32_t CA = 16 / IW;  // column indices per 16 bytes
    SlotView v;
    v.rp = slot + SL.rp_off - (D.row0 & ~3u) * 4u;
    v.col = slot + SL.col_off - (D.nz0 & ~(CA - 1)) * IW;
    v.val = slot + SL.val_off - (D.nz0 & ~(VA - 1)) * ES;
    v.ne = slot + SL.ne_off + (D.ne0 & 7u) * 2u;
    return v;
}

// Column index of entry k of a slot (IW-byte indices).
template <uint32_t IW>
__device__ __forceinline__ uint32_t col_at(const SlotView& v, uint32_t k) {
    return IW == 4 ? dev::lds_u32(v.col + 4 * k) : dev::lds_u16(v.col + 2 * k);
}
template <uint32_t IW>
__device__ __forceinline__ uint32_t col_at_lt(uint32_t k, uint32_t ke, const SlotView& v) {
    if (IW == 4) return dev::lds_u32_lt(k, ke, v.col + 4 * k);
    return dev::lds_u16_lt(k, ke, v.col + 2 * k);
}
// Column indices of the four entries k .. k + 3 (k a multiple of 4), loaded
// only when p (zeros otherwise): one 16-byte or 8-byte load.
template <uint32_t IW>
__device__ __forceinline__ uint4 col4_if(bool p, const SlotView& v, uint32_t k) {
    if (IW == 4) return dev::lds_v4_if(p, v.col + 4 * k);
    const uint2 q = dev::lds_v2_if(p, v.col + 2 * k);
    return make_uint4(q.x & 0xFFFFu, q.x >> 16, q.y & 0xFFFFu, q.y >> 16);
}

// Sum of a[k] * x[col[k]] over k = kb, kb + STEP, ... < ke with four
// independent FP32 accumulators (combined as (a0 + a1) + (a2 + a3)).  STEP is a
// compile-time power of two, so successive entries are immediate offsets from
// two walking shared addresses.
template <int FMT, uint32_t STEP, uint32_t IW = 4>
__device__ __forceinline__ float dot_fixed(const SlotView& v, uint32_t xs, uint32_t kb, uint32_t ke) {
    constexpr uint32_t ES = (uint32_t)sizeof(typename Fmt<FMT>::T);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (kb < ke) {
        uint32_t n = (ke - kb + STEP - 1) / STEP;  // entries of this lane
        uint32_t ca = v.col + IW * kb, va = v.val + ES * kb;
        for (; n >= 4; n -= 4) {
            auto ldc = [](uint32_t a) { return IW == 4 ? dev::lds_u32(a) : dev::lds_u16(a); };
            const uint32_t c0 = ldc(ca), c1 = ldc(ca + IW * STEP);
            const uint32_t c2 = ldc(ca + 2 * IW * STEP), c3 = ldc(ca + 3 * IW * STEP);
            const float w0 = Fmt<FMT>::lds(va), w1 = Fmt<FMT>::lds(va + ES * STEP);
            const float w2 = Fmt<FMT>::lds(va + 2 * ES * STEP), w3 = Fmt<FMT>::lds(va + 3 * ES * STEP);
            a0 = __fmaf_rn(w0, dev::lds_f32(xs + 4 * c0), a0);
            a1 = __fmaf_rn(w1, dev::lds_f32(xs + 4 * c1), a1);
            a2 = __fmaf_rn(w2, dev::lds_f32(xs + 4 * c2), a2);
            a3 = __fmaf_rn(w3, dev::lds_f32(xs + 4 * c3), a3);
            ca += 4 * IW * STEP;
            va += 4 * ES * STEP;
        }
        auto ldc = [](uint32_t a) { return IW == 4 ? dev::lds_u32(a) : dev::lds_u16(a); };
        if (n > 0) a0 = __fmaf_rn(Fmt<FMT>::lds(va), dev::lds_f32(xs + 4 * ldc(ca)), a0);
        if (n > 1) a1 = __fmaf_rn(Fmt<FMT>::lds(va + ES * STEP), dev::lds_f32(xs + 4 * ldc(ca + IW * STEP)), a1);
        if (n > 2)
            a2 = __fmaf_rn(Fmt<FMT>::lds(va + 2 * ES * STEP), dev::lds_f32(xs + 4 * ldc(ca + 2 * IW * STEP)), a2);
    }
    return __fadd_rn(__fadd_rn(a0, a1), __fadd_rn(a2, a3));
}

// ---- one step over a group of four consecutive entries of a row
//
// A lane's group holds the entries at positions off .. off + 3 of a row of len
// entries (positions counted from the row's first entry; a row's first group
// starts at the 4-aligned entry at or below it, so off may be -1..-3 there).
// An entry takes part iff 0 <= position < len, tested as one unsigned compare;
// that predicate guards its gather, its FMA and (scatter) its store, so no
// loaded value needs a default and masked entries cost no select.

// Column indices (one 16-byte load) and stored values (8 bytes; 4 for FP8, 16 for F32)
// of the group at shared addresses ca / va, loaded only if the group reaches
// into the row (off < len), decoded to FP32.  Registers of a group that is not
// loaded hold unspecified values that no guarded access ever uses.
template <int FMT>
__device__ __forceinline__ void load_group(int off, int len, uint32_t ca, uint32_t va, uint32_t (&c)[4],
                                           float (&a)[4]) {
    if constexpr (sizeof(typename Fmt<FMT>::T) == 4) {
        uint32_t q[4];
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.lt.s32 p, %8, %9;\n\t"
            "@p ld.shared.v4.u32 {%0, %1, %2, %3}, [%10];\n\t"
            "@p ld.shared.v4.u32 {%4, %5, %6, %7}, [%11];\n\t}"
            : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3])
            : "r"(off), "r"(len), "r"(ca), "r"(va));
        for (int u = 0; u < 4; ++u) a[u] = __uint_as_float(q[u]);
        return;
    } else {
    uint32_t q0, q1 = 0;
    if (sizeof(typename Fmt<FMT>::T) == 2) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.lt.s32 p, %6, %7;\n\t"
            "@p ld.shared.v4.u32 {%0, %1, %2, %3}, [%8];\n\t"
            "@p ld.shared.v2.u32 {%4, %5}, [%9];\n\t}"
            : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(q0), "=r"(q1)
            : "r"(off), "r"(len), "r"(ca), "r"(va));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.lt.s32 p, %5, %6;\n\t"
            "@p ld.shared.v4.u32 {%0, %1, %2, %3}, [%7];\n\t"
            "@p ld.shared.u32 %4, [%8];\n\t}"
            : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(q0)
            : "r"(off), "r"(len), "r"(ca), "r"(va));
    }
    Fmt<FMT>::dec4(q0, q1, a);
    }
}

// acc[u] += a[u] * x[c[u]] for the group's entries inside the row; x at shared
// address xs + 4 * column.
__device__ __forceinline__ void dot_group(int off, int len, uint32_t xs, const uint32_t (&c)[4], const float (&a)[4],
                                          float (&acc)[4]) {
    asm volatile(
        "{\n\t.reg .pred p0, p1, p2, p3;\n\t.reg .b32 t1, t2, t3, g0, g1, g2, g3;\n\t"
        ".reg .f32 x0, x1, x2, x3;\n\t"
        "setp.lt.u32 p0, %4, %5;\n\t"
        "add.s32 t1, %4, 1;\n\tsetp.lt.u32 p1, t1, %5;\n\t"
        "add.s32 t2, %4, 2;\n\tsetp.lt.u32 p2, t2, %5;\n\t"
        "add.s32 t3, %4, 3;\n\tsetp.lt.u32 p3, t3, %5;\n\t"
        "mad.lo.u32 g0, %7, 4, %6;\n\tmad.lo.u32 g1, %8, 4, %6;\n\t"
        "mad.lo.u32 g2, %9, 4, %6;\n\tmad.lo.u32 g3, %10, 4, %6;\n\t"
        "@p0 ld.shared.f32 x0, [g0];\n\t@p1 ld.shared.f32 x1, [g1];\n\t"
        "@p2 ld.shared.f32 x2, [g2];\n\t@p3 ld.shared.f32 x3, [g3];\n\t"
        "@p0 fma.rn.f32 %0, %11, x0, %0;\n\t@p1 fma.rn.f32 %1, %12, x1, %1;\n\t"
        "@p2 fma.rn.f32 %2, %13, x2, %2;\n\t@p3 fma.rn.f32 %3, %14, x3, %3;\n\t}"
        : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
        : "r"(off), "r"(len), "r"(xs), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "f"(a[0]), "f"(a[1]),
          "f"(a[2]), "f"(a[3]));
}

// g[c[u]] += a[u] * r for the group's entries inside the row; g at shared
// address gw + 4 * column.  The columns of a row are distinct, so the four
// loads may precede the four stores, and no two lanes of the warp touch one
// word.
__device__ __forceinline__ void scatter_group(int off, int len, uint32_t gw, const uint32_t (&c)[4],
                                              const float (&a)[4], float r) {
    asm volatile(
        "{\n\t.reg .pred p0, p1, p2, p3;\n\t.reg .b32 t1, t2, t3, g0, g1, g2, g3;\n\t"
        ".reg .f32 v0, v1, v2, v3;\n\t"
        "setp.lt.u32 p0, %0, %1;\n\t"
        "add.s32 t1, %0, 1;\n\tsetp.lt.u32 p1, t1, %1;\n\t"
        "add.s32 t2, %0, 2;\n\tsetp.lt.u32 p2, t2, %1;\n\t"
        "add.s32 t3, %0, 3;\n\tsetp.lt.u32 p3, t3, %1;\n\t"
        "mad.lo.u32 g0, %3, 4, %2;\n\tmad.lo.u32 g1, %4, 4, %2;\n\t"
        "mad.lo.u32 g2, %5, 4, %2;\n\tmad.lo.u32 g3, %6, 4, %2;\n\t"
        "@p0 ld.shared.f32 v0, [g0];\n\t@p1 ld.shared.f32 v1, [g1];\n\t"
        "@p2 ld.shared.f32 v2, [g2];\n\t@p3 ld.shared.f32 v3, [g3];\n\t"
        "@p0 fma.rn.f32 v0, %7, %11, v0;\n\t@p1 fma.rn.f32 v1, %8, %11, v1;\n\t"
        "@p2 fma.rn.f32 v2, %9, %11, v2;\n\t@p3 fma.rn.f32 v3, %10, %11, v3;\n\t"
        "@p0 st.shared.f32 [g0], v0;\n\t@p1 st.shared.f32 [g1], v1;\n\t"
        "@p2 st.shared.f32 [g2], v2;\n\t@p3 st.shared.f32 [g3], v3;\n\t}"
        ::"r"(off), "r"(len), "r"(gw), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "f"(a[0]), "f"(a[1]),
          "f"(a[2]), "f"(a[3]), "f"(r)
        : "memory");
}

// Plain typed pointers to a slot's column indices and values, indexed by the
// global entry index (the slot holds [nz0 & ~(16/IW - 1), ...) and
// [nz0 & ~(kAlign - 1), ...)).
template <int FMT, uint32_t IW>
struct SlotPtrs {
    const void* col;
    const typename Fmt<FMT>::T* val;
};
template <int FMT, uint32_t IW>
__device__ __forceinline__ SlotPtrs<FMT, IW> slot_ptrs(const unsigned char* slotp, const SlotLayout& SL,
                                                       const StageDesc& D) {
    using T = typename Fmt<FMT>::T;
    SlotPtrs<FMT, IW> q;
    q.col = slotp + SL.col_off - (size_t)(D.nz0 & ~(16 / IW - 1)) * IW;
    q.val = reinterpret_cast<const T*>(slotp + SL.val_off) - (D.nz0 & ~(Fmt<FMT>::kAlign - 1));
    return q;
}

// Lane li of an L-lane group takes the groups of four consecutive entries at
// (kb & ~3) + 4 li + 4 L s, `iters` steps (the same for the whole warp).  A
// group is loaded whole (one 16- or 8-byte load of indices, one of values);
// a group past the row's end loads the row's first group instead (always in
// the slot), and every entry outside [kb, ke) reads x at the zero element zc
// with weight 0, so it adds exactly nothing.  Plain typed shared-memory loads
// (the slot's data were released by an mbarrier wait, a compiler barrier), so
// the compiler may overlap steps.
template <int FMT, uint32_t L, uint32_t IW>
__device__ __forceinline__ float dot_vec_p(const SlotPtrs<FMT, IW>& sp, const float* __restrict__ xsp, uint32_t zc,
                                           uint32_t kb, uint32_t ke, uint32_t li, uint32_t iters) {
    using T = typename Fmt<FMT>::T;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
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
            acc[u] = __fmaf_rn(m ? a[u] : 0.f, xsp[m ? c[u] : zc], acc[u]);
        }
    }
    return __fadd_rn(__fadd_rn(acc[0], acc[1]), __fadd_rn(acc[2], acc[3]));
}

// Same with a run-time stride (the whole-CTA reduction of long rows).
template <int FMT, uint32_t IW = 4>
__device__ __forceinline__ float dot_strided(const SlotView& v, uint32_t xs, uint32_t kb, uint32_t ke,
                                             uint32_t step) {
    constexpr uint32_t ES = (uint32_t)sizeof(typename Fmt<FMT>::T);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    uint32_t k = kb;
    for (; k + 3 * step < ke; k += 4 * step) {
        const uint32_t k1 = k + step, k2 = k + 2 * step, k3 = k + 3 * step;
        const uint32_t c0 = col_at<IW>(v, k), c1 = col_at<IW>(v, k1);
        const uint32_t c2 = col_at<IW>(v, k2), c3 = col_at<IW>(v, k3);
        const float w0 = Fmt<FMT>::lds(v.val + ES * k), w1 = Fmt<FMT>::lds(v.val + ES * k1);
        const float w2 = Fmt<FMT>::lds(v.val + ES * k2), w3 = Fmt<FMT>::lds(v.val + ES * k3);
        a0 = __fmaf_rn(w0, dev::lds_f32(xs + 4 * c0), a0);
        a1 = __fmaf_rn(w1, dev::lds_f32(xs + 4 * c1), a1);
        a2 = __fmaf_rn(w2, dev::lds_f32(xs + 4 * c2), a2);
        a3 = __fmaf_rn(w3, dev::lds_f32(xs + 4 * c3), a3);
    }
    if (k < ke) a0 = __fmaf_rn(Fmt<FMT>::lds(v.val + ES * k), dev::lds_f32(xs + 4 * col_at<IW>(v, k)), a0);
    k += step;
    if (k < ke) a1 = __fmaf_rn(Fmt<FMT>::lds(v.val + ES * k), dev::lds_f32(xs + 4 * col_at<IW>(v, k)), a1);
    k += step;
    if (k < ke) a2 = __fmaf_rn(Fmt<FMT>::lds(v.val + ES * k), dev::lds_f32(xs + 4 * col_at<IW>(v, k)), a2);
    return __fadd_rn(__fadd_rn(a0, a1), __fadd_rn(a2, a3));
}

// Compensated version (Dot2 of Ogita, Rump and Oishi, 2005): returns (s, c)
// with s + c the dot product to about twice the working precision.
template <int FMT, uint32_t IW = 4>
__device__ __forceinline__ void dot_strided_comp(const SlotView& v, uint32_t xs, const float* __restrict__ xg,
                                                 bool xsmem, uint32_t kb, uint32_t ke, uint32_t step, float& s,
                                                 float& c) {
    constexpr uint32_t ES = (uint32_t)sizeof(typename Fmt<FMT>::T);
    for (uint32_t k = kb; k < ke; k += step) {
        const float a = Fmt<FMT>::lds(v.val + ES * k);
        const uint32_t j = col_at<IW>(v, k);
        const float xv = xsmem ? dev::lds_f32(xs + 4 * j) : __ldg(xg + j);
        float pr, ep, t, es;
        dev::two_prod(a, xv, pr, ep);
        dev::two_sum(s, pr, t, es);
        s = t;
        c = __fadd_rn(c, __fadd_rn(es, ep));
    }
}

// Plain sum with x read from global memory (x too large for shared memory).
template <int FMT, uint32_t IW = 4>
__device__ __forceinline__ float dot_strided_gx(const SlotView& v, const float* __restrict__ xg, uint32_t kb,
                                                uint32_t ke, uint32_t step) {
    constexpr uint32_t ES = (uint32_t)sizeof(typename Fmt<FMT>::T);
    float a0 = 0.f, a1 = 0.f;
    uint32_t k = kb;
    for (; k + step < ke; k += 2 * step) {
        const uint32_t k1 = k + step;
        const uint32_t c0 = col_at<IW>(v, k), c1 = col_at<IW>(v, k1);
        const float w0 = Fmt<FMT>::lds(v.val + ES * k), w1 = Fmt<FMT>::lds(v.val + ES * k1);
        a0 = __fmaf_rn(w0, __ldg(xg + c0), a0);
        a1 = __fmaf_rn(w1, __ldg(xg + c1), a1);
    }
    if (k < ke) a0 = __fmaf_rn(Fmt<FMT>::lds(v.val + ES * k), __ldg(xg + col_at<IW>(v, k)), a0);
    return __fadd_rn(a0, a1);
}

#endif

}  // namespace dose
