// FP64-vector accumulation shared by the dose SpMVs with FP64 x and d
// (dose_spmv_f64: spmv_f64_kernel.cu on CSR, rg_spmm.cu on the row-group
// layout).  Double-float (default): x_j arrives as an FP32 pair (hi, lo) with
// hi + lo = x_j to 2^-48 relative; a decoded value a times x_j is formed as
// p + e with p = fl(a hi) and e = fma(a, lo, fma(a, hi, -p)); accumulators are
// pairs (s, c) updated by TwoSum (Knuth) with the rounding errors and e
// collected in c (Dot2 of Ogita, Rump and Oishi); pairs combine the same way
// and a row's result is one FP64 addition.  FP64-FMA (the paper's arithmetic):
// x_j as a double, one FP64 FMA per term.
#pragma once

#include "stage_common.cuh"

namespace dose {

constexpr int F64_DF = 0;  // double-float accumulation (FP32 pairs)
constexpr int F64_DP = 1;  // native FP64 FMA accumulation

// (s, c) += a * (hi + lo)
__device__ __forceinline__ void df_mac(float a, float2 x, float& s, float& c) {
    const float p = __fmul_rn(a, x.x);
    const float e = __fmaf_rn(a, x.y, __fmaf_rn(a, x.x, -p));
    float t, err;
    dev::two_sum(s, p, t, err);
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}

// (s, c) += (s2, c2)
__device__ __forceinline__ void df_add(float& s, float& c, float s2, float c2) {
    float t, e;
    dev::two_sum(s, s2, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, e));
}

// Accumulator of one lane: a double-float pair or a double.
template <int MODE>
struct Acc;
template <>
struct Acc<F64_DF> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void mac(float a, const uint2* xsp, uint32_t j) {
        const uint2 q = xsp[j];
        df_mac(a, make_float2(__uint_as_float(q.x), __uint_as_float(q.y)), s, c);
    }
    __device__ __forceinline__ void add(const Acc& o) { df_add(s, c, o.s, o.c); }
    __device__ __forceinline__ Acc shfl_xor(uint32_t off) const {
        Acc o;
        o.s = __shfl_xor_sync(0xffffffffu, s, off);
        o.c = __shfl_xor_sync(0xffffffffu, c, off);
        return o;
    }
    // d = sc * (s + c) in FP64 (sc = 1: no scale)
    __device__ __forceinline__ double result(bool scaled, float sc) const {
        if (!scaled) return __dadd_rn((double)s, (double)c);
        const float p = __fmul_rn(sc, s);
        const float e = __fmaf_rn(sc, c, __fmaf_rn(sc, s, -p));
        return __dadd_rn((double)p, (double)e);
    }
    __device__ __forceinline__ uint2 pack() const { return make_uint2(__float_as_uint(s), __float_as_uint(c)); }
    __device__ __forceinline__ static Acc unpack(uint2 q) {
        Acc a;
        a.s = __uint_as_float(q.x);
        a.c = __uint_as_float(q.y);
        return a;
    }
};
template <>
struct Acc<F64_DP> {
    double v = 0.0;
    __device__ __forceinline__ void mac(float a, const uint2* xsp, uint32_t j) {
        const uint2 q = xsp[j];
        v = __fma_rn((double)a, __hiloint2double((int)q.y, (int)q.x), v);
    }
    __device__ __forceinline__ void add(const Acc& o) { v = __dadd_rn(v, o.v); }
    __device__ __forceinline__ Acc shfl_xor(uint32_t off) const {
        Acc o;
        o.v = __shfl_xor_sync(0xffffffffu, v, off);
        return o;
    }
    __device__ __forceinline__ double result(bool scaled, float sc) const {
        return scaled ? __dmul_rn((double)sc, v) : v;
    }
    __device__ __forceinline__ uint2 pack() const {
        return make_uint2((uint32_t)__double2loint(v), (uint32_t)__double2hiint(v));
    }
    __device__ __forceinline__ static Acc unpack(uint2 q) {
        Acc a;
        a.v = __hiloint2double((int)q.y, (int)q.x);
        return a;
    }
};

}  // namespace dose
