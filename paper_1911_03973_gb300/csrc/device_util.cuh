// Small device helpers shared by the kernels of libebe.so.
#pragma once

#include <cstdint>

namespace ebe {

__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// float -> double and double -> float by integer operations on the IEEE-754
// bit layouts, so that the conversions stay off the FP64 pipe (GB300 runs
// FP64 at 1/64 of the FP32 rate).  f2d is exact (normal numbers: rebias the
// exponent by 1023 - 127 = 896 and shift the mantissa up by 29 bits); d2f
// rounds to nearest, ties to even (round bit 28, sticky bits 0..27; a carry
// out of the mantissa correctly bumps the exponent).  Signed zeros map to
// signed zeros; subnormals, infinities, NaNs and results outside the normal
// FP32 range take the hardware conversion.
// The rare cases call out of line: an inlined fallback would be if-converted
// and the hardware conversion executed for every element.
static __device__ __noinline__ double f2d_rare(float f) { return double(f); }
static __device__ __noinline__ float d2f_rare(double v) { return float(v); }

__device__ __forceinline__ double f2d(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double(static_cast<long long>(uint64_t(u) << 32));
    if (e == 0u || e == 0xffu) return f2d_rare(f);
    const uint64_t d = (uint64_t(u & 0x80000000u) << 32) | (uint64_t(e + 896u) << 52) | (uint64_t(u & 0x7fffffu) << 29);
    return __longlong_as_double(static_cast<long long>(d));
}
__device__ __forceinline__ float d2f(double v) {
    const uint64_t u = static_cast<uint64_t>(__double_as_longlong(v));
    if ((u & 0x7fffffffffffffffull) == 0ull) return __uint_as_float(uint32_t(u >> 32));
    const int e = int((u >> 52) & 0x7ffu) - 896;
    if (e <= 0 || e >= 254) return d2f_rare(v);
    uint32_t bits = (uint32_t(e) << 23) | uint32_t((u >> 29) & 0x7fffffu);
    const uint32_t rnd = uint32_t(u >> 28) & 1u;
    const uint32_t sticky = (u & 0x0fffffffull) != 0ull ? 1u : 0u;
    bits += rnd & (sticky | (bits & 1u));
    return __uint_as_float((uint32_t(u >> 32) & 0x80000000u) | bits);
}

// Programmatic dependent launch.  pdl_trigger: once every CTA of this grid has
// executed it (or exited), the next kernel in the stream may start launching
// into free SM slots.  pdl_wait: blocks until the previous kernel has
// completed and its memory is visible; code before it must not read that
// kernel's results.  Both are no-ops for kernels launched without the
// programmatic-serialisation attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Neumaier-compensated FP32 sum: s + c carries the sum to about FP32^2.
struct CompSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// Knuth's TwoSum: returns fl(a + b) and sets e to its rounding error, so that
// the result plus e equals a + b exactly (FP32 arithmetic only).  The error of
// a rounded sum is unique, so swapping a and b gives the same pair.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float t = a + b;
    const float bp = t - a;
    e = (a - (t - bp)) + (b - bp);
    return t;
}

// Sum of a compensated FP32 value over a warp in a fixed butterfly order,
// all in FP32 (GB300 runs FP64 at 1/64 of the FP32 rate): each level adds the
// two partners' leading parts with TwoSum and carries the rounding error and
// the partners' error terms in c.  Every lane ends with the same total.
__device__ __forceinline__ void warp_sum(CompSum& v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, v.s, o), c2 = __shfl_xor_sync(0xffffffffu, v.c, o);
        float e;
        v.s = two_sum(v.s, s2, e);
        v.c = (v.c + c2) + e;
    }
}

__device__ __forceinline__ CompSum comp_of(float2 v) {
    CompSum c;
    c.s = v.x;
    c.c = v.y;
    return c;
}

// a += b for compensated FP32 values (TwoSum of the leading parts, errors
// carried in c); the same result in either order of a and b.
__device__ __forceinline__ void merge(CompSum& a, const CompSum& b) {
    float e;
    a.s = two_sum(a.s, b.s, e);
    a.c = (a.c + b.c) + e;
}

// Sum over each group of 8 consecutive lanes (butterfly offsets 4, 2, 1),
// compensated FP32; every lane of a group ends with its group's total.
__device__ __forceinline__ void group8_sum(CompSum& v) {
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, v.s, o), c2 = __shfl_xor_sync(0xffffffffu, v.c, o);
        float e;
        v.s = two_sum(v.s, s2, e);
        v.c = (v.c + c2) + e;
    }
}

// Sum over a warp in a fixed butterfly order with plain FP32 additions (the
// lane's compensation term is folded in first; the total comes back with
// c = 0).  Five roundings of partial sums of a few terms each: about 3e-7 of
// the warp's sum of magnitudes, random in sign across warps, whose totals
// are then added in compensated form.  Every lane ends with the same total.
__device__ __forceinline__ void warp_sum_plain(CompSum& v) {
    float t = v.s + v.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    v.s = t;
    v.c = 0.0f;
}

// K compensated FP32 sums over a block of NT threads, entirely in FP32:
// warp butterflies, then thread 0 merges the per-warp totals in warp order.
// Every thread must call it; out is valid in thread 0.  red: K * NT / 32
// float2 of shared memory.
template <int K, int NT>
__device__ __forceinline__ void block_sums_f32(CompSum (&v)[K], CompSum (&out)[K], float2* red) {
    constexpr int NW = NT / 32;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * NW + w] = make_float2(v[k].s, v[k].c);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        CompSum t;
        if (threadIdx.x == 0)
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                const float2 r = red[k * NW + i];
                CompSum x;
                x.s = r.x;
                x.c = r.y;
                merge(t, x);
            }
        out[k] = t;
    }
}

// K compensated FP32 sums over a block of NT threads: warp butterflies in
// FP32, then thread 0 adds the per-warp totals (converted to FP64 once per
// warp) in warp order.  Every thread must call it; the results are valid in
// thread 0.  red: K * NT / 32 doubles of shared memory.
template <int K, int NT>
__device__ __forceinline__ void block_sums_comp(CompSum (&v)[K], double (&out)[K], double* red) {
    constexpr int NW = NT / 32;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * NW + w] = v[k].value();
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double t = 0.0;
        if (threadIdx.x == 0)
#pragma unroll
            for (int i = 0; i < NW; ++i) t += red[k * NW + i];
        out[k] = t;
    }
}

// Double-word (pairs of FP32) arithmetic for FP64-accurate sums on the FP32
// pipe (Dekker 1971; Hida, Li and Bailey 2001, "sloppy" addition): a value is
// hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits.

// x = hi + lo to 48 bits: hi is x rounded to FP32, lo the remainder x - hi
// (exact in FP64) rounded to FP32, both formed on the integer pipe (the
// remainder of the 53-bit mantissa after its top 24 bits is an integer of at
// most 29 bits, converted and scaled).  Zeros, subnormals and values whose hi
// or lo leaves the normal FP32 range take the hardware conversions.
static __device__ __noinline__ void split_rare(double v, float& hi, float& lo) {
    hi = float(v);
    lo = float(v - double(hi));
}
__device__ __forceinline__ void split_dw(double v, float& hi, float& lo) {
    const uint64_t u = static_cast<uint64_t>(__double_as_longlong(v));
    const int e = int((u >> 52) & 0x7ffu);                  // biased FP64 exponent
    if (e < 1023 - 126 + 53 || e > 1023 + 126) { split_rare(v, hi, lo); return; }
    hi = d2f(v);
    const uint32_t hb = __float_as_uint(hi);
    const int eh = int((hb >> 23) & 0xffu) - 127;           // hi's exponent: e - 1023 or one more
    const int64_t m = int64_t((u & 0xfffffffffffffull) | 0x10000000000000ull);
    const int64_t mh = int64_t((hb & 0x7fffffu) | 0x800000u) << (29 + eh - (e - 1023));
    const int32_t d = int32_t(m - mh);                      // |d| <= 2^28
    // lo = d * 2^(e - 1075), the scale a normal FP32 power of two here
    const float scale = __uint_as_float(uint32_t(e - 1075 + 127) << 23);
    const float l = __int2float_rn(d) * scale;
    lo = (u >> 63) ? -l : l;
}

// p + e = a * b exactly (fused multiply-add gives the rounding error).
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
    const float p = a * b;
    e = __fmaf_rn(a, b, -p);
    return p;
}

// (s, c) += (ah + al) * (xh + xl): the leading product exactly (two_prod),
// the cross terms in FP32 (the al * xl term is below the 48-bit precision).
__device__ __forceinline__ void dw_fma(float ah, float al, float xh, float xl, float& s, float& c) {
    float e;
    const float p = two_prod(ah, xh, e);
    const float t = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
    float e2;
    s = two_sum(s, p, e2);
    c = c + (t + e2);
}

// (s, c) = (ah + al) * (xh + xl): the first product of a sum, the same
// pair dw_fma gives from (0, 0) without its TwoSum with zero.
__device__ __forceinline__ void dw_mul(float ah, float al, float xh, float xl, float& s, float& c) {
    float e;
    s = two_prod(ah, xh, e);
    c = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
}

// (s, c) += (s2, c2).
__device__ __forceinline__ void dw_add(float& s, float& c, float s2, float c2) {
    float e;
    s = two_sum(s, s2, e);
    c = c + (c2 + e);
}

}  // namespace ebe
