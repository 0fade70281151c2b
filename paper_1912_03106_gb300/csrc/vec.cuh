// Vector loads/stores of work vectors and the ELL row product, shared by the
// step-solver kernels.  Work vectors are written by other CTAs between phases
// that are separated by barriers with acquire semantics (cluster barriers, or
// kernel boundaries), so loads either bypass L1 (ld.global.cg, the default) or
// are ordinary L1-cached loads (MG_L1 = 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#ifndef MG_L1
#define MG_L1 0
#endif

namespace mgv {

constexpr int WMAX = 8;  // ELL entries handled fully unrolled; wider rows loop

template <class T, int V>
struct VT;
template <>
struct VT<float, 1> { using t = float; };
template <>
struct VT<float, 2> { using t = float2; };
template <>
struct VT<float, 4> { using t = float4; };
template <>
struct VT<double, 1> { using t = double; };
template <>
struct VT<double, 2> { using t = double2; };

template <class T, int V>
__device__ __forceinline__ void vld(const T* p, T (&o)[V]) {
    if constexpr (std::is_same<T, double>::value && V == 4) {
        double2 a = __ldcg(reinterpret_cast<const double2*>(p));
        double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
        o[0] = a.x;
        o[1] = a.y;
        o[2] = b.x;
        o[3] = b.y;
    } else {
#if MG_L1
        typename VT<T, V>::t v = *reinterpret_cast<const typename VT<T, V>::t*>(p);
#else
        typename VT<T, V>::t v = __ldcg(reinterpret_cast<const typename VT<T, V>::t*>(p));
#endif
        const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int q = 0; q < V; ++q) o[q] = e[q];
    }
}

template <class T, int V>
__device__ __forceinline__ void vst(T* p, const T (&o)[V]) {
    if constexpr (std::is_same<T, double>::value && V == 4) {
        __stcg(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
        __stcg(reinterpret_cast<double2*>(p) + 1, make_double2(o[2], o[3]));
    } else {
        typename VT<T, V>::t v;
        T* e = reinterpret_cast<T*>(&v);
#pragma unroll
        for (int q = 0; q < V; ++q) e[q] = o[q];
#if MG_L1
        *reinterpret_cast<typename VT<T, V>::t*>(p) = v;
#else
        __stcg(reinterpret_cast<typename VT<T, V>::t*>(p), v);
#endif
    }
}

template <class T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }
template <class T>
__device__ __forceinline__ void stcg(T* p, T v) { __stcg(p, v); }

// acc[e] = sum_w val[w, i] * v[col[w, i]][c0 + e]  (v tile-major with KT columns)
template <int KT, int V, class A, class VAL, class X>
__device__ __forceinline__ void ell_vec(const int32_t* __restrict__ col, const VAL* __restrict__ val, int n, int W,
                                        int i, const X* v, int c0, A (&acc)[V]) {
#pragma unroll
    for (int e = 0; e < V; ++e) acc[e] = 0;
    int32_t j[WMAX];
    VAL a[WMAX];
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < W) {
            j[w] = __ldg(col + w * n + i);
            a[w] = __ldg(val + w * n + i);
        }
#pragma unroll
    for (int w = 0; w < WMAX; ++w)
        if (w < W) {
            X xv[V];
            vld<X, V>(v + j[w] * KT + c0, xv);
#pragma unroll
            for (int e = 0; e < V; ++e) acc[e] += (A)a[w] * (A)xv[e];
        }
    for (int w = WMAX; w < W; ++w) {
        X xv[V];
        vld<X, V>(v + __ldg(col + w * n + i) * KT + c0, xv);
        const A aw = (A)__ldg(val + w * n + i);
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] += aw * (A)xv[e];
    }
}

// |x| as a float, by integer instructions (exponent rebiased, mantissa truncated:
// at most 2^-23 below |x|; 0 below the float range, infinity above it).  Used for
// magnitude estimates, which need no FP64 arithmetic: on GB300 the FP64 pipe, which
// also converts between double and float, runs at a small fraction of FP32's rate.
__device__ __forceinline__ float abs_to_float(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    const int e = (int)(u >> 52) - 1023 + 127;
    if (e <= 0) return 0.0f;
    if (e >= 255) return __uint_as_float(0x7f800000u);
    return __uint_as_float(((unsigned)e << 23) | (unsigned)((u >> 29) & 0x7fffffull));
}

// Exact float -> double conversion with integer instructions: on GB300 the F2F
// conversion issues on the FP64 pipe, whose rate is a small fraction of FP32's.
// Normal numbers and zeros convert by moving bits; infinities stay infinities and
// NaNs stay NaNs (exponent all ones maps to all ones, the mantissa bits are kept),
// so a poisoned preconditioner output reaches the convergence test instead of
// turning into a large finite number; the rare denormals take the hardware path.
__device__ __forceinline__ double f2d_int(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u && (u & 0x7fffffu)) return (double)f;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned long long mant = (unsigned long long)(u & 0x7fffffu) << 29;
    const unsigned long long ex = (unsigned long long)(e == 0xffu ? 0x7ffu : e + (1023u - 127u)) << 52;
    return __longlong_as_double((long long)(e ? (sign | ex | mant) : sign));
}

// x split into two floats, x ~ h + l, by integer instructions: h is x with its
// significand truncated to 24 bits (exact), l the remaining 29 bits truncated to
// 24 (|x - h - l| <= 2^-47 |x|).  Magnitudes below the float range give h = l = 0
// (their products sit far below the sums they enter); infinities and NaNs give
// h = x as a float (NaN stays NaN) and l = 0, so poisoned inputs stay visible.
__device__ __forceinline__ void split_d2f(double x, float& h, float& l) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ffull);
    l = 0.0f;
    if (e == 0x7ff) {
        h = __uint_as_float(sign | 0x7f800000u | ((u & 0xfffffffffffffull) ? 0x400000u : 0u));
        return;
    }
    const int eh = e - 1023 + 127;
    if (eh <= 0) {
        h = 0.0f;
        return;
    }
    if (eh >= 255) {  // beyond the float range
        h = __uint_as_float(sign | 0x7f800000u);
        return;
    }
    h = __uint_as_float(sign | ((unsigned)eh << 23) | (unsigned)((u >> 29) & 0x7fffffull));
    const unsigned rem = (unsigned)(u & 0x1fffffffull);  // value rem * 2^(e - 1075)
    if (!rem) return;
    const int top = 31 - __clz(rem);  // leading one of rem, 0 .. 28
    const int el = top + e - 1075 + 127;
    if (el <= 0) return;
    const unsigned frac = top >= 23 ? (rem >> (top - 23)) & 0x7fffffu : (rem << (23 - top)) & 0x7fffffu;
    l = __uint_as_float(sign | ((unsigned)el << 23) | frac);
}

// Double-float accumulator of products in FP32 arithmetic: hi holds the running
// sum of the rounded leading products (each addition's rounding error is kept by
// two-sum), lo the FP32 sum of those errors, of the products' own FMA error terms
// and of the small products al * z; value() widens both and adds them once in FP64.
struct DfAcc {
    float hi = 0.0f, lo = 0.0f;
    // += (ah + al) z
    __device__ __forceinline__ void add(float ah, float al, float z) {
        const float p = __fmul_rn(ah, z);
        const float pe = __fmaf_rn(ah, z, -p);  // ah * z = p + pe exactly
        const float s = __fadd_rn(hi, p);
        const float bp = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));  // hi + p = s + err
        hi = s;
        lo = __fmaf_rn(al, z, __fadd_rn(lo, __fadd_rn(err, pe)));
    }
    // += (ah + al) (xh + xl), dropping al * xl
    __device__ __forceinline__ void add(float ah, float al, float xh, float xl) {
        const float p = __fmul_rn(ah, xh);
        const float pe = __fmaf_rn(ah, xh, -p);  // ah * xh = p + pe exactly
        const float s = __fadd_rn(hi, p);
        const float bp = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));  // hi + p = s + err
        hi = s;
        lo = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, __fadd_rn(lo, __fadd_rn(err, pe))));
    }
    __device__ __forceinline__ double value() const { return f2d_int(hi) + f2d_int(lo); }
};

}  // namespace mgv
