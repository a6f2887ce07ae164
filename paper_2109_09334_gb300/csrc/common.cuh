// common.cuh -- device helpers shared by the SFFT kernels (sm_103a).
//
// Complex numbers, compensated (two-sum) accumulators, monomial ordering
// and the normalised pixel coordinate used by every kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfft {

template <typename T>
struct alignas(2 * sizeof(T)) cpx {
    T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T r, T i) {
    cpx<T> c;
    c.re = r;
    c.im = i;
    return c;
}
template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// acc + a * b and acc - a * b as four fused multiply-adds each (the
// products are not rounded separately, so the results differ from
// acc +- cmul(a, b) in the last bits; both are single-rounding-per-term sums)
template <typename T>
__device__ __forceinline__ cpx<T> cfma(cpx<T> acc, cpx<T> a, cpx<T> b) {
    T re = fma(a.re, b.re, acc.re);
    re = fma(-a.im, b.im, re);
    T im = fma(a.re, b.im, acc.im);
    im = fma(a.im, b.re, im);
    return mk(re, im);
}
template <typename T>
__device__ __forceinline__ cpx<T> cfms(cpx<T> acc, cpx<T> a, cpx<T> b) {
    T re = fma(-a.re, b.re, acc.re);
    re = fma(a.im, b.im, re);
    T im = fma(-a.re, b.im, acc.im);
    im = fma(-a.im, b.re, im);
    return mk(re, im);
}
// conj(a) * b
template <typename T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
    return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
template <typename T>
__device__ __forceinline__ cpx<T> conj(cpx<T> a) { return mk(a.re, -a.im); }
template <typename T>
__device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk(a.re * s, a.im * s); }
// multiply by +i (sgn > 0) or -i (sgn < 0)
template <typename T>
__device__ __forceinline__ cpx<T> mul_i(cpx<T> a, int sgn) {
    return sgn > 0 ? mk(-a.im, a.re) : mk(a.im, -a.re);
}

// ---- compensated accumulation ----------------------------------------------
// Acc<float> keeps an unevaluated sum hi + lo; each add is Knuth's two-sum, so
// the rounding error of every addition is carried in lo.  This gives the
// frequency sums near double accuracy on the FP32 pipes (the FP64 rate of
// the part is too low for these sums).  Acc<double> is a plain double.
// These kernels must be compiled without fast-math (no reassociation).
template <typename T>
struct Acc;

template <>
struct Acc<double> {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add(double b) { v += b; }
    __device__ __forceinline__ void add(const Acc<double> &o) { v += o.v; }
    __device__ __forceinline__ double value() const { return v; }
    __device__ __forceinline__ double wide() const { return v; }
};

template <>
struct Acc<float> {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
    __device__ __forceinline__ void add(float b) {
        float s = __fadd_rn(hi, b);
        float bb = __fsub_rn(s, hi);
        float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    __device__ __forceinline__ void add(const Acc<float> &o) {
        add(o.hi);
        lo = __fadd_rn(lo, o.lo);
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(hi, lo); }
    __device__ __forceinline__ double wide() const { return (double)hi + (double)lo; }
};

template <typename T>
struct CAcc {
    Acc<T> re, im;
    __device__ __forceinline__ void zero() { re.zero(); im.zero(); }
    __device__ __forceinline__ void add(cpx<T> v) { re.add(v.re); im.add(v.im); }
};

// shuffle helpers for accumulators
__device__ __forceinline__ void shfl_add(Acc<float> &a, int mask, int width = 32) {
    Acc<float> o;
    o.hi = __shfl_xor_sync(0xffffffffu, a.hi, mask, width);
    o.lo = __shfl_xor_sync(0xffffffffu, a.lo, mask, width);
    a.add(o);
}
__device__ __forceinline__ void shfl_add(Acc<double> &a, int mask, int width = 32) {
    a.v += __shfl_xor_sync(0xffffffffu, a.v, mask, width);
}

// ---- geometry ------------------------------------------------------------------
// normalised coordinate xt = (2x - (n-1)) / (n-1) in [-1, 1]
template <typename T>
__device__ __forceinline__ T coord(int x, int n) {
    return (T)(2 * x - (n - 1)) / (T)(n - 1);
}

template <typename T>
__device__ __forceinline__ T ipow(T v, int e) {
    T r = (T)1;
    for (int k = 0; k < e; ++k) r *= v;
    return r;
}

// monomial k -> (i, j) with i + j <= d: by total degree, then descending i
__host__ __device__ __forceinline__ void term_ij(int k, int *i, int *j) {
    int deg = 0, start = 0;
    while (start + deg + 1 <= k) {
        start += deg + 1;
        ++deg;
    }
    *i = deg - (k - start);
    *j = k - start;
}
__host__ __device__ __forceinline__ int term_index(int i, int j) {
    int deg = i + j;
    return deg * (deg + 1) / 2 + j;
}
__host__ __device__ __forceinline__ int n_terms(int d) { return (d + 1) * (d + 2) / 2; }

__device__ __forceinline__ int imod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

}  // namespace sfft
