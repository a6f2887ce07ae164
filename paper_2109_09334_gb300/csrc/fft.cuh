// fft.cuh -- block-cooperative FFTs in shared memory (power-of-two lengths).
//
// Stockham auto-sort formulation: every stage reads the whole vector from one
// shared buffer and writes it in natural order to the other, so no bit
// reversal pass is needed.  Radix-4 stages, plus one radix-2 stage when
// log2(n) is odd.  Twiddles come from a table tw[q] = exp(-2 pi i q / n_tab)
// that the plan computes in FP64 (sincospi) and rounds to T; a transform of
// length n reads it with stride n_tab / n.
#pragma once

#include "common.cuh"

namespace sfft {

// exp(sgn * 2 pi i q / n) from the forward table (sgn = -1 forward, +1 inverse)
template <typename T>
__device__ __forceinline__ cpx<T> twiddle(const cpx<T> *__restrict__ tw, int q, int stride, int sgn) {
    cpx<T> w = tw[q * stride];
    return sgn < 0 ? w : mk(w.re, -w.im);
}

// 4-point DFT with sign sgn on (v0..v3) in place
template <typename T>
__device__ __forceinline__ void dft4(cpx<T> &v0, cpx<T> &v1, cpx<T> &v2, cpx<T> &v3, int sgn) {
    cpx<T> a = v0 + v2, b = v0 - v2, c = v1 + v3, d = mul_i(v1 - v3, sgn);
    v0 = a + c;
    v2 = a - c;
    v1 = b + d;
    v3 = b - d;
}

// 8-point DFT with sign sgn on v (natural order in and out): a radix-2 split
// into two 4-point DFTs.
template <typename T>
__device__ __forceinline__ void dft8(cpx<T> (&v)[8], int sgn) {
    const T c = (T)0.70710678118654752440;
    cpx<T> a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = v[k] + v[k + 4];
        b[k] = v[k] - v[k + 4];
    }
    // b[k] *= exp(sgn 2 pi i k / 8)
    b[1] = cmul(b[1], mk(c, sgn * c));
    b[2] = mul_i(b[2], sgn);
    b[3] = cmul(b[3], mk(-c, sgn * c));
    dft4(a[0], a[1], a[2], a[3], sgn);
    dft4(b[0], b[1], b[2], b[3], sgn);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = a[k];
        v[2 * k + 1] = b[k];
    }
}

// Transform the n values in buf (shared memory); scratch is another n-element
// shared buffer.  All threads of the block participate (tid, nthr) and must
// call it together.  Returns the buffer that holds the result (buf or
// scratch).  Ends with __syncthreads.
template <typename T>
__device__ cpx<T> *block_fft(cpx<T> *buf, cpx<T> *scratch, int n, const cpx<T> *__restrict__ tw,
                             int tw_n, int sgn, int tid, int nthr) {
    cpx<T> *src = buf, *dst = scratch;
    int log2n = 31 - __clz(n);
    int ns = 1;
    if (log2n & 1) {
        int h = n >> 1;
        for (int j = tid; j < h; j += nthr) {
            cpx<T> u0 = src[j], u1 = src[j + h];
            dst[2 * j] = u0 + u1;
            dst[2 * j + 1] = u0 - u1;
        }
        __syncthreads();
        cpx<T> *t = src;
        src = dst;
        dst = t;
        ns = 2;
    }
    int q = n >> 2;
    for (; ns < n; ns <<= 2) {
        int twstep = (tw_n / n) * (n / (4 * ns));  // table index per unit of r*k
        for (int j = tid; j < q; j += nthr) {
            int k = j & (ns - 1);
            cpx<T> v0 = src[j], v1 = src[j + q], v2 = src[j + 2 * q], v3 = src[j + 3 * q];
            if (ns > 1) {
                v1 = cmul(v1, twiddle(tw, k, twstep, sgn));
                v2 = cmul(v2, twiddle(tw, 2 * k, twstep, sgn));
                v3 = cmul(v3, twiddle(tw, 3 * k, twstep, sgn));
            }
            dft4(v0, v1, v2, v3, sgn);
            int o = (j - k) * 4 + k;
            dst[o] = v0;
            dst[o + ns] = v1;
            dst[o + 2 * ns] = v2;
            dst[o + 3 * ns] = v3;
        }
        __syncthreads();
        cpx<T> *t = src;
        src = dst;
        dst = t;
    }
    return src;
}

}  // namespace sfft
