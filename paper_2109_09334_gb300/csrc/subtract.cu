// subtract.cu -- difference image of Eq. 12-13 from the solved coefficients.
//
// D = S - sum_t sum_(a,b) c_t(a,b) g_t(x - a, y - b) - sum_pq b_pq T^pq, with
// g_t = xt^i yt^j R and the per-term kernel c_t of the delta basis (Eq. 3-4):
// c_t(a,b) = a_t,ab for (a,b) != 0 and c_t(0,0) = a_t,00 - sum_(a,b)!=0 a_t,ab.
// Along y the convolution is taken in Fourier space (Eq. 13): with the row
// transforms G~_t(x, m) of the build, the row transform of D is
//   D~(x, m) = S~(x, m) - sum_t sum_a kap_t(a, m) G~_t(x - a, m) - B~(x, m),
//   kap_t(a, m) = sum_b c_t(a, b) exp(-2 pi i m b / N1),
// an L0-tap circular stencil along x per frequency column m; one inverse
// real FFT per row then gives D.
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft.cuh"
#include "fft16.cuh"
#include "internal.h"

namespace sfft {

__device__ __forceinline__ int unknown_index(int t, int a, int b, int w0, int w1, int cpr) {
    const int L1 = 2 * w1 + 1, L = (2 * w0 + 1) * L1;
    const int off = (a + w0) * L1 + (b + w1);
    if (t == 0) return off;
    const int ctr = (L - 1) / 2;
    if (cpr) {
        if (off == ctr) return -1;
        return L + (t - 1) * (L - 1) + (off > ctr ? off - 1 : off);
    }
    return L + (t - 1) * L + off;
}

// ksum[t] = sum over (a,b) != 0 of a_t,ab  (FP64)
__global__ void k_kernel_sums(int w0, int w1, int cpr, const double *__restrict__ x, double *__restrict__ ksum) {
    const int t = blockIdx.x;
    double s = 0.0;
    const int L1 = 2 * w1 + 1, L = (2 * w0 + 1) * L1;
    for (int off = threadIdx.x; off < L; off += blockDim.x) {
        const int a = off / L1 - w0, b = off % L1 - w1;
        if (a == 0 && b == 0) continue;
        s += x[unknown_index(t, a, b, w0, w1, cpr)];
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        ksum[t] = v;
    }
}

// kap[t][a + w0][m]
template <typename T>
__global__ void k_kernel_table(int n1, int nk, int w0, int w1, int cpr, const double *__restrict__ x,
                               const double *__restrict__ ksum, const cpx<T> *__restrict__ tw1,
                               cpx<T> *__restrict__ kap) {
    const int h1c = n1 / 2 + 1, L0 = 2 * w0 + 1;
    const size_t total = (size_t)nk * L0 * h1c;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(e % h1c);
        const int ta = (int)(e / h1c);
        const int t = ta / L0, a = ta % L0 - w0;
        T re = (T)0, im = (T)0;
        for (int b = -w1; b <= w1; ++b) {
            double c;
            if (a == 0 && b == 0) {
                const int u = unknown_index(t, 0, 0, w0, w1, cpr);
                c = (u >= 0 ? x[u] : 0.0) - ksum[t];
            } else {
                c = x[unknown_index(t, a, b, w0, w1, cpr)];
            }
            cpx<T> w = tw1[imod(m * b, n1)];  // exp(-2 pi i m b / n1)
            re += (T)c * w.re;
            im += (T)c * w.im;
        }
        kap[e] = mk(re, im);
    }
}

// One block per column m: D~(., m) into Dt[m][x].  For each y-power j the
// row transforms of yt^j R are staged in shared memory; the kernel row
// spectra of the terms (i, j) are combined per tap by Horner's rule in the
// source row's coordinate, sum_i kap_(i,j)(a, m) xt(x - a)^i.
template <typename T>
__global__ void k_sub_cols(int n0, int n1, int dk, int db, int w0, int nbkg_off, const cpx<T> *__restrict__ F,
                           const cpx<T> *__restrict__ kap, const cpx<T> *__restrict__ yhat,
                           const double *__restrict__ x, cpx<T> *__restrict__ Dt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *col = reinterpret_cast<cpx<T> *>(smem_raw);  // n0
    cpx<T> *kp = col + n0;                                // nk * L0
    T *xts = reinterpret_cast<T *>(kp + n_terms(dk) * (2 * w0 + 1));  // n0 coordinates
    constexpr int kMaxPer = 32;
    const int m = blockIdx.x, tid = threadIdx.x, nthr = blockDim.x;
    const int h1c = n1 / 2 + 1, L0 = 2 * w0 + 1;
    const int nk = n_terms(dk), nbt = n_terms(db);
    const int per = n0 / nthr;  // outputs per thread (n0 multiple of nthr)
    const int msk = n0 - 1;     // n0 is a power of two
    for (int e = tid; e < nk * L0; e += nthr) kp[e] = kap[(size_t)e * h1c + m];
    for (int e = tid; e < n0; e += nthr) {
        xts[e] = coord<T>(e, n0);
        col[e] = F[((size_t)(dk + 1) * h1c + m) * n0 + e];
    }
    __syncthreads();
    cpx<T> acc[kMaxPer];
    // S~ minus the background B~(x, m) = sum_pq b_pq xt^p Y^q(m)
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) {
        if (k < per) {
            const int x0 = tid + k * nthr;
            cpx<T> v = col[x0];
            const T xt = xts[x0];
            for (int s = 0; s < nbt; ++s) {
                int p, q;
                term_ij(s, &p, &q);
                const T bpq = (T)x[nbkg_off + s];
                v = v - scale(yhat[(size_t)q * h1c + m], bpq * ipow(xt, p));
            }
            acc[k] = v;
        }
    }
    __syncthreads();
    for (int j = 0; j <= dk; ++j) {
        const int deg = dk - j;  // terms (i, j) for i = 0..deg
        for (int e = tid; e < n0; e += nthr) col[e] = F[((size_t)j * h1c + m) * n0 + e];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kMaxPer; ++k) {
            if (k < per) {
                const int x0 = tid + k * nthr;
                cpx<T> v = acc[k];
                for (int a = -w0; a <= w0; ++a) {
                    const int src = (x0 - a) & msk;
                    const cpx<T> g = col[src];
                    const T xs = xts[src];
                    cpx<T> kv = kp[term_index(deg, j) * L0 + (a + w0)];
                    for (int i = deg - 1; i >= 0; --i) kv = scale(kv, xs) + kp[term_index(i, j) * L0 + (a + w0)];
                    v = v - cmul(kv, g);
                }
                acc[k] = v;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k)
        if (k < per) Dt[(size_t)m * n0 + tid + k * nthr] = acc[k];
}

// Inverse real FFT of rows: NG groups of G = n1/16 threads per block, each
// group transforms two rows at once (real and imaginary part of one complex
// FFT of the Hermitian-extended row spectra).
template <typename T, typename I>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) k_rows_inv(int n0, int n1, int NG, const cpx<T> *__restrict__ Dt,
                                                   const cpx<T> *__restrict__ tw1g, I *__restrict__ D) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = n1 / 16;
    const int np = padded_len(n1);
    cpx<T> *tw = reinterpret_cast<cpx<T> *>(smem_raw);  // n1
    cpx<T> *Z = tw + n1;                                 // NG * np
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int grp = tid / G, gt = tid - grp * G;
    const int half = n1 / 2;
    const T inv = (T)1 / (T)n1;
    const int xa = (blockIdx.x * NG + grp) * 2, xb = xa + 1;
    for (int q = tid; q < n1; q += nthr) tw[q] = tw1g[q];
    cpx<T> *zr = Z + (size_t)grp * np;
    for (int mm = gt; mm < n1; mm += G) {
        cpx<T> A, B;
        if (mm <= half) {
            A = Dt[(size_t)mm * n0 + xa];
            B = Dt[(size_t)mm * n0 + xb];
        } else {
            A = conj(Dt[(size_t)(n1 - mm) * n0 + xa]);
            B = conj(Dt[(size_t)(n1 - mm) * n0 + xb]);
        }
        zr[pad16(mm)] = A + mul_i(B, 1);
    }
    __syncthreads();
    group_fft(zr, n1, 1, tw, n1, gt, G);
    for (int y = gt; y < n1; y += G) {
        const cpx<T> z = zr[pad16(y)];
        D[(size_t)xa * n1 + y] = (I)(z.re * inv);
        D[(size_t)xb * n1 + y] = (I)(z.im * inv);
    }
}

template <typename T>
static cudaError_t sub_t(Plan *p, const double *x, void *diff, cudaStream_t s) {
    cudaError_t err;
    double *ksum = p->xw + p->n + 700;  // after the solve's statistics and partial sums
    p->launches += 4;
    k_kernel_sums<<<p->nk, 256, 0, s>>>(p->cfg.w0, p->cfg.w1, p->cfg.const_phot_ratio, x, ksum);
    const size_t tot = (size_t)p->nk * p->L0 * p->h1c;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    k_kernel_table<T><<<blocks, 256, 0, s>>>(p->n1, p->nk, p->cfg.w0, p->cfg.w1, p->cfg.const_phot_ratio, x,
                                             ksum, (const cpx<T> *)p->tw1, (cpx<T> *)p->kap);
    if ((err = cudaGetLastError())) return err;
    {
        int nthr = 256;
        while (p->n0 / nthr > 32) nthr *= 2;
        if (nthr > p->n0) nthr = p->n0;
        size_t smem = ((size_t)p->n0 + (size_t)p->nk * p->L0) * sizeof(cpx<T>) + (size_t)p->n0 * sizeof(T);
        cudaFuncSetAttribute(k_sub_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int nbkg_off = p->n - p->nb;
        k_sub_cols<T><<<p->h1c, nthr, smem, s>>>(p->n0, p->n1, p->cfg.dk, p->cfg.db, p->cfg.w0, nbkg_off,
                                                 (const cpx<T> *)p->F, (const cpx<T> *)p->kap,
                                                 (const cpx<T> *)p->yhat, x, (cpx<T> *)p->U);
        if ((err = cudaGetLastError())) return err;
    }
    {
        const int G = p->n1 / 16;
        int NG = (sizeof(T) == 4 ? 1024 : 512) / G;
        if (NG > 4) NG = 4;
        if (NG > p->n0 / 2) NG = p->n0 / 2;
        size_t smem = ((size_t)p->n1 + (size_t)NG * padded_len(p->n1)) * sizeof(cpx<T>);
        while (NG > 1 && smem > 200 * 1024) {
            NG /= 2;
            smem = ((size_t)p->n1 + (size_t)NG * padded_len(p->n1)) * sizeof(cpx<T>);
        }
        const int blocks = p->n0 / (2 * NG);
        if (p->cfg.dtype == SFFT_F64) {
            cudaFuncSetAttribute(k_rows_inv<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_rows_inv<T, double><<<blocks, NG * G, smem, s>>>(p->n0, p->n1, NG, (const cpx<T> *)p->U,
                                                                (const cpx<T> *)p->tw1, (double *)diff);
        } else {
            cudaFuncSetAttribute(k_rows_inv<T, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_rows_inv<T, float><<<blocks, NG * G, smem, s>>>(p->n0, p->n1, NG, (const cpx<T> *)p->U,
                                                               (const cpx<T> *)p->tw1, (float *)diff);
        }
    }
    return cudaGetLastError();
}

cudaError_t subtract_from_rows(Plan *p, const double *x, void *diff, cudaStream_t s) {
    return p->fp64 ? sub_t<double>(p, x, diff, s) : sub_t<float>(p, x, diff, s);
}

}  // namespace sfft
