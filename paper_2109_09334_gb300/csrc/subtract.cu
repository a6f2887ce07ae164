// subtract.cu -- difference image of Eq. 12-13 from the solved coefficients.
//
// D = S - sum_t sum_(a,b) c_t(a,b) g_t(x - a, y - b) - sum_s b_s T^s, with
// g_t = xt^i yt^j R (Eq. 10-11) or B_i(xt) B_j(yt) R (Eq. 8), T^s the
// background basis, and the per-term kernel c_t of the delta basis (Eq. 3-4):
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

// ksum[t] = sum over (a,b) != 0 of a_t,ab  (FP64)
__global__ void k_kernel_sums(BasisView bv, const double *__restrict__ x, double *__restrict__ ksum) {
    const int t = blockIdx.x;
    double s = 0.0;
    const int L1 = 2 * bv.w1 + 1, L = (2 * bv.w0 + 1) * L1;
    for (int off = threadIdx.x; off < L; off += blockDim.x) {
        const int a = off / L1 - bv.w0, b = off % L1 - bv.w1;
        if (a == 0 && b == 0) continue;
        const int u = bv.unknown(t, a, b);
        if (u >= 0) s += x[u];
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
__global__ void k_kernel_table(int n1, BasisView bv, const double *__restrict__ x, const double *__restrict__ ksum,
                               const cpx<T> *__restrict__ tw1, cpx<T> *__restrict__ kap) {
    const int w0 = bv.w0, w1 = bv.w1;
    const int h1c = n1 / 2 + 1, L0 = 2 * w0 + 1;
    const size_t total = (size_t)bv.nk * L0 * h1c;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(e % h1c);
        const int ta = (int)(e / h1c);
        const int t = ta / L0, a = ta % L0 - w0;
        T re = (T)0, im = (T)0;
        for (int b = -w1; b <= w1; ++b) {
            const int u = bv.unknown(t, a, b);
            double c = u >= 0 ? x[u] : 0.0;
            if (a == 0 && b == 0) c -= ksum[t];
            cpx<T> w = tw1[imod(m * b, n1)];  // exp(-2 pi i m b / n1)
            re += (T)c * w.re;
            im += (T)c * w.im;
        }
        kap[e] = mk(re, im);
    }
}

// One block per column m: D~(., m) into Dt[m][x].  Thread t computes the Q
// consecutive outputs x0 = Q t .. Q t + Q - 1.  For each kernel term (i, j)
// the weighted column W(x) = xt^i F_j(x, m) is staged in shared memory (one
// pad element after every Q, so the threads' strided accesses hit distinct
// banks) and the L0 taps slide a Q-value window over it: one shared load and
// Q complex multiply-adds per tap.  Q = 4 for FP32, 8 for FP64, so that
// n0 = 4096 needs at most 1024 (FP32) or 512 (FP64) threads.
template <typename T>
__host__ __device__ constexpr int sub_q() { return sizeof(T) == 4 ? 4 : 8; }

// W0 >= 0: the kernel half-width is the compile-time W0 (the tap loop unrolls
// completely, so the window shifts are register renames); W0 < 0: w0 at run time.
template <typename T, bool P2, int W0>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) k_sub_cols(int n0, int n1, BasisView bv, FTab<T> ft,
                                                                         int w0, int nbkg_off,
                                                                         const cpx<T> *__restrict__ F,
                                                                         const cpx<T> *__restrict__ kap,
                                                                         const cpx<T> *__restrict__ yhat,
                                                                         const double *__restrict__ x,
                                                                         cpx<T> *__restrict__ Dt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = bv.nk, nbt = bv.nb;
    if (W0 >= 0) w0 = W0;
    const int L0 = 2 * w0 + 1;
    cpx<T> *kp = reinterpret_cast<cpx<T> *>(smem_raw);  // nk * L0
    constexpr int Q = sub_q<T>();
    cpx<T> *Wb = kp + nk * L0;  // two buffers of n0 + n0 / Q (padded), alternating by term
    auto padq = [](int v) { return v + v / Q; };
    const int m = blockIdx.x, tid = threadIdx.x, nthr = blockDim.x;
    const int h1c = n1 / 2 + 1;
    const int msk = n0 - 1;
    // index mod n0 for -n0 <= v < 2 n0 (P2: n0 is a power of two)
    auto wrapx = [&](int v) { return P2 ? (v & msk) : (v < 0 ? v + n0 : (v >= n0 ? v - n0 : v)); };
    const int x0 = Q * tid;  // outputs x0 .. x0 + Q - 1 below n0
    for (int e = tid; e < nk * L0; e += nthr) kp[e] = kap[(size_t)e * h1c + m];
    T xt[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) xt[q] = coord<T>(x0 + q, n0);
    // S~ minus the background B~(x, m) = sum_s b_s bx_p(x) Y_q(m)
    cpx<T> acc[Q];
    {
        const cpx<T> *Sc = F + ((size_t)bv.nfy * h1c + m) * n0 + x0;
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] = (P2 || x0 + q < n0) ? Sc[q] : mk((T)0, (T)0);
        for (int s = 0; s < nbt; ++s) {
            const int p = bv.sp(s), qq = bv.sq(s);
            const cpx<T> yq = yhat[(size_t)qq * h1c + m];
            const T bpq = (T)x[nbkg_off + s];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const T wx = ft.bx ? ((P2 || x0 + q < n0) ? ft.bx[(size_t)p * n0 + x0 + q] : (T)0) : ipow(xt[q], p);
                acc[q] = acc[q] - scale(yq, bpq * wx);
            }
        }
    }
    // terms grouped by their y-function j: F_j is loaded once per group.  The
    // weighted columns alternate between two buffers, so one barrier per term
    // separates a buffer's fill from its reads and from its refill two terms on.
    const int wlen = n0 + (n0 + Q - 1) / Q;
    int nterm = 0;
    for (int j = 0; j < bv.nfy; ++j) {
        const int ncj = bv.jcnt(j);
        if (ncj == 0) continue;
        cpx<T> f[Q];
        const cpx<T> *Fj = F + ((size_t)j * h1c + m) * n0 + x0;
#pragma unroll
        for (int q = 0; q < Q; ++q) f[q] = (P2 || x0 + q < n0) ? Fj[q] : mk((T)0, (T)0);
        for (int k = 0; k < ncj; ++k) {
            const int t = bv.jterm(j, k), i = bv.ti(t);
            cpx<T> *W = Wb + (size_t)(nterm++ & 1) * wlen;
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (P2 || x0 + q < n0) {
                    const T wx = ft.fx ? ft.fx[(size_t)i * n0 + x0 + q] : ipow(xt[q], i);
                    W[padq(x0 + q)] = scale(f[q], wx);
                }
            __syncthreads();  // this buffer is filled; the other one's reads (two terms ago) are done
            const cpx<T> *kt = kp + t * L0;
            cpx<T> win[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) win[q] = W[padq(wrapx(x0 - w0 + q))];
#pragma unroll
            for (int a = (W0 >= 0 ? W0 : w0); a >= -(W0 >= 0 ? W0 : w0); --a) {
                const cpx<T> kv = kt[a + w0];
#pragma unroll
                for (int q = 0; q < Q; ++q) acc[q] = cfms(acc[q], kv, win[q]);
#pragma unroll
                for (int q = 0; q + 1 < Q; ++q) win[q] = win[q + 1];
                win[Q - 1] = W[padq(wrapx(x0 + Q - a))];
            }
        }
    }
    cpx<T> *out = Dt + (size_t)m * n0 + x0;
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (P2 || x0 + q < n0) out[q] = acc[q];
}

// two consecutive complex values from global memory (16-byte aligned for
// float: one 16-byte load)
__device__ __forceinline__ void load_pair(const cpx<float> *p, cpx<float> &a, cpx<float> &b) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    a = mk(v.x, v.y);
    b = mk(v.z, v.w);
}
__device__ __forceinline__ void load_pair(const cpx<double> *p, cpx<double> &a, cpx<double> &b) {
    a = p[0];
    b = p[1];
}

// Inverse real FFT of rows: NG groups of G = n1/16 threads per block, each
// group transforms two rows at once (real and imaginary part of one complex
// FFT of the Hermitian-extended row spectra).
template <typename T, typename I>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) k_rows_inv(int n0, int n1, int NG, const cpx<T> *__restrict__ Dt,
                                                   const cpx<T> *__restrict__ tw1g, I *__restrict__ D) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = n1 / 16;
    const int np = padded_len(n1);
    cpx<T> *Z = reinterpret_cast<cpx<T> *>(smem_raw);  // NG * np
    const int tid = threadIdx.x;
    const int grp = tid / G, gt = tid - grp * G;
    const int half = n1 / 2;
    const T inv = (T)1 / (T)n1;
    const int xa = (blockIdx.x * NG + grp) * 2, xb = xa + 1;
    const cpx<T> *tw = tw1g;  // pass-ordered twiddles, read through L1
    cpx<T> *zr = Z + (size_t)grp * np;
    {
        // 16 frequencies per thread, all loads in flight; rows xa, xb are
        // adjacent, so with an even n0 both come in one 2-element load
        cpx<T> A[16], B[16];
        if (xb < n0 && (n0 & 1) == 0) {
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int mm = gt + c * G;
                const int mr = (mm <= half) ? mm : n1 - mm;
                load_pair(Dt + (size_t)mr * n0 + xa, A[c], B[c]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int mm = gt + c * G;
                const int mr = (mm <= half) ? mm : n1 - mm;
                A[c] = xa < n0 ? Dt[(size_t)mr * n0 + xa] : mk((T)0, (T)0);
                B[c] = xb < n0 ? Dt[(size_t)mr * n0 + xb] : mk((T)0, (T)0);
            }
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int mm = gt + c * G;
            const cpx<T> a = (mm <= half) ? A[c] : conj(A[c]);
            const cpx<T> b = (mm <= half) ? B[c] : conj(B[c]);
            zr[pad16(mm)] = a + mul_i(b, 1);
        }
    }
    __syncthreads();
    group_fft(zr, n1, 1, tw, gt, G);
    for (int y = gt; y < n1; y += G) {
        const cpx<T> z = zr[pad16(y)];
        if (xa < n0) D[(size_t)xa * n1 + y] = (I)(z.re * inv);
        if (xb < n0) D[(size_t)xb * n1 + y] = (I)(z.im * inv);
    }
}

// Inverse real transform of rows for a row length n1 that is not a power of
// two: as k_rows_inv, with Bluestein DFTs of length n1 (FFTs of length m1).
template <typename T, typename I>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) k_rows_inv_blu(int n0, int n1, int m1, int NG,
                                                       const cpx<T> *__restrict__ Dt,
                                                       const cpx<T> *__restrict__ chirp,
                                                       const cpx<T> *__restrict__ bfilt,
                                                       const cpx<T> *__restrict__ twpm, I *__restrict__ D) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = m1 / 16;
    const int np = padded_len(m1);
    cpx<T> *Z = reinterpret_cast<cpx<T> *>(smem_raw);  // NG * np
    const int tid = threadIdx.x;
    const int grp = tid / G, gt = tid - grp * G;
    const int half = n1 / 2;
    const T inv = (T)1 / (T)n1;
    const int xa = (blockIdx.x * NG + grp) * 2, xb = xa + 1;
    cpx<T> *zr = Z + (size_t)grp * np;
    for (int mm = gt; mm < n1; mm += G) {
        const int mr = (mm <= half) ? mm : n1 - mm;
        cpx<T> a = xa < n0 ? Dt[(size_t)mr * n0 + xa] : mk((T)0, (T)0);
        cpx<T> b = xb < n0 ? Dt[(size_t)mr * n0 + xb] : mk((T)0, (T)0);
        if (mm > half) {
            a = conj(a);
            b = conj(b);
        }
        zr[pad16(mm)] = a + mul_i(b, 1);
    }
    __syncthreads();
    bluestein(zr, n1, m1, 1, chirp, bfilt, twpm, gt, G);
    for (int y = gt; y < n1; y += G) {
        const cpx<T> z = zr[pad16(y)];
        if (xa < n0) D[(size_t)xa * n1 + y] = (I)(z.re * inv);
        if (xb < n0) D[(size_t)xb * n1 + y] = (I)(z.im * inv);
    }
}

// D from its row transforms in p->U (layout [m][x]): the inverse real FFT of
// every row, two rows per complex transform.
template <typename T>
static cudaError_t launch_rows_inv(Plan *p, void *diff, cudaStream_t s) {
    if (p->gen1) {
        const int G = p->m1 / 16;
        int NG = (sizeof(T) == 4 ? 1024 : 512) / G;
        if (NG < 1) NG = 1;
        if (NG > 4) NG = 4;
        if (NG > (p->n0 + 1) / 2) NG = (p->n0 + 1) / 2;
        size_t smem = (size_t)NG * padded_len(p->m1) * sizeof(cpx<T>);
        while (NG > 1 && smem > 200 * 1024) {
            NG /= 2;
            smem = (size_t)NG * padded_len(p->m1) * sizeof(cpx<T>);
        }
        if (p->tune_ng > 0 && p->tune_ng < NG) {
            NG = p->tune_ng;
            smem = (size_t)NG * padded_len(p->m1) * sizeof(cpx<T>);
        }
        const int blocks = (p->n0 + 2 * NG - 1) / (2 * NG);
        const cpx<T> *ch = (const cpx<T> *)p->chirp1, *bf = (const cpx<T> *)p->bfilt1, *tw = (const cpx<T> *)p->twpm1;
        if (p->cfg.dtype == SFFT_F64) {
            cudaFuncSetAttribute(k_rows_inv_blu<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_rows_inv_blu<T, double><<<blocks, NG * G, smem, s>>>(p->n0, p->n1, p->m1, NG, (const cpx<T> *)p->U,
                                                                    ch, bf, tw, (double *)diff);
        } else {
            cudaFuncSetAttribute(k_rows_inv_blu<T, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_rows_inv_blu<T, float><<<blocks, NG * G, smem, s>>>(p->n0, p->n1, p->m1, NG, (const cpx<T> *)p->U,
                                                                   ch, bf, tw, (float *)diff);
        }
    } else {
        const int G = p->n1 / 16;
        // at most 512 (FP32) / 256 (FP64) threads and about 100 KB of shared
        // memory per block, so that two blocks share an SM
        int NG = (sizeof(T) == 4 ? 512 : 256) / G;
        if (NG < 1) NG = 1;
        if (NG > 4) NG = 4;
        if (NG > (p->n0 + 1) / 2) NG = (p->n0 + 1) / 2;
        size_t smem = (size_t)NG * padded_len(p->n1) * sizeof(cpx<T>);
        while (NG > 1 && smem > 110 * 1024) {
            NG /= 2;
            smem = (size_t)NG * padded_len(p->n1) * sizeof(cpx<T>);
        }
        if (p->tune_ng > 0 && p->tune_ng < NG) {
            NG = p->tune_ng;
            smem = (size_t)NG * padded_len(p->n1) * sizeof(cpx<T>);
        }
        const int blocks = (p->n0 + 2 * NG - 1) / (2 * NG);
        if (p->cfg.dtype == SFFT_F64) {
            cudaFuncSetAttribute(k_rows_inv<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_rows_inv<T, double><<<blocks, NG * G, smem, s>>>(p->n0, p->n1, NG, (const cpx<T> *)p->U,
                                                                (const cpx<T> *)p->twp1, (double *)diff);
        } else {
            cudaFuncSetAttribute(k_rows_inv<T, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_rows_inv<T, float><<<blocks, NG * G, smem, s>>>(p->n0, p->n1, NG, (const cpx<T> *)p->U,
                                                               (const cpx<T> *)p->twp1, (float *)diff);
        }
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t sub_t(Plan *p, const double *x, void *diff, cudaStream_t s) {
    cudaError_t err;
    double *ksum = p->xw + p->n + kSolveTail;  // after the solve's statistics and partial sums
    p->launches += 4;
    k_kernel_sums<<<p->nk, 256, 0, s>>>(p->bv, x, ksum);
    const size_t tot = (size_t)p->nk * p->L0 * p->h1c;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 8192) blocks = 8192;
    k_kernel_table<T><<<blocks, 256, 0, s>>>(p->n1, p->bv, x, ksum, (const cpx<T> *)p->tw1, (cpx<T> *)p->kap);
    if ((err = cudaGetLastError())) return err;
    {
        const int nthr = (p->n0 + sub_q<T>() - 1) / sub_q<T>();
        const size_t smem = ((size_t)p->nk * p->L0 + 2 * (size_t)(p->n0 + (p->n0 + sub_q<T>() - 1) / sub_q<T>())) *
                            sizeof(cpx<T>);
        const int nbkg_off = p->n - p->nb;
        auto kern = p->gen0 ? k_sub_cols<T, false, -1> : k_sub_cols<T, true, -1>;
        switch (p->cfg.w0) {  // the half-widths of the workloads, unrolled
            case 4: kern = p->gen0 ? k_sub_cols<T, false, 4> : k_sub_cols<T, true, 4>; break;
            case 5: kern = p->gen0 ? k_sub_cols<T, false, 5> : k_sub_cols<T, true, 5>; break;
            case 6: kern = p->gen0 ? k_sub_cols<T, false, 6> : k_sub_cols<T, true, 6>; break;
            case 7: kern = p->gen0 ? k_sub_cols<T, false, 7> : k_sub_cols<T, true, 7>; break;
            case 8: kern = p->gen0 ? k_sub_cols<T, false, 8> : k_sub_cols<T, true, 8>; break;
            default: break;
        }
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<p->h1c, nthr, smem, s>>>(p->n0, p->n1, p->bv, ftab_of<T>(p), p->cfg.w0, nbkg_off,
                                        (const cpx<T> *)p->F, (const cpx<T> *)p->kap, (const cpx<T> *)p->yhat, x,
                                        (cpx<T> *)p->U);
        if ((err = cudaGetLastError())) return err;
    }
    if ((err = launch_rows_inv<T>(p, diff, s))) return err;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Noise decorrelation (App. C, Eq. 21-24) for one pair.  The spatial
// variation of the kernel is ignored there, so the matching kernel of Eq. 6
// is taken at one normalised position (xt0, yt0):
//     K(a, b) = sum_t xt0^i yt0^j c_t(a, b)            (kernel image, FP64)
// and the real filter of Eq. 24, normalised to unit kernel sum,
//     Q(l, m) = sqrt((s_S^2 + s_R^2 K^(0,0)^2) / (s_S^2 + s_R^2 |K^(l, m)|^2)),
// multiplies the 2-D transform of D:  D_dc = D (*) Q.  K^ is separable in the
// same way as the subtraction: kappa(a, m) = sum_b K(a, b) exp(-2 pi i m b / N1)
// and K^(l, m) = sum_a kappa(a, m) exp(-2 pi i l a / N0).

// Term weights at one normalised position (host-computed): xt0^i yt0^j,
// B_i(xt0) B_j(yt0), or 1 for the constant term.
struct TermWeights {
    double w[kMaxKTerms];
};

__global__ void k_kernel_image(BasisView bv, TermWeights tw, const double *__restrict__ x, double *__restrict__ kimg) {
    const int w0 = bv.w0, w1 = bv.w1;
    const int L1 = 2 * w1 + 1, L = (2 * w0 + 1) * L1;
    for (int e = threadIdx.x; e < L; e += blockDim.x) {
        const int a = e / L1 - w0, b = e % L1 - w1;
        double v = 0.0;
        for (int t = 0; t < bv.nk; ++t) {
            const double wt = tw.w[t];
            if (a != 0 || b != 0) {
                const int u = bv.unknown(t, a, b);
                if (u >= 0) v += wt * x[u];
            } else {
                const int u0 = bv.unknown(t, 0, 0);
                double c = u0 >= 0 ? x[u0] : 0.0;
                for (int o = 0; o < L; ++o) {
                    const int aa = o / L1 - w0, bb = o % L1 - w1;
                    if (aa == 0 && bb == 0) continue;
                    const int u = bv.unknown(t, aa, bb);
                    if (u >= 0) c -= x[u];
                }
                v += wt * c;
            }
        }
        kimg[e] = v;
    }
}

// kap[a + w0][m] = sum_b K(a, b) exp(-2 pi i m b / N1)
// for nkern centred kernels of half-widths w0, w1 (kernel c at kimg_a for
// c < na, else kimg_b): kap[c][a + w0][m] = sum_b k_c(a, b) exp(-2 pi i m b / N1)
template <typename T>
__global__ void k_decorr_kappa(int n1, int nkern, int na, int w0, int w1, const double *__restrict__ kimg_a,
                               const double *__restrict__ kimg_b, const cpx<T> *__restrict__ tw1,
                               cpx<T> *__restrict__ kap) {
    const int h1c = n1 / 2 + 1, L0 = 2 * w0 + 1, L1 = 2 * w1 + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nkern * L0 * h1c; e += gridDim.x * blockDim.x) {
        const int ca = e / h1c, m = e - ca * h1c;
        const int c = ca / L0, a = ca - c * L0;
        const double *k = c < na ? kimg_a + (size_t)c * L0 * L1 : kimg_b + (size_t)(c - na) * L0 * L1;
        cpx<T> v = mk((T)0, (T)0);
        for (int bi = 0; bi < L1; ++bi) v = v + scale(tw1[imod(m * (bi - w1), n1)], (T)k[a * L1 + bi]);
        kap[e] = v;
    }
}

// The co-added form of Eq. 21: ns science kernels G_j then nr reference
// kernels H_i (half-widths g0 along x), their noise variances s2[0 .. ns+nr).
struct CoaddDesc {
    int ns, nr, g0;
    double s2[2 * kMaxCoadd];
};

// Forward real transform of the rows of D, two rows per complex transform,
// written as Dt[m][x] (m < N1/2 + 1): pow2 n1 by the radix-16 FFT, other n1
// by Bluestein.
template <typename T, typename I, bool BLU>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) k_decorr_rows(int n0, int n1, int mlen, int NG,
                                                      const I *__restrict__ D, const cpx<T> *__restrict__ twg,
                                                      const cpx<T> *__restrict__ chirp,
                                                      const cpx<T> *__restrict__ bfilt, cpx<T> *__restrict__ Dt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = mlen / 16;
    const int np = padded_len(mlen);
    const int ntw = BLU ? 0 : pass_table_len(n1);
    cpx<T> *tw = reinterpret_cast<cpx<T> *>(smem_raw);  // pass table (pow2)
    cpx<T> *Z = tw + ntw;                                // NG * np
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int grp = tid / G, gt = tid - grp * G;
    const int xa = (blockIdx.x * NG + grp) * 2, xb = xa + 1;
    for (int q = tid; q < ntw; q += nthr) tw[q] = twg[q];
    cpx<T> *zr = Z + (size_t)grp * np;
    for (int y = gt; y < n1; y += G) {
        const T a = xa < n0 ? (T)D[(size_t)xa * n1 + y] : (T)0;
        const T b = xb < n0 ? (T)D[(size_t)xb * n1 + y] : (T)0;
        zr[pad16(y)] = mk(a, b);
    }
    __syncthreads();
    if (BLU) bluestein(zr, n1, mlen, -1, chirp, bfilt, twg, gt, G);
    else group_fft(zr, n1, -1, tw, gt, G);
    const int h1c = n1 / 2 + 1;
    for (int m = gt; m < h1c; m += G) {
        const cpx<T> z = zr[pad16(m)];
        const cpx<T> zc = conj(zr[pad16(m == 0 ? 0 : n1 - m)]);
        if (xa < n0) Dt[(size_t)m * n0 + xa] = scale(z + zc, (T)0.5);
        if (xb < n0) Dt[(size_t)m * n0 + xb] = mul_i(scale(z - zc, (T)0.5), -1);
    }
}

// Per frequency column m: transform along x, multiply by Q(l, m), transform
// back (scaled by 1/N0), in place in Dt[m][x].
template <typename T, bool BLU>
__global__ void __launch_bounds__(512) k_decorr_cols(int n0, int n1, int mlen, int w0,
                                                      double sigma_ref, double sigma_sci,
                                                      const cpx<T> *__restrict__ kap, const cpx<T> *__restrict__ tw0,
                                                      const cpx<T> *__restrict__ twg, const cpx<T> *__restrict__ chirp,
                                                      const cpx<T> *__restrict__ bfilt, cpx<T> *__restrict__ Dt,
                                                      CoaddDesc cd, const cpx<T> *__restrict__ gam) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = mlen / 16;
    const int ntw = BLU ? 0 : pass_table_len(n0);
    const int L0 = 2 * w0 + 1;
    const int nc = cd.ns + cd.nr, Lg = 2 * cd.g0 + 1;  // nc = 0: the one-pair form
    cpx<T> *tw = reinterpret_cast<cpx<T> *>(smem_raw);  // pass table (pow2)
    cpx<T> *kp = tw + ntw;                               // L0: kappa(a, m)
    cpx<T> *gp = kp + L0;                                // nc * Lg: gamma_c(a, m)
    cpx<T> *zr = gp + nc * Lg;                           // padded mlen
    const int tid = threadIdx.x, m = blockIdx.x;
    const int h1c = n1 / 2 + 1;
    for (int q = tid; q < ntw; q += G) tw[q] = twg[q];
    for (int a = tid; a < L0; a += G) kp[a] = kap[(size_t)a * h1c + m];
    for (int e = tid; e < nc * Lg; e += G) gp[e] = gam[(size_t)e * h1c + m];
    double k00 = 0.0;  // K^(0, 0): the kernel sum
    for (int a = 0; a < L0; ++a) k00 += (double)kap[(size_t)a * h1c].re;
    cpx<T> *col = Dt + (size_t)m * n0;
    for (int x = tid; x < n0; x += G) zr[pad16(x)] = col[x];
    __syncthreads();
    if (BLU) bluestein(zr, n0, mlen, -1, chirp, bfilt, twg, tid, G);
    else group_fft(zr, n0, -1, tw, tid, G);
    if (nc == 0) {
        const double ss2 = sigma_sci * sigma_sci, sr2 = sigma_ref * sigma_ref;
        const T num = (T)(ss2 + sr2 * k00 * k00);
        for (int l = tid; l < n0; l += G) {
            cpx<T> kh = mk((T)0, (T)0);
            for (int a = 0; a < L0; ++a) kh = kh + cmul(kp[a], tw0[imod(l * (a - w0), n0)]);
            const T q = sqrt(num / ((T)ss2 + (T)sr2 * (kh.re * kh.re + kh.im * kh.im)));
            zr[pad16(l)] = scale(zr[pad16(l)], q);
        }
    } else {
        // Eq. 23-24 in full: den = sum_j s_Sj^2 |G^_j|^2 + |K^|^2 sum_i s_Ri^2 |H^_i|^2,
        // normalised by its value at frequency 0 (unit kernel sum)
        double ds = 0.0, dr = 0.0;
        for (int c = 0; c < nc; ++c) {
            double g00 = 0.0;
            for (int a = 0; a < Lg; ++a) g00 += (double)gam[((size_t)c * Lg + a) * h1c].re;
            (c < cd.ns ? ds : dr) += cd.s2[c] * g00 * g00;
        }
        const T num = (T)(ds + k00 * k00 * dr);
        for (int l = tid; l < n0; l += G) {
            cpx<T> kh = mk((T)0, (T)0);
            for (int a = 0; a < L0; ++a) kh = kh + cmul(kp[a], tw0[imod(l * (a - w0), n0)]);
            T es = (T)0, er = (T)0;
            for (int c = 0; c < nc; ++c) {
                cpx<T> gh = mk((T)0, (T)0);
                for (int a = 0; a < Lg; ++a) gh = gh + cmul(gp[c * Lg + a], tw0[imod(l * (a - cd.g0), n0)]);
                const T e2 = (T)cd.s2[c] * (gh.re * gh.re + gh.im * gh.im);
                if (c < cd.ns) es += e2;
                else er += e2;
            }
            const T q = sqrt(num / (es + (kh.re * kh.re + kh.im * kh.im) * er));
            zr[pad16(l)] = scale(zr[pad16(l)], q);
        }
    }
    __syncthreads();
    if (BLU) bluestein(zr, n0, mlen, 1, chirp, bfilt, twg, tid, G);
    else group_fft(zr, n0, 1, tw, tid, G);
    const T inv = (T)1 / (T)n0;
    for (int x = tid; x < n0; x += G) col[x] = scale(zr[pad16(x)], inv);
}

template <typename T>
static cudaError_t decorr_t(Plan *p, const double *x, double xt0, double yt0, double sr, double ss,
                            const void *diff, void *out, const Coadd *co, cudaStream_t s) {
    cudaError_t err;
    const int w0 = p->cfg.w0, w1 = p->cfg.w1;
    TermWeights tw;
    basis_term_weights(p, xt0, yt0, tw.w);
    k_kernel_image<<<1, 256, 0, s>>>(p->bv, tw, x, p->kimg);
    const int tot = p->L0 * p->h1c;
    k_decorr_kappa<T><<<(tot + 255) / 256, 256, 0, s>>>(p->n1, 1, 1, w0, w1, p->kimg, nullptr,
                                                        (const cpx<T> *)p->tw1, (cpx<T> *)p->kap);
    p->launches += 2;
    CoaddDesc cd{};
    if (co) {  // row spectra of the homogenisation kernels, science then reference
        cd.ns = co->ns;
        cd.nr = co->nr;
        cd.g0 = co->g0;
        for (int c = 0; c < co->ns + co->nr; ++c) cd.s2[c] = co->sigma2[c];
        const int totc = (co->ns + co->nr) * (2 * co->g0 + 1) * p->h1c;
        k_decorr_kappa<T><<<(totc + 255) / 256, 256, 0, s>>>(p->n1, co->ns + co->nr, co->ns, co->g0, co->g1,
                                                             co->G, co->H, (const cpx<T> *)p->tw1,
                                                             (cpx<T> *)p->gam);
        p->launches++;
    }
    if ((err = cudaGetLastError())) return err;
    {  // rows
        const int G = p->m1 / 16;
        int NG = (sizeof(T) == 4 ? 1024 : 512) / G;
        if (NG < 1) NG = 1;
        if (NG > 4) NG = 4;
        if (NG > (p->n0 + 1) / 2) NG = (p->n0 + 1) / 2;
        const int ntw = p->gen1 ? 0 : pass_table_len(p->n1);
        auto smem_of = [&](int ng) { return ((size_t)ntw + (size_t)ng * padded_len(p->m1)) * sizeof(cpx<T>); };
        while (NG > 1 && smem_of(NG) > 200 * 1024) NG /= 2;
        const size_t smem = smem_of(NG);
        const int blocks = (p->n0 + 2 * NG - 1) / (2 * NG);
        const cpx<T> *twg = (const cpx<T> *)(p->gen1 ? p->twpm1 : p->twp1);
        const cpx<T> *ch = (const cpx<T> *)p->chirp1, *bf = (const cpx<T> *)p->bfilt1;
        cpx<T> *Dt = (cpx<T> *)p->U;
#define SFFT_DROWS(I, BLU)                                                                                    \
    do {                                                                                                      \
        cudaFuncSetAttribute(k_decorr_rows<T, I, BLU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k_decorr_rows<T, I, BLU><<<blocks, NG * G, smem, s>>>(p->n0, p->n1, p->m1, NG, (const I *)diff, twg, ch, \
                                                              bf, Dt);                                        \
    } while (0)
        if (p->cfg.dtype == SFFT_F64) {
            if (p->gen1) SFFT_DROWS(double, true);
            else SFFT_DROWS(double, false);
        } else {
            if (p->gen1) SFFT_DROWS(float, true);
            else SFFT_DROWS(float, false);
        }
#undef SFFT_DROWS
        p->launches++;
        if ((err = cudaGetLastError())) return err;
    }
    {  // columns
        const int G = p->m0 / 16;
        const int ntw = p->gen0 ? 0 : pass_table_len(p->n0);
        const int ncg = (cd.ns + cd.nr) * (2 * cd.g0 + 1);
        const size_t smem = ((size_t)ntw + p->L0 + ncg + padded_len(p->m0)) * sizeof(cpx<T>);
        auto kern = p->gen0 ? k_decorr_cols<T, true> : k_decorr_cols<T, false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<p->h1c, G, smem, s>>>(p->n0, p->n1, p->m0, w0, sr, ss, (const cpx<T> *)p->kap, (const cpx<T> *)p->tw0,
                                     (const cpx<T> *)(p->gen0 ? p->twpm0 : p->twp0), (const cpx<T> *)p->chirp0,
                                     (const cpx<T> *)p->bfilt0, (cpx<T> *)p->U, cd, (const cpx<T> *)p->gam);
        p->launches++;
        if ((err = cudaGetLastError())) return err;
    }
    p->launches++;
    return launch_rows_inv<T>(p, out, s);
}

cudaError_t decorrelate(Plan *p, const double *x, double xt0, double yt0, double sigma_ref, double sigma_sci,
                        const void *diff, void *out, const Coadd *co, cudaStream_t s) {
    return p->fp64 ? decorr_t<double>(p, x, xt0, yt0, sigma_ref, sigma_sci, diff, out, co, s)
                   : decorr_t<float>(p, x, xt0, yt0, sigma_ref, sigma_sci, diff, out, co, s);
}

cudaError_t subtract_from_rows(Plan *p, const double *x, void *diff, cudaStream_t s) {
    return p->fp64 ? sub_t<double>(p, x, diff, s) : sub_t<float>(p, x, diff, s);
}

}  // namespace sfft
