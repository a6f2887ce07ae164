// solve.cu -- solution of the normal equations M theta = rhs (Eq. 18).
//
// The paper names no solver.  M = C^T C is symmetric positive semidefinite;
// we take Cholesky of the Jacobi-scaled matrix A = D M D, D = diag(M)^-1/2,
// in the plan's compute type (FP32 for the mixed path, FP64 for the plain
// path), followed by iterative refinement with FP64 residuals:
//     r = rhs - M x (FP64),  solve (L L^T) z = D r,  x += D z.
// Every kernel reads the device status word first and returns at once after
// a failure or after convergence, so the whole sequence is enqueued without
// host synchronisation.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace sfft {

constexpr int kNB = 32;        // Cholesky panel width
constexpr int kMaxIters = 30;  // refinement iterations
constexpr double kTol = 1e-12; // ||r|| / ||rhs||

// flag[0]: 0 running, 1 converged, <0 failure status; flag[1]: iterations
// flag[2..3]: spare.  dvals (double) live in xw's tail: see solve_system.

__global__ void k_solve_init(int n, const double *__restrict__ M, double *__restrict__ dsc,
                             double *__restrict__ x, int *flag, double *stats) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = M[(size_t)i * n + i];
        if (!(d > 0.0)) {
            flag[0] = SFFT_ERR_SINGULAR;
            dsc[i] = 0.0;
        } else {
            dsc[i] = 1.0 / sqrt(d);
        }
        x[i] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        stats[0] = 1e300;  // min pivot
        stats[1] = 0.0;    // ||rhs||^2
        stats[2] = 0.0;    // last ||r||^2
        flag[1] = 0;
    }
}

template <typename T>
__global__ void k_scale(int n, const double *__restrict__ M, const double *__restrict__ dsc,
                        T *__restrict__ A, const int *flag) {
    if (flag[0] < 0) return;
    const size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        A[e] = (T)(M[e] * dsc[i] * dsc[j]);
    }
}

// Factor the diagonal block A[k0:k0+nb, k0:k0+nb] in shared memory.
template <typename T>
__global__ void k_potrf_diag(int n, int k0, T *__restrict__ A, int *flag, double *stats) {
    if (flag[0] < 0) return;
    __shared__ T a[kNB][kNB + 1];
    const int nb = min(kNB, n - k0);
    const int tid = threadIdx.x;
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        a[i][j] = A[(size_t)(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    __shared__ int bad;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (tid == 0) {
            T d = a[j][j];
            if (!(d > (T)0)) bad = 1;
            else {
                double dd = (double)d;
                if (dd < stats[0]) stats[0] = dd;
                a[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad) break;
        const T l = a[j][j];
        for (int i = j + 1 + tid; i < nb; i += blockDim.x) a[i][j] /= l;
        __syncthreads();
        for (int e = tid; e < (nb - j - 1) * (nb - j - 1); e += blockDim.x) {
            const int i = j + 1 + e / (nb - j - 1), c = j + 1 + e % (nb - j - 1);
            if (c <= i) a[i][c] -= a[i][j] * a[c][j];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) flag[0] = SFFT_ERR_SINGULAR;
        return;
    }
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        A[(size_t)(k0 + i) * n + k0 + j] = (j <= i) ? a[i][j] : (T)0;
    }
}

// Rows below the diagonal block: L[i, k0:k0+nb] = A[i, k0:k0+nb] * L_kk^-T
template <typename T>
__global__ void k_trsm(int n, int k0, T *__restrict__ A, const int *flag) {
    if (flag[0] < 0) return;
    __shared__ T l[kNB][kNB + 1];
    const int nb = min(kNB, n - k0);
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        l[i][j] = A[(size_t)(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    const int i = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T row[kNB];
    T *Ai = A + (size_t)i * n + k0;
#pragma unroll
    for (int c = 0; c < kNB; ++c)
        if (c < nb) row[c] = Ai[c];
#pragma unroll
    for (int c = 0; c < kNB; ++c) {
        if (c < nb) {
            T s = row[c];
#pragma unroll
            for (int p = 0; p < kNB; ++p)
                if (p < c) s -= row[p] * l[c][p];
            row[c] = s / l[c][c];
        }
    }
#pragma unroll
    for (int c = 0; c < kNB; ++c)
        if (c < nb) Ai[c] = row[c];
}

// Trailing update of the lower triangle: A[i][j] -= sum_p L[i][k0+p] L[j][k0+p],
// i >= j >= k0+nb, in 64x64 tiles (256 threads, 4x4 per thread).
template <typename T>
__global__ void k_syrk(int n, int k0, T *__restrict__ A, const int *flag) {
    if (flag[0] < 0) return;
    const int nb = min(kNB, n - k0);
    const int base = k0 + nb;
    // map blockIdx.x to a lower tile (ti >= tj)
    int t = blockIdx.x, ti = 0;
    while (t > ti) {
        t -= ti + 1;
        ++ti;
    }
    const int tj = t;
    const int i0 = base + ti * 64, j0 = base + tj * 64;
    __shared__ T Li[64][kNB + 1], Lj[64][kNB + 1];
    for (int e = threadIdx.x; e < 64 * kNB; e += blockDim.x) {
        const int r = e / kNB, p = e % kNB;
        Li[r][p] = (i0 + r < n && p < nb) ? A[(size_t)(i0 + r) * n + k0 + p] : (T)0;
        Lj[r][p] = (j0 + r < n && p < nb) ? A[(size_t)(j0 + r) * n + k0 + p] : (T)0;
    }
    __syncthreads();
    const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
#pragma unroll 8
    for (int p = 0; p < kNB; ++p) {
        T x[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) x[a] = Li[tr * 4 + a][p];
#pragma unroll
        for (int b = 0; b < 4; ++b) y[b] = Lj[tc + 16 * b][p];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += x[a] * y[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + tr * 4 + a;
        if (i >= n) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + tc + 16 * b;
            if (j < n && j <= i) A[(size_t)i * n + j] -= acc[a][b];
        }
    }
}

// r = rhs - M x in FP64; per-block partial sums of ||r||^2 (and ||rhs||^2).
__global__ void k_residual(int n, const double *__restrict__ M, const double *__restrict__ rhs,
                           const double *__restrict__ x, double *__restrict__ r, double *__restrict__ part,
                           const int *flag) {
    if (flag[0] != 0) return;
    __shared__ double red[2][32];
    double s_r = 0.0, s_b = 0.0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = blockIdx.x * nw + warp; i < n; i += gridDim.x * nw) {
        const double *Mi = M + (size_t)i * n;
        double acc = 0.0;
        for (int j = lane; j < n; j += 32) acc += Mi[j] * x[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const double ri = rhs[i] - acc;
        if (lane == 0) {
            r[i] = ri;
            s_r += ri * ri;
            s_b += rhs[i] * rhs[i];
        }
    }
    if (lane == 0) {
        red[0][warp] = s_r;
        red[1][warp] = s_b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < nw; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// Single block: convergence test, then (L L^T) z = D r and x += D z.
template <typename T>
__global__ void k_refine(int n, const T *__restrict__ L, const double *__restrict__ dsc,
                         const double *__restrict__ r, double *__restrict__ x, T *__restrict__ z,
                         const double *__restrict__ part, int nparts, int *flag, double *stats,
                         int last) {
    if (flag[0] != 0) return;
    __shared__ double s_rr, s_bb;
    __shared__ T zb[kNB];
    const int tid = threadIdx.x, nthr = blockDim.x;
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < nparts; ++k) {
            a += part[2 * k];
            b += part[2 * k + 1];
        }
        s_rr = a;
        s_bb = b;
        stats[1] = b;
        stats[2] = a;
    }
    __syncthreads();
    const double rel = (s_bb > 0.0) ? sqrt(s_rr / s_bb) : sqrt(s_rr);
    if (rel <= kTol || s_rr == 0.0) {
        if (tid == 0) flag[0] = 1;
        return;
    }
    if (last) {
        if (tid == 0) flag[0] = SFFT_ERR_NOT_CONVERGED;
        return;
    }
    for (int i = tid; i < n; i += nthr) z[i] = (T)(dsc[i] * r[i]);
    __syncthreads();
    // forward: L y = z
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int nb = min(kNB, n - k0);
        if (tid < 32) {
            T v = (tid < nb) ? z[k0 + tid] : (T)0;
            for (int c = 0; c < nb; ++c) {
                // lane c holds the fully updated right-hand side of row k0+c
                const T zc = __shfl_sync(0xffffffffu, v, c) / L[(size_t)(k0 + c) * n + k0 + c];
                if (tid == c) v = zc;
                if (tid > c && tid < nb) v -= L[(size_t)(k0 + tid) * n + k0 + c] * zc;
            }
            if (tid < nb) {
                z[k0 + tid] = v;
                zb[tid] = v;
            }
        }
        __syncthreads();
        for (int i = k0 + nb + tid; i < n; i += nthr) {
            const T *Li = L + (size_t)i * n + k0;
            T s = (T)0;
            for (int c = 0; c < nb; ++c) s += Li[c] * zb[c];
            z[i] -= s;
        }
        __syncthreads();
    }
    // backward: L^T w = y
    for (int kend = n; kend > 0; kend -= kNB) {
        const int k0 = max(0, kend - kNB), nb = kend - k0;
        if (tid < 32) {
            T v = (tid < nb) ? z[k0 + tid] : (T)0;
            for (int c = nb - 1; c >= 0; --c) {
                T wc = __shfl_sync(0xffffffffu, v, c) / L[(size_t)(k0 + c) * n + k0 + c];
                if (tid == c) v = wc;
                if (tid < c) v -= L[(size_t)(k0 + c) * n + k0 + tid] * wc;
            }
            if (tid < nb) {
                z[k0 + tid] = v;
                zb[tid] = v;
            }
        }
        __syncthreads();
        for (int i = tid; i < k0; i += nthr) {
            T s = (T)0;
            for (int c = 0; c < nb; ++c) s += L[(size_t)(k0 + c) * n + i] * zb[c];
            z[i] -= s;
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += nthr) x[i] += dsc[i] * (double)z[i];
    if (tid == 0) flag[1] += 1;
}

__global__ void k_solve_finish(int n, const double *x, double *xout, const int *flag, const double *stats,
                               sfft_solve_info *info) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) xout[i] = x[i];
    if (info && blockIdx.x == 0 && threadIdx.x == 0) {
        const int f = flag[0];
        info->status = (f == 1) ? SFFT_OK : (f == 0 ? SFFT_ERR_NOT_CONVERGED : f);
        info->iters = flag[1];
        info->rel_residual = (stats[1] > 0.0) ? sqrt(stats[2] / stats[1]) : sqrt(stats[2]);
        info->min_pivot = stats[0];
    }
}

template <typename T>
static cudaError_t solve_t(Plan *p, const double *M, const double *rhs, double *x, sfft_solve_info *info,
                           cudaStream_t s) {
    const int n = p->n;
    T *A = (T *)p->A;
    double *stats = p->xw + n;        // [0] min pivot, [1] ||rhs||^2, [2] ||r||^2
    double *part = p->xw + n + 8;     // residual partials
    const int rblocks = 128;
    cudaMemsetAsync(p->flag, 0, 4 * sizeof(int), s);
    k_solve_init<<<(n + 255) / 256, 256, 0, s>>>(n, M, p->dscale, p->xw, p->flag, stats);
    int sb = (int)(((size_t)n * n + 255) / 256);
    if (sb > 4096) sb = 4096;
    k_scale<T><<<sb, 256, 0, s>>>(n, M, p->dscale, A, p->flag);
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int nb = min(kNB, n - k0);
        k_potrf_diag<T><<<1, 256, 0, s>>>(n, k0, A, p->flag, stats);
        const int rows = n - k0 - nb;
        if (rows > 0) {
            k_trsm<T><<<(rows + 127) / 128, 128, 0, s>>>(n, k0, A, p->flag);
            const int tiles = (rows + 63) / 64;
            k_syrk<T><<<tiles * (tiles + 1) / 2, 256, 0, s>>>(n, k0, A, p->flag);
        }
    }
    for (int it = 0; it <= kMaxIters; ++it) {
        k_residual<<<rblocks, 256, 0, s>>>(n, M, rhs, p->xw, p->r, part, p->flag);
        k_refine<T><<<1, 1024, 0, s>>>(n, A, p->dscale, p->r, p->xw, (T *)p->zv, part, rblocks, p->flag,
                                       stats, it == kMaxIters);
    }
    k_solve_finish<<<(n + 255) / 256, 256, 0, s>>>(n, p->xw, x, p->flag, stats, info);
    return cudaGetLastError();
}

cudaError_t solve_system(Plan *p, const double *M, const double *rhs, double *x, sfft_solve_info *info,
                         cudaStream_t s) {
    return p->fp64 ? solve_t<double>(p, M, rhs, x, info, s) : solve_t<float>(p, M, rhs, x, info, s);
}

}  // namespace sfft
