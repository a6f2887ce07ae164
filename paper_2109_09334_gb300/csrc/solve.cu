// solve.cu -- solution of the normal equations M theta = rhs (Eq. 18).
//
// The paper names no solver.  M = C^T C is symmetric positive semidefinite;
// we factor the Jacobi-scaled matrix A = D M D (D = diag(M)^-1/2) by Cholesky
// in the plan's compute type (FP32 for the mixed path, FP64 for the plain
// path), form W = L^-1 explicitly, and refine with FP64 residuals:
//     r = rhs - M x (FP64),  x += D W^T W D r,
// until ||r|| / ||rhs|| <= 1e-12.
//
// Everything runs in one cooperative (grid-synchronised) kernel with one
// block per SM, so the ~n/32 dependent block steps cost a grid barrier each
// instead of a kernel launch:
//   * Cholesky, right-looking with 32-wide panels: phase P solves for the
//     panel L_ik = A_ik L_kk^-T, one thread per row; phase U applies
//     A_ij -= L_ik L_jk^T to the trailing lower triangle in 64x64 tiles.  The
//     block that updates the tile holding the next diagonal block factors it
//     right away (one warp, registers and shuffles).
//   * W = L^-1 is formed in the same sweep (forward elimination applied to
//     the identity): phase P also sets W_k = L_kk^-1 W_k for block row k (one
//     thread per column) and phase U applies W_i -= L_ik W_k below.
//   * refinement: residual GEMV in FP64 and two GEMVs with W.
// Every control decision after a barrier uses values written before it, so
// all blocks execute the same sequence of barriers.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace sfft {

constexpr int kNB = 32;         // Cholesky panel width / diagonal block size
constexpr int kTile = 64;       // trailing-update and GEMM output tile
constexpr int kMaxIters = 12;   // refinement iterations
constexpr double kTol = 1e-12;  // ||r|| / ||rhs||
constexpr int kThreads = 256;
constexpr int kSeg = 8;         // row segments of the W^T y product

template <typename T>
struct SolveArgs {
    int n, nblk;
    const double *M, *rhs;
    double *dsc, *x, *r, *part, *stats;  // part: 2 * gridDim doubles; stats[0..3]
    T *A, *W, *z, *y, *wseg;
    int *flag;  // [0] status (0 running, 1 converged, <0 failure), [1] iterations
    double *xout;
    sfft_solve_info *info;
};

template <typename T>
struct TileSmem {
    T a[kTile][kNB + 1];
    T b[kNB][kTile + 1];
};

// 64x64 tile:  acc(i, j) += sum_{k0 <= k < k1} a(i, k) b(k, j)
//   a(i, k) = Ag[(arow0 + i) * lda + k]
//   b(k, j) = transB ? Bg[(bcol0 + j) * ldb + k] : Bg[k * ldb + bcol0 + j]
// rows i >= arows and columns j >= bcols read as zero.
template <typename T>
__device__ void tile_gemm(T (&acc)[4][4], TileSmem<T> &sm, const T *Ag, int lda, int arow0, int arows,
                          const T *Bg, int ldb, int bcol0, int bcols, bool transB, int k0, int k1) {
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;
    for (int kk = k0; kk < k1; kk += kNB) {
        const int kn = min(kNB, k1 - kk);
        for (int e = tid; e < kTile * kNB; e += kThreads) {
            const int i = e / kNB, p = e % kNB;
            sm.a[i][p] = (i < arows && p < kn) ? Ag[(size_t)(arow0 + i) * lda + kk + p] : (T)0;
        }
        if (transB) {
            for (int e = tid; e < kTile * kNB; e += kThreads) {
                const int j = e / kNB, p = e % kNB;
                sm.b[p][j] = (j < bcols && p < kn) ? Bg[(size_t)(bcol0 + j) * ldb + kk + p] : (T)0;
            }
        } else {
            for (int e = tid; e < kTile * kNB; e += kThreads) {
                const int p = e / kTile, j = e % kTile;
                sm.b[p][j] = (j < bcols && p < kn) ? Bg[(size_t)(kk + p) * ldb + bcol0 + j] : (T)0;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int p = 0; p < kNB; ++p) {
            T av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = sm.a[tr * 4 + u][p];
#pragma unroll
            for (int v = 0; v < 4; ++v) bv[v] = sm.b[p][tc + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
        }
        __syncthreads();
    }
}

// One warp factors the 32x32 diagonal block kb (already fully updated) in
// registers: lane t holds row t; column steps broadcast by shuffles.  Writes
// L_kk into A (zeros above the diagonal) and flags a non-positive pivot.
template <typename T>
__device__ __noinline__ void factor_diag(const SolveArgs<T> &s, int kb) {
    const int t = threadIdx.x & 31;
    const int n = s.n, k0 = kb * kNB;
    const int nb = min(kNB, n - k0);
    T a[kNB];
#pragma unroll
    for (int c = 0; c < kNB; ++c) {
        T v = (T)0;
        if (t < nb && c < nb) v = s.A[(size_t)(k0 + t) * n + k0 + c];
        if (t >= nb && c == t) v = (T)1;  // identity beyond the matrix edge
        a[c] = v;
    }
    bool bad = false;
    T minpiv = (T)1e30;
#pragma unroll
    for (int j = 0; j < kNB; ++j) {
        const T d = __shfl_sync(0xffffffffu, a[j], j);
        if (!(d > (T)0)) bad = true;
        const T l = sqrt(d > (T)0 ? d : (T)1);
        if (j < nb && d < minpiv) minpiv = d;
        if (t == j) a[j] = l;
        if (t > j) a[j] = a[j] / l;
#pragma unroll
        for (int c = j + 1; c < kNB; ++c) {
            const T lcj = __shfl_sync(0xffffffffu, a[j], c);
            if (t >= c) a[c] -= a[j] * lcj;
        }
    }
    if (bad) {
        if (t == 0) s.flag[0] = SFFT_ERR_SINGULAR;
        return;
    }
    if (t == 0 && (double)minpiv < s.stats[0]) s.stats[0] = (double)minpiv;
    if (t < nb) {
#pragma unroll
        for (int c = 0; c < kNB; ++c)
            if (c < nb) s.A[(size_t)(k0 + t) * n + k0 + c] = (c <= t) ? a[c] : (T)0;
    }
}

// Forward substitution L_kk y = b for one right-hand side held in registers
// (L_kk in shared memory, lower triangular, padded rows).
template <typename T>
__device__ __forceinline__ void trsv_lower(T (&b)[kNB], const T (*L)[kNB + 1]) {
#pragma unroll
    for (int c = 0; c < kNB; ++c) {
        T v = b[c];
#pragma unroll
        for (int p = 0; p < c; ++p) v -= L[c][p] * b[p];
        b[c] = v / L[c][c];
    }
}

// Panel row i: L[i, k0:k0+kn] = solution of L_kk x = A[i, k0:k0+kn]^T
template <typename T>
__device__ __noinline__ void panel_row(T *Ai, int kn, const T (*L)[kNB + 1]) {
    T b[kNB];
#pragma unroll
    for (int c = 0; c < kNB; ++c) b[c] = (c < kn) ? Ai[c] : (T)0;
    trsv_lower(b, L);
#pragma unroll
    for (int c = 0; c < kNB; ++c)
        if (c < kn) Ai[c] = b[c];
}

// Column c of W's block row k: W[k0:k0+kn, c] = L_kk^-1 W[k0:k0+kn, c] for
// c < k0, or column c - k0 of L_kk^-1 for c >= k0.
template <typename T>
__device__ __noinline__ void wcol(T *W, int n, int k0, int kn, int c, const T (*L)[kNB + 1]) {
    T b[kNB];
#pragma unroll
    for (int r = 0; r < kNB; ++r) {
        T v;
        if (c < k0) v = (r < kn) ? W[(size_t)(k0 + r) * n + c] : (T)0;
        else v = (r == c - k0) ? (T)1 : (T)0;
        b[r] = v;
    }
    trsv_lower(b, L);
#pragma unroll
    for (int r = 0; r < kNB; ++r)
        if (r < kn) W[(size_t)(k0 + r) * n + c] = b[r];
}

// trailing-update tile tt -> (ti, tj), ti >= tj
__device__ __forceinline__ void lower_tile(int tt, int *ti, int *tj) {
    int t = tt, i = 0;
    while (t > i) {
        t -= i + 1;
        ++i;
    }
    *ti = i;
    *tj = t;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_solve_coop(SolveArgs<T> s) {
    cg::grid_group grid = cg::this_grid();
    __shared__ TileSmem<T> sm;
    __shared__ T Ls[kNB][kNB + 1];
    __shared__ double red[2][kThreads / 32];
    const int tid = threadIdx.x, bid = blockIdx.x, nbk = gridDim.x;
    const int gtid = bid * kThreads + tid, gthreads = nbk * kThreads;
    const int n = s.n, nblk = s.nblk;
    const int tr = tid / 16, tc = tid % 16;
    const int warp = tid >> 5, lane = tid & 31, nw = kThreads / 32;

    // ---- Jacobi scaling, zero W and x --------------------------------------
    for (int i = gtid; i < n; i += gthreads) {
        const double d = s.M[(size_t)i * n + i];
        if (!(d > 0.0)) s.flag[0] = SFFT_ERR_SINGULAR;
        s.dsc[i] = (d > 0.0) ? 1.0 / sqrt(d) : 0.0;
        s.x[i] = 0.0;
    }
    for (size_t e = gtid; e < (size_t)n * n; e += gthreads) s.W[e] = (T)0;
    grid.sync();
    for (int i = bid; i < n; i += nbk) {
        const double di = s.dsc[i];
        const double *Mi = s.M + (size_t)i * n;
        T *Ai = s.A + (size_t)i * n;
        for (int j = tid; j < n; j += kThreads) Ai[j] = (T)(Mi[j] * di * s.dsc[j]);
    }
    grid.sync();

    // ---- Cholesky and W = L^-1 ----------------------------------------------
    if (s.flag[0] == 0 && bid == 0 && warp == 0) factor_diag(s, 0);
    grid.sync();
    for (int kb = 0; kb < nblk; ++kb) {
        if (s.flag[0] < 0) break;  // written before the last barrier: same value everywhere
        const int k0 = kb * kNB;
        const int kn = min(kNB, n - k0);
        const int base = k0 + kNB;  // first trailing row
        const int rows = n - base;  // may be <= 0 on the last block
        // phase P: L_kk to shared memory; then, one thread per right-hand side,
        // the panel rows L[i, k0:k0+32] = A[i, k0:k0+32] L_kk^-T (i >= k0+32)
        // and the block row k of W: W_k[:, c] = L_kk^-1 W_k[:, c] for c < k0,
        // W_kk = L_kk^-1 (identity right-hand sides)
        {
            for (int e = tid; e < kNB * kNB; e += kThreads) {
                const int i = e / kNB, c = e % kNB;
                Ls[i][c] = (i < kn && c < kn) ? s.A[(size_t)(k0 + i) * n + k0 + c] : (i == c ? (T)1 : (T)0);
            }
            __syncthreads();
            const int nrow = rows > 0 ? rows : 0;
            const int ncol = k0 + kn;
            for (int task = gtid; task < nrow + ncol; task += gthreads) {
                if (task < nrow) panel_row(s.A + (size_t)(base + task) * n + k0, kn, Ls);
                else wcol(s.W, n, k0, kn, task - nrow, Ls);
            }
        }
        grid.sync();
        if (rows <= 0) break;  // last block: nothing below (same in every block)
        // phase U: the trailing lower triangle of A in 64x64 tiles, and the
        // block rows of W below: W_i[:, 0:k0+32] -= L_ik W_k.  Block 0 takes
        // tile 0 (it holds the next diagonal block) and factors that block at
        // once; all other tasks go to the other blocks.
        {
            const int nt = (rows + kTile - 1) / kTile;
            const int ntiles = nt * (nt + 1) / 2;
            const int ncw = (k0 + kNB + kTile - 1) / kTile;
            const int ntask = ntiles + nt * ncw;
            const int first = (nbk == 1) ? 0 : (bid == 0 ? 0 : bid);
            const int step = (nbk == 1) ? 1 : (bid == 0 ? ntask : nbk - 1);
            for (int task = first; task < ntask; task += step) {
                T acc[4][4] = {};
                if (task < ntiles) {
                    int ti, tj;
                    lower_tile(task, &ti, &tj);
                    const int i0 = base + ti * kTile, j0 = base + tj * kTile;
                    const int ni = min(kTile, n - i0), nj = min(kTile, n - j0);
                    tile_gemm(acc, sm, s.A + k0, n, i0, ni, s.A + k0, n, j0, nj, true, 0, kNB);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int i = i0 + tr * 4 + u, j = j0 + tc + 16 * v;
                            if (i < n && j < n && j <= i) s.A[(size_t)i * n + j] -= acc[u][v];
                        }
                    if (task == 0) {
                        __syncthreads();  // the tile's writes are visible to the block
                        if (warp == 0) factor_diag(s, kb + 1);
                        __syncthreads();
                    }
                } else {
                    const int q = task - ntiles, ti = q / ncw, tj = q % ncw;
                    const int i0 = base + ti * kTile, j0 = tj * kTile;
                    const int ni = min(kTile, n - i0), nj = min(kTile, k0 + kNB - j0);
                    // a(i, p) = L[i0 + i][k0 + p], b(p, j) = W[k0 + p][j0 + j]
                    tile_gemm(acc, sm, s.A + k0, n, i0, ni, s.W + (size_t)k0 * n, n, j0, nj, false, 0, kNB);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int i = i0 + tr * 4 + u, j = j0 + tc + 16 * v;
                            if (i < n && j < k0 + kNB) s.W[(size_t)i * n + j] -= acc[u][v];
                        }
                }
            }
        }
        grid.sync();
    }

    // ---- refinement ---------------------------------------------------------
    for (int it = 0; it <= kMaxIters; ++it) {
        if (s.flag[0] != 0) break;  // same value in every block
        // r = rhs - M x (FP64); z = D r; per-block partial norms
        double pr = 0.0, pb = 0.0;
        for (int i = bid * nw + warp; i < n; i += nbk * nw) {
            const double *Mi = s.M + (size_t)i * n;
            double a = 0.0;
            for (int j = lane; j < n; j += 32) a += Mi[j] * s.x[j];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            const double ri = s.rhs[i] - a;
            if (lane == 0) {
                s.r[i] = ri;
                s.z[i] = (T)(s.dsc[i] * ri);
                pr += ri * ri;
                pb += s.rhs[i] * s.rhs[i];
            }
        }
        if (lane == 0) {
            red[0][warp] = pr;
            red[1][warp] = pb;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < nw; ++w) {
                a += red[0][w];
                b += red[1][w];
            }
            s.part[2 * bid] = a;
            s.part[2 * bid + 1] = b;
        }
        grid.sync();
        // every block sums the partials in the same order: the same decision everywhere
        double rr = 0.0, bb = 0.0;
        for (int k = 0; k < nbk; ++k) {
            rr += s.part[2 * k];
            bb += s.part[2 * k + 1];
        }
        const double rel = (bb > 0.0) ? sqrt(rr / bb) : sqrt(rr);
        if (bid == 0 && tid == 0) {
            s.stats[1] = bb;
            s.stats[2] = rr;
        }
        if (rel <= kTol || rr == 0.0) {
            if (bid == 0 && tid == 0) s.flag[0] = 1;
            break;
        }
        if (it == kMaxIters) {
            if (bid == 0 && tid == 0) s.flag[0] = SFFT_ERR_NOT_CONVERGED;
            break;
        }
        // y = W z  (W lower triangular)
        for (int i = bid * nw + warp; i < n; i += nbk * nw) {
            const T *Wi = s.W + (size_t)i * n;
            T a = (T)0;
            for (int j = lane; j <= i; j += 32) a += Wi[j] * s.z[j];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) s.y[i] = a;
        }
        grid.sync();
        // w = W^T y in kSeg row segments (coalesced rows of W), summed in a fixed order
        {
            const int segrows = (n + kSeg - 1) / kSeg;
            const int nchunk = (n + 31) / 32;
            for (int task = bid * nw + warp; task < nchunk * kSeg; task += nbk * nw) {
                const int ch = task / kSeg, sg = task % kSeg;
                const int i = ch * 32 + lane;
                const int k0 = max(ch * 32, sg * segrows), k1 = min(n, (sg + 1) * segrows);
                T a = (T)0;
                if (i < n)
                    for (int k = k0; k < k1; ++k) a += s.W[(size_t)k * n + i] * s.y[k];
                if (i < n) s.wseg[(size_t)sg * n + i] = a;
            }
        }
        grid.sync();
        for (int i = gtid; i < n; i += gthreads) {
            T a = (T)0;
#pragma unroll
            for (int sg = 0; sg < kSeg; ++sg) a += s.wseg[(size_t)sg * n + i];
            s.x[i] += s.dsc[i] * (double)a;
        }
        if (bid == 0 && tid == 0) s.flag[1] += 1;
        grid.sync();
    }
    // ---- results ------------------------------------------------------------
    for (int i = gtid; i < n; i += gthreads) s.xout[i] = s.x[i];
    if (s.info && bid == 0 && tid == 0) {
        const int f = s.flag[0];
        s.info->status = (f == 1) ? SFFT_OK : (f == 0 ? SFFT_ERR_NOT_CONVERGED : f);
        s.info->iters = s.flag[1];
        s.info->rel_residual = (s.stats[1] > 0.0) ? sqrt(s.stats[2] / s.stats[1]) : sqrt(s.stats[2]);
        s.info->min_pivot = s.stats[0];
    }
}

__global__ void k_solve_reset(int *flag, double *stats) {
    flag[0] = flag[1] = flag[2] = flag[3] = 0;
    stats[0] = 1e300;
    stats[1] = stats[2] = stats[3] = 0.0;
}

static size_t solve_dyn_smem(bool fp64);

template <typename T>
static cudaError_t solve_t(Plan *p, const double *M, const double *rhs, double *x, sfft_solve_info *info,
                           cudaStream_t st) {
    SolveArgs<T> a;
    a.n = p->n;
    a.nblk = (p->n + kNB - 1) / kNB;
    a.M = M;
    a.rhs = rhs;
    a.dsc = p->dscale;
    a.x = p->xw;
    a.r = p->r;
    a.stats = p->xw + p->n;
    a.part = p->xw + p->n + 8;
    a.A = (T *)p->A;
    a.W = (T *)p->Wm;
    a.z = (T *)p->zv;
    a.y = (T *)p->zv + p->n;
    a.wseg = (T *)p->zv + 2 * (size_t)p->n;
    a.flag = p->flag;
    a.xout = x;
    a.info = info;
    k_solve_reset<<<1, 1, 0, st>>>(p->flag, a.stats);
    cudaError_t err = cudaGetLastError();
    if (err) return err;
    void *args[] = {&a};
    const size_t dsm = solve_dyn_smem(p->fp64);
    err = cudaLaunchCooperativeKernel(p->fp64 ? (void *)k_solve_coop<double> : (void *)k_solve_coop<float>,
                                      p->solve_grid, kThreads, args, dsm, st);
    p->launches += 2;
    return err;
}

static size_t solve_dyn_smem(bool) { return 0; }

int solve_grid_size(bool fp64) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t dsm = solve_dyn_smem(fp64);
    if (fp64) {
        cudaFuncSetAttribute(k_solve_coop<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_coop<double>, kThreads, dsm);
    } else {
        cudaFuncSetAttribute(k_solve_coop<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_coop<float>, kThreads, dsm);
    }
    if (per < 1 || sms < 1) return 0;
    return sms;  // one block per SM; partial sums sized for at most 256 blocks
}

size_t solve_vec_elems(int n) { return (size_t)(2 + kSeg) * n; }

cudaError_t solve_system(Plan *p, const double *M, const double *rhs, double *x, sfft_solve_info *info,
                         cudaStream_t s) {
    return p->fp64 ? solve_t<double>(p, M, rhs, x, info, s) : solve_t<float>(p, M, rhs, x, info, s);
}

template <typename T>
static cudaError_t solve_buf_t(const SolveBuffers &b, const double *M, const double *rhs, double *x,
                               sfft_solve_info *info, cudaStream_t st) {
    SolveArgs<T> a;
    a.n = b.n;
    a.nblk = (b.n + kNB - 1) / kNB;
    a.M = M;
    a.rhs = rhs;
    a.dsc = b.dsc;
    a.x = b.xw;
    a.r = b.r;
    a.stats = b.xw + b.n;
    a.part = b.xw + b.n + 8;
    a.A = (T *)b.A;
    a.W = (T *)b.W;
    a.z = (T *)b.zv;
    a.y = (T *)b.zv + b.n;
    a.wseg = (T *)b.zv + 2 * (size_t)b.n;
    a.flag = b.flag;
    a.xout = x;
    a.info = info;
    k_solve_reset<<<1, 1, 0, st>>>(b.flag, a.stats);
    cudaError_t err = cudaGetLastError();
    if (err) return err;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((void *)k_solve_coop<T>, b.grid, kThreads, args, solve_dyn_smem(b.fp64), st);
}

cudaError_t solve_on_buffers(const SolveBuffers &b, const double *M, const double *rhs, double *x,
                             sfft_solve_info *info, cudaStream_t s) {
    return b.fp64 ? solve_buf_t<double>(b, M, rhs, x, info, s) : solve_buf_t<float>(b, M, rhs, x, info, s);
}

}  // namespace sfft
