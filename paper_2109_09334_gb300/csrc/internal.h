// internal.h -- plan layout and kernel launchers shared by the SFFT sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sfft.h"

namespace sfft {

// Inner length of the split pruned inverse DFT along x (frequency l = lb + NB*r,
// r in [0, NA)): min(64, n0).
constexpr int kMaxNA = 64;

// Cooperative solve grid: at most kMaxSolveGrid blocks.  The plan's vector
// xw holds x (n), then the solve's statistics (8) and per-block partial sums
// (2 per block), then the subtraction's kernel sums.
constexpr int kMaxSolveGrid = 512;
constexpr int kSolveTail = 8 + 2 * kMaxSolveGrid;
// Systems solved together by one launch of the batched solve.
constexpr int kMaxSolveBatch = 8;

enum PairKind { PK_OMEGA = 0, PK_LAMBDA = 1, PK_THETA = 2 };

// One spectrum product transformed in the gather: conj(U_a) * V_b where V_b
// is an image spectrum (Omega: b = R-term, Theta: b = S) or the 1-D spectrum
// of x^p (Lambda).  h0 = lag half-range along x.
struct PairDesc {
    int kind, a, b, h0;
    int row0;  // first row of this pair in the stage-1 table Q[row][m]
};

struct Plan {
    sfft_config cfg;
    int n0, n1, h1c;       // h1c = n1/2 + 1 half-spectrum columns
    int nk, nb, n;         // kernel terms, background terms, unknowns
    int L0, L1;            // 2w+1
    int na, nbk;           // split: n0 = na * nbk
    int nimg;              // R-terms + S
    int npairs, nrows;     // gather pairs; stage-1 rows (sum of 2*h0+1)
    int nmom;              // per-row moment values
    bool fp64;             // compute in double
    size_t csz;            // sizeof(cpx<compute type>)

    // device workspace
    void *tw0, *tw1;       // twiddle tables exp(-2 pi i q / n), length n0 and n1 (compute type)
    void *twp0, *twp1;     // the same twiddles in pass order for the FFTs (fft16.cuh)
    // Sizes that are not powers of two.  gen1: the row transforms are
    // Bluestein DFTs of length n1 through FFTs of length m1; gen0: the lag
    // sums along x are direct circular correlations (k_xcorr), no column FFT.
    int gen0, gen1, m0, m1;
    void *chirp1, *bfilt1, *twpm1;  // Bluestein tables for n1 (compute type)
    void *chirp0, *bfilt0, *twpm0;  // Bluestein tables for n0 (noise decorrelation only)
    double *kimg;                   // L0 x L1 kernel image (noise decorrelation)
    // launch shapes chosen by sfft_plan_autotune (0: the built-in choice)
    int tune_tr, tune_gi, tune_ng, tune_sgrid;
    void *xhat;            // [p][lb][r] 1-D spectra of x^p, permuted (compute type), p <= db
    void *yhat;            // [q][m] 1-D spectra of y^q, m < h1c (compute type)
    void *F;               // [(dk+2)][m][x] row transforms (compute type)
    void *U;               // [nimg][m][lb][r] full spectra, permuted (compute type); reused for Dt
    void *Q;               // [nrows][m] stage-1 results (compute type complex)
    PairDesc *pairs;       // device copy
    double *rowmom;        // [n0][nmom] per-row moment sums
    double *mom;           // moments table (see build.cu)
    double *lag;           // lag tables (Omega, Lambda, Theta), FP64
    int lag_om, lag_la, lag_th;  // offsets into lag
    // solve workspace
    void *A;               // n*n factor (compute type)
    void *Wm;              // n*n: W = L^-1 (compute type)
    int solve_grid;        // blocks of the cooperative solve kernel (one per SM)
    double *dscale;        // n Jacobi scales
    double *r, *xw;        // n residual, n iterate
    void *zv;              // n vector (compute type)
    int *flag;             // device status word for the solve
    // owned buffers for run_pair(_host)
    double *M_own, *rhs_own, *x_own;
    sfft_solve_info *info_own;
    void *img_ref, *img_sci, *img_diff;
    uint8_t *img_mask;
    void *kap;             // [nk][L0][m] kernel row spectra (compute type)
    size_t ws_bytes;
    uint64_t launches;     // kernels this plan has enqueued
    // buffers of the most recent run_pair (for sfft_replay_stage)
    const void *last_ref, *last_sci;
    const uint8_t *last_mask;
    double *last_M, *last_rhs, *last_x;
    sfft_solve_info *last_info;
    void *last_diff;
    cudaStream_t last_stream;
    PairDesc host_pairs[256];
};

// plans (api.cu): validation, allocation + tables, release
int plan_validate(const sfft_config *c);
int plan_new(const sfft_config *cfg, cudaStream_t s, Plan **out);  // cfg already validated
void plan_free(Plan *p);
int status_of(cudaError_t e);

// launchers (return cudaError_t of the last launch)
cudaError_t build_system(Plan *p, const void *ref, const void *sci, const uint8_t *mask, double *M,
                         double *rhs, cudaStream_t s);
cudaError_t row_transform(Plan *p, const void *ref, const void *sci, const uint8_t *mask,
                          bool moments, cudaStream_t s);
cudaError_t build_stage(Plan *p, int stage, double *M, double *rhs, cudaStream_t s);
cudaError_t solve_system(Plan *p, const double *M, const double *rhs, double *x,
                         sfft_solve_info *info, cudaStream_t s);
// Solve the systems of `count` (1..8) plans of the same size together in
// one cooperative launch (on the grid of plans[0]).
cudaError_t solve_batch(Plan *const *plans, int count, const double *const *M, const double *const *rhs,
                        double *const *x, sfft_solve_info *const *info, cudaStream_t s);
int solve_grid_size(bool fp64);
size_t solve_vec_elems(int n);
// Solve workspace given by the caller instead of a plan (sizes for n
// unknowns in the compute type: A, W n*n; zv solve_vec_elems(n); dsc, r n
// doubles; xw n + 8 + 2*grid doubles; flag 4 ints).
struct SolveBuffers {
    int n, grid;
    bool fp64;
    void *A, *W, *zv;
    double *dsc, *r, *xw;
    int *flag;
};
cudaError_t solve_on_buffers(const SolveBuffers &b, const double *M, const double *rhs, double *x,
                             sfft_solve_info *info, cudaStream_t s);
cudaError_t decorrelate(Plan *p, const double *x, double xt0, double yt0, double sigma_ref, double sigma_sci,
                        const void *diff, void *out, cudaStream_t s);
cudaError_t subtract_from_rows(Plan *p, const double *x, void *diff, cudaStream_t s);
cudaError_t plan_tables(Plan *p, cudaStream_t s);

}  // namespace sfft
