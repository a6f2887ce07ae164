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

enum PairKind { PK_OMEGA = 0, PK_LAMBDA = 1, PK_THETA = 2, PK_OMEGA2 = 3 };

// One spectrum product transformed in the gather: conj(U_a) * V_b where V_b
// is an image spectrum (Omega: b = R-term, Theta: b = S) or the 1-D spectrum
// of x^p (Lambda).  h0 = lag half-range along x.
// PK_OMEGA2 (gather only): the two auto-products Omega_aa and Omega_bb,
// whose spectrum products |U_a|^2, |U_b|^2 are real, transformed together as
// the one complex sequence |U_a|^2 + i |U_b|^2; rows row0 (a) and row1 (b).
struct PairDesc {
    int kind, a, b, h0;
    int row0;  // first row of this pair in the stage-1 table Q[row][m]
    int row1;  // PK_OMEGA2: first row of the second auto-product
};

// Spatial-variation basis (Eq. 2 and 6, or Eq. 7-9).  Kernel term t weights
// R by fx_i(x) fy_j(y) with i = ti[t], j = tj[t]; background term s is
// bx_p(x) by_q(y) with p = sp[s], q = sq[s].  Polynomial: fx_i = xt^i etc.,
// computed in the kernels; B-spline: tabulated functions (ftab).  The int
// tables live in one array; BasisView holds their offsets.
struct BasisView {
    const int *d;  // int tables (device)
    int nk, nb, nfx, nfy, nbx, nby;
    int o_ti, o_tj, o_fl, o_uoff, o_sp, o_sq, o_lamn, o_lams, o_lamq, o_jcnt, o_jterm, total;
    int w0, w1;
    __host__ __device__ int ti(int t) const { return d[o_ti + t]; }
    __host__ __device__ int tj(int t) const { return d[o_tj + t]; }
    // bit 0: the term has the (0,0) offset; bit 1: it has the other offsets
    __host__ __device__ int flags(int t) const { return d[o_fl + t]; }
    __host__ __device__ int sp(int s) const { return d[o_sp + s]; }
    __host__ __device__ int sq(int s) const { return d[o_sq + s]; }
    // background terms whose x-function is p: lamn(p) of them, lams/lamq(p, k)
    __host__ __device__ int lamn(int p) const { return d[o_lamn + p]; }
    __host__ __device__ int lams(int p, int k) const { return d[o_lams + p * nby + k]; }
    __host__ __device__ int lamq(int p, int k) const { return d[o_lamq + p * nby + k]; }
    // kernel terms whose y-function is j: jcnt(j) of them, jterm(j, k)
    __host__ __device__ int jcnt(int j) const { return d[o_jcnt + j]; }
    __host__ __device__ int jterm(int j, int k) const { return d[o_jterm + j * nk + k]; }
    // unknown index of offset (a, b) of kernel term t, or -1 if the term lacks it
    __host__ __device__ int unknown(int t, int a, int b) const {
        const int L1 = 2 * w1 + 1, L = (2 * w0 + 1) * L1;
        const int off = (a + w0) * L1 + (b + w1), ctr = (L - 1) / 2;
        const int f = flags(t), u0 = d[o_uoff + t];
        if (off == ctr) return (f & 1) ? ((f & 2) ? u0 + off : u0) : -1;
        if (!(f & 2)) return -1;
        return u0 + ((f & 1) ? off : (off > ctr ? off - 1 : off));
    }
};

// Tabulated basis functions in the compute type (B-spline functions, or the
// monomials xt^i, yt^j of the polynomial basis; null only before the plan's
// tables exist): fx [nfx][n0], fy [nfy][n1], bx [nbx][n0], by [nby][n1].
template <typename T>
struct FTab {
    const T *fx, *fy, *bx, *by;
};

// Largest basis sizes (kernel terms, functions per axis).
constexpr int kMaxKTerms = 40;
constexpr int kMaxFun = 8;
// Largest number of science (and of reference) images in the co-added form of the decorrelation.
constexpr int kMaxCoadd = 16;

struct Plan {
    sfft_config cfg;
    int n0, n1, h1c;       // h1c = n1/2 + 1 half-spectrum columns
    int nk, nb, n;         // kernel terms, background terms, unknowns
    int L0, L1;            // 2w+1
    int na, nbk;           // split: n0 = na * nbk
    int nimg;              // R-terms + S
    int npairs, nrows;     // stage-1 products (one per row range); stage-1 rows (sum of 2*h0+1)
    int ngpairs;           // the gather's product list (auto-products packed in pairs where it can)
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
    // tune_tc: 0 or 1 the solve's tile products on the CUDA cores, 2 on the
    // tensor cores (FP32 plans only; see solve.cu)
    int tune_tr, tune_gi, tune_ng, tune_sgrid, tune_tc;
    // panel width of the FP32 blocked Cholesky: 32 (default) or 64 (solve.cu)
    int solve_panel;
    int sms;  // multiprocessors of the device the plan was created on
    // basis (see BasisView); the tables are built at plan creation
    int bspline;           // 0 polynomial, 1 B-spline
    int nfx, nfy, nbx, nby;
    BasisView bv;          // offsets; bv.d points to d_int
    int *h_int, *d_int;    // int tables (host copy, device copy)
    void *ftab;            // B-spline function tables, compute type: fx | fy | bx | by
    double *ftab64;        // FP64 x-functions for the zero-lag sums: [nallx][n0]
    double *bxy64;         // FP64 background functions bx [nbx][n0] then by [nby][n1] (for their spectra)
    int nallx;
    int nzm;               // zero-lag values: Omega(0,0) of each pair, Lambda(0,0), Theta(0,0), E
    int *d_zdesc;          // [nzm][3] (row moment, x-function a, x-function b or -1)
    int *d_rdesc;          // [nmom][3] B-spline row moments (kind, y-function a, b or -1)
    double *z0;            // [nzm] zero-lag values (FP64)
    double *cmat;          // C of Eq. B11, [nb][nb] (FP64, depends on the basis only)
    int4 *unk;             // [n] decoded unknowns: (kernel term?, term, alpha, beta)
    // Polynomial basis: Lambda in closed form (k_lambda_closed) instead of the
    // gather; z_mu: offset of the 2-D moments mu(u, v), u, v <= dk + db, in z0;
    // bnd: FP64 column moments of the 2 w1 boundary columns and the masked R
    // in the 2 w0 x 2 w1 corner pixels.
    int lam_closed, z_mu;
    double *bnd;
    void *xhat;            // [p][lb][r] 1-D spectra of the background x-functions, permuted (compute
                           // type); only where Lambda goes through the gather (not lam_closed)
    void *yhat;            // [q][m] 1-D spectra of the background y-functions, m < h1c (compute type)
    void *F;               // [(nfy+1)][m][x] row transforms (compute type)
    void *U;               // [nimg][m][lb][r] full spectra, permuted (compute type); reused for Dt
    void *Q;               // [nrows][m] stage-1 results (compute type complex)
    PairDesc *pairs;       // device copy: npairs products, then the gather's ngpairs (gpairs)
    PairDesc *gpairs;
    double *rowmom;        // [n0][nmom] per-row moment sums
    double *lag;           // lag tables (Omega, Lambda, Theta), FP64
    int lag_om, lag_la, lag_th;  // offsets into lag
    // solve workspace
    void *A;               // n*n factor (compute type)
    void *Wm;              // n*n: W = L^-1 (compute type)
    int solve_grid;        // blocks of the cooperative solve kernel
    int solve_grid_tc;     // blocks of its tensor-core variant (one per SM), 0 for FP64
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
    void *gam;             // co-added decorrelation: row spectra of the homogenisation kernels
    size_t gam_bytes;
    size_t ws_bytes;
    uint64_t launches;     // kernels this plan has enqueued
    // buffers of the most recent run_pair (for sfft_replay_stage)
    const void *last_ref, *last_sci;
    const uint8_t *last_mask;
    double *last_M, *last_rhs, *last_x;
    sfft_solve_info *last_info;
    void *last_diff;
    cudaStream_t last_stream;
    PairDesc *host_pairs;  // [npairs]
};

// Device images and masks are read with 16-byte vector loads: every entry
// point checks their alignment before any launch.
inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
inline bool images_aligned(const void *ref, const void *sci, const void *mask) {
    return aligned16(ref) && aligned16(sci) && (mask == nullptr || aligned16(mask));
}

// plans (api.cu): validation, allocation + tables, release
int plan_validate(const sfft_config *c);
int plan_new(const sfft_config *cfg, cudaStream_t s, Plan **out);  // cfg already validated
void plan_free(Plan *p);
int status_of(cudaError_t e);

// the function tables of a plan in the compute type (B-spline functions or
// monomials of the normalised coordinates); ftab holds fx | bx | fy | by
template <typename T>
inline FTab<T> ftab_of(const Plan *p) {
    FTab<T> f{nullptr, nullptr, nullptr, nullptr};
    if (!p->ftab) return f;
    f.fx = (const T *)p->ftab;
    f.bx = f.fx + (size_t)p->nfx * p->n0;
    f.fy = f.bx + (size_t)p->nbx * p->n0;
    f.by = f.fy + (size_t)p->nfy * p->n1;
    return f;
}

// basis (basis.cu)
int basis_validate(const sfft_config *c);
int basis_unknowns(const sfft_config *c);
int basis_terms(const sfft_config *c, int *nk, int *nb);
int basis_build(Plan *p, cudaStream_t s);  // p->n, sizes and cfg set; allocations owned by p
// weights of the kernel terms at one normalised position (w: nk values)
void basis_term_weights(const Plan *p, double xt0, double yt0, double *w);

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
int solve_grid_size(bool fp64, bool tc = false);
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
// The co-added form of App. C (Eq. 21): ns science and nr reference
// homogenisation kernels (FP64 device images, half-widths g0, g1) and their
// noise variances sigma2[0 .. ns+nr).  Null: the one-pair form.
struct Coadd {
    int ns, nr, g0, g1;
    const double *G, *H;
    double sigma2[2 * kMaxCoadd];
};
cudaError_t decorrelate(Plan *p, const double *x, double xt0, double yt0, double sigma_ref, double sigma_sci,
                        const void *diff, void *out, const Coadd *co, cudaStream_t s);
cudaError_t subtract_from_rows(Plan *p, const double *x, void *diff, cudaStream_t s);
cudaError_t plan_tables(Plan *p, cudaStream_t s);

}  // namespace sfft
