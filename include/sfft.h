/*
 * sfft.h -- C ABI of the GB300 (sm_103a) implementation of the SFFT hot path:
 * Fourier-space construction of the delta-function-basis least-squares
 * system, its solution, and the spatially varying convolve-and-subtract
 * (Hu et al., "Image Subtraction in Fourier Space", arXiv:2109.09334).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Images are row-major [x][y] arrays of n0 x n1 pixels: x is axis 0 (rows,
 * length n0), y is axis 1 (contiguous), as in Eq. 1.  Pixel coordinates in
 * the polynomials of Eq. 2 and Eq. 6 are normalised to [-1, 1]:
 *     xt = (2x - (n0-1)) / (n0-1),   yt = (2y - (n1-1)) / (n1-1),
 * which spans the same polynomial space as the raw indices.  Shifts and
 * convolutions are circular (Eq. 12), every index taken mod n0, n1.
 *
 * Unknowns are in real-space units (the a-ring of Eq. 6; Eq. 13's
 * a = n0*n1*a-ring is a uniform rescaling that is not applied), ordered:
 *   kernel block first -- for each kernel term (i,j) with i+j <= dk, ordered
 *   by total degree then descending i: (0,0),(1,0),(0,1),(2,0),(1,1),(0,2),...
 *   -- the offsets (alpha,beta) row-major, alpha from -w0 to w0 (outer), beta
 *   from -w1 to w1; with a constant photometric ratio the offset (0,0) of
 *   every term other than (0,0) is omitted; then the background terms (p,q)
 *   with p+q <= db in the same monomial order.  n = nk*L + nb, or
 *   nk*(L-1) + 1 + nb with a constant photometric ratio, where L =
 *   (2w0+1)(2w1+1), nk = (dk+1)(dk+2)/2, nb = (db+1)(db+2)/2.
 *
 * B-spline basis (Eq. 7-9, cfg.basis = SFFT_BASIS_BSPLINE): the polynomials
 * are replaced by tensor products of B-splines on the normalised
 * coordinates, the same basis along x and y, with clamped uniform knots on
 * [-1, 1]: degree kdeg and kint interior knots give K = kint + kdeg + 1
 * functions B_0..B_(K-1) per axis (the right end xt = 1 belongs to the last
 * knot span).  Kernel terms are (i,j), i,j < K, ordered i outer, weight
 * B_i(xt) B_j(yt), each with all L offsets; with a constant photometric
 * ratio a first term of weight 1 carries the (0,0) offset alone (one
 * unknown: the kernel sum) and the K*K spline terms omit that offset.  The
 * background terms are (p,q), p,q < K' = bint + bdeg + 1, p outer, weight
 * B'_p(xt) B'_q(yt).  n = K*K*L + K'*K', or 1 + K*K*(L-1) + K'*K'.
 *
 * Memory: every pointer named d_* is device memory owned by the caller; h_*
 * is host memory owned by the caller (page-locked for asynchronous copies).
 * Device images R, S and masks are read with 16-byte vector loads: d_ref,
 * d_sci and d_mask must be 16-byte aligned (cudaMalloc and PyTorch
 * allocations are); the calls return SFFT_ERR_INVALID before any launch
 * otherwise.
 * A plan owns its workspace; it is not thread-safe and serves one pair at a
 * time on the stream it is used with.
 *
 * Errors: calls are asynchronous on the given stream.  A negative return
 * value reports an invalid argument, an allocation failure or a launch
 * failure, synchronously, and nothing was enqueued past the failing launch.
 * Numerical failures (matrix not positive definite, refinement not
 * converged) are written to sfft_solve_info.status in device memory.
 * No exception crosses this interface.
 */
#ifndef SFFT_H
#define SFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFFT_OK = 0,
    SFFT_ERR_INVALID = -1,       /* bad argument or configuration */
    SFFT_ERR_OOM = -2,           /* device or host allocation failed */
    SFFT_ERR_CUDA = -3,          /* a CUDA call or kernel launch failed */
    SFFT_ERR_SINGULAR = -4,      /* normal matrix not positive definite (device status) */
    SFFT_ERR_NOT_CONVERGED = -5, /* iterative refinement did not reach tolerance (device status) */
    SFFT_ERR_TIMEOUT = -6,       /* a bounded wait ran out */
    SFFT_ERR_BUSY = -7,          /* no free slot / memory for a request right now */
    SFFT_ERR_UNSUPPORTED = -8    /* valid but not implemented (e.g. image size) */
} sfft_status;

typedef enum { SFFT_F32 = 0, SFFT_F64 = 1 } sfft_dtype;

typedef enum {
    SFFT_PREC_FP64 = 0,  /* plain path: FP64 FFTs, products, sums and Cholesky */
    SFFT_PREC_MIXED = 1  /* FP32 FFTs and products with compensated (two-sum)
                            accumulation of the frequency sums, FP32 Cholesky of
                            the Jacobi-scaled matrix, FP64 residual refinement */
} sfft_precision;

typedef enum {
    SFFT_BASIS_POLY = 0,    /* polynomial variation (Eq. 2 and 6), degrees dk and db */
    SFFT_BASIS_BSPLINE = 1  /* tensor-product B-splines (Eq. 7-9), see the unknown order above */
} sfft_basis;

/* Fit parameters of one image pair (Sec. 3.3 and Table A1). */
typedef struct {
    int32_t n0, n1;           /* image size, each in [16, 4096] (any length) */
    int32_t w0, w1;           /* kernel half-widths: L0 = 2*w0+1, L1 = 2*w1+1 (Eq. 3-4) */
    int32_t dk;               /* kernel polynomial degree D_K (Eq. 6), 0..3; 0 for B-splines */
    int32_t db;               /* background polynomial degree D_B (Eq. 2), 0..3; 0 for B-splines */
    int32_t const_phot_ratio; /* 1: kernel sum constant over the field (Sec. 2.2) */
    int32_t dtype;            /* sfft_dtype of the images R, S and of the output D */
    int32_t precision;        /* sfft_precision */
    int32_t basis;            /* sfft_basis; the fields below are used by SFFT_BASIS_BSPLINE only */
    int32_t kdeg, kint;       /* kernel B-splines: degree 0..3, interior knots; K = kint+kdeg+1 <= 6 */
    int32_t bdeg, bint;       /* background B-splines: degree 0..3, interior knots; K' <= 6 */
} sfft_config;

/* Written by sfft_solve in device memory. */
typedef struct {
    int32_t status;       /* SFFT_OK, SFFT_ERR_SINGULAR or SFFT_ERR_NOT_CONVERGED */
    int32_t iters;        /* refinement iterations performed */
    double rel_residual;  /* ||rhs - M x||_2 / ||rhs||_2 of the returned x (FP64) */
    double min_pivot;     /* smallest Cholesky pivot of the Jacobi-scaled matrix */
} sfft_solve_info;

typedef struct sfft_plan_s *sfft_plan_t;
typedef void *sfft_stream_t; /* a cudaStream_t; NULL is the legacy default stream */

/* Human-readable name of a status code.  Never NULL. */
const char *sfft_status_string(int status);

/* Number of unknowns n of Eq. 18 for this configuration (no GPU use). */
int sfft_num_unknowns(const sfft_config *cfg, int32_t *n);

/*
 * Create a plan for one configuration: validates it, allocates the device
 * workspace, and computes on `stream` the twiddle tables and the 1-D spectra
 * of the background monomials (T^pq of Eq. 2 is separable, so its DFT is the
 * outer product of two 1-D DFTs).  *out is NULL on failure.
 */
int sfft_plan_create(const sfft_config *cfg, sfft_stream_t stream, sfft_plan_t *out);

/*
 * Waits for all work on the device (the plan's buffers may be in use on any
 * stream the caller gave it, or in a captured batch), then frees its
 * workspace.  NULL is a no-op.
 */
int sfft_plan_destroy(sfft_plan_t plan);

/* Device bytes the plan holds. */
int sfft_plan_workspace_bytes(sfft_plan_t plan, uint64_t *bytes);

/*
 * Panel width of the blocked Cholesky factorisation of the FP32 solve (the
 * solve of Eq. 18; FP64 plans always use 32): 32 (the default) or 64.  With
 * 64 a solve needs half the grid barriers and half the passes over the
 * trailing matrix but a longer serial chain per diagonal block: faster when
 * several systems share a launch (sfft_run_pairs, batches, servers), slower
 * for one system alone.  The widths round differently (both meet the
 * solve's tolerance); systems solved in one launch must share the width
 * (SFFT_ERR_INVALID otherwise).  Server slots and pool lanes that batch
 * four or more pairs (batch >= 4) use 64.  SFFT_ERR_INVALID for another width.
 */
int sfft_plan_set_solve_panel(sfft_plan_t plan, int32_t width);
int sfft_plan_solve_panel(sfft_plan_t plan, int32_t *width);

/*
 * Build the normal equations M theta = rhs of Eq. 18 (blocks Eq. 19-24) from
 * the reference R and science S, through the lag tables of App. B
 * (Eq. B5-B16): forward FFTs of the monomial-weighted images R^ij = xt^i yt^j R
 * and of S, spectrum products, a pruned inverse DFT evaluated only at the lags
 * |rho| <= 2w (Omega) and |rho| <= w (Lambda, Theta), and the index maps of
 * Eq. B5/B7/B9/B13 into M and rhs.  C and E (Eq. B11, B15) are moment sums.
 *   d_ref, d_sci : n0*n1 images of cfg.dtype.
 *   d_mask       : n0*n1 bytes or NULL; 0 marks a pixel excluded from the fit
 *                  (R and S zero-filled there, Sec. 3); NULL uses every pixel.
 *   d_M          : n*n doubles, row-major, symmetric (both triangles written).
 *   d_rhs        : n doubles.
 */
int sfft_build_system(sfft_plan_t plan, const void *d_ref, const void *d_sci,
                      const uint8_t *d_mask, double *d_M, double *d_rhs,
                      sfft_stream_t stream);

/*
 * Solve M theta = rhs (Eq. 18; the paper names no solver).  FP64 precision:
 * Cholesky in FP64.  Mixed precision: Jacobi scaling, Cholesky in FP32, then
 * iterative refinement with FP64 residuals r = rhs - M theta until
 * ||r|| / ||rhs|| <= 1e-12, at most 12 iterations (else SFFT_ERR_NOT_CONVERGED).
 *   d_M, d_rhs : as written by sfft_build_system (read only).
 *   d_x        : n doubles, the coefficients theta in the unknown order above.
 *   d_info     : device sfft_solve_info, or NULL.
 */
int sfft_solve(sfft_plan_t plan, const double *d_M, const double *d_rhs, double *d_x,
               sfft_solve_info *d_info, sfft_stream_t stream);

/*
 * Several systems of Eq. 18 in one launch: system i is M_i theta_i = rhs_i on
 * plans[i]'s workspace, solved exactly as sfft_solve would solve it alone
 * (bit for bit), up to 8 systems of any sizes side by side.
 *   plans[count] : distinct plans of one precision (and, for FP32, one solve
 *                  panel width); count 1..8.
 *   d_M[i], d_rhs[i], d_x[i], d_info[i] : as for sfft_solve (d_info may be
 *                  NULL, or any of its entries).
 * SFFT_ERR_INVALID for count outside 1..8, a NULL plan, matrix, right-hand
 * side or solution, a plan listed twice, or a mismatch, before any CUDA call.
 */
int sfft_solve_batch(const sfft_plan_t *plans, int32_t count, const double *const *d_M,
                     const double *const *d_rhs, double *const *d_x, sfft_solve_info *const *d_info,
                     sfft_stream_t stream);

/*
 * sfft_solve without a plan and without allocating: the paper has no
 * counterpart; this is an engineering variant of sfft_solve for callers that
 * cannot allocate device memory at call time.  Examples are a pipeline that
 * has handed all of the device's memory to its own pool, where a cudaMalloc
 * would fail, and a service that keeps other streams busy, where cudaFree
 * would synchronise the device and stall them.  It is also for a system
 * assembled elsewhere, which would otherwise need a plan whose creation
 * allocates the whole image workspace.  Same algorithm and results as
 * sfft_solve.
 *   d_M, d_rhs : n*n and n doubles in device memory (read only).
 *   n          : 1 <= n <= SFFT_SOLVE_STATIC_MAX_N; larger n returns
 *                SFFT_ERR_UNSUPPORTED before any device work.
 *   precision  : SFFT_PREC_FP64 or SFFT_PREC_MIXED (as sfft_config.precision).
 *   d_x        : n doubles.  d_info : device sfft_solve_info, or NULL.
 * Workspace: one file-scope device array per device, 16.25 MiB
 * (2 SFFT_SOLVE_STATIC_MAX_N^2 doubles + 256 KiB), placed by the CUDA driver
 * when the library's module is loaded.  Nothing in it needs to start at
 * zero, because each call resets its own status flags first.  Calls whose
 * executions overlap on one device share the array and race: order them on
 * one stream, or make one wait for the other.  The first call on each device
 * (made with that device current) does one-time setup.  It looks up the
 * array's address and sizes the cooperative grid, checking both results.
 * Make that call before any stream capture begins.  The setup is kept for
 * the life of the process and belongs to the device's context at that time:
 * calls must not span a cudaDeviceReset of the device (or any other end of
 * its primary context), after which the recorded address is stale.
 */
#define SFFT_SOLVE_STATIC_MAX_N 1024
int sfft_solve_static(const double *d_M, const double *d_rhs, int32_t n, int32_t precision,
                      double *d_x, sfft_solve_info *d_info, sfft_stream_t stream);

/*
 * Difference image of Eq. 12-13 from the UNMASKED pair (two-step process of
 * Sec. 3): D = S - sum_ij (R^ij o k_ij) - sum_pq b_pq T^pq, evaluated in
 * Fourier space along y and as an L0-tap circular stencil along x.
 *   d_x    : n doubles from sfft_solve.
 *   d_diff : n0*n1 output image of cfg.dtype (may not alias d_ref or d_sci).
 */
int sfft_subtract(sfft_plan_t plan, const void *d_ref, const void *d_sci, const double *d_x,
                  void *d_diff, sfft_stream_t stream);

/*
 * Noise decorrelation of a difference image (App. C, Eq. 21-24) for one
 * pair: D_dc = D (*) Q with the real filter of Eq. 24,
 *     Q^(p) = sqrt(sigma_D^2 / (sigma_sci^2 + sigma_ref^2 |K^(p)|^2)),
 * normalised to unit kernel sum (sigma_D^2 = sigma_sci^2 + sigma_ref^2 K^(0)^2,
 * the flux-preserving choice), as a circular convolution.  App. C ignores the
 * spatial variation of the kernel: K is the matching kernel of Eq. 6 at the
 * normalised position (xt0, yt0) in [-1, 1]^2, built from the coefficients
 * d_x of sfft_solve (the delta basis of Eq. 3-4).
 *   sigma_ref >= 0, sigma_sci > 0 : noise of R and S (their ratio matters).
 *   d_diff : n0*n1 image of cfg.dtype (read);  d_out : n0*n1 image of
 *            cfg.dtype (written; may equal d_diff).
 * Uses the plan's workspace: it overwrites the row transforms of the last
 * build, so call it after sfft_subtract / sfft_run_pair of that pair.
 */
int sfft_decorrelate(sfft_plan_t plan, const double *d_x, double xt0, double yt0, double sigma_ref,
                     double sigma_sci, const void *d_diff, void *d_out, sfft_stream_t stream);

/*
 * Noise decorrelation in the co-added form of App. C (Eq. 21-24 in full):
 * the difference image was made as D = sum_j S_j (*) G_j - [sum_i R_i (*) H_i] (*) K
 * from M science and N reference exposures with white noise sigma_Sj,
 * sigma_Ri, homogenised by the kernels G_j, H_i (divided by M and N, as
 * Eq. 21 states) and co-added.  The real filter
 *     Q^ = sqrt(s_D^2 / (sum_j s_Sj^2 |G^_j|^2 + |K^|^2 sum_i s_Ri^2 |H^_i|^2)),
 * normalised to unit kernel sum (s_D^2 = the denominator at frequency 0),
 * is applied as in sfft_decorrelate, with K the kernel of this plan's
 * coefficients d_x at (xt0, yt0).
 *   n_sci, n_ref     : M and N, each 1..16.
 *   d_G, d_H         : device FP64 kernel images, centred, [n_sci][2g0+1][2g1+1]
 *                      and [n_ref][2g0+1][2g1+1] (row-major, offset a = -g0 first).
 *   h_sigma_sci/_ref : host arrays of the noise levels (>= 0; not all science ones 0).
 *   g0, g1           : half-widths of G and H, 0..32, 2g+1 at most the image size.
 * Where the denominator vanishes (every G^_j and H^_i zero at a frequency)
 * the output is not finite.  Allocates the plan's table of the kernels' row
 * spectra on first use (or when larger kernels are given); otherwise as
 * sfft_decorrelate (asynchronous on `stream`, d_out may equal d_diff).
 */
int sfft_decorrelate_coadd(sfft_plan_t plan, const double *d_x, double xt0, double yt0,
                           int32_t n_sci, const double *d_G, const double *h_sigma_sci,
                           int32_t n_ref, const double *d_H, const double *h_sigma_ref,
                           int32_t g0, int32_t g1, const void *d_diff, void *d_out,
                           sfft_stream_t stream);

/*
 * Crowded-flavor mask (Sec. 3.1): the pixels affected by saturated sources,
 * for the d_mask argument of sfft_build_system / sfft_run_pair.  A pixel is
 * masked (0) when R reaches sat_ref or S reaches sat_sci anywhere within the
 * square of half-width `grow` around it (Chebyshev distance, clipped at the
 * image edges), or when d_mask_in (NULL: none) masks it; else 1.  Needs no
 * plan.
 *   n0, n1        : image size (>= 1); dtype: sfft_dtype of d_ref, d_sci.
 *   grow          : 0..16.
 *   d_mask_out    : n0*n1 bytes, device; may equal d_mask_in.
 * Asynchronous on `stream`; SFFT_ERR_INVALID for bad arguments.
 */
int sfft_saturation_mask(int32_t n0, int32_t n1, int32_t dtype, const void *d_ref, const void *d_sci,
                         double sat_ref, double sat_sci, int32_t grow, const uint8_t *d_mask_in,
                         uint8_t *d_mask_out, sfft_stream_t stream);

/*
 * One whole pair on device buffers: build, solve and subtract.  d_M, d_rhs,
 * d_x and d_info may be NULL, in which case plan-owned buffers are used.
 */
int sfft_run_pair(sfft_plan_t plan, const void *d_ref, const void *d_sci,
                  const uint8_t *d_mask, double *d_M, double *d_rhs, double *d_x,
                  sfft_solve_info *d_info, void *d_diff, sfft_stream_t stream);

/*
 * Several whole pairs on device buffers, pair i with its own plan plans[i]
 * (Sec. 3 subtracts the pairs of a survey one by one; the pairs here may
 * differ in size and basis).  Every pair's system (Eq. 18) is built, the
 * systems are then solved up to eight per launch of the batched solve
 * (grouped by number of unknowns, largest first), and every pair is
 * subtracted (Eq. 3).  Per pair the results equal those of
 * sfft_run_pair on the same plan and inputs, bit for bit.
 *   plans[count]   : distinct plans sharing cfg.precision (and, for FP32,
 *                    the solve panel width); a plan listed twice, or a
 *                    mismatch, is SFFT_ERR_INVALID.
 *   d_refs, d_scis, d_diffs : count device image pointers, each as in
 *                    sfft_run_pair (d_diffs[i] distinct from the inputs).
 *   d_masks        : NULL, or count pointers, each NULL or a mask.
 *   d_xs, d_infos  : NULL, or count pointers, each NULL (plan-owned buffer)
 *                    or a device buffer as in sfft_run_pair.
 * The normal matrices land in the plans' own buffers.  Errors found on the
 * host return before any launch; a launch error stops the sequence and is
 * returned.  Solve failures are reported per pair in its sfft_solve_info.
 */
int sfft_run_pairs(const sfft_plan_t *plans, int32_t count, const void *const *d_refs,
                   const void *const *d_scis, const uint8_t *const *d_masks, double *const *d_xs,
                   sfft_solve_info *const *d_infos, void *const *d_diffs, sfft_stream_t stream);

/*
 * The pairs of sfft_run_pairs captured once into a CUDA graph, replayed as
 * one launch (the batched-sectors workload: a survey's uneven CCD sectors,
 * Sec. 3 and the timings of Sec. 4 over many pairs).  Creation records, for
 * the given plans and device buffers, every kernel of the whole sequence
 * (builds, solves `solve_group` systems per cooperative launch, largest
 * first, subtractions) into a graph on a private stream; each
 * sfft_batch_launch then enqueues all of it on `stream` with one call.
 * Arguments as sfft_run_pairs; the plans and every buffer must stay valid,
 * at the same addresses, until sfft_batch_destroy (the graph holds them).
 * New data is processed by writing new images into the same input buffers
 * before a launch.  Per pair the results equal sfft_run_pair's bit for bit.
 *   solve_group : 1..8 systems per solve launch, or 0 to autotune: the batch
 *                 is captured with groups of 8, 4, 2 and 1, each replayed
 *                 (once untimed, then three times timed, CUDA events) on the
 *                 buffers' current contents, and the fastest is kept;
 *                 creation then runs the batch 16 times and synchronises.
 * Creation synchronises its private stream; it may not run inside another
 * stream capture.  A plan must not be used by other calls while a launch of
 * a batch that holds it is in flight.
 */
typedef struct sfft_batch_s *sfft_batch_t;
int sfft_batch_create(const sfft_plan_t *plans, int32_t count, const void *const *d_refs,
                      const void *const *d_scis, const uint8_t *const *d_masks, double *const *d_xs,
                      sfft_solve_info *const *d_infos, void *const *d_diffs, int32_t solve_group,
                      sfft_batch_t *out);

/* Enqueue the whole captured batch on `stream` (one graph launch). */
int sfft_batch_launch(sfft_batch_t batch, sfft_stream_t stream);

/*
 * The batch's solve grouping, its number of kernel launches per replay, and
 * (autotuned batches; NULL to skip) the replay times in ms of groups 8, 4,
 * 2 and 1.
 */
int sfft_batch_info(sfft_batch_t batch, int32_t *solve_group, int32_t *launches, float *tune_ms4);

/* Frees the graph (NULL is a no-op); the plans and buffers stay the caller's. */
int sfft_batch_destroy(sfft_batch_t batch);

/*
 * One whole pair from and to host memory: copies h_ref, h_sci (and h_mask if
 * not NULL) to plan-owned device buffers, runs build, solve and subtract,
 * copies the coefficients, the solve status and the difference image back,
 * and synchronises the stream before returning.
 *   h_x    : n doubles or NULL.  h_info : host sfft_solve_info or NULL.
 *   h_diff : n0*n1 image of cfg.dtype.
 */
int sfft_run_pair_host(sfft_plan_t plan, const void *h_ref, const void *h_sci,
                       const uint8_t *h_mask, double *h_x, sfft_solve_info *h_info,
                       void *h_diff, sfft_stream_t stream);

/* ---- serving: several pairs in flight ------------------------------------ */
/*
 * The paper subtracts pair after pair (Sec. 3); a server keeps up to `depth`
 * pairs of one configuration in flight and solves their systems `batch` at a
 * time in one launch.  The solve is a latency-bound chain of small steps, so
 * a batch of systems costs little more than one.  Each pair runs the kernels
 * of sfft_run_pair on its own workspace, and the batched solve performs, for
 * each system, the operations of the single solve in the same order, so the
 * results equal sfft_run_pair's.  Requests complete in submission order.
 */
typedef struct sfft_server_s *sfft_server_t;

typedef enum { SFFT_REQ_DEVICE = 0, SFFT_REQ_HOST = 1 } sfft_request_memory;

typedef struct {
    int32_t memory;         /* sfft_request_memory: where all six buffers below live */
    const void *ref;        /* n0*n1 image of cfg.dtype */
    const void *sci;        /* n0*n1 image of cfg.dtype */
    const uint8_t *mask;    /* n0*n1 bytes or NULL (as sfft_build_system) */
    double *x;              /* n doubles or NULL */
    sfft_solve_info *info;  /* or NULL */
    void *diff;             /* n0*n1 output image; may not alias ref or sci */
    sfft_stream_t stream;   /* SFFT_REQ_DEVICE: ref, sci and mask are ready in this
                               stream's order (NULL: the legacy default stream).
                               Ignored for SFFT_REQ_HOST. */
} sfft_request;

typedef struct {
    uint64_t seq; /* submission number, from 0 */
} sfft_ticket;

/*
 * Create a server with `depth` (1..8) slots, each a full plan workspace plus
 * staging buffers for host requests (sfft_server_workspace_bytes), and its
 * own streams; systems are solved `batch` (1..depth) at a time.
 * Synchronises once its tables are ready.
 */
int sfft_server_create(const sfft_config *cfg, int32_t depth, int32_t batch, sfft_server_t *out);

/* Waits for all submitted requests, then frees everything.  NULL is a no-op. */
int sfft_server_destroy(sfft_server_t server);

/* Device bytes held by the server. */
int sfft_server_workspace_bytes(sfft_server_t server, uint64_t *bytes);

/*
 * Enqueue one pair and return at once with its ticket.  Its build starts at
 * once; its solve and subtraction are enqueued when its batch is complete, on
 * sfft_flush, or when the caller polls or waits for it.  The caller keeps
 * every buffer of the request valid and unchanged (outputs unread) until the
 * ticket completes; host buffers should be pinned for the copies to overlap.
 * Blocks only while 64 requests are already pending.  Thread-safe.
 */
int sfft_submit(sfft_server_t server, const sfft_request *req, sfft_ticket *ticket);

/* Enqueue the solves and subtractions of an incomplete batch now. */
int sfft_flush(sfft_server_t server);

/*
 * SFFT_OK if the ticket's request has completed, SFFT_ERR_BUSY if not yet,
 * SFFT_ERR_CUDA if a completion query reported a CUDA error (sticky: every
 * later submit, poll and wait on this server returns it; destroy it).
 */
int sfft_poll(sfft_server_t server, const sfft_ticket *ticket);

/*
 * Wait until the ticket's request has completed: SFFT_OK, or
 * SFFT_ERR_TIMEOUT after timeout_us microseconds (timeout_us < 0: no limit),
 * or SFFT_ERR_CUDA as soon as a completion query reports a CUDA error (as
 * for sfft_poll; the wait never spins on a failed query).  Numerical
 * failures are reported in the request's info, as for sfft_solve.
 */
int sfft_wait(sfft_server_t server, const sfft_ticket *ticket, int64_t timeout_us);

/*
 * Continuous batching policy, off by default.  With enable != 0 a batch that
 * is not yet full is solved at once (without waiting for `batch` requests,
 * sfft_flush, poll or wait) whenever every request flushed before it has
 * completed: a request that arrives while the server is idle starts its
 * solve as soon as its build is done, and the requests that arrive while the
 * server is busy gather into the next batch.  Results are unchanged (each
 * system's solve does not depend on its batch partners).
 */
int sfft_server_set_eager(sfft_server_t server, int32_t enable);

/*
 * Testing hook, off by default: with enable != 0 the server's completion
 * queries report a CUDA error (as a failed device would) without asking the
 * device, so that the error paths of sfft_poll, sfft_wait and sfft_submit can
 * be exercised with no fault on the GPU.  The work already enqueued still
 * runs; sfft_server_destroy waits for it as usual.
 */
int sfft_server_debug_fail_queries(sfft_server_t server, int32_t enable);

/*
 * Make `stream` wait (on the device, without blocking the host) until the
 * ticket's request has completed, e.g. before a kernel that reads its diff.
 */
int sfft_stream_wait_ticket(sfft_server_t server, const sfft_ticket *ticket, sfft_stream_t stream);

/* ---- pool: pairs of many configurations under one memory budget -------- */
/*
 * A pool holds one server (lane) per configuration it has seen, each with
 * `depth` slots and solve batches of `batch`, created on first use and kept
 * with their plans and spectra on the device.  Lanes of different
 * configurations run on their own streams, so their work overlaps on the
 * GPU.  Admission by memory footprint: a new configuration is admitted only
 * if its lane fits in `budget_bytes` together with the lanes held; idle lanes
 * (every request completed, nobody waiting) are released, least recently used
 * first, to make room.  Results equal sfft_run_pair's on the same inputs.
 */
typedef struct sfft_pool_s *sfft_pool_t;

typedef struct {
    uint64_t lane; /* lane id, from 1 */
    uint64_t seq;  /* submission number within the lane */
} sfft_pool_ticket;

/* budget_bytes > 0; 1 <= batch <= depth <= 8. */
int sfft_pool_create(uint64_t budget_bytes, int32_t depth, int32_t batch, sfft_pool_t *out);

/* Waits for every request, then frees all lanes.  NULL is a no-op. */
int sfft_pool_destroy(sfft_pool_t pool);

/*
 * Enqueue one pair of configuration *cfg (as sfft_submit, same request
 * rules).  SFFT_ERR_BUSY: the configuration's lane does not fit the budget
 * even after releasing the idle lanes; wait for some ticket and retry.
 * Thread-safe.
 */
int sfft_pool_submit(sfft_pool_t pool, const sfft_config *cfg, const sfft_request *req,
                     sfft_pool_ticket *ticket);

/* As sfft_poll / sfft_wait for a pool ticket. */
int sfft_pool_poll(sfft_pool_t pool, const sfft_pool_ticket *ticket);
int sfft_pool_wait(sfft_pool_t pool, const sfft_pool_ticket *ticket, int64_t timeout_us);

/*
 * The continuous batching policy of sfft_server_set_eager for every lane of
 * the pool, current and future; with it set, sfft_pool_wait first starts the
 * open batches of all idle lanes before it blocks.
 */
int sfft_pool_set_eager(sfft_pool_t pool, int32_t enable);

/* Device bytes held by the pool's lanes and their number. */
int sfft_pool_usage(sfft_pool_t pool, uint64_t *bytes, int32_t *lanes);

/* ---- diagnostics -------------------------------------------------------- */

/* Stages of one pair, as re-enqueued by sfft_replay_stage. */
typedef enum {
    SFFT_STAGE_ROWS = 0,     /* masked row FFTs of yt^j R and S, per-row moments */
    SFFT_STAGE_COLS = 1,     /* moment sums and column FFTs of xt^i (row transforms) */
    SFFT_STAGE_GATHER = 2,   /* spectrum products and pruned inverse DFT along x */
    SFFT_STAGE_LAGS = 3,     /* frequency sums along y to the lag tables; assembly of M, rhs */
    SFFT_STAGE_SOLVE = 4,    /* Cholesky and refinement */
    SFFT_STAGE_SUBTRACT = 5  /* the difference image (after a masked build, preceded by
                                the row FFTs of the unmasked pair) */
} sfft_stage;

/*
 * Autotuning of launch shapes (no counterpart in the paper): runs one pair on
 * the given device buffers with sfft_run_pair, then times each tunable stage
 * (sfft_replay_stage) over candidate launch shapes and keeps the fastest:
 * rows per block of the row FFT, images per block of the column FFT and
 * row pairs per block of the inverse row FFT (the solve grid and the
 * solve's tensor-core tile products stay as set: a single system's time does
 * not predict batched solves, and the tensor-core products round
 * differently).  The shapes change how the work is split into blocks, not
 * the arithmetic, so results are unchanged.  They stay with the plan and are
 * remembered for later plans (and server slots, pool lanes) of the same image
 * size, types and D_K in this process.  Synchronises the stream.
 */
int sfft_plan_autotune(sfft_plan_t plan, const void *d_ref, const void *d_sci, void *d_diff,
                       sfft_stream_t stream);

/*
 * Launch shapes, SFFT_TUNING_LEN values, 0 = built-in choice:
 *   [0] rows per block of the row FFT (0 or a power of two <= 16; capped by
 *       the block size),
 *   [1] images per block of the column FFT (0..4),
 *   [2] row pairs per block of the inverse row FFT (0..4),
 *   [3] blocks of the solve grid (0 or up to 512; used only when it exceeds
 *       the systems in the launch and is at most the built-in grid),
 *   [4] the FP32 solve's 64x64x32 trailing-update tile products: 0 or 1 on
 *       the CUDA cores, 2 on the tensor cores (tcgen05.mma kind::tf32 with a
 *       3xTF32 split, accumulator in tensor memory; that kernel variant runs
 *       one block per SM).  The built-in choice is the CUDA cores, measured
 *       faster for these latency-bound tiles; the tensor-core products round
 *       differently (the refined solution meets the same tolerance).
 *       Ignored by FP64 plans.
 */
#define SFFT_TUNING_LEN 5

/* The plan's launch shapes (shapes: SFFT_TUNING_LEN values, written). */
int sfft_plan_tuning(sfft_plan_t plan, int32_t *shapes);

/*
 * Set the plan's launch shapes (SFFT_TUNING_LEN values, read), e.g. to
 * reproduce an earlier sfft_plan_autotune; like the autotuner, this also
 * sets the shapes later plans (server slots, pool lanes) of the same
 * configuration start with in this process.  Results do not depend on them.
 * SFFT_ERR_INVALID for a value outside the ranges above (nothing changed).
 */
int sfft_plan_set_tuning(sfft_plan_t plan, const int32_t *shapes);

/* Number of kernels this plan has enqueued since it was created. */
int sfft_plan_launch_count(sfft_plan_t plan, uint64_t *count);

/* Number of kernels a server's slots have enqueued since it was created. */
int sfft_server_launch_count(sfft_server_t server, uint64_t *count);

/*
 * Enqueue one stage of the most recent sfft_run_pair on this plan again, on
 * the same buffers (which must still be valid), for timing a stage alone.
 * Stages after the replayed one are not re-run; a replayed stage overwrites
 * the same intermediate and output buffers with the same values.
 * SFFT_ERR_INVALID if no pair has run on the plan or stage is unknown.
 */
int sfft_replay_stage(sfft_plan_t plan, int stage, sfft_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SFFT_H */
