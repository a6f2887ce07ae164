// api.cu -- the extern "C" entry points declared in include/sfft.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>

#include "common.cuh"
#include "fft16.cuh"
#include "internal.h"

namespace sfft {

// exp(-2 pi i q / n) in FP64
__global__ void k_twiddle64(int n, cpx<double> *tw) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)q / (double)n, &s, &c);
        tw[q] = mk(c, s);
    }
}

// Pass-ordered twiddles of a length-n transform (fft16.cuh): for the
// radix-16 pass of stride ns, entry (r - 1) * ns + k holds
// exp(-2 pi i r k / (16 ns)) = tw64[r k n / (16 ns)] rounded to T.
template <typename T>
__global__ void k_pass_table(int n, int ns, const cpx<double> *tw64, cpx<T> *out) {
    const int cnt = 15 * ns;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
        const int r = 1 + e / ns, k = e % ns;
        const cpx<double> w = tw64[r * k * (n / (16 * ns))];  // r k < 16 ns, so the index is below n
        out[e] = mk((T)w.re, (T)w.im);
    }
}

template <typename T>
static void pass_tables(int n, const cpx<double> *tw64, cpx<T> *out, cudaStream_t s) {
    int e = 0;
    while ((1 << e) < n) ++e;
    int off = 0;
    for (int ns = 1 << (e & 3); ns < n; ns *= 16) {
        if (ns == 1) continue;
        k_pass_table<T><<<(15 * ns + 255) / 256, 256, 0, s>>>(n, ns, tw64, out + off);
        off += 15 * ns;
    }
}

// Bluestein chirp c_t = exp(-i pi t^2 / n), t < n, in FP64; t^2 is reduced
// mod 2n exactly in integers first.
__global__ void k_chirp64(int n, cpx<double> *c) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const long long q = ((long long)t * t) % (2LL * n);
        double sn, cs;
        sincospi(-(double)q / (double)n, &sn, &cs);
        c[t] = mk(cs, sn);
    }
}

// Bluestein filter: the length-m FFT of b_t = conj(c_|t|), |t| < n, placed at
// t mod m, by direct FP64 summation with the FP64 twiddles of length m.
template <typename T>
__global__ void k_bfilt(int n, int m, const cpx<double> *twm, const cpx<double> *c, cpx<T> *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int t = -(n - 1); t < n; ++t) {
            const cpx<double> ct = c[t < 0 ? -t : t];
            const int tm = t < 0 ? t + m : t;
            const cpx<double> w = twm[(int)(((long long)tm * k) & (m - 1))];
            // conj(ct) * w
            re += ct.re * w.re + ct.im * w.im;
            im += ct.re * w.im - ct.im * w.re;
        }
        out[k] = mk((T)re, (T)im);
    }
}

template <typename T>
__global__ void k_round(int n, const cpx<double> *src, cpx<T> *dst) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        dst[q] = mk((T)src[q].re, (T)src[q].im);
}

// 1-D DFT of the background functions of one axis (FP64, direct sum with the
// FP64 table), written in the compute type: function p is xt^p, or row p of
// tab (FP64, [nfun][n]) when tab is not null.  perm: output index of bin l
// (permuted layout for x, natural for y).
template <typename T>
__global__ void k_poly_dft(int n, int nout, int nfun, const cpx<double> *tw, int na, int nbk, int permute,
                           const double *tab, cpx<T> *out) {
    const int total = nfun * nout;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int p = e / nout, l = e % nout;
        double re = 0.0, im = 0.0;
        int q = 0;  // l x mod n, stepped by l
        for (int x = 0; x < n; ++x) {
            const double v = tab ? tab[(size_t)p * n + x] : ipow(coord<double>(x, n), p);
            const cpx<double> w = tw[q];
            re += v * w.re;
            im += v * w.im;
            q += l;
            if (q >= n) q -= n;
        }
        int o = l;
        if (permute) o = (l % nbk) * na + l / nbk;
        out[(size_t)p * nout + o] = mk((T)re, (T)im);
    }
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int plan_validate(const sfft_config *c) {
    if (!c) return SFFT_ERR_INVALID;
    if (c->n0 < 16 || c->n1 < 16 || c->n0 > 4096 || c->n1 > 4096) return SFFT_ERR_UNSUPPORTED;
    if (c->w0 < 0 || c->w1 < 0) return SFFT_ERR_INVALID;
    const int bvr = basis_validate(c);
    if (bvr) return bvr;
    // lag ranges: |rho| <= 2w must stay inside one period; along x the split
    // pruned transform of power-of-two n0 further needs 4 w0 + 1 <= NA
    const int na = !is_pow2(c->n0) ? c->n0 : (c->n0 < kMaxNA ? c->n0 : kMaxNA);
    if (4 * c->w0 + 1 > na || 4 * c->w1 + 1 > c->n1) return SFFT_ERR_UNSUPPORTED;
    if (c->dtype != SFFT_F32 && c->dtype != SFFT_F64) return SFFT_ERR_INVALID;
    if (c->precision != SFFT_PREC_FP64 && c->precision != SFFT_PREC_MIXED) return SFFT_ERR_INVALID;
    return SFFT_OK;
}

void plan_free(Plan *p) {
    void *bufs[] = {p->tw0, p->tw1, p->twp0, p->twp1, p->chirp1, p->bfilt1, p->twpm1, p->chirp0, p->bfilt0,
                    p->twpm0, p->kimg, p->xhat, p->yhat, p->F, p->U, p->Q, p->pairs, p->rowmom, p->lag, p->A,
                    p->Wm, p->dscale, p->r, p->xw, p->zv, p->flag, p->M_own, p->rhs_own, p->x_own, p->info_own,
                    p->img_ref, p->img_sci, p->img_diff, p->img_mask, p->kap, p->d_int, p->ftab, p->ftab64,
                    p->bxy64, p->d_zdesc, p->d_rdesc, p->z0, p->cmat, p->unk, p->gam, p->bnd};
    for (void *b : bufs)
        if (b) cudaFree(b);
    free(p->h_int);
    free(p->host_pairs);
    delete p;
}

#define SFFT_ALLOC(ptr, bytes)                                        \
    do {                                                              \
        if (cudaMalloc((void **)&(ptr), (bytes)) != cudaSuccess) {    \
            cudaGetLastError();                                       \
            plan_free(p);                                             \
            return SFFT_ERR_OOM;                                      \
        }                                                             \
        p->ws_bytes += (bytes);                                       \
    } while (0)

// Launch shapes found by sfft_plan_autotune, kept for later plans of the same
// image size, types and kernel degree (server slots, pool lanes).
struct TuneEntry {
    int n0, n1, dtype, precision, dk, basis, kdeg, kint;
    int32_t shapes[SFFT_TUNING_LEN];
};

static void get_shapes(const Plan *p, int32_t *v) {
    v[0] = p->tune_tr;
    v[1] = p->tune_gi;
    v[2] = p->tune_ng;
    v[3] = p->tune_sgrid;
    v[4] = p->tune_tc;
}

static void set_shapes(Plan *p, const int32_t *v) {
    p->tune_tr = v[0];
    p->tune_gi = v[1];
    p->tune_ng = v[2];
    p->tune_sgrid = v[3];
    p->tune_tc = v[4];
}
constexpr int kTuneCache = 64;
static TuneEntry g_tune[kTuneCache];
static int g_ntune = 0;
static std::mutex g_tune_mu;

static bool tune_key_eq(const TuneEntry &e, const sfft_config *c) {
    return e.n0 == c->n0 && e.n1 == c->n1 && e.dtype == c->dtype && e.precision == c->precision && e.dk == c->dk &&
           e.basis == c->basis && e.kdeg == c->kdeg && e.kint == c->kint;
}

static void tune_lookup(Plan *p) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (int k = 0; k < g_ntune; ++k)
        if (tune_key_eq(g_tune[k], &p->cfg)) set_shapes(p, g_tune[k].shapes);
}

static void tune_store(const Plan *p) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    int k = 0;
    while (k < g_ntune && !tune_key_eq(g_tune[k], &p->cfg)) ++k;
    if (k == g_ntune) {
        if (g_ntune == kTuneCache) k = 0;  // full: overwrite the oldest slot
        else ++g_ntune;
    }
    const sfft_config &c = p->cfg;
    g_tune[k] = TuneEntry{c.n0, c.n1, c.dtype, c.precision, c.dk, c.basis, c.kdeg, c.kint, {}};
    get_shapes(p, g_tune[k].shapes);
}

int plan_new(const sfft_config *cfg, cudaStream_t s, Plan **out) {
    Plan *p = new (std::nothrow) Plan();
    if (!p) return SFFT_ERR_OOM;
    memset((void *)p, 0, sizeof(Plan));
    p->solve_panel = 32;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            p->sms = 0;
        cudaGetLastError();
    }
    p->cfg = *cfg;
    p->n0 = cfg->n0;
    p->n1 = cfg->n1;
    p->h1c = cfg->n1 / 2 + 1;
    basis_terms(cfg, &p->nk, &p->nb);
    p->n = basis_unknowns(cfg);
    p->L0 = 2 * cfg->w0 + 1;
    p->L1 = 2 * cfg->w1 + 1;
    p->gen0 = !is_pow2(cfg->n0);
    p->gen1 = !is_pow2(cfg->n1);
    p->m1 = p->gen1 ? bluestein_len(cfg->n1) : cfg->n1;
    p->m0 = p->gen0 ? bluestein_len(cfg->n0) : cfg->n0;
    p->na = p->gen0 ? cfg->n0 : (cfg->n0 < kMaxNA ? cfg->n0 : kMaxNA);
    p->nbk = cfg->n0 / p->na;
    p->nimg = p->nk + 1;
    p->fp64 = cfg->precision == SFFT_PREC_FP64;
    p->csz = p->fp64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
    p->last_stream = s;
    {
        const int rc = basis_build(p, s);
        if (rc != SFFT_OK) {
            cudaGetLastError();
            plan_free(p);
            return rc;
        }
    }
    // gather pairs
    const int maxp = p->nk * (p->nk + 1) / 2 + p->nk * p->nbx + p->nk;
    p->host_pairs = (PairDesc *)malloc((size_t)2 * maxp * sizeof(PairDesc));
    if (!p->host_pairs) {
        plan_free(p);
        return SFFT_ERR_OOM;
    }
    int np = 0, rows = 0;
    auto push = [&](int kind, int a, int b, int h0) {
        PairDesc d;
        d.kind = kind;
        d.a = a;
        d.b = b;
        d.h0 = h0;
        d.row0 = rows;
        d.row1 = -1;
        rows += 2 * h0 + 1;
        p->host_pairs[np++] = d;
    };
    for (int a = 0; a < p->nk; ++a)
        for (int b = a; b < p->nk; ++b) push(PK_OMEGA, a, b, 2 * cfg->w0);
    if (!p->lam_closed)  // otherwise Lambda is evaluated in closed form (k_lambda_closed)
        for (int a = 0; a < p->nk; ++a)
            for (int q = 0; q < p->nbx; ++q) push(PK_LAMBDA, a, q, cfg->w0);
    for (int a = 0; a < p->nk; ++a) push(PK_THETA, a, p->nk, cfg->w0);
    p->npairs = np;
    p->nrows = rows;
    {
        // The gather's list.  Its lag-range-16 variant (NA = 64, |rho| <= 16)
        // transforms the real auto-products Omega_tt two at a time (PK_OMEGA2);
        // the other variants take the products one by one.
        PairDesc *g = p->host_pairs + np;
        int ng = 0, pending = -1;
        const bool pack = !p->gen0 && p->na == 64 && 2 * cfg->w0 <= 16;
        for (int k = 0; k < np; ++k) {
            const PairDesc &d = p->host_pairs[k];
            if (pack && d.kind == PK_OMEGA && d.a == d.b) {
                if (pending < 0) {
                    pending = k;
                    continue;
                }
                PairDesc q = p->host_pairs[pending];
                q.kind = PK_OMEGA2;
                q.b = d.a;
                q.row1 = d.row0;
                g[ng++] = q;
                pending = -1;
                continue;
            }
            g[ng++] = d;
        }
        if (pending >= 0) g[ng++] = p->host_pairs[pending];
        p->ngpairs = ng;
    }

    const size_t P = (size_t)p->n0 * p->n1;
    const size_t half = (size_t)p->h1c * p->n0;
    const size_t csz = p->csz;
    const size_t rsz = p->fp64 ? sizeof(double) : sizeof(float);
    const int npo = p->nk * (p->nk + 1) / 2;
    const size_t lom = (size_t)(4 * cfg->w0 + 1) * (4 * cfg->w1 + 1);
    const size_t lla = (size_t)(2 * cfg->w0 + 1) * (2 * cfg->w1 + 1);
    p->lag_om = 0;
    p->lag_la = (int)(npo * lom);
    p->lag_th = (int)(p->lag_la + (size_t)p->nk * p->nb * lla);
    const size_t nlag = p->lag_th + (size_t)p->nk * lla;
    const size_t n = p->n;
    (void)P;

    SFFT_ALLOC(p->tw0, p->n0 * csz);
    SFFT_ALLOC(p->tw1, p->n1 * csz);
    SFFT_ALLOC(p->twp0, p->n0 * csz);
    SFFT_ALLOC(p->twp1, p->n1 * csz);
    if (!p->lam_closed) SFFT_ALLOC(p->xhat, (size_t)p->nbx * p->n0 * csz);
    SFFT_ALLOC(p->yhat, (size_t)p->nby * p->h1c * csz);
    SFFT_ALLOC(p->F, (size_t)(p->nfy + 1) * half * csz);
    // the column spectra (power-of-two n0); the subtraction reuses U for D~
    SFFT_ALLOC(p->U, (size_t)(p->gen0 ? 1 : p->nimg) * half * csz);
    SFFT_ALLOC(p->kimg, (size_t)p->L0 * p->L1 * sizeof(double));
    if (p->gen0) {
        SFFT_ALLOC(p->chirp0, (size_t)p->n0 * csz);
        SFFT_ALLOC(p->bfilt0, (size_t)p->m0 * csz);
        SFFT_ALLOC(p->twpm0, (size_t)p->m0 * csz);
    }
    if (p->gen1) {
        SFFT_ALLOC(p->chirp1, (size_t)p->n1 * csz);
        SFFT_ALLOC(p->bfilt1, (size_t)p->m1 * csz);
        SFFT_ALLOC(p->twpm1, (size_t)p->m1 * csz);
    }
    SFFT_ALLOC(p->Q, (size_t)p->nrows * p->h1c * csz);
    SFFT_ALLOC(p->pairs, (size_t)(np + p->ngpairs) * sizeof(PairDesc));
    p->gpairs = p->pairs + np;
    SFFT_ALLOC(p->rowmom, (size_t)p->n0 * p->nmom * sizeof(double));
    SFFT_ALLOC(p->lag, nlag * sizeof(double));
    SFFT_ALLOC(p->A, n * n * rsz);
    SFFT_ALLOC(p->Wm, n * n * rsz);
    p->solve_grid = solve_grid_size(p->fp64);
    p->solve_grid_tc = p->fp64 ? 0 : solve_grid_size(false, true);
    if (p->solve_grid <= 0 || p->solve_grid > kMaxSolveGrid) {
        plan_free(p);
        return SFFT_ERR_CUDA;
    }
    SFFT_ALLOC(p->dscale, n * sizeof(double));
    SFFT_ALLOC(p->r, n * sizeof(double));
    SFFT_ALLOC(p->xw, (n + kSolveTail + 64) * sizeof(double));  // x, stats, per-block partials, kernel sums
    SFFT_ALLOC(p->zv, solve_vec_elems((int)n) * rsz);
    SFFT_ALLOC(p->flag, 4 * sizeof(int));
    SFFT_ALLOC(p->M_own, n * n * sizeof(double));
    SFFT_ALLOC(p->rhs_own, n * sizeof(double));
    SFFT_ALLOC(p->x_own, n * sizeof(double));
    SFFT_ALLOC(p->info_own, sizeof(sfft_solve_info));
    SFFT_ALLOC(p->kap, (size_t)p->nk * p->L0 * p->h1c * csz);

    // constant tables
    cudaError_t err;
    if ((err = cudaMemcpyAsync(p->pairs, p->host_pairs, (np + p->ngpairs) * sizeof(PairDesc), cudaMemcpyHostToDevice,
                               s))) {
        plan_free(p);
        return SFFT_ERR_CUDA;
    }
    cpx<double> *t64a = nullptr, *t64b = nullptr;
    if (cudaMalloc((void **)&t64a, p->n0 * sizeof(cpx<double>)) != cudaSuccess ||
        cudaMalloc((void **)&t64b, p->n1 * sizeof(cpx<double>)) != cudaSuccess) {
        cudaGetLastError();
        if (t64a) cudaFree(t64a);
        plan_free(p);
        return SFFT_ERR_OOM;
    }
    k_twiddle64<<<(p->n0 + 255) / 256, 256, 0, s>>>(p->n0, t64a);
    k_twiddle64<<<(p->n1 + 255) / 256, 256, 0, s>>>(p->n1, t64b);
    const int bx = (p->nbx * p->n0 + 127) / 128, by = (p->nby * p->h1c + 127) / 128;
    // the tabulated background functions (FP64)
    const double *tbx = p->bxy64, *tby = p->bxy64 + (size_t)p->nbx * p->n0;
    if (p->fp64) {
        k_round<double><<<(p->n0 + 255) / 256, 256, 0, s>>>(p->n0, t64a, (cpx<double> *)p->tw0);
        k_round<double><<<(p->n1 + 255) / 256, 256, 0, s>>>(p->n1, t64b, (cpx<double> *)p->tw1);
        if (!p->gen0) pass_tables<double>(p->n0, t64a, (cpx<double> *)p->twp0, s);
        if (!p->gen1) pass_tables<double>(p->n1, t64b, (cpx<double> *)p->twp1, s);
        if (p->xhat)
            k_poly_dft<double><<<bx, 128, 0, s>>>(p->n0, p->n0, p->nbx, t64a, p->na, p->nbk, 1, tbx,
                                                  (cpx<double> *)p->xhat);
        k_poly_dft<double><<<by, 128, 0, s>>>(p->n1, p->h1c, p->nby, t64b, 0, 1, 0, tby, (cpx<double> *)p->yhat);
    } else {
        k_round<float><<<(p->n0 + 255) / 256, 256, 0, s>>>(p->n0, t64a, (cpx<float> *)p->tw0);
        k_round<float><<<(p->n1 + 255) / 256, 256, 0, s>>>(p->n1, t64b, (cpx<float> *)p->tw1);
        if (!p->gen0) pass_tables<float>(p->n0, t64a, (cpx<float> *)p->twp0, s);
        if (!p->gen1) pass_tables<float>(p->n1, t64b, (cpx<float> *)p->twp1, s);
        if (p->xhat)
            k_poly_dft<float><<<bx, 128, 0, s>>>(p->n0, p->n0, p->nbx, t64a, p->na, p->nbk, 1, tbx,
                                                 (cpx<float> *)p->xhat);
        k_poly_dft<float><<<by, 128, 0, s>>>(p->n1, p->h1c, p->nby, t64b, 0, 1, 0, tby, (cpx<float> *)p->yhat);
    }
    for (int ax = 0; ax < 2; ++ax) {  // Bluestein tables of the axes that are not powers of two
        const bool gen = ax == 0 ? p->gen0 : p->gen1;
        if (!gen) continue;
        const int nn = ax == 0 ? p->n0 : p->n1, mm = ax == 0 ? p->m0 : p->m1;
        void *chirp = ax == 0 ? p->chirp0 : p->chirp1, *bfilt = ax == 0 ? p->bfilt0 : p->bfilt1;
        void *twpm = ax == 0 ? p->twpm0 : p->twpm1;
        cpx<double> *tm64 = nullptr, *c64 = nullptr;
        if (cudaMalloc((void **)&tm64, mm * sizeof(cpx<double>)) != cudaSuccess ||
            cudaMalloc((void **)&c64, nn * sizeof(cpx<double>)) != cudaSuccess) {
            cudaGetLastError();
            if (tm64) cudaFree(tm64);
            cudaFree(t64a);
            cudaFree(t64b);
            plan_free(p);
            return SFFT_ERR_OOM;
        }
        k_twiddle64<<<(mm + 255) / 256, 256, 0, s>>>(mm, tm64);
        k_chirp64<<<(nn + 255) / 256, 256, 0, s>>>(nn, c64);
        if (p->fp64) {
            k_round<double><<<(nn + 255) / 256, 256, 0, s>>>(nn, c64, (cpx<double> *)chirp);
            k_bfilt<double><<<(mm + 127) / 128, 128, 0, s>>>(nn, mm, tm64, c64, (cpx<double> *)bfilt);
            pass_tables<double>(mm, tm64, (cpx<double> *)twpm, s);
        } else {
            k_round<float><<<(nn + 255) / 256, 256, 0, s>>>(nn, c64, (cpx<float> *)chirp);
            k_bfilt<float><<<(mm + 127) / 128, 128, 0, s>>>(nn, mm, tm64, c64, (cpx<float> *)bfilt);
            pass_tables<float>(mm, tm64, (cpx<float> *)twpm, s);
        }
        cudaStreamSynchronize(s);
        cudaFree(tm64);
        cudaFree(c64);
    }
    err = cudaGetLastError();
    cudaStreamSynchronize(s);
    cudaFree(t64a);
    cudaFree(t64b);
    if (err != cudaSuccess) {
        plan_free(p);
        return SFFT_ERR_CUDA;
    }
    tune_lookup(p);
    *out = p;
    return SFFT_OK;
}

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return SFFT_OK;
    if (e == cudaErrorMemoryAllocation) return SFFT_ERR_OOM;
    return SFFT_ERR_CUDA;
}

static size_t img_bytes(const Plan *p) {
    return (size_t)p->n0 * p->n1 * (p->cfg.dtype == SFFT_F64 ? sizeof(double) : sizeof(float));
}

static int run_pair(Plan *p, const void *ref, const void *sci, const uint8_t *mask, double *M, double *rhs,
                    double *x, sfft_solve_info *info, void *diff, cudaStream_t s) {
    if (!M) M = p->M_own;
    if (!rhs) rhs = p->rhs_own;
    if (!x) x = p->x_own;
    if (!info) info = p->info_own;
    p->last_ref = ref;
    p->last_sci = sci;
    p->last_mask = mask;
    p->last_M = M;
    p->last_rhs = rhs;
    p->last_x = x;
    p->last_info = info;
    p->last_diff = diff;
    cudaError_t e = build_system(p, ref, sci, mask, M, rhs, s);
    if (e == cudaSuccess) e = solve_system(p, M, rhs, x, info, s);
    if (e == cudaSuccess && mask) e = row_transform(p, ref, sci, nullptr, false, s);
    if (e == cudaSuccess) e = subtract_from_rows(p, x, diff, s);
    p->last_stream = s;
    return status_of(e);
}

}  // namespace sfft

using namespace sfft;

extern "C" {

const char *sfft_status_string(int status) {
    switch (status) {
        case SFFT_OK: return "ok";
        case SFFT_ERR_INVALID: return "invalid argument";
        case SFFT_ERR_OOM: return "out of memory";
        case SFFT_ERR_CUDA: return "CUDA error";
        case SFFT_ERR_SINGULAR: return "normal matrix not positive definite";
        case SFFT_ERR_NOT_CONVERGED: return "iterative refinement did not converge";
        case SFFT_ERR_TIMEOUT: return "timed out";
        case SFFT_ERR_BUSY: return "busy";
        case SFFT_ERR_UNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

int sfft_num_unknowns(const sfft_config *cfg, int32_t *n) {
    if (!cfg || !n) return SFFT_ERR_INVALID;
    if (cfg->w0 < 0 || cfg->w1 < 0) return SFFT_ERR_INVALID;
    const int v = basis_validate(cfg);
    if (v == SFFT_ERR_INVALID) return v;
    *n = basis_unknowns(cfg);
    return SFFT_OK;
}

int sfft_plan_create(const sfft_config *cfg, sfft_stream_t stream, sfft_plan_t *out) {
    if (!out) return SFFT_ERR_INVALID;
    *out = nullptr;
    int v = plan_validate(cfg);
    if (v) return v;
    Plan *p = nullptr;
    int rc = plan_new(cfg, (cudaStream_t)stream, &p);
    if (rc == SFFT_OK) *out = (sfft_plan_t)p;
    return rc;
}

int sfft_plan_destroy(sfft_plan_t plan) {
    if (!plan) return SFFT_OK;
    Plan *p = (Plan *)plan;
    // the streams the plan last ran on may have been destroyed since
    cudaDeviceSynchronize();
    plan_free(p);
    return SFFT_OK;
}

int sfft_plan_set_solve_panel(sfft_plan_t plan, int32_t width) {
    if (!plan || (width != 32 && width != 64)) return SFFT_ERR_INVALID;
    ((Plan *)plan)->solve_panel = width;
    return SFFT_OK;
}

int sfft_plan_solve_panel(sfft_plan_t plan, int32_t *width) {
    if (!plan || !width) return SFFT_ERR_INVALID;
    *width = ((Plan *)plan)->solve_panel;
    return SFFT_OK;
}

int sfft_plan_workspace_bytes(sfft_plan_t plan, uint64_t *bytes) {
    if (!plan || !bytes) return SFFT_ERR_INVALID;
    *bytes = ((Plan *)plan)->ws_bytes;
    return SFFT_OK;
}

int sfft_plan_launch_count(sfft_plan_t plan, uint64_t *count) {
    if (!plan || !count) return SFFT_ERR_INVALID;
    *count = ((Plan *)plan)->launches;
    return SFFT_OK;
}

int sfft_replay_stage(sfft_plan_t plan, int stage, sfft_stream_t stream) {
    if (!plan) return SFFT_ERR_INVALID;
    Plan *p = (Plan *)plan;
    if (!p->last_ref || !p->last_diff) return SFFT_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    cudaError_t e;
    switch (stage) {
        case SFFT_STAGE_ROWS: e = row_transform(p, p->last_ref, p->last_sci, p->last_mask, true, s); break;
        case SFFT_STAGE_COLS:
        case SFFT_STAGE_GATHER:
        case SFFT_STAGE_LAGS: e = build_stage(p, stage, p->last_M, p->last_rhs, s); break;
        case SFFT_STAGE_SOLVE: e = solve_system(p, p->last_M, p->last_rhs, p->last_x, p->last_info, s); break;
        case SFFT_STAGE_SUBTRACT:  // as in sfft_run_pair: unmasked row FFTs only after a masked build
            e = p->last_mask ? row_transform(p, p->last_ref, p->last_sci, nullptr, false, s) : cudaSuccess;
            if (e == cudaSuccess) e = subtract_from_rows(p, p->last_x, p->last_diff, s);
            break;
        default: return SFFT_ERR_INVALID;
    }
    return status_of(e);
}

int sfft_build_system(sfft_plan_t plan, const void *d_ref, const void *d_sci, const uint8_t *d_mask,
                      double *d_M, double *d_rhs, sfft_stream_t stream) {
    if (!plan || !d_ref || !d_sci || !d_M || !d_rhs) return SFFT_ERR_INVALID;
    if (!images_aligned(d_ref, d_sci, d_mask)) return SFFT_ERR_INVALID;
    Plan *p = (Plan *)plan;
    p->last_stream = (cudaStream_t)stream;
    return status_of(build_system(p, d_ref, d_sci, d_mask, d_M, d_rhs, (cudaStream_t)stream));
}

int sfft_solve(sfft_plan_t plan, const double *d_M, const double *d_rhs, double *d_x, sfft_solve_info *d_info,
               sfft_stream_t stream) {
    if (!plan || !d_M || !d_rhs || !d_x) return SFFT_ERR_INVALID;
    Plan *p = (Plan *)plan;
    p->last_stream = (cudaStream_t)stream;
    return status_of(solve_system(p, d_M, d_rhs, d_x, d_info, (cudaStream_t)stream));
}

int sfft_solve_batch(const sfft_plan_t *plans, int32_t count, const double *const *d_M,
                     const double *const *d_rhs, double *const *d_x, sfft_solve_info *const *d_info,
                     sfft_stream_t stream) {
    if (!plans || count < 1 || count > kMaxSolveBatch || !d_M || !d_rhs || !d_x) return SFFT_ERR_INVALID;
    Plan *ps[kMaxSolveBatch];
    sfft_solve_info *inf[kMaxSolveBatch];
    for (int i = 0; i < count; ++i) {  // pointers only: no plan is read before all pass
        if (!plans[i] || !d_M[i] || !d_rhs[i] || !d_x[i]) return SFFT_ERR_INVALID;
        ps[i] = (Plan *)plans[i];
        inf[i] = d_info ? d_info[i] : nullptr;
        for (int k = 0; k < i; ++k)
            if (ps[k] == ps[i]) return SFFT_ERR_INVALID;  // one workspace per system
    }
    for (int i = 1; i < count; ++i)
        if (ps[i]->fp64 != ps[0]->fp64 || (!ps[0]->fp64 && ps[i]->solve_panel != ps[0]->solve_panel))
            return SFFT_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) ps[i]->last_stream = s;
    return status_of(solve_batch(ps, count, d_M, d_rhs, d_x, inf, s));
}

int sfft_subtract(sfft_plan_t plan, const void *d_ref, const void *d_sci, const double *d_x, void *d_diff,
                  sfft_stream_t stream) {
    if (!plan || !d_ref || !d_sci || !d_x || !d_diff) return SFFT_ERR_INVALID;
    if (d_diff == d_ref || d_diff == d_sci) return SFFT_ERR_INVALID;
    if (!images_aligned(d_ref, d_sci, nullptr)) return SFFT_ERR_INVALID;
    Plan *p = (Plan *)plan;
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    cudaError_t e = row_transform(p, d_ref, d_sci, nullptr, false, s);
    if (e == cudaSuccess) e = subtract_from_rows(p, d_x, d_diff, s);
    return status_of(e);
}

int sfft_plan_autotune(sfft_plan_t plan, const void *d_ref, const void *d_sci, void *d_diff,
                       sfft_stream_t stream) {
    if (!plan || !d_ref || !d_sci || !d_diff) return SFFT_ERR_INVALID;
    if (d_diff == d_ref || d_diff == d_sci) return SFFT_ERR_INVALID;
    if (!images_aligned(d_ref, d_sci, nullptr)) return SFFT_ERR_INVALID;
    Plan *p = (Plan *)plan;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = run_pair(p, d_ref, d_sci, nullptr, nullptr, nullptr, nullptr, nullptr, d_diff, s);
    if (rc != SFFT_OK) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SFFT_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SFFT_ERR_CUDA;
    }
    // time one stage (one warm-up, then 5 replays) with the plan's current shapes
    auto time_stage = [&](int stage, float *ms) -> int {
        int r = sfft_replay_stage(plan, stage, stream);
        if (r != SFFT_OK) return r;
        cudaEventRecord(e0, s);
        for (int k = 0; k < 5 && r == SFFT_OK; ++k) r = sfft_replay_stage(plan, stage, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return SFFT_ERR_CUDA;
        cudaEventElapsedTime(ms, e0, e1);
        return r;
    };
    struct Knob {
        int *field;
        int stage;
        int cand[5];
    } knobs[] = {
        {&p->tune_tr, SFFT_STAGE_ROWS, {0, 4, 2, 1, -1}},
        {&p->tune_gi, SFFT_STAGE_COLS, {0, 3, 2, 1, -1}},
        {&p->tune_ng, SFFT_STAGE_SUBTRACT, {0, 2, 1, -1, -1}},
    };
    // (the tensor-core tile products of the solve, tune_tc, are not chosen
    // here: they round differently, and tuning must not change results)
    // The solve grid is not tuned here: a single system's time does not
    // predict the batched solves of the serving path (sfft_plan_set_tuning
    // sets it by hand).
    for (Knob &kb : knobs) {
        if (kb.stage == SFFT_STAGE_COLS && p->gen0) continue;  // no column FFT
        int best = 0;
        float best_ms = 1e30f;
        for (int c : kb.cand) {
            if (c < 0) continue;
            *kb.field = c;
            float ms = 0.f;
            rc = time_stage(kb.stage, &ms);
            if (rc != SFFT_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        *kb.field = best;
        if (rc != SFFT_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == SFFT_OK) tune_store(p);
    return rc;
}

int sfft_plan_tuning(sfft_plan_t plan, int32_t *shapes) {
    if (!plan || !shapes) return SFFT_ERR_INVALID;
    get_shapes((const Plan *)plan, shapes);
    return SFFT_OK;
}

int sfft_plan_set_tuning(sfft_plan_t plan, const int32_t *shapes) {
    if (!plan || !shapes) return SFFT_ERR_INVALID;
    const int32_t tr = shapes[0];
    if (tr < 0 || tr > 16 || (tr & (tr - 1)) != 0) return SFFT_ERR_INVALID;  // 0 or a power of two
    if (shapes[1] < 0 || shapes[1] > 4 || shapes[2] < 0 || shapes[2] > 4) return SFFT_ERR_INVALID;
    if (shapes[3] < 0 || shapes[3] > kMaxSolveGrid) return SFFT_ERR_INVALID;
    if (shapes[4] < 0 || shapes[4] > 2) return SFFT_ERR_INVALID;
    set_shapes((Plan *)plan, shapes);
    tune_store((Plan *)plan);  // later plans of this configuration start with them
    return SFFT_OK;
}

int sfft_decorrelate(sfft_plan_t plan, const double *d_x, double xt0, double yt0, double sigma_ref,
                     double sigma_sci, const void *d_diff, void *d_out, sfft_stream_t stream) {
    if (!plan || !d_x || !d_diff || !d_out) return SFFT_ERR_INVALID;
    if (!(sigma_sci > 0.0) || !(sigma_ref >= 0.0)) return SFFT_ERR_INVALID;
    if (!(xt0 >= -1.0 && xt0 <= 1.0) || !(yt0 >= -1.0 && yt0 <= 1.0)) return SFFT_ERR_INVALID;
    Plan *p = (Plan *)plan;
    p->last_stream = (cudaStream_t)stream;
    return status_of(
        decorrelate(p, d_x, xt0, yt0, sigma_ref, sigma_sci, d_diff, d_out, nullptr, (cudaStream_t)stream));
}

int sfft_decorrelate_coadd(sfft_plan_t plan, const double *d_x, double xt0, double yt0, int32_t n_sci,
                           const double *d_G, const double *h_sigma_sci, int32_t n_ref, const double *d_H,
                           const double *h_sigma_ref, int32_t g0, int32_t g1, const void *d_diff, void *d_out,
                           sfft_stream_t stream) {
    if (!plan || !d_x || !d_diff || !d_out || !d_G || !d_H || !h_sigma_sci || !h_sigma_ref) return SFFT_ERR_INVALID;
    if (!(xt0 >= -1.0 && xt0 <= 1.0) || !(yt0 >= -1.0 && yt0 <= 1.0)) return SFFT_ERR_INVALID;
    if (n_sci < 1 || n_ref < 1 || n_sci > kMaxCoadd || n_ref > kMaxCoadd) return SFFT_ERR_INVALID;
    Plan *p = (Plan *)plan;
    if (g0 < 0 || g1 < 0 || g0 > 32 || g1 > 32 || 2 * g0 + 1 > p->n0 || 2 * g1 + 1 > p->n1) return SFFT_ERR_INVALID;
    Coadd co{};
    co.ns = n_sci;
    co.nr = n_ref;
    co.g0 = g0;
    co.g1 = g1;
    co.G = d_G;
    co.H = d_H;
    double ssum = 0.0;
    for (int j = 0; j < n_sci; ++j) {
        if (!(h_sigma_sci[j] >= 0.0)) return SFFT_ERR_INVALID;
        co.sigma2[j] = h_sigma_sci[j] * h_sigma_sci[j];
        ssum += co.sigma2[j];
    }
    for (int i = 0; i < n_ref; ++i) {
        if (!(h_sigma_ref[i] >= 0.0)) return SFFT_ERR_INVALID;
        co.sigma2[n_sci + i] = h_sigma_ref[i] * h_sigma_ref[i];
    }
    if (!(ssum > 0.0)) return SFFT_ERR_INVALID;
    const size_t need = (size_t)(n_sci + n_ref) * (2 * g0 + 1) * p->h1c * p->csz;
    if (need > p->gam_bytes) {  // plan-owned table, grown on demand
        if (p->gam) cudaFree(p->gam);
        p->gam = nullptr;
        p->gam_bytes = 0;
        if (cudaMalloc(&p->gam, need) != cudaSuccess) {
            cudaGetLastError();
            return SFFT_ERR_OOM;
        }
        p->gam_bytes = need;
    }
    p->last_stream = (cudaStream_t)stream;
    return status_of(decorrelate(p, d_x, xt0, yt0, 0.0, 1.0, d_diff, d_out, &co, (cudaStream_t)stream));
}

int sfft_run_pair(sfft_plan_t plan, const void *d_ref, const void *d_sci, const uint8_t *d_mask, double *d_M,
                  double *d_rhs, double *d_x, sfft_solve_info *d_info, void *d_diff, sfft_stream_t stream) {
    if (!plan || !d_ref || !d_sci || !d_diff) return SFFT_ERR_INVALID;
    if (d_diff == d_ref || d_diff == d_sci) return SFFT_ERR_INVALID;
    if (!images_aligned(d_ref, d_sci, d_mask)) return SFFT_ERR_INVALID;
    return run_pair((Plan *)plan, d_ref, d_sci, d_mask, d_M, d_rhs, d_x, d_info, d_diff, (cudaStream_t)stream);
}

namespace {

// Host-side checks of a set of pairs (sfft_run_pairs, sfft_batch_create).
int check_pairs(const sfft_plan_t *plans, int32_t count, const void *const *d_refs, const void *const *d_scis,
                const uint8_t *const *d_masks, void *const *d_diffs) {
    if (!plans || count < 1 || !d_refs || !d_scis || !d_diffs) return SFFT_ERR_INVALID;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !d_refs[i] || !d_scis[i] || !d_diffs[i]) return SFFT_ERR_INVALID;
        if (d_diffs[i] == d_refs[i] || d_diffs[i] == d_scis[i]) return SFFT_ERR_INVALID;
        if (!images_aligned(d_refs[i], d_scis[i], d_masks ? d_masks[i] : nullptr)) return SFFT_ERR_INVALID;
        if (((Plan *)plans[i])->fp64 != ((Plan *)plans[0])->fp64) return SFFT_ERR_INVALID;
        if (!((Plan *)plans[0])->fp64 && ((Plan *)plans[i])->solve_panel != ((Plan *)plans[0])->solve_panel)
            return SFFT_ERR_INVALID;  // one solve kernel per launch
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return SFFT_ERR_INVALID;  // one workspace per pair
    }
    return SFFT_OK;
}

// Enqueue the pairs on s: every build, the systems solved `group` (1..8) per
// launch, largest first, then every subtraction.
cudaError_t enqueue_pairs(const sfft_plan_t *plans, int32_t count, const void *const *d_refs,
                          const void *const *d_scis, const uint8_t *const *d_masks, double *const *d_xs,
                          sfft_solve_info *const *d_infos, void *const *d_diffs, int group, cudaStream_t s);

}  // namespace

int sfft_run_pairs(const sfft_plan_t *plans, int32_t count, const void *const *d_refs, const void *const *d_scis,
                   const uint8_t *const *d_masks, double *const *d_xs, sfft_solve_info *const *d_infos,
                   void *const *d_diffs, sfft_stream_t stream) {
    const int rc = check_pairs(plans, count, d_refs, d_scis, d_masks, d_diffs);
    if (rc != SFFT_OK) return rc;
    return status_of(enqueue_pairs(plans, count, d_refs, d_scis, d_masks, d_xs, d_infos, d_diffs, kMaxSolveBatch,
                                   (cudaStream_t)stream));
}

namespace {

cudaError_t enqueue_pairs(const sfft_plan_t *plans, int32_t count, const void *const *d_refs,
                          const void *const *d_scis, const uint8_t *const *d_masks, double *const *d_xs,
                          sfft_solve_info *const *d_infos, void *const *d_diffs, int group, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        Plan *p = (Plan *)plans[i];
        p->last_ref = d_refs[i];
        p->last_sci = d_scis[i];
        p->last_mask = d_masks ? d_masks[i] : nullptr;
        p->last_M = p->M_own;
        p->last_rhs = p->rhs_own;
        p->last_x = (d_xs && d_xs[i]) ? d_xs[i] : p->x_own;
        p->last_info = (d_infos && d_infos[i]) ? d_infos[i] : p->info_own;
        p->last_diff = d_diffs[i];
        p->last_stream = s;
        e = build_system(p, p->last_ref, p->last_sci, p->last_mask, p->M_own, p->rhs_own, s);
    }
    // A launch lasts as long as its largest system: group the systems by
    // size, largest first (the order of the systems in a launch does not
    // change their results).
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return ((Plan *)plans[a])->n > ((Plan *)plans[b])->n; });
    for (int g = 0; g < count && e == cudaSuccess; g += group) {
        const int cnt = count - g < group ? count - g : group;
        Plan *ps[kMaxSolveBatch];
        const double *M[kMaxSolveBatch], *rhs[kMaxSolveBatch];
        double *x[kMaxSolveBatch];
        sfft_solve_info *info[kMaxSolveBatch];
        for (int b = 0; b < cnt; ++b) {
            ps[b] = (Plan *)plans[order[g + b]];
            M[b] = ps[b]->last_M;
            rhs[b] = ps[b]->last_rhs;
            x[b] = ps[b]->last_x;
            info[b] = ps[b]->last_info;
        }
        e = solve_batch(ps, cnt, M, rhs, x, info, s);
    }
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        Plan *p = (Plan *)plans[i];
        if (p->last_mask) e = row_transform(p, p->last_ref, p->last_sci, nullptr, false, s);
        if (e == cudaSuccess) e = subtract_from_rows(p, p->last_x, p->last_diff, s);
    }
    return e;
}

}  // namespace

// ---- a batch of pairs captured once into a CUDA graph -------------------------

struct sfft_batch_s {
    cudaGraphExec_t exec = nullptr;
    int count = 0, group = 0, launches = 0;
    float tune_ms[4] = {0, 0, 0, 0};  // replay time of groups 8, 4, 2, 1 (autotune only)
};

namespace {

// Capture the batch with solve groups of `group` on a private stream.
cudaError_t capture_batch(const sfft_plan_t *plans, int32_t count, const void *const *d_refs,
                          const void *const *d_scis, const uint8_t *const *d_masks, double *const *d_xs,
                          sfft_solve_info *const *d_infos, void *const *d_diffs, int group, cudaStream_t cs,
                          cudaGraphExec_t *exec, int *launches) {
    uint64_t l0 = 0, l1 = 0;
    for (int i = 0; i < count; ++i) l0 += ((Plan *)plans[i])->launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t ee = enqueue_pairs(plans, count, d_refs, d_scis, d_masks, d_xs, d_infos, d_diffs, group, cs);
    e = cudaStreamEndCapture(cs, &graph);
    if (ee != cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    for (int i = 0; i < count; ++i) l1 += ((Plan *)plans[i])->launches;
    *launches = (int)(l1 - l0);
    return e;
}

}  // namespace

int sfft_batch_create(const sfft_plan_t *plans, int32_t count, const void *const *d_refs, const void *const *d_scis,
                      const uint8_t *const *d_masks, double *const *d_xs, sfft_solve_info *const *d_infos,
                      void *const *d_diffs, int32_t solve_group, sfft_batch_t *out) {
    if (!out) return SFFT_ERR_INVALID;
    *out = nullptr;
    if (solve_group < 0 || solve_group > kMaxSolveBatch) return SFFT_ERR_INVALID;
    const int rc = check_pairs(plans, count, d_refs, d_scis, d_masks, d_diffs);
    if (rc != SFFT_OK) return rc;
    sfft_batch_s *b = new (std::nothrow) sfft_batch_s();
    if (!b) return SFFT_ERR_OOM;
    b->count = count;
    // the capture runs on a stream of its own, destroyed below: the plans
    // keep the stream they last ran on
    std::vector<cudaStream_t> prev(count);
    for (int i = 0; i < count; ++i) prev[i] = ((Plan *)plans[i])->last_stream;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess && solve_group > 0) {
        b->group = solve_group;
        e = capture_batch(plans, count, d_refs, d_scis, d_masks, d_xs, d_infos, d_diffs, solve_group, cs, &b->exec,
                          &b->launches);
    } else if (e == cudaSuccess) {
        // autotune: capture with solve groups of 8, 4, 2 and 1, replay each
        // (after one untimed replay) three times on the caller's data and
        // keep the fastest; the results do not depend on the grouping
        const int groups[4] = {8, 4, 2, 1};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        float best = 0.f;
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            cudaGraphExec_t ex = nullptr;
            int nl = 0;
            e = capture_batch(plans, count, d_refs, d_scis, d_masks, d_xs, d_infos, d_diffs, groups[k], cs, &ex, &nl);
            if (e == cudaSuccess) e = cudaGraphLaunch(ex, cs);
            if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = cudaGraphLaunch(ex, cs);
            if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                if (ex) cudaGraphExecDestroy(ex);
                break;
            }
            b->tune_ms[k] = ms / 3.f;
            if (!b->exec || ms < best) {
                if (b->exec) cudaGraphExecDestroy(b->exec);
                b->exec = ex;
                b->group = groups[k];
                b->launches = nl;
                best = ms;
            } else {
                cudaGraphExecDestroy(ex);
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
    if (cs) {
        const cudaError_t es = cudaStreamSynchronize(cs);
        if (e == cudaSuccess) e = es;
        cudaStreamDestroy(cs);
    }
    for (int i = 0; i < count; ++i) ((Plan *)plans[i])->last_stream = prev[i];
    if (e != cudaSuccess) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        delete b;
        return status_of(e);
    }
    *out = b;
    return SFFT_OK;
}

int sfft_batch_launch(sfft_batch_t batch, sfft_stream_t stream) {
    if (!batch) return SFFT_ERR_INVALID;
    return status_of(cudaGraphLaunch(batch->exec, (cudaStream_t)stream));
}

int sfft_batch_info(sfft_batch_t batch, int32_t *solve_group, int32_t *launches, float *tune_ms4) {
    if (!batch) return SFFT_ERR_INVALID;
    if (solve_group) *solve_group = batch->group;
    if (launches) *launches = batch->launches;
    if (tune_ms4)
        for (int k = 0; k < 4; ++k) tune_ms4[k] = batch->tune_ms[k];
    return SFFT_OK;
}

int sfft_batch_destroy(sfft_batch_t batch) {
    if (!batch) return SFFT_OK;
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    delete batch;
    return SFFT_OK;
}

int sfft_run_pair_host(sfft_plan_t plan, const void *h_ref, const void *h_sci, const uint8_t *h_mask,
                       double *h_x, sfft_solve_info *h_info, void *h_diff, sfft_stream_t stream) {
    if (!plan || !h_ref || !h_sci || !h_diff) return SFFT_ERR_INVALID;
    Plan *p = (Plan *)plan;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ib = img_bytes(p);
    const size_t P = (size_t)p->n0 * p->n1;
    if (!p->img_ref) {
        if (cudaMalloc(&p->img_ref, ib) != cudaSuccess || cudaMalloc(&p->img_sci, ib) != cudaSuccess ||
            cudaMalloc(&p->img_diff, ib) != cudaSuccess || cudaMalloc((void **)&p->img_mask, P) != cudaSuccess) {
            cudaGetLastError();
            return SFFT_ERR_OOM;
        }
        p->ws_bytes += 3 * ib + P;
    }
    cudaError_t e = cudaMemcpyAsync(p->img_ref, h_ref, ib, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->img_sci, h_sci, ib, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && h_mask) e = cudaMemcpyAsync(p->img_mask, h_mask, P, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return status_of(e);
    int rc = run_pair(p, p->img_ref, p->img_sci, h_mask ? p->img_mask : nullptr, nullptr, nullptr, nullptr,
                      nullptr, p->img_diff, s);
    if (rc) return rc;
    e = cudaMemcpyAsync(h_diff, p->img_diff, ib, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_x) e = cudaMemcpyAsync(h_x, p->x_own, p->n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_info)
        e = cudaMemcpyAsync(h_info, p->info_own, sizeof(sfft_solve_info), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return status_of(e);
}

}  // extern "C"
