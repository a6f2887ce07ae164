/*
 * sfft_oracle.c -- plain, slow FP64 CPU oracle for the SFFT hot path
 * (Hu et al., "Image Subtraction in Fourier Space", arXiv:2109.09334).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU library never
 * links or calls it, and it shares no code, header or table with the GPU path.
 *
 * What it computes (all in real-space units, double precision):
 *   - the delta-function-basis least-squares system of Eq. 18, with the block
 *     entries of Eq. 19-24 expressed through the lag tables of App. B
 *     (Eq. B5-B16), each lag value evaluated by a direct circular spatial sum
 *     (no FFT anywhere in this file);
 *   - its solution by a hand-written Cholesky factorisation;
 *   - the difference image of Eq. 12 by a literal circular convolution.
 *
 * Readings of the paper this file adopts (each is listed in the design notes):
 *   - Eq. 12 is a circular convolution; every shift wraps mod N0, N1.
 *   - x is axis 0 (rows, length N0), y is axis 1 (length N1), row-major.
 *   - Polynomial coordinates are normalised: xt = (2x - (N0-1)) / (N0-1),
 *     likewise yt; this is the same polynomial space as Eq. 2 / Eq. 6.
 *   - Unknowns are in real-space units (a-ring of Eq. 6); Eq. 13's
 *     a = N0*N1*a-ring is a uniform rescaling and is not applied.
 *   - Omega(rho) = sum_x g_row(x) g_col(x + rho)   (Eq. B6 read in real space),
 *     Lambda(rho) = sum_x g_row(x) T(x + rho)      (Eq. B8),
 *     Theta(rho)  = sum_x g_row(x) S(x + rho)      (Eq. B14 read via Eq. 23),
 *     C = sum_x T T (Eq. B11), E = sum_x T S (Eq. B15 read via Eq. 24).
 *   - Optional mask: the system is built from R*m and S*m (zero fill); the
 *     subtraction uses the unmasked R and S (two-step process of Sec. 3).
 *   - Unknown order: kernel block first, terms (i,j) by total degree then
 *     descending i; within a term, offsets (alpha,beta) row-major with alpha
 *     from -w0 to w0 outer; with a constant photometric ratio the offsets
 *     (alpha,beta)=(0,0) of terms other than (0,0) are omitted; then the
 *     background terms (p,q) in the same monomial order.
 *   - B-spline bases (Eq. 7-9): the same basis along x and y, on the
 *     normalised coordinates, clamped uniform knots on [-1, 1] (degree k,
 *     n_int interior knots, K = n_int + k + 1 functions, evaluated by the
 *     Cox-de Boor recursion; the right end x = 1 belongs to the last knot
 *     span).  Kernel terms (i, j), i, j < K, ordered i outer, weight
 *     B_i(xt) B_j(yt); background terms (p, q) likewise with their own degree
 *     and knots.  With a constant photometric ratio the (0,0) offset of the
 *     kernel has one unknown whose weight is 1 (the sum of all B_i B_j), put
 *     first as term 0; the spline terms then omit that offset.
 *
 * Pins (tests, on the CPU): brute-force design matrix and least squares on
 * tiny images, the closed-form w=0 regression, the one-pixel shift case,
 * exact recovery of an injected kernel/scale/background, symmetry, positive
 * semidefiniteness, structural zeros, Toeplitz structure, flux conservation
 * and a frequency-domain evaluation of Eq. 19-24.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_NOMEM (-2)
#define ORC_ERR_NOT_PD (-4)

/* Configuration as passed in by the caller: 12 ints
 *   n0, n1, w0, w1, dk, db, cpr, basis (0 polynomial, 1 B-spline),
 *   kdeg, kint (kernel spline degree, interior knots),
 *   bdeg, bint (background spline degree, interior knots). */
#define ORC_CFG_LEN 12

typedef struct {
    int n0, n1, w0, w1, dk, db, cpr;
    int basis, kdeg, kint, bdeg, bint;
} orc_cfg;

static orc_cfg cfg_from(const int *v) {
    orc_cfg c;
    c.n0 = v[0]; c.n1 = v[1]; c.w0 = v[2]; c.w1 = v[3]; c.dk = v[4]; c.db = v[5];
    c.cpr = v[6] ? 1 : 0; c.basis = v[7]; c.kdeg = v[8]; c.kint = v[9]; c.bdeg = v[10]; c.bint = v[11];
    return c;
}

/* ---- indexing ---------------------------------------------------------- */

static int n_terms(int d) { return (d + 1) * (d + 2) / 2; }

/* number of B-spline functions per axis */
static int n_spl(int deg, int nint) { return nint + deg + 1; }

/* kernel terms: polynomial terms, or the B-spline products (plus the constant
 * term 0 when the photometric ratio is constant) */
static int kernel_terms(const orc_cfg *c) {
    if (c->basis == 0) return n_terms(c->dk);
    int K = n_spl(c->kdeg, c->kint);
    return K * K + (c->cpr ? 1 : 0);
}

static int background_terms(const orc_cfg *c) {
    if (c->basis == 0) return n_terms(c->db);
    int K = n_spl(c->bdeg, c->bint);
    return K * K;
}

/* which offsets a kernel term carries: the (0,0) offset and/or the others */
static int term_has00(const orc_cfg *c, int t) { return c->cpr ? t == 0 : 1; }
static int term_hasother(const orc_cfg *c, int t) { return (c->basis == 1 && c->cpr) ? t != 0 : 1; }

/* k-th monomial (i,j) with i+j <= d, ordered by total degree, then i descending */
static void term_ij(int k, int *i, int *j) {
    int deg = 0, start = 0;
    while (start + deg + 1 <= k) { start += deg + 1; deg++; }
    int off = k - start;
    *i = deg - off;
    *j = off;
}

static double ipow(double v, int e) {
    double r = 1.0;
    for (int k = 0; k < e; k++) r *= v;
    return r;
}

static double coord(int x, int n) { return (2.0 * x - (n - 1)) / (double)(n - 1); }

/* knot r of the clamped uniform knot vector on [-1, 1] (r = 0 .. nint + 2 deg + 1) */
static double knot(int deg, int nint, int r) {
    if (r <= deg) return -1.0;
    if (r >= nint + deg + 1) return 1.0;
    return -1.0 + 2.0 * (double)(r - deg) / (double)(nint + 1);
}

/* B-spline basis function i of degree deg at u in [-1, 1], by the Cox-de Boor
 * recursion B_{i,0} = [t_i <= u < t_{i+1}],
 * B_{i,d} = (u - t_i)/(t_{i+d} - t_i) B_{i,d-1} + (t_{i+d+1} - u)/(t_{i+d+1} - t_{i+1}) B_{i+1,d-1},
 * with 0/0 terms taken as 0 and u = 1 placed in the last non-empty span. */
static double bspline(int deg, int nint, int i, double u) {
    int K = n_spl(deg, nint);
    double b[64];
    if (i < 0 || i >= K || deg + 1 > 32) return 0.0;
    /* degree 0 functions i .. i + deg (those that feed B_{i,deg}) */
    for (int r = 0; r <= deg; r++) {
        int q = i + r;
        double t0 = knot(deg, nint, q), t1 = knot(deg, nint, q + 1);
        int in = (u >= t0 && u < t1);
        if (u >= 1.0 && t1 >= 1.0 && t0 < 1.0) in = 1;  /* right end: last non-empty span */
        b[r] = in ? 1.0 : 0.0;
    }
    for (int d = 1; d <= deg; d++) {
        for (int r = 0; r + d <= deg; r++) {
            int q = i + r;
            double tq = knot(deg, nint, q), tqd = knot(deg, nint, q + d);
            double tq1 = knot(deg, nint, q + 1), tqd1 = knot(deg, nint, q + d + 1);
            double left = (tqd > tq) ? (u - tq) / (tqd - tq) * b[r] : 0.0;
            double right = (tqd1 > tq1) ? (tqd1 - u) / (tqd1 - tq1) * b[r + 1] : 0.0;
            b[r] = left + right;
        }
    }
    return b[0];
}

double orc_bspline(int deg, int nint, int i, double u) { return bspline(deg, nint, i, u); }

/* weight of kernel term t at pixel (x, y) */
static double kernel_weight(const orc_cfg *c, int t, int x, int y) {
    double xt = coord(x, c->n0), yt = coord(y, c->n1);
    if (c->basis == 0) {
        int i, j;
        term_ij(t, &i, &j);
        return ipow(xt, i) * ipow(yt, j);
    }
    if (c->cpr) {
        if (t == 0) return 1.0;
        t -= 1;
    }
    int K = n_spl(c->kdeg, c->kint);
    return bspline(c->kdeg, c->kint, t / K, xt) * bspline(c->kdeg, c->kint, t % K, yt);
}

/* weight of background term s at pixel (x, y) */
static double background_weight(const orc_cfg *c, int s, int x, int y) {
    double xt = coord(x, c->n0), yt = coord(y, c->n1);
    if (c->basis == 0) {
        int p, q;
        term_ij(s, &p, &q);
        return ipow(xt, p) * ipow(yt, q);
    }
    int K = n_spl(c->bdeg, c->bint);
    return bspline(c->bdeg, c->bint, s / K, xt) * bspline(c->bdeg, c->bint, s % K, yt);
}

static int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

/* unknowns of kernel term t: its (0,0) offset and/or the L-1 others */
static int term_unknowns(const orc_cfg *c, int t) {
    int L = (2 * c->w0 + 1) * (2 * c->w1 + 1);
    return (term_has00(c, t) ? 1 : 0) + (term_hasother(c, t) ? L - 1 : 0);
}

static int num_unknowns(const orc_cfg *c) {
    int n = 0, nk = kernel_terms(c);
    for (int t = 0; t < nk; t++) n += term_unknowns(c, t);
    return n + background_terms(c);
}

int orc_num_unknowns(const int *cfg) {
    orc_cfg c = cfg_from(cfg);
    return num_unknowns(&c);
}

/* Decode unknown index u into (is_kernel, term, alpha, beta) */
static void decode_unknown(const orc_cfg *c, int u, int *is_k, int *t, int *a, int *b) {
    int L1 = 2 * c->w1 + 1;
    int L = (2 * c->w0 + 1) * L1;
    int centre = (L - 1) / 2;          /* row-major position of (alpha,beta)=(0,0) */
    int nk = kernel_terms(c);
    for (int k = 0; k < nk; k++) {
        int cnt = term_unknowns(c, k);
        if (u < cnt) {
            int off;
            if (!term_hasother(c, k)) off = centre;          /* only the (0,0) offset */
            else if (!term_has00(c, k)) off = u >= centre ? u + 1 : u;  /* all but (0,0) */
            else off = u;
            *is_k = 1;
            *t = k;
            *a = off / L1 - c->w0;
            *b = off % L1 - c->w1;
            return;
        }
        u -= cnt;
    }
    *is_k = 0; *t = u; *a = 0; *b = 0;
}

static int check_cfg(const orc_cfg *c) {
    if (c->n0 < 2 || c->n1 < 2) return ORC_ERR_INVALID;
    if (c->w0 < 0 || c->w1 < 0 || c->dk < 0 || c->db < 0) return ORC_ERR_INVALID;
    if (2 * c->w0 + 1 > c->n0 || 2 * c->w1 + 1 > c->n1) return ORC_ERR_INVALID;
    if (c->basis != 0 && c->basis != 1) return ORC_ERR_INVALID;
    if (c->basis == 1 && (c->kdeg < 0 || c->kint < 0 || c->bdeg < 0 || c->bint < 0 || c->kdeg > 8 ||
                          c->bdeg > 8 || c->kint > 30 || c->bint > 30))
        return ORC_ERR_INVALID;
    return ORC_OK;
}

/* ---- images ------------------------------------------------------------ */

/* g_t = w_t * Rm for every kernel term t, w_t = xt^i yt^j (Eq. 10-11:
 * R^{ij} = T^{ij} R) or B_i(xt) B_j(yt) (Eq. 8) */
static double *make_weighted(const orc_cfg *c, const double *Rm, int t) {
    size_t P = (size_t)c->n0 * c->n1;
    double *g = (double *)malloc(P * sizeof(double));
    if (!g) return NULL;
    for (int x = 0; x < c->n0; x++)
        for (int y = 0; y < c->n1; y++)
            g[(size_t)x * c->n1 + y] = kernel_weight(c, t, x, y) * Rm[(size_t)x * c->n1 + y];
    return g;
}

/* background basis image T^{pq} = xt^p yt^q (Eq. 2) or B'_p(xt) B'_q(yt) (Eq. 9) */
static double *make_poly(const orc_cfg *c, int s) {
    size_t P = (size_t)c->n0 * c->n1;
    double *T = (double *)malloc(P * sizeof(double));
    if (!T) return NULL;
    for (int x = 0; x < c->n0; x++)
        for (int y = 0; y < c->n1; y++) T[(size_t)x * c->n1 + y] = background_weight(c, s, x, y);
    return T;
}

static double *masked_copy(const orc_cfg *c, const double *img, const uint8_t *mask) {
    size_t P = (size_t)c->n0 * c->n1;
    double *o = (double *)malloc(P * sizeof(double));
    if (!o) return NULL;
    for (size_t k = 0; k < P; k++) o[k] = (mask && mask[k] == 0) ? 0.0 : img[k];
    return o;
}

/* sum_x f(x) g((x + rho) mod N): the circular cross-correlation at one lag */
double orc_lag_sum(int n0, int n1, const double *f, const double *g, int r0, int r1) {
    double s = 0.0;
    for (int x = 0; x < n0; x++) {
        const double *fr = f + (size_t)x * n1;
        const double *gr = g + (size_t)imod(x + r0, n0) * n1;
        for (int y = 0; y < n1; y++) s += fr[y] * gr[imod(y + r1, n1)];
    }
    return s;
}

/* ---- lag tables (App. B) ---------------------------------------------- */

typedef struct {
    orc_cfg c;
    int nk, nb;
    int h0, h1;        /* Omega lag half-ranges: 2w0, 2w1 */
    double **g;        /* nk weighted images */
    double **T;        /* nb background monomials */
    double *Sm;        /* masked science image */
    double *om;        /* Omega[t][u][lag] for t <= u (upper-triangular pairs) */
    double *la;        /* Lambda[t][s][lag], lag in [-w0,w0]x[-w1,w1] */
    double *th;        /* Theta[t][lag] */
    double *cc;        /* C[s][s'] */
    double *ee;        /* E[s] */
} tables;

static int pair_index(int nk, int t, int u) { /* t <= u */
    return t * nk - t * (t - 1) / 2 + (u - t);
}

static size_t om_lags(const tables *tb) { return (size_t)(2 * tb->h0 + 1) * (2 * tb->h1 + 1); }
static size_t la_lags(const tables *tb) { return (size_t)(2 * tb->c.w0 + 1) * (2 * tb->c.w1 + 1); }

/* Omega_{t u}(rho) for any ordered pair; Omega_{u t}(rho) = Omega_{t u}(-rho) */
static double omega(const tables *tb, int t, int u, int r0, int r1) {
    if (t > u) { int z = t; t = u; u = z; r0 = -r0; r1 = -r1; }
    size_t lag = (size_t)(r0 + tb->h0) * (2 * tb->h1 + 1) + (r1 + tb->h1);
    return tb->om[(size_t)pair_index(tb->nk, t, u) * om_lags(tb) + lag];
}
static double lambda_(const tables *tb, int t, int s, int r0, int r1) {
    size_t lag = (size_t)(r0 + tb->c.w0) * (2 * tb->c.w1 + 1) + (r1 + tb->c.w1);
    return tb->la[((size_t)t * tb->nb + s) * la_lags(tb) + lag];
}
static double theta(const tables *tb, int t, int r0, int r1) {
    size_t lag = (size_t)(r0 + tb->c.w0) * (2 * tb->c.w1 + 1) + (r1 + tb->c.w1);
    return tb->th[(size_t)t * la_lags(tb) + lag];
}

static void free_tables(tables *tb) {
    if (tb->g) { for (int t = 0; t < tb->nk; t++) free(tb->g[t]); free(tb->g); }
    if (tb->T) { for (int s = 0; s < tb->nb; s++) free(tb->T[s]); free(tb->T); }
    free(tb->Sm); free(tb->om); free(tb->la); free(tb->th); free(tb->cc); free(tb->ee);
    memset(tb, 0, sizeof(*tb));
}

/* Images only (no lag sums yet) */
static int make_images(tables *tb, const orc_cfg *c, const double *R, const double *S,
                       const uint8_t *mask) {
    memset(tb, 0, sizeof(*tb));
    tb->c = *c;
    tb->nk = kernel_terms(c);
    tb->nb = background_terms(c);
    tb->h0 = 2 * c->w0;
    tb->h1 = 2 * c->w1;
    double *Rm = masked_copy(c, R, mask);
    tb->Sm = masked_copy(c, S, mask);
    tb->g = (double **)calloc(tb->nk, sizeof(double *));
    tb->T = (double **)calloc(tb->nb, sizeof(double *));
    if (!Rm || !tb->Sm || !tb->g || !tb->T) { free(Rm); free_tables(tb); return ORC_ERR_NOMEM; }
    for (int t = 0; t < tb->nk; t++)
        if (!(tb->g[t] = make_weighted(c, Rm, t))) { free(Rm); free_tables(tb); return ORC_ERR_NOMEM; }
    for (int s = 0; s < tb->nb; s++)
        if (!(tb->T[s] = make_poly(c, s))) { free(Rm); free_tables(tb); return ORC_ERR_NOMEM; }
    free(Rm);
    return ORC_OK;
}

static int fill_tables(tables *tb) {
    const orc_cfg *c = &tb->c;
    int nk = tb->nk, nb = tb->nb;
    int npair = nk * (nk + 1) / 2;
    size_t nom = om_lags(tb), nla = la_lags(tb);
    size_t P = (size_t)c->n0 * c->n1;
    tb->om = (double *)malloc((size_t)npair * nom * sizeof(double));
    tb->la = (double *)malloc((size_t)nk * nb * nla * sizeof(double));
    tb->th = (double *)malloc((size_t)nk * nla * sizeof(double));
    tb->cc = (double *)malloc((size_t)nb * nb * sizeof(double));
    tb->ee = (double *)malloc((size_t)nb * sizeof(double));
    if (!tb->om || !tb->la || !tb->th || !tb->cc || !tb->ee) return ORC_ERR_NOMEM;

    /* Omega: every pair t <= u, every lag in [-2w0,2w0] x [-2w1,2w1] */
    long long nwork = (long long)npair * (long long)nom;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long k = 0; k < nwork; k++) {
        int pr = (int)(k / (long long)nom);
        int lag = (int)(k % (long long)nom);
        int t = 0, u = 0, acc = 0;
        for (t = 0; t < nk; t++) {
            if (pr < acc + (nk - t)) { u = t + (pr - acc); break; }
            acc += nk - t;
        }
        int r0 = lag / (2 * tb->h1 + 1) - tb->h0;
        int r1 = lag % (2 * tb->h1 + 1) - tb->h1;
        tb->om[(size_t)pr * nom + lag] = orc_lag_sum(c->n0, c->n1, tb->g[t], tb->g[u], r0, r1);
    }
    /* Lambda and Theta: lags in [-w0,w0] x [-w1,w1] */
    long long nwl = (long long)nk * (nb + 1) * (long long)nla;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long k = 0; k < nwl; k++) {
        int which = (int)(k / (long long)nla);
        int lag = (int)(k % (long long)nla);
        int t = which / (nb + 1), s = which % (nb + 1);
        int r0 = lag / (2 * c->w1 + 1) - c->w0;
        int r1 = lag % (2 * c->w1 + 1) - c->w1;
        if (s < nb)
            tb->la[((size_t)t * nb + s) * nla + lag] =
                orc_lag_sum(c->n0, c->n1, tb->g[t], tb->T[s], r0, r1);
        else
            tb->th[(size_t)t * nla + lag] = orc_lag_sum(c->n0, c->n1, tb->g[t], tb->Sm, r0, r1);
    }
    /* C and E: plain spatial dot products (Eq. B11, B15 at lag zero) */
    for (int s = 0; s < nb; s++) {
        for (int s2 = 0; s2 < nb; s2++) {
            double acc = 0.0;
            for (size_t p = 0; p < P; p++) acc += tb->T[s][p] * tb->T[s2][p];
            tb->cc[s * nb + s2] = acc;
        }
        double acc = 0.0;
        for (size_t p = 0; p < P; p++) acc += tb->T[s][p] * tb->Sm[p];
        tb->ee[s] = acc;
    }
    return ORC_OK;
}

/* One entry of the normal matrix [A B; B~ C] from the tables (Eq. B5, B7, B9, B11) */
static double entry_from_tables(const tables *tb, int row, int col) {
    int rk, rt, ra, rb, ck, ct, ca, cb;
    decode_unknown(&tb->c, row, &rk, &rt, &ra, &rb);
    decode_unknown(&tb->c, col, &ck, &ct, &ca, &cb);
    if (rk && ck) {
        int rz = (ra == 0 && rb == 0), cz = (ca == 0 && cb == 0);
        if (!rz && !cz)
            return omega(tb, rt, ct, ra - ca, rb - cb) - omega(tb, rt, ct, ra, rb) -
                   omega(tb, rt, ct, -ca, -cb) + omega(tb, rt, ct, 0, 0);
        if (rz && !cz) return omega(tb, rt, ct, -ca, -cb) - omega(tb, rt, ct, 0, 0);
        if (!rz && cz) return omega(tb, rt, ct, ra, rb) - omega(tb, rt, ct, 0, 0);
        return omega(tb, rt, ct, 0, 0);
    }
    if (rk && !ck) { /* B (Eq. B7) */
        if (ra == 0 && rb == 0) return lambda_(tb, rt, ct, 0, 0);
        return lambda_(tb, rt, ct, ra, rb) - lambda_(tb, rt, ct, 0, 0);
    }
    if (!rk && ck) { /* B~ (Eq. B9): Psi_{s t}(rho) = Lambda_{t s}(-rho) */
        if (ca == 0 && cb == 0) return lambda_(tb, ct, rt, 0, 0);
        return lambda_(tb, ct, rt, ca, cb) - lambda_(tb, ct, rt, 0, 0);
    }
    return tb->cc[rt * tb->nb + ct]; /* C (Eq. B11) */
}

static double rhs_from_tables(const tables *tb, int row) {
    int rk, rt, ra, rb;
    decode_unknown(&tb->c, row, &rk, &rt, &ra, &rb);
    if (rk) { /* D (Eq. B13) */
        if (ra == 0 && rb == 0) return theta(tb, rt, 0, 0);
        return theta(tb, rt, ra, rb) - theta(tb, rt, 0, 0);
    }
    return tb->ee[rt]; /* E (Eq. B15) */
}

/* Full system: M (n*n row-major) and rhs (n) */
int orc_build_system(const int *cfg, const double *R, const double *S, const uint8_t *mask, double *M,
                     double *rhs) {
    orc_cfg c = cfg_from(cfg);
    int rc = check_cfg(&c);
    if (rc) return rc;
    tables tb;
    if ((rc = make_images(&tb, &c, R, S, mask))) return rc;
    if ((rc = fill_tables(&tb))) { free_tables(&tb); return rc; }
    int n = num_unknowns(&c);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; r++) {
        for (int k = 0; k < n; k++) M[(size_t)r * n + k] = entry_from_tables(&tb, r, k);
        rhs[r] = rhs_from_tables(&tb, r);
    }
    free_tables(&tb);
    return ORC_OK;
}

/*
 * Selected entries only: for each requested (row, col) the needed lag values
 * are computed by direct spatial sums on the spot.  Used to check the full
 * 4096^2 system at sampled positions.  col < 0 requests rhs[row].
 */
static double lag_value(const tables *tb, int kind, int t, int u, int r0, int r1) {
    const orc_cfg *c = &tb->c;
    if (kind == 0) return orc_lag_sum(c->n0, c->n1, tb->g[t], tb->g[u], r0, r1);
    if (kind == 1) return orc_lag_sum(c->n0, c->n1, tb->g[t], tb->T[u], r0, r1);
    return orc_lag_sum(c->n0, c->n1, tb->g[t], tb->Sm, r0, r1);
}

int orc_system_entries(const int *cfg, const double *R, const double *S, const uint8_t *mask, int count,
                       const int *rows, const int *cols, double *out) {
    orc_cfg c = cfg_from(cfg);
    int rc = check_cfg(&c);
    if (rc) return rc;
    tables tb;
    if ((rc = make_images(&tb, &c, R, S, mask))) return rc;
    int n = num_unknowns(&c);
    size_t P = (size_t)c.n0 * c.n1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < count; q++) {
        int row = rows[q], col = cols[q];
        if (row < 0 || row >= n || col >= n) { out[q] = NAN; continue; }
        int rk, rt, ra, rb, ck, ct, ca, cb;
        decode_unknown(&c, row, &rk, &rt, &ra, &rb);
        double v;
        if (col < 0) {
            if (rk) {
                v = (ra == 0 && rb == 0) ? lag_value(&tb, 2, rt, 0, 0, 0)
                                         : lag_value(&tb, 2, rt, 0, ra, rb) - lag_value(&tb, 2, rt, 0, 0, 0);
            } else {
                double acc = 0.0;
                for (size_t p = 0; p < P; p++) acc += tb.T[rt][p] * tb.Sm[p];
                v = acc;
            }
            out[q] = v;
            continue;
        }
        decode_unknown(&c, col, &ck, &ct, &ca, &cb);
        if (rk && ck) {
            int rz = (ra == 0 && rb == 0), cz = (ca == 0 && cb == 0);
            /* Omega_{rt ct}(rho) = sum g_rt(x) g_ct(x+rho) */
            if (!rz && !cz)
                v = lag_value(&tb, 0, rt, ct, ra - ca, rb - cb) - lag_value(&tb, 0, rt, ct, ra, rb) -
                    lag_value(&tb, 0, rt, ct, -ca, -cb) + lag_value(&tb, 0, rt, ct, 0, 0);
            else if (rz && !cz)
                v = lag_value(&tb, 0, rt, ct, -ca, -cb) - lag_value(&tb, 0, rt, ct, 0, 0);
            else if (!rz && cz)
                v = lag_value(&tb, 0, rt, ct, ra, rb) - lag_value(&tb, 0, rt, ct, 0, 0);
            else
                v = lag_value(&tb, 0, rt, ct, 0, 0);
        } else if (rk && !ck) {
            v = (ra == 0 && rb == 0) ? lag_value(&tb, 1, rt, ct, 0, 0)
                                     : lag_value(&tb, 1, rt, ct, ra, rb) - lag_value(&tb, 1, rt, ct, 0, 0);
        } else if (!rk && ck) {
            v = (ca == 0 && cb == 0) ? lag_value(&tb, 1, ct, rt, 0, 0)
                                     : lag_value(&tb, 1, ct, rt, ca, cb) - lag_value(&tb, 1, ct, rt, 0, 0);
        } else {
            double acc = 0.0;
            for (size_t p = 0; p < P; p++) acc += tb.T[rt][p] * tb.T[ct][p];
            v = acc;
        }
        out[q] = v;
    }
    free_tables(&tb);
    return ORC_OK;
}

/* ---- solve -------------------------------------------------------------- */

/* Cholesky M = L L^T (lower, in place on a copy), then two triangular solves.
 * Returns ORC_ERR_NOT_PD if a pivot is not positive. */
int orc_cholesky_solve(int n, const double *M, const double *rhs, double *x) {
    if (n <= 0) return ORC_ERR_INVALID;
    double *L = (double *)malloc((size_t)n * n * sizeof(double));
    double *z = (double *)malloc((size_t)n * sizeof(double));
    if (!L || !z) { free(L); free(z); return ORC_ERR_NOMEM; }
    memcpy(L, M, (size_t)n * n * sizeof(double));
    for (int j = 0; j < n; j++) {
        double d = L[(size_t)j * n + j];
        for (int k = 0; k < j; k++) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0)) { free(L); free(z); return ORC_ERR_NOT_PD; }
        double ljj = sqrt(d);
        L[(size_t)j * n + j] = ljj;
#pragma omp parallel for schedule(static)
        for (int i = j + 1; i < n; i++) {
            double s = L[(size_t)i * n + j];
            for (int k = 0; k < j; k++) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = s / ljj;
        }
    }
    for (int i = 0; i < n; i++) { /* L z = rhs */
        double s = rhs[i];
        for (int k = 0; k < i; k++) s -= L[(size_t)i * n + k] * z[k];
        z[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) { /* L^T x = z */
        double s = z[i];
        for (int k = i + 1; k < n; k++) s -= L[(size_t)k * n + i] * x[k];
        x[i] = s / L[(size_t)i * n + i];
    }
    free(L);
    free(z);
    return ORC_OK;
}

/* ---- subtract (Eq. 12) -------------------------------------------------- */

/* D(x) at one pixel: S - sum_{t,ab} a_{t,ab} (g_t o K_ab)(x) - sum_s b_s T^s(x),
 * with (g o K_ab)(x) = g(x - ab) - g(x) for ab != 0 and g(x) for ab = 0. */
static double diff_pixel(const orc_cfg *c, const double *R, const double *S, const double *x,
                         int px, int py) {
    int nk = kernel_terms(c), nb = background_terms(c);
    double d = S[(size_t)px * c->n1 + py];
    int u = 0;
    for (int t = 0; t < nk; t++) {
        double g0 = kernel_weight(c, t, px, py) * R[(size_t)px * c->n1 + py];
        for (int a = -c->w0; a <= c->w0; a++) {
            for (int b = -c->w1; b <= c->w1; b++) {
                int zero = (a == 0 && b == 0);
                if (zero ? !term_has00(c, t) : !term_hasother(c, t)) continue;
                double coef = x[u++];
                if (zero) { d -= coef * g0; continue; }
                int qx = imod(px - a, c->n0), qy = imod(py - b, c->n1);
                double gs = kernel_weight(c, t, qx, qy) * R[(size_t)qx * c->n1 + qy];
                d -= coef * (gs - g0);
            }
        }
    }
    for (int s = 0; s < nb; s++) d -= x[u++] * background_weight(c, s, px, py);
    return d;
}

int orc_subtract(const int *cfg, const double *R, const double *S, const double *x, double *D) {
    orc_cfg c = cfg_from(cfg);
    int rc = check_cfg(&c);
    if (rc) return rc;
#pragma omp parallel for schedule(static)
    for (int px = 0; px < c.n0; px++)
        for (int py = 0; py < c.n1; py++) D[(size_t)px * c.n1 + py] = diff_pixel(&c, R, S, x, px, py);
    return ORC_OK;
}

/* D at a list of flat pixel indices */
int orc_subtract_pixels(const int *cfg, const double *R, const double *S, const double *x, int count,
                        const long long *pix, double *out) {
    orc_cfg c = cfg_from(cfg);
    int rc = check_cfg(&c);
    if (rc) return rc;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < count; k++) {
        long long p = pix[k];
        if (p < 0 || p >= (long long)c.n0 * c.n1) { out[k] = NAN; continue; }
        out[k] = diff_pixel(&c, R, S, x, (int)(p / c.n1), (int)(p % c.n1));
    }
    return ORC_OK;
}

/* Decoded unknown: kind (1 kernel, 0 background), term, alpha, beta */
int orc_decode_unknown(const int *cfg, int u, int *out4) {
    orc_cfg c = cfg_from(cfg);
    int n = num_unknowns(&c);
    if (u < 0 || u >= n) return ORC_ERR_INVALID;
    decode_unknown(&c, u, &out4[0], &out4[1], &out4[2], &out4[3]);
    return ORC_OK;
}

int orc_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
