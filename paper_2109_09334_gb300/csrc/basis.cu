// basis.cu -- the spatial-variation basis of a plan: polynomial (Eq. 2, 6)
// or tensor-product B-splines (Eq. 7-9), as term tables, function tables and
// the descriptors of the zero-lag sums.  Host code, run once per plan.
//
// Term structure (BasisView): kernel term t weights R by fx_i(x) fy_j(y),
// background term s is bx_p(x) by_q(y).
//   Polynomial: fx_i = xt^i (i <= dk), fy_j = yt^j, terms (i, j), i + j <= dk,
//   by total degree then descending i; background likewise with db.
//   B-spline: K = kint + kdeg + 1 functions B_0..B_(K-1) per axis on the
//   normalised coordinate (clamped uniform knots on [-1, 1]); with a constant
//   photometric ratio a constant function (index K) is added.  Terms: the
//   constant term (K, K) first if the ratio is constant, carrying only the
//   (0,0) offset; then (i, j), i, j < K, i outer, carrying all offsets but
//   (0,0) when the ratio is constant.  Background: (p, q), p, q < K', p outer.
//
// Zero-lag values (Eq. B5-B16 at rho = 0, and E of Eq. B15) are FP64 sums
//   Omega_tu(0,0) = sum_x fx_i fx_i' RR_jj'(x),   RR_jj'(x) = sum_y fy_j fy_j' Rm^2
//   Lambda_ts(0,0) = sum_x fx_i bx_p RB_jq(x),    RB_jq(x) = sum_y fy_j by_q Rm
//   Theta_t(0,0)  = sum_x fx_i RS_j(x),           RS_j(x) = sum_y fy_j Rm Sm
//   E_s           = sum_x bx_p SB_q(x),           SB_q(x) = sum_y by_q Sm
// of per-row moments.  For the polynomial basis the products collapse to
// powers (the per-row power sums of k_row_moments, the x-table xt^u); for
// B-splines every product is kept.  C (Eq. B11) needs no image:
// C_ss' = (sum_x bx_p bx_p')(sum_y by_q by_q').
#include <cuda_runtime.h>

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sfft {

namespace {

int spl_count(int deg, int nint) { return nint + deg + 1; }

// knot r of the clamped uniform knot vector on [-1, 1] with K functions
double spl_knot(int deg, int K, int r) {
    if (r <= deg) return -1.0;
    if (r >= K) return 1.0;
    return -1.0 + 2.0 * (double)(r - deg) / (double)(K - deg);
}

// All K basis functions at u (out[0..K)), by the triangular scheme that
// builds the deg+1 functions nonzero on u's knot span from degree 0 upward
// (L. Piegl and W. Tiller, The NURBS Book, Algorithm A2.2); u = 1 belongs
// to the last span.
void spl_eval(int deg, int nint, double u, double *out) {
    const int K = spl_count(deg, nint);
    for (int i = 0; i < K; ++i) out[i] = 0.0;
    int span = K - 1;
    for (int r = deg; r < K; ++r)
        if (u < spl_knot(deg, K, r + 1)) {
            span = r;
            break;
        }
    double N[kMaxFun + 1], left[kMaxFun + 1], right[kMaxFun + 1];
    N[0] = 1.0;
    for (int j = 1; j <= deg; ++j) {
        left[j] = u - spl_knot(deg, K, span + 1 - j);
        right[j] = spl_knot(deg, K, span + j) - u;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            const double tmp = N[r] / (right[r + 1] + left[j - r]);
            N[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        N[j] = saved;
    }
    for (int r = 0; r <= deg; ++r) out[span - deg + r] = N[r];
}

double coord64(int x, int n) { return (2.0 * x - (n - 1)) / (double)(n - 1); }

double ipow64(double v, int e) {
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= v;
    return r;
}

// Monomial k of degree <= d: by total degree, then descending i.
void mono_ij(int k, int *i, int *j) { term_ij(k, i, j); }

// Row values of the function tables: fill out[f * n + x] for f < count of
// the axis functions (xt^f or B_f), plus the constant 1 at index `cst` if >= 0.
void axis_table(int poly, int deg, int nint, int count, int cst, int n, std::vector<double> &out) {
    out.assign((size_t)count * n, 0.0);
    std::vector<double> b(kMaxFun + 1);
    for (int x = 0; x < n; ++x) {
        const double u = coord64(x, n);
        if (!poly) spl_eval(deg, nint, u, b.data());
        for (int f = 0; f < count; ++f) {
            double v;
            if (f == cst) v = 1.0;
            else v = poly ? ipow64(u, f) : b[f];
            out[(size_t)f * n + x] = v;
        }
    }
}

}  // namespace

int basis_validate(const sfft_config *c) {
    if (c->basis == SFFT_BASIS_POLY) {
        if (c->dk < 0 || c->db < 0) return SFFT_ERR_INVALID;
        if (c->dk > 3 || c->db > 3) return SFFT_ERR_UNSUPPORTED;
        return SFFT_OK;
    }
    if (c->basis != SFFT_BASIS_BSPLINE) return SFFT_ERR_INVALID;
    if (c->dk != 0 || c->db != 0) return SFFT_ERR_INVALID;
    if (c->kdeg < 0 || c->kint < 0 || c->bdeg < 0 || c->bint < 0) return SFFT_ERR_INVALID;
    if (c->kdeg > 3 || c->bdeg > 3) return SFFT_ERR_UNSUPPORTED;
    if (spl_count(c->kdeg, c->kint) > 6 || spl_count(c->bdeg, c->bint) > 6) return SFFT_ERR_UNSUPPORTED;
    return SFFT_OK;
}

int basis_unknowns(const sfft_config *c) {
    const int L = (2 * c->w0 + 1) * (2 * c->w1 + 1);
    if (c->basis == SFFT_BASIS_POLY) {
        const int nk = n_terms(c->dk), nb = n_terms(c->db);
        return c->const_phot_ratio ? nk * (L - 1) + 1 + nb : nk * L + nb;
    }
    const int K = spl_count(c->kdeg, c->kint), Kb = spl_count(c->bdeg, c->bint);
    return c->const_phot_ratio ? 1 + K * K * (L - 1) + Kb * Kb : K * K * L + Kb * Kb;
}

int basis_terms(const sfft_config *c, int *nk, int *nb) {
    if (c->basis == SFFT_BASIS_POLY) {
        *nk = n_terms(c->dk);
        *nb = n_terms(c->db);
    } else {
        const int K = spl_count(c->kdeg, c->kint), Kb = spl_count(c->bdeg, c->bint);
        *nk = K * K + (c->const_phot_ratio ? 1 : 0);
        *nb = Kb * Kb;
    }
    return SFFT_OK;
}

// Host tables of a validated configuration (allocated into p; freed by plan_free).
int basis_build(Plan *p, cudaStream_t s) {
    const sfft_config &c = p->cfg;
    const bool poly = c.basis == SFFT_BASIS_POLY;
    const int cpr = c.const_phot_ratio ? 1 : 0;
    const int L1 = 2 * c.w1 + 1, L = (2 * c.w0 + 1) * L1;
    int nk = 0, nb = 0;
    basis_terms(&c, &nk, &nb);
    p->nk = nk;
    p->nb = nb;
    p->bspline = poly ? 0 : 1;
    int K = 0, Kb = 0;
    if (poly) {
        p->nfx = p->nfy = c.dk + 1;
        p->nbx = p->nby = c.db + 1;
    } else {
        K = spl_count(c.kdeg, c.kint);
        Kb = spl_count(c.bdeg, c.bint);
        p->nfx = p->nfy = K + cpr;
        p->nbx = p->nby = Kb;
    }
    const int nfx = p->nfx, nfy = p->nfy, nbx = p->nbx, nby = p->nby;

    // ---- int tables -------------------------------------------------------
    BasisView &bv = p->bv;
    bv.nk = nk;
    bv.nb = nb;
    bv.nfx = nfx;
    bv.nfy = nfy;
    bv.nbx = nbx;
    bv.nby = nby;
    bv.w0 = c.w0;
    bv.w1 = c.w1;
    int o = 0;
    bv.o_ti = o; o += nk;
    bv.o_tj = o; o += nk;
    bv.o_fl = o; o += nk;
    bv.o_uoff = o; o += nk;
    bv.o_sp = o; o += nb;
    bv.o_sq = o; o += nb;
    bv.o_lamn = o; o += nbx;
    bv.o_lams = o; o += nbx * nby;
    bv.o_lamq = o; o += nbx * nby;
    bv.o_jcnt = o; o += nfy;
    bv.o_jterm = o; o += nfy * nk;
    bv.total = o;
    p->h_int = (int *)calloc((size_t)o, sizeof(int));
    if (!p->h_int) return SFFT_ERR_OOM;
    int *h = p->h_int;
    int uoff = 0;
    for (int t = 0; t < nk; ++t) {
        int i, j, fl;
        if (poly) {
            mono_ij(t, &i, &j);
            fl = (cpr && t != 0) ? 2 : 3;
        } else if (cpr && t == 0) {
            i = j = K;  // the constant function
            fl = 1;
        } else {
            const int u = t - cpr;
            i = u / K;
            j = u % K;
            fl = cpr ? 2 : 3;
        }
        h[bv.o_ti + t] = i;
        h[bv.o_tj + t] = j;
        h[bv.o_fl + t] = fl;
        h[bv.o_uoff + t] = uoff;
        uoff += ((fl & 1) ? 1 : 0) + ((fl & 2) ? L - 1 : 0);
    }
    for (int sidx = 0; sidx < nb; ++sidx) {
        int pp, qq;
        if (poly) mono_ij(sidx, &pp, &qq);
        else {
            pp = sidx / Kb;
            qq = sidx % Kb;
        }
        h[bv.o_sp + sidx] = pp;
        h[bv.o_sq + sidx] = qq;
        const int k = h[bv.o_lamn + pp]++;
        h[bv.o_lams + pp * nby + k] = sidx;
        h[bv.o_lamq + pp * nby + k] = qq;
    }
    for (int t = 0; t < nk; ++t) {
        const int j = h[bv.o_tj + t];
        const int k = h[bv.o_jcnt + j]++;
        h[bv.o_jterm + j * nk + k] = t;
    }
    if (uoff + nb != p->n) return SFFT_ERR_INVALID;  // the two counts must agree
    if (cudaMalloc((void **)&p->d_int, (size_t)o * sizeof(int)) != cudaSuccess) return SFFT_ERR_OOM;
    p->ws_bytes += (size_t)o * sizeof(int);
    bv.d = p->d_int;

    // ---- decoded unknowns ---------------------------------------------------
    std::vector<int4> unk((size_t)p->n);
    {
        int u = 0;
        const int ctr = (L - 1) / 2;
        for (int t = 0; t < nk; ++t) {
            const int fl = h[bv.o_fl + t];
            for (int off = 0; off < L; ++off) {
                if (off == ctr ? !(fl & 1) : !(fl & 2)) continue;
                unk[u++] = make_int4(1, t, off / L1 - c.w0, off % L1 - c.w1);
            }
        }
        for (int sidx = 0; sidx < nb; ++sidx) unk[u++] = make_int4(0, sidx, 0, 0);
    }
    if (cudaMalloc((void **)&p->unk, (size_t)p->n * sizeof(int4)) != cudaSuccess) return SFFT_ERR_OOM;
    p->ws_bytes += (size_t)p->n * sizeof(int4);

    // ---- function tables in the compute type, x-functions then y: the
    // B-spline functions, or the monomials xt^i, yt^j of the polynomial
    // basis (evaluated in FP64 and rounded once, so the row, column and
    // subtraction passes read a weight instead of dividing and raising a
    // coordinate to a power per pixel) -----------------------------------------
    std::vector<double> tfx, tfy, tbx, tby;
    axis_table(poly, c.kdeg, c.kint, nfx, poly ? -1 : (cpr ? K : -1), p->n0, tfx);
    axis_table(poly, c.kdeg, c.kint, nfy, poly ? -1 : (cpr ? K : -1), p->n1, tfy);
    axis_table(poly, c.bdeg, c.bint, nbx, -1, p->n0, tbx);
    axis_table(poly, c.bdeg, c.bint, nby, -1, p->n1, tby);
    const size_t nft = tfx.size() + tbx.size() + tfy.size() + tby.size();
    std::vector<double> all;
    all.reserve(nft);
    all.insert(all.end(), tfx.begin(), tfx.end());
    all.insert(all.end(), tbx.begin(), tbx.end());
    all.insert(all.end(), tfy.begin(), tfy.end());
    all.insert(all.end(), tby.begin(), tby.end());
    {
        const size_t esz = p->fp64 ? sizeof(double) : sizeof(float);
        if (cudaMalloc(&p->ftab, nft * esz) != cudaSuccess) return SFFT_ERR_OOM;
        p->ws_bytes += nft * esz;
        cudaError_t e;
        if (p->fp64) {
            e = cudaMemcpy(p->ftab, all.data(), nft * sizeof(double), cudaMemcpyHostToDevice);
        } else {
            std::vector<float> f32(all.begin(), all.end());
            e = cudaMemcpy(p->ftab, f32.data(), nft * sizeof(float), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return SFFT_ERR_CUDA;
    }
    {  // FP64 background functions, bx then by, for their 1-D spectra (both bases)
        const size_t nbg = tbx.size() + tby.size();
        if (cudaMalloc((void **)&p->bxy64, nbg * sizeof(double)) != cudaSuccess) return SFFT_ERR_OOM;
        p->ws_bytes += nbg * sizeof(double);
        if (cudaMemcpy(p->bxy64, tbx.data(), tbx.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p->bxy64 + tbx.size(), tby.data(), tby.size() * sizeof(double), cudaMemcpyHostToDevice) !=
                cudaSuccess)
            return SFFT_ERR_CUDA;
    }

    // ---- FP64 x-functions of the zero-lag sums -----------------------------
    std::vector<double> x64;
    if (poly) {
        const int umax = (2 * c.dk > c.dk + c.db ? 2 * c.dk : c.dk + c.db);
        p->nallx = umax + 1;
        axis_table(1, 0, 0, p->nallx, -1, p->n0, x64);
    } else {
        p->nallx = nfx + nbx;
        x64.insert(x64.end(), tfx.begin(), tfx.end());
        x64.insert(x64.end(), tbx.begin(), tbx.end());
    }
    if (cudaMalloc((void **)&p->ftab64, x64.size() * sizeof(double)) != cudaSuccess) return SFFT_ERR_OOM;
    p->ws_bytes += x64.size() * sizeof(double);
    if (cudaMemcpy(p->ftab64, x64.data(), x64.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return SFFT_ERR_CUDA;

    // ---- row moments and zero-lag descriptors -------------------------------
    const int npo = nk * (nk + 1) / 2;
    p->nzm = npo + nk * nb + nk + nb;
    // polynomial basis: Lambda in closed form from the 2-D moments
    // mu(u, v) = sum x^u y^v Rm, u, v <= dk + db, appended to z0
    const int Dm = c.dk + c.db;
    p->lam_closed = (poly && c.w0 <= 16 && c.w1 <= 16) ? 1 : 0;  // half-widths of k_lambda_closed's tables
    p->z_mu = p->nzm;
    if (poly) p->nzm += (Dm + 1) * (Dm + 1);
    std::vector<int> zd((size_t)p->nzm * 3);
    std::vector<int> rd;
    // row-moment indices
    int fRR = 0, fR = 0, fRS = 0, fS = 0, nrr = 0, nrb = 0;
    if (poly) {
        fRR = 0;
        fR = 2 * c.dk + 1;
        fRS = fR + c.dk + c.db + 1;
        fS = fRS + c.dk + 1;
        p->nmom = fS + c.db + 1;
    } else {
        nrr = nfy * (nfy + 1) / 2;
        nrb = nfy * nby;
        p->nmom = nrr + nrb + nfy + nby;
        rd.resize((size_t)p->nmom * 3);
        int d = 0;
        for (int j = 0; j < nfy; ++j)
            for (int j2 = j; j2 < nfy; ++j2) {
                rd[3 * d] = 0, rd[3 * d + 1] = j, rd[3 * d + 2] = j2;
                ++d;
            }
        for (int j = 0; j < nfy; ++j)
            for (int q = 0; q < nby; ++q) {
                rd[3 * d] = 1, rd[3 * d + 1] = j, rd[3 * d + 2] = nfy + q;
                ++d;
            }
        for (int j = 0; j < nfy; ++j) {
            rd[3 * d] = 2, rd[3 * d + 1] = j, rd[3 * d + 2] = -1;
            ++d;
        }
        for (int q = 0; q < nby; ++q) {
            rd[3 * d] = 3, rd[3 * d + 1] = nfy + q, rd[3 * d + 2] = -1;
            ++d;
        }
    }
    auto rr_idx = [&](int j, int j2) {
        if (j > j2) {
            const int z = j;
            j = j2;
            j2 = z;
        }
        return j * nfy - j * (j - 1) / 2 + (j2 - j);
    };
    auto put = [&](int e, int d, int xa, int xb) {
        zd[3 * e] = d;
        zd[3 * e + 1] = xa;
        zd[3 * e + 2] = xb;
    };
    int e = 0;
    for (int t = 0; t < nk; ++t)
        for (int u = t; u < nk; ++u) {
            const int it = h[bv.o_ti + t], jt = h[bv.o_tj + t], iu = h[bv.o_ti + u], ju = h[bv.o_tj + u];
            if (poly) put(e++, fRR + jt + ju, it + iu, -1);
            else put(e++, rr_idx(jt, ju), it, iu);
        }
    for (int t = 0; t < nk; ++t)
        for (int sidx = 0; sidx < nb; ++sidx) {
            const int it = h[bv.o_ti + t], jt = h[bv.o_tj + t];
            const int pp = h[bv.o_sp + sidx], qq = h[bv.o_sq + sidx];
            if (poly) put(e++, fR + jt + qq, it + pp, -1);
            else put(e++, nrr + jt * nby + qq, it, nfx + pp);
        }
    for (int t = 0; t < nk; ++t) {
        const int it = h[bv.o_ti + t], jt = h[bv.o_tj + t];
        if (poly) put(e++, fRS + jt, it, -1);
        else put(e++, nrr + nrb + jt, it, -1);
    }
    for (int sidx = 0; sidx < nb; ++sidx) {
        const int pp = h[bv.o_sp + sidx], qq = h[bv.o_sq + sidx];
        if (poly) put(e++, fS + qq, pp, -1);
        else put(e++, nrr + nrb + nfy + qq, nfx + pp, -1);
    }
    if (poly)
        for (int u = 0; u <= Dm; ++u)
            for (int v = 0; v <= Dm; ++v) put(e++, fR + v, u, -1);
    if (p->lam_closed) {  // 16 row-chunk partial sums of the boundary column moments, then the corners
        const size_t nbnd = (size_t)16 * 2 * c.w1 * (Dm + 1) + (size_t)4 * c.w0 * c.w1 + 1;
        if (cudaMalloc((void **)&p->bnd, nbnd * sizeof(double)) != cudaSuccess) return SFFT_ERR_OOM;
        p->ws_bytes += nbnd * sizeof(double);
    }
    if (cudaMalloc((void **)&p->d_zdesc, zd.size() * sizeof(int)) != cudaSuccess) return SFFT_ERR_OOM;
    if (cudaMalloc((void **)&p->z0, (size_t)p->nzm * sizeof(double)) != cudaSuccess) return SFFT_ERR_OOM;
    p->ws_bytes += zd.size() * sizeof(int) + (size_t)p->nzm * sizeof(double);
    if (cudaMemcpy(p->d_zdesc, zd.data(), zd.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return SFFT_ERR_CUDA;
    if (!poly) {
        if (cudaMalloc((void **)&p->d_rdesc, rd.size() * sizeof(int)) != cudaSuccess) return SFFT_ERR_OOM;
        p->ws_bytes += rd.size() * sizeof(int);
        if (cudaMemcpy(p->d_rdesc, rd.data(), rd.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            return SFFT_ERR_CUDA;
    }

    // ---- C (Eq. B11): separable sums of the background functions ------------
    std::vector<double> cm((size_t)nb * nb);
    for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b) {
            const int pa = h[bv.o_sp + a], qa = h[bv.o_sq + a], pb = h[bv.o_sp + b], qb = h[bv.o_sq + b];
            double sx = 0.0, sy = 0.0;
            for (int x = 0; x < p->n0; ++x) sx += tbx[(size_t)pa * p->n0 + x] * tbx[(size_t)pb * p->n0 + x];
            for (int y = 0; y < p->n1; ++y) sy += tby[(size_t)qa * p->n1 + y] * tby[(size_t)qb * p->n1 + y];
            cm[(size_t)a * nb + b] = sx * sy;
        }
    if (cudaMalloc((void **)&p->cmat, cm.size() * sizeof(double)) != cudaSuccess) return SFFT_ERR_OOM;
    p->ws_bytes += cm.size() * sizeof(double);
    if (cudaMemcpy(p->cmat, cm.data(), cm.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return SFFT_ERR_CUDA;

    // ---- device int tables and unknowns (after the host tables are final) ----
    if (cudaMemcpy(p->d_int, h, (size_t)o * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return SFFT_ERR_CUDA;
    if (cudaMemcpy(p->unk, unk.data(), unk.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
        return SFFT_ERR_CUDA;
    (void)s;
    return SFFT_OK;
}

void basis_term_weights(const Plan *p, double xt0, double yt0, double *w) {
    const sfft_config &c = p->cfg;
    const BasisView &bv = p->bv;
    double bx[kMaxFun + 1], by[kMaxFun + 1];
    const bool poly = !p->bspline;
    if (!poly) {
        spl_eval(c.kdeg, c.kint, xt0, bx);
        spl_eval(c.kdeg, c.kint, yt0, by);
        const int K = spl_count(c.kdeg, c.kint);
        bx[K] = by[K] = 1.0;  // the constant function of a constant photometric ratio
    }
    for (int t = 0; t < bv.nk; ++t) {
        const int i = p->h_int[bv.o_ti + t], j = p->h_int[bv.o_tj + t];
        w[t] = poly ? ipow64(xt0, i) * ipow64(yt0, j) : bx[i] * by[j];
    }
}

}  // namespace sfft
