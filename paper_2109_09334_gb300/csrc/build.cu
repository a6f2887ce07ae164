// build.cu -- construction of the normal equations (Eq. 18-24 via App. B).
//
// Pipeline (all on the plan's stream):
//   k_rows     row pass: zero-fill with the mask, weight by yt^j, real FFT of
//              every row along y for j = 0..dk and of S; writes the row
//              transforms transposed ([image][m][x], x contiguous) and the
//              per-row moment sums used for the lag-zero entries.
//   k_moments  FP64 moments sum_x xt^u * (row moment) (Eq. B11, B15 and the
//              lag-zero values of Omega, Lambda, Theta).
//   k_cols     column pass: weight by xt^i, FFT along x, and store every
//              spectrum permuted so that the bins l = lb + NB*r (r < NA) of one
//              residue class lb are contiguous.
//   k_gather   for each column m and residue class lb: spectrum products
//              conj(U_a) U_b with the DC bin removed, an NA-point inverse DFT
//              over r, and the outer sum over lb with twiddles exp(2 pi i lb
//              rho/N0), accumulated with two-sum compensation (pruned inverse
//              DFT along x, only |rho| <= 2w (Omega) or w (Lambda, Theta)).
//   k_stage2   the remaining sum over m with exp(2 pi i m rho/N1) (and the
//              1-D spectrum of y^q for Lambda), compensated, to FP64 lag tables.
//   k_assemble the index maps of Eq. B5, B7, B9, B11, B13, B15 into M and rhs.
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft.cuh"
#include "fft16.cuh"
#include "internal.h"

namespace sfft {

constexpr int kMaxMom = 24;  // per-row moments for dk, db <= 3

struct MomLayout {
    int fRR, fR, fRS, fS, n;
};
__host__ __device__ inline MomLayout mom_layout(int dk, int db) {
    MomLayout m;
    m.fRR = 0;
    m.fR = 2 * dk + 1;
    m.fRS = m.fR + dk + db + 1;
    m.fS = m.fRS + dk + 1;
    m.n = m.fS + db + 1;
    return m;
}

template <typename I>
__device__ __forceinline__ double load_img(const I *p, size_t k) { return (double)p[k]; }

// ---------------------------------------------------------------------------
// Row pass.  Block: TR rows, one group of G = n1/16 threads per row.  The two
// real sequences of a packed complex FFT (yt^j * Rm for j <= dk, then Sm) are
// transformed together and separated after; the transforms are written
// transposed ([image][m][x]) for the column pass.
template <typename T, typename I>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) k_rows(int n0, int n1, int nfy, int TR, const I *__restrict__ R,
                                               const I *__restrict__ S, const uint8_t *__restrict__ mask,
                                               cpx<T> *__restrict__ F, const cpx<T> *__restrict__ tw1g,
                                               const T *__restrict__ fy, int pf_dist) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = n1 / 16;
    const int np = padded_len(n1) + 4;  // +4: rows start in different banks
    // the pass-ordered twiddles are read through L1 (a shared copy per block
    // cost more than it saved)
    const cpx<T> *tw = tw1g;
    cpx<T> *Z = reinterpret_cast<cpx<T> *>(smem_raw);  // TR * np
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int grp = tid / G, gt = tid - grp * G;
    const int nseq = nfy + 1;
    const int nfft = (nseq + 1) / 2;
    // packed pair index fastest: blocks that read the same rows run together
    const int f = blockIdx.x % nfft;
    const int x0b = (blockIdx.x / nfft) * TR;
    const int sa = 2 * f, sb = 2 * f + 1;
    cpx<T> *zr = Z + (size_t)grp * np;
    if (x0b + grp < n0) {
        // thread gt loads pixels [16 gt, 16 gt + 16) of its row (all loads in flight)
        const size_t rowoff = (size_t)(x0b + grp) * n1;
        const int y0 = 16 * gt;
        T rv[16], sv[16];
        load16<T, I>(R + rowoff + y0, rv);
        load16<T, I>(S + rowoff + y0, sv);
        // the rows of the block pf_dist launches later (about one wave of
        // resident blocks) into L2, so that its loads need not wait for HBM
        if (pf_dist > 0) {
            const int xp = ((blockIdx.x + pf_dist) / nfft) * TR + grp;
            if (xp < n0) {
                const size_t po = (size_t)xp * n1 + y0;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(R + po));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(S + po));
                if (mask != nullptr && (gt & 7) == 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(mask + po));
            }
        }
        if (mask != nullptr) {
            const uint4 mv = __ldg(reinterpret_cast<const uint4 *>(mask + rowoff + y0));
            const unsigned mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const bool keep = ((mw[c >> 2] >> (8 * (c & 3))) & 0xffu) != 0u;
                rv[c] = keep ? rv[c] : (T)0;
                sv[c] = keep ? sv[c] : (T)0;
            }
        }
        const T inv = (T)1 / (T)(n1 - 1);  // yt = (2y - (n1 - 1)) / (n1 - 1), by one multiply
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const T yt = (T)(2 * (y0 + c) - (n1 - 1)) * inv;
            // weights yt^j (polynomial) or the tabulated y-functions (B-spline)
            const T wa = fy ? (sa < nfy ? fy[(size_t)sa * n1 + y0 + c] : (T)0) : ipow(yt, sa);
            const T wb = fy ? (sb < nfy ? fy[(size_t)sb * n1 + y0 + c] : (T)0) : ipow(yt, sb);
            const T va = (sa < nfy) ? rv[c] * wa : sv[c];
            const T vb = (sb < nfy) ? rv[c] * wb : (sb == nfy ? sv[c] : (T)0);
            zr[pad16(y0 + c)] = mk(va, vb);
        }
    }
    __syncthreads();
    group_fft(zr, n1, -1, tw, gt, G);
    // separate the two real transforms and write them transposed: thread tid
    // takes row r = tid mod TR and frequencies m = tid / TR + k * (nthr / TR),
    // so its addresses advance by constant steps
    const int h1c = n1 / 2 + 1;
    const int ltr = __ffs(TR) - 1;  // TR is a power of two
    const int r = tid & (TR - 1);
    if (x0b + r < n0) {  // rows past the end (n0 not a multiple of TR)
        const int mstep = nthr >> ltr;
        const size_t ostep = (size_t)mstep * n0;
        const cpx<T> *zz = Z + (size_t)r * np;
        int m = tid >> ltr;
        cpx<T> *fa = F + (size_t)sa * h1c * n0 + x0b + r + (size_t)m * n0;
        cpx<T> *fb = F + (size_t)sb * h1c * n0 + x0b + r + (size_t)m * n0;
        const bool two = sb < nseq;
        for (; m < h1c; m += mstep, fa += ostep, fb += ostep) {
            const cpx<T> z = zz[pad16(m)];
            const cpx<T> zc = conj(zz[pad16((n1 - m) & (n1 - 1))]);
            *fa = scale(z + zc, (T)0.5);
            if (two) *fb = mul_i(scale(z - zc, (T)0.5), -1);
        }
    }
}

// Row pass for a row length n1 that is not a power of two: Bluestein DFTs of
// length n1 through FFTs of length m1 (fft16.cuh); one group of m1/16
// threads per row, TR rows per block, otherwise as k_rows (two real
// sequences per complex transform, transposed output).
template <typename T, typename I>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) k_rows_blu(int n0, int n1, int m1, int nfy, int TR,
                                               const I *__restrict__ R, const I *__restrict__ S,
                                               const uint8_t *__restrict__ mask, cpx<T> *__restrict__ F,
                                               const cpx<T> *__restrict__ chirp, const cpx<T> *__restrict__ bfilt,
                                               const cpx<T> *__restrict__ twpm, const T *__restrict__ fy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = m1 / 16;
    const int np = padded_len(m1) + 4;
    cpx<T> *Z = reinterpret_cast<cpx<T> *>(smem_raw);  // TR * np
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int grp = tid / G, gt = tid - grp * G;
    const int nseq = nfy + 1;
    const int nfft = (nseq + 1) / 2;
    const int f = blockIdx.x % nfft;
    const int x0b = (blockIdx.x / nfft) * TR;
    const int sa = 2 * f, sb = 2 * f + 1;
    cpx<T> *zr = Z + (size_t)grp * np;
    if (x0b + grp < n0) {
        const size_t rowoff = (size_t)(x0b + grp) * n1;
        for (int y = gt; y < n1; y += G) {
            const bool keep = mask == nullptr || mask[rowoff + y] != 0;
            const T rv = keep ? (T)R[rowoff + y] : (T)0;
            const T sv = keep ? (T)S[rowoff + y] : (T)0;
            const T yt = coord<T>(y, n1);
            const T wa = fy ? (sa < nfy ? fy[(size_t)sa * n1 + y] : (T)0) : ipow(yt, sa);
            const T wb = fy ? (sb < nfy ? fy[(size_t)sb * n1 + y] : (T)0) : ipow(yt, sb);
            const T va = (sa < nfy) ? rv * wa : sv;
            const T vb = (sb < nfy) ? rv * wb : (sb == nfy ? sv : (T)0);
            zr[pad16(y)] = mk(va, vb);
        }
    }
    __syncthreads();
    bluestein(zr, n1, m1, -1, chirp, bfilt, twpm, gt, G);
    // separate the two real transforms and write them transposed
    const int h1c = n1 / 2 + 1;
    const int total = h1c * TR;
    cpx<T> *Fa = F + (size_t)sa * h1c * n0 + x0b;
    cpx<T> *Fb = F + (size_t)sb * h1c * n0 + x0b;
    for (int idx = tid; idx < total; idx += nthr) {
        const int m = idx / TR, r = idx - m * TR;
        if (x0b + r >= n0) continue;
        const cpx<T> *zz = Z + (size_t)r * np;
        const cpx<T> z = zz[pad16(m)];
        const cpx<T> zc = conj(zz[pad16(m == 0 ? 0 : n1 - m)]);
        const size_t o = (size_t)m * n0 + r;
        Fa[o] = scale(z + zc, (T)0.5);
        if (sb < nseq) Fb[o] = mul_i(scale(z - zc, (T)0.5), -1);
    }
}

// ---------------------------------------------------------------------------
// Per-row moment sums (for the lag-zero entries, C and E): one block per row,
// plain per-thread partials, then a two-sum reduction across the block.
//   RR_v = sum_y Rm^2 yt^v (v <= 2dk), R_v = sum_y Rm yt^v (v <= dk+db),
//   RS_v = sum_y Rm Sm yt^v (v <= dk), S_v = sum_y Sm yt^v (v <= db).
// NRR, NR, NRS, NS: the powers accumulated of each kind (the largest needed
// for any degrees: 7, 7, 4, 4; D_K = D_B = 2 needs 5, 5, 3, 3)
template <typename T, typename I, int NRR = 7, int NR = 7, int NRS = 4, int NS = 4>
__global__ void __launch_bounds__(256) k_row_moments(int n1, int dk, int db, const I *__restrict__ R,
                                                     const I *__restrict__ S, const uint8_t *__restrict__ mask,
                                                     double *__restrict__ rowmom) {
    __shared__ T part_s[kMaxMom][256];  // plain per-thread partials, transposed for the reduction
    const int x0 = blockIdx.x, tid = threadIdx.x, nthr = blockDim.x;
    const size_t rowoff = (size_t)x0 * n1;
    const MomLayout ml = mom_layout(dk, db);
    T pRR[7], pR[7], pRS[4], pS[4];
#pragma unroll
    for (int v = 0; v < 7; ++v) pRR[v] = pR[v] = (T)0;
#pragma unroll
    for (int v = 0; v < 4; ++v) pRS[v] = pS[v] = (T)0;
    const T inv = (T)1 / (T)(n1 - 1);  // yt = (2y - (n1 - 1)) / (n1 - 1)
    auto accum = [&](int y, T r, T sval, bool keep) {
        const T rv = keep ? r : (T)0, sv = keep ? sval : (T)0;
        const T yt = (T)(2 * y - (n1 - 1)) * inv;
        T p = (T)1;
#pragma unroll
        for (int v = 0; v < 7; ++v) {
            if (v < NRR) pRR[v] += rv * rv * p;
            if (v < NR) pR[v] += rv * p;
            if (v < NRS) pRS[v] += rv * sv * p;
            if (v < NS) pS[v] += sv * p;
            p *= yt;
        }
    };
    if (sizeof(I) == 4 && (n1 & 3) == 0) {
        // rows of 16-byte-aligned float images: four pixels per load, all of a
        // thread's loads in flight
        const float4 *R4 = reinterpret_cast<const float4 *>(R + rowoff);
        const float4 *S4 = reinterpret_cast<const float4 *>(S + rowoff);
        const uchar4 *M4 = mask ? reinterpret_cast<const uchar4 *>(mask + rowoff) : nullptr;
#pragma unroll 4
        for (int c = tid; c < (n1 >> 2); c += nthr) {
            const float4 r = __ldg(R4 + c), sv = __ldg(S4 + c);
            const uchar4 m = M4 ? M4[c] : make_uchar4(1, 1, 1, 1);
            accum(4 * c, (T)r.x, (T)sv.x, m.x != 0);
            accum(4 * c + 1, (T)r.y, (T)sv.y, m.y != 0);
            accum(4 * c + 2, (T)r.z, (T)sv.z, m.z != 0);
            accum(4 * c + 3, (T)r.w, (T)sv.w, m.w != 0);
        }
    } else {
#pragma unroll 4
        for (int y = tid; y < n1; y += nthr)
            accum(y, (T)R[rowoff + y], (T)S[rowoff + y], mask == nullptr || mask[rowoff + y] != 0);
    }
    // the partials that are needed, at their moment index
#pragma unroll
    for (int k = 0; k < 22; ++k) {
        T val;
        int dst;
        if (k < 7) { val = pRR[k]; dst = (k <= 2 * dk) ? ml.fRR + k : -1; }
        else if (k < 14) { val = pR[k - 7]; dst = (k - 7 <= dk + db) ? ml.fR + k - 7 : -1; }
        else if (k < 18) { val = pRS[k - 14]; dst = (k - 14 <= dk) ? ml.fRS + k - 14 : -1; }
        else { val = pS[k - 18]; dst = (k - 18 <= db) ? ml.fS + k - 18 : -1; }
        if (dst >= 0) part_s[dst][tid] = val;
    }
    __syncthreads();
    // warp w reduces moments w, w + nw, ...: each lane a two-sum over its
    // threads' partials, then across the warp, in a fixed order
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    for (int d = warp; d < ml.n; d += nw) {
        Acc<T> a;
        a.zero();
        for (int k = lane; k < nthr; k += 32) a.add(part_s[d][k]);
        for (int o = 16; o > 0; o >>= 1) shfl_add(a, o);
        if (lane == 0) rowmom[(size_t)x0 * ml.n + d] = a.wide();
    }
}

// Per-row moments of the B-spline basis: moment d of row x is
//   sum_y v_kind(y) ytab[ya](y) (ytab[yb](y) if yb >= 0),
// v = Rm^2 (kind 0), Rm (1), Rm Sm (2), Sm (3); ytab = [fy | by] rows.
// Block (row, chunk of kMomChunk moments): plain per-thread partials, then a
// two-sum reduction across the block, as in k_row_moments.
constexpr int kMomChunk = 12;

template <typename T, typename I>
__global__ void k_row_moments_tab(int n1, int nmom, const int *__restrict__ rdesc, const T *__restrict__ ytab,
                                  const I *__restrict__ R, const I *__restrict__ S,
                                  const uint8_t *__restrict__ mask, double *__restrict__ rowmom) {
    __shared__ Acc<T> red[32][kMomChunk];
    const int x0 = blockIdx.x, d0 = blockIdx.y * kMomChunk, tid = threadIdx.x, nthr = blockDim.x;
    const size_t rowoff = (size_t)x0 * n1;
    int kind[kMomChunk], ya[kMomChunk], yb[kMomChunk];
    T part[kMomChunk];
#pragma unroll
    for (int k = 0; k < kMomChunk; ++k) {
        const bool ok = d0 + k < nmom;
        kind[k] = ok ? rdesc[3 * (d0 + k)] : -1;
        ya[k] = ok ? rdesc[3 * (d0 + k) + 1] : 0;
        yb[k] = ok ? rdesc[3 * (d0 + k) + 2] : -1;
        part[k] = (T)0;
    }
    for (int y = tid; y < n1; y += nthr) {
        const T keep = (mask == nullptr || mask[rowoff + y] != 0) ? (T)1 : (T)0;
        const T rv = (T)R[rowoff + y] * keep;
        const T sv = (T)S[rowoff + y] * keep;
#pragma unroll
        for (int k = 0; k < kMomChunk; ++k) {
            if (kind[k] < 0) continue;
            T w = ytab[(size_t)ya[k] * n1 + y];
            if (yb[k] >= 0) w *= ytab[(size_t)yb[k] * n1 + y];
            const T v = kind[k] == 0 ? rv * rv : (kind[k] == 1 ? rv : (kind[k] == 2 ? rv * sv : sv));
            part[k] += v * w;
        }
    }
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
#pragma unroll
    for (int k = 0; k < kMomChunk; ++k) {
        Acc<T> a;
        a.zero();
        a.add(part[k]);
        for (int o = 16; o > 0; o >>= 1) shfl_add(a, o);
        if (lane == 0) red[warp][k] = a;
    }
    __syncthreads();
    if (tid < kMomChunk && d0 + tid < nmom) {
        Acc<T> a = red[0][tid];
        for (int w = 1; w < nw; ++w) a.add(red[w][tid]);
        rowmom[(size_t)x0 * nmom + d0 + tid] = a.wide();
    }
}

// ---------------------------------------------------------------------------
// Boundary data of the closed-form Lambda (polynomial basis), FP64, in
// kBndChunks partial sums over row chunks (added in order by the consumer):
//   bnd[(h * 2 w1 + c) * (D+1) + u] = sum over rows x of chunk h of xt^u Rm(x, y_c)
//       for the 2 w1 boundary columns y_c = c (c < w1) or n1 - 2 w1 + c,
//   bnd[kBndChunks * 2 w1 (D+1) + r * 2 w1 + c] = Rm(x_r, y_c) for the
//       2 w0 boundary rows x_r = r (r < w0) or n0 - 2 w0 + r.
// Grid (2 w1 + 1, kBndChunks): block (c, h) one column and row chunk; blocks
// (2 w1, 0) the corner pixels.
constexpr int kMaxDm = 6;  // dk + db
constexpr int kBndChunks = 16;
constexpr int kMaxWClosed = 16;  // kernel half-widths of the closed-form Lambda

template <typename I>
__global__ void __launch_bounds__(256) k_boundary(int n0, int n1, int w0, int w1, int D, const I *__restrict__ R,
                                                  const uint8_t *__restrict__ mask, double *__restrict__ bnd) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nbc = 2 * w1;
    const int c = blockIdx.x, h = blockIdx.y;
    if (c == nbc) {
        if (h != 0) return;
        for (int e = tid; e < 2 * w0 * nbc; e += nthr) {
            const int r = e / nbc, cc = e - r * nbc;
            const int x = r < w0 ? r : n0 - 2 * w0 + r, y = cc < w1 ? cc : n1 - 2 * w1 + cc;
            const size_t k = (size_t)x * n1 + y;
            bnd[(size_t)kBndChunks * nbc * (D + 1) + e] = (mask == nullptr || mask[k] != 0) ? (double)R[k] : 0.0;
        }
        return;
    }
    const int y = c < w1 ? c : n1 - 2 * w1 + c;
    const int per = (n0 + kBndChunks - 1) / kBndChunks;
    const int xa = h * per, xb = min(n0, xa + per);
    double acc[kMaxDm + 1];
#pragma unroll
    for (int u = 0; u <= kMaxDm; ++u) acc[u] = 0.0;
    for (int x = xa + tid; x < xb; x += nthr) {
        const size_t k = (size_t)x * n1 + y;
        const double v = (mask == nullptr || mask[k] != 0) ? (double)R[k] : 0.0;
        const double xt = coord<double>(x, n0);
        double pw = v;
#pragma unroll
        for (int u = 0; u <= kMaxDm; ++u) {
            if (u <= D) acc[u] += pw;
            pw *= xt;
        }
    }
    __shared__ double red[8][kMaxDm + 1];
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int u = 0; u <= kMaxDm; ++u) {
        double v = acc[u];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][u] = v;
    }
    __syncthreads();
    if (tid <= D) {
        double v = 0.0;
        for (int w = 0; w < (nthr >> 5); ++w) v += red[w][tid];
        bnd[((size_t)h * nbc + c) * (D + 1) + tid] = v;
    }
}

// Lambda_ts(rho) = sum_x g_t(x) T_s((x + rho) mod N) in closed form for the
// polynomial basis, g_t = xt^i yt^j Rm, T_s = xt^p yt^q (Eq. B8), FP64.
// With X_e(x) = (xt + 2 rho0/(N0-1))^p, the shifted monomial as if it did not
// wrap, and dX = X_wrapped - X_e (non-zero only on the |rho0| rows where x +
// rho0 wraps), likewise Y_e, dY along y:
//   Lambda = sum g X_e Y_e + sum g dX Y_e + sum g X_e dY + sum g dX dY,
// the first term by binomial expansion over the 2-D moments mu(u, v), the
// second from the per-row moments of the wrapping rows, the third from the
// column moments of the wrapping columns, the last over the corner pixels.
// One block per (t, s): the per-row and per-column pieces that do not depend
// on both lags are built once in shared memory; thread e then takes lag e.
__device__ __forceinline__ double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

__global__ void __launch_bounds__(256) k_lambda_closed(int n0, int n1, int w0, int w1, int D, BasisView bv,
                                                       const double *__restrict__ rowmom, int nmom, int fR,
                                                       const double *__restrict__ mu, const double *__restrict__ bnd,
                                                       double *__restrict__ lagla) {
    constexpr int W = kMaxWClosed, NR = 2 * W + 1;
    __shared__ double sbx[NR][kMaxDm + 1], sby[NR][kMaxDm + 1];  // C(p,k) h0^(p-k), C(q,l) h1^(q-l)
    __shared__ double sdx[NR][W], sdy[NR][W];                    // dX(rho0, k-th wrapping row), dY
    __shared__ double srow[NR][2 * W];  // [rho1][r]: sum_y (Y_e Rm yt^j)(x_r) + sum over wrapping y of Rm yt^j dY
    __shared__ double scol[NR][2 * W];  // [rho0][c]: sum_x X_e Rm xt^i at boundary column c
    __shared__ double sxi[2 * W], syj[2 * W];  // xt^i at the boundary rows, yt^j at the boundary columns
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int L0 = 2 * w0 + 1, L1 = 2 * w1 + 1;
    const int ts = blockIdx.x, t = ts / bv.nb, s = ts - t * bv.nb;
    const int i = bv.ti(t), j = bv.tj(t), p = bv.sp(s), q = bv.sq(s);
    const int nbc = 2 * w1, nbr = 2 * w0;
    const double *corner = bnd + (size_t)kBndChunks * nbc * (D + 1);
    auto xrow = [&](int r) { return r < w0 ? r : n0 - 2 * w0 + r; };
    auto ycol = [&](int c) { return c < w1 ? c : n1 - 2 * w1 + c; };
    // rows (columns) where x + rho0 (y + rho1) wraps: k-th of them
    auto wrow = [&](int rho0, int k) { return rho0 > 0 ? n0 - rho0 + k : k; };
    auto wcol = [&](int rho1, int k) { return rho1 > 0 ? n1 - rho1 + k : k; };
    for (int e = tid; e < L0 * (kMaxDm + 1); e += nthr) {
        const int a = e / (kMaxDm + 1), k = e - a * (kMaxDm + 1);
        const double h0 = 2.0 * (a - w0) / (double)(n0 - 1);
        sbx[a][k] = k <= p ? binom(p, k) * ipow(h0, p - k) : 0.0;
    }
    for (int e = tid; e < L1 * (kMaxDm + 1); e += nthr) {
        const int b = e / (kMaxDm + 1), l = e - b * (kMaxDm + 1);
        const double h1 = 2.0 * (b - w1) / (double)(n1 - 1);
        sby[b][l] = l <= q ? binom(q, l) * ipow(h1, q - l) : 0.0;
    }
    for (int e = tid; e < L0 * w0; e += nthr) {
        const int a = e / max(w0, 1), k = e - a * max(w0, 1);
        const int rho0 = a - w0, nx = rho0 > 0 ? rho0 : -rho0;
        double d = 0.0;
        if (k < nx) {
            const int x = wrow(rho0, k);
            const int xw = x + rho0 >= n0 ? x + rho0 - n0 : (x + rho0 < 0 ? x + rho0 + n0 : x + rho0);
            d = ipow(coord<double>(xw, n0), p) - ipow(coord<double>(x, n0) + 2.0 * rho0 / (double)(n0 - 1), p);
        }
        sdx[a][k] = d;
    }
    for (int e = tid; e < L1 * w1; e += nthr) {
        const int b = e / max(w1, 1), k = e - b * max(w1, 1);
        const int rho1 = b - w1, ny = rho1 > 0 ? rho1 : -rho1;
        double d = 0.0;
        if (k < ny) {
            const int y = wcol(rho1, k);
            const int yw = y + rho1 >= n1 ? y + rho1 - n1 : (y + rho1 < 0 ? y + rho1 + n1 : y + rho1);
            d = ipow(coord<double>(yw, n1), q) - ipow(coord<double>(y, n1) + 2.0 * rho1 / (double)(n1 - 1), q);
        }
        sdy[b][k] = d;
    }
    for (int r = tid; r < nbr; r += nthr) sxi[r] = ipow(coord<double>(xrow(r), n0), i);
    for (int c = tid; c < nbc; c += nthr) syj[c] = ipow(coord<double>(ycol(c), n1), j);
    __syncthreads();
    // srow[rho1][r] = sum_l by[l] rowmom(x_r, j + l) + sum_(wrapping y) Rm(x_r, y) yt^j dY(y)
    for (int e = tid; e < L1 * nbr; e += nthr) {
        const int b = e / nbr, r = e - b * nbr;
        const int rho1 = b - w1, ny = rho1 > 0 ? rho1 : -rho1;
        const int x = xrow(r);
        double v = 0.0;
        for (int l = 0; l <= q; ++l) v += sby[b][l] * rowmom[(size_t)x * nmom + fR + j + l];
        for (int k = 0; k < ny; ++k) {
            const int y = wcol(rho1, k);
            const int c = y < w1 ? y : y - (n1 - nbc);
            v += corner[r * nbc + c] * syj[c] * sdy[b][k];
        }
        srow[b][r] = v;
    }
    // scol[rho0][c] = sum_k bx[k] (column moment of y_c at i + k), chunks added in order
    for (int e = tid; e < L0 * nbc; e += nthr) {
        const int a = e / nbc, c = e - a * nbc;
        double v = 0.0;
        for (int k = 0; k <= p; ++k) {
            double cm = 0.0;
            for (int h = 0; h < kBndChunks; ++h) cm += bnd[((size_t)h * nbc + c) * (D + 1) + i + k];
            v += sbx[a][k] * cm;
        }
        scol[a][c] = v;
    }
    __syncthreads();
    for (int e = tid; e < L0 * L1; e += nthr) {
        const int a = e / L1, b = e - a * L1;
        const int rho0 = a - w0, rho1 = b - w1;
        const int nx = rho0 > 0 ? rho0 : -rho0, ny = rho1 > 0 ? rho1 : -rho1;
        double A = 0.0;  // sum g X_e Y_e by binomial expansion over mu
        for (int k = 0; k <= p; ++k)
            for (int l = 0; l <= q; ++l) A += sbx[a][k] * sby[b][l] * mu[(i + k) * (D + 1) + (j + l)];
        double BD = 0.0;  // wrapping rows: sum dX xt^i (Y_e-weighted row sums + corner dY part)
        for (int k = 0; k < nx; ++k) {
            const int x = wrow(rho0, k);
            const int r = x < w0 ? x : x - (n0 - nbr);
            BD += sdx[a][k] * sxi[r] * srow[b][r];
        }
        double Cc = 0.0;  // wrapping columns: sum dY yt^j (X_e-weighted column sums)
        for (int k = 0; k < ny; ++k) {
            const int y = wcol(rho1, k);
            const int c = y < w1 ? y : y - (n1 - nbc);
            Cc += sdy[b][k] * syj[c] * scol[a][c];
        }
        lagla[(size_t)ts * L0 * L1 + e] = A + BD + Cc;
    }
}

// ---------------------------------------------------------------------------
// Zero-lag values (FP64): z0[e] = sum_x xtab[xa](x) (xtab[xb](x) if xb >= 0)
// rowmom[x][d] for descriptor e = (d, xa, xb).
__global__ void k_zero_lag(int n0, int nmom, const int *__restrict__ zdesc, const double *__restrict__ xtab,
                           const double *__restrict__ rowmom, double *__restrict__ z0) {
    const int e = blockIdx.x;
    const int d = zdesc[3 * e], xa = zdesc[3 * e + 1], xb = zdesc[3 * e + 2];
    double acc = 0.0;
    for (int x = threadIdx.x; x < n0; x += blockDim.x) {
        double w = xtab[(size_t)xa * n0 + x];
        if (xb >= 0) w *= xtab[(size_t)xb * n0 + x];
        acc += w * rowmom[(size_t)x * nmom + d];
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
        z0[e] = v;
    }
}

// ---------------------------------------------------------------------------
// Column pass.  Block (chunk, m): GI output images in parallel, one group of
// G = n0/16 threads each; the chunks of one column are neighbours in launch
// order, so the row transforms they share are read from L2.  Image t < nk is
// the term (i, j): the row transform of yt^j * Rm weighted by xt^i; t = nk
// is Sm.  Output layout U[t][m][lb*NA + r] = spectrum at l = lb + NB*r.
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) k_cols(int n0, int n1, BasisView bv, int na, int nbk, int GI,
                                               const cpx<T> *__restrict__ F, cpx<T> *__restrict__ U,
                                               const cpx<T> *__restrict__ tw0g, const T *__restrict__ fx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = n0 / 16;
    const int np = padded_len(n0);
    cpx<T> *Z = reinterpret_cast<cpx<T> *>(smem_raw);  // GI * np
    const int tid = threadIdx.x;
    const int grp = tid / G, gt = tid - grp * G;
    const int m = blockIdx.y;
    const int h1c = n1 / 2 + 1;
    const int nk = bv.nk;
    const int t = blockIdx.x * GI + grp;
    const bool act = t <= nk;
    // the pass-ordered twiddles are read through L1 (the whole table is
    // 8 n0 bytes and every block of the launch reads it)
    const cpx<T> *tw = tw0g;
    cpx<T> *zr = Z + (size_t)grp * np;
    if (act) {
        // thread gt loads elements gt + G c, c < 16: coalesced, all in flight
        int i = 0, j = bv.nfy;  // t = nk: Sm, weight 1
        if (t < nk) {
            i = bv.ti(t);
            j = bv.tj(t);
        }
        const cpx<T> *col = F + ((size_t)j * h1c + m) * n0 + gt;
        cpx<T> v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = col[G * c];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int x = gt + G * c;
            const T wx = (fx && t < nk) ? fx[(size_t)i * n0 + x] : ipow(coord<T>(x, n0), i);
            zr[pad16(x)] = scale(v[c], wx);
        }
    }
    __syncthreads();
    // the last pass stores bin l = lb + NB*r at lb*(NA+1) + r (NA, NB powers of two)
    const int lna = __ffs(na) - 1, lnb = __ffs(nbk) - 1;
    group_fft(zr, n0, -1, tw, gt, G, lnb, na);
    if (act) {
        // element o = gt + G k sits at (o / na) (na + 1) + o mod na in the
        // residue-class layout; with na | G that advances by (G / na)(na + 1)
        cpx<T> *out = U + ((size_t)t * h1c + m) * n0;
        if ((G & (na - 1)) == 0) {
            const cpx<T> *src = zr + (gt >> lna) * (na + 1) + (gt & (na - 1));
            const int sstep = (G >> lna) * (na + 1);
            for (int o = gt; o < n0; o += G, src += sstep) out[o] = *src;
        } else {
            for (int o = gt; o < n0; o += G) {
                const int lb = o >> lna, r = o & (na - 1);
                out[o] = zr[lb * (na + 1) + r];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Gather: products and the split pruned inverse DFT along x.
//
// NA = 8*G.  Group of G lanes per product; lane r1 holds P(r1 + G*r2) for
// r2 = 0..7.  Y(s2 + 8*s1) = sum_r1 wG^(r1 s1) w^(r1 s2) sum_r2 w8^(r2 s2) P(r1 + G r2),
// w = exp(2 pi i / NA): an 8-point DFT in registers, a twiddle, a transpose
// through shared memory and a G-point DFT.
template <typename T, int G>
__device__ __forceinline__ void dftG(cpx<T> (&v)[G], int sgn) {
    if constexpr (G == 1) {
    } else if constexpr (G == 2) {
        cpx<T> a = v[0] + v[1], b = v[0] - v[1];
        v[0] = a;
        v[1] = b;
    } else if constexpr (G == 4) {
        dft4(v[0], v[1], v[2], v[3], sgn);
    } else {
        dft8(v, sgn);
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// One block per column m; one group of G lanes per spectrum product.  The
// residue-class tiles (NA bins of every image and of the x^p spectra) are
// double-buffered in shared memory with cp.async; image tiles are padded so
// that the groups of a warp read different banks, and the 8x8 transposes are
// XOR-swizzled.  Outer twiddles exp(2 pi i lb rho / N0) come from a per-block
// shared table.  Each output keeps a plain FP32 partial over kFold residue
// classes that is folded into a two-sum accumulator.
constexpr int kPad = 8;   // complex elements of padding per image tile / transpose region
// threads per block of the gather: the FP32 lag-range-16 variant runs blocks
// of 28 product groups, with registers for two blocks per SM (at four, the
// register cap of 72 spilled the accumulators: 0.54 -> 0.45 ms at 4096^2);
// the others take up to 48 groups
template <typename T, int NS>
__host__ __device__ constexpr int kGatherThreads() { return (sizeof(T) == 4 && NS == 5) ? 224 : 384; }
constexpr int kFold = 4;  // residue classes per plain partial sum (a power of two)

// NS output slots per lane: 8 in general; 5 when every lag half-range is at most
// 16 and G = 8 (then only s1 in {0, 1, 2, 6, 7} can be needed).
template <int G, int NS>
__device__ __forceinline__ int out_slot(int c, int s1) {
    if constexpr (NS == 8) return c * G + s1;
    else return s1 < 3 ? s1 : (s1 >= 6 ? s1 - 3 : -1);
}

template <typename T, int G, int NS>
__global__ void __launch_bounds__(kGatherThreads<T, NS>(), (sizeof(T) == 4 && NS == 5) ? 2 : 1) k_gather(int n0, int n1, int nk, int nxp, int nbk, int npairs, int hmax,
                                                const PairDesc *__restrict__ pairs, const cpx<T> *__restrict__ U,
                                                const cpx<T> *__restrict__ xhat, const cpx<T> *__restrict__ tw0,
                                                cpx<T> *__restrict__ Q) {
    constexpr int NA = 8 * G;
    constexpr int NAP = NA + kPad;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nimg = nk + 1;
    const int tile = (nimg + nxp) * NAP;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ngroups = nthr / G;
    cpx<T> *sU = reinterpret_cast<cpx<T> *>(smem_raw);  // 2 * tile (double buffer)
    cpx<T> *sT = sU + 2 * (size_t)tile;                 // ngroups * NAP (transposes)
    cpx<T> *sW = sT + (size_t)ngroups * NAP;            // nbk * (2 hmax + 1) outer twiddles
    const int grp = tid / G, lane = tid - grp * G;
    const int m = blockIdx.x;
    const int h1c = n1 / 2 + 1;
    const size_t colstride = (size_t)h1c * n0;
    const int pidx = blockIdx.y * ngroups + grp;  // products split over blockIdx.y chunks
    const bool act = pidx < npairs;
    PairDesc pd;
    if (act) pd = pairs[pidx];
    else {
        pd.kind = 0;
        pd.a = pd.b = pd.h0 = pd.row0 = pd.row1 = 0;
    }
    const int h0 = pd.h0;
    const int wrow = 2 * hmax + 1;
    for (int e = tid; e < nbk * wrow; e += nthr) {
        const int lb = e / wrow, rho = e - lb * wrow - hmax;
        sW[e] = conj(tw0[(lb * rho) & (n0 - 1)]);
    }
    // inner twiddles w^(r1 s2), w = exp(2 pi i / NA), for this lane (r1 = lane)
    cpx<T> wi[8];
#pragma unroll
    for (int s2 = 0; s2 < 8; ++s2) wi[s2] = conj(tw0[(lane * s2) * (n0 / NA)]);
    CAcc<T> acc[NS];
    cpx<T> part[NS];
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        acc[o].zero();
        part[o] = mk((T)0, (T)0);
    }
    cpx<T> *tg = sT + (size_t)grp * NAP;
    // NS = 5 (G = 8, lags <= 16): validity and lag of each output slot
    bool o_ok[NS];
    int o_rho[NS];
#pragma unroll
    for (int o = 0; o < NS; ++o) {
        const int s1 = o < 3 ? o : o + 3;
        const int rp = lane + 8 * s1;
        o_ok[o] = rp <= h0 || rp >= NA - h0;
        o_rho[o] = rp <= h0 ? rp : rp - NA;
    }
    constexpr int kPer16 = 16 / (int)sizeof(cpx<T>);
    constexpr int kChunksPerImg = NA / kPer16;
    const int chunks = (nimg + nxp) * kChunksPerImg;
    // 16-byte chunk c of a residue-class tile: its source for class 0 and its
    // place in the tile (the source of class lb is lb * NA elements further)
    auto chunk_src = [&](int c) {
        const int img = c / kChunksPerImg, r = (c - img * kChunksPerImg) * kPer16;
        return (img < nimg) ? U + (size_t)img * colstride + (size_t)m * n0 + r : xhat + (size_t)(img - nimg) * n0 + r;
    };
    auto chunk_dst = [&](int c) {
        const int img = c / kChunksPerImg, r = (c - img * kChunksPerImg) * kPer16;
        return img * NAP + r;
    };
    // this thread's first two chunks, kept (most launches have no others)
    const cpx<T> *src0 = tid < chunks ? chunk_src(tid) : U, *src1 = tid + nthr < chunks ? chunk_src(tid + nthr) : U;
    const int dst0 = tid < chunks ? chunk_dst(tid) : 0, dst1 = tid + nthr < chunks ? chunk_dst(tid + nthr) : 0;
    auto prefetch = [&](int lb, int buf) {
        cpx<T> *dst = sU + (size_t)buf * tile;
        const size_t off = (size_t)lb * NA;
        if (tid < chunks) cp_async16(dst + dst0, src0 + off);
        if (tid + nthr < chunks) cp_async16(dst + dst1, src1 + off);
        for (int c = tid + 2 * nthr; c < chunks; c += nthr) cp_async16(dst + chunk_dst(c), chunk_src(c) + off);
        cp_async_commit();
    };
    prefetch(0, 0);
    for (int lb = 0; lb < nbk; ++lb) {
        if (lb + 1 < nbk) {
            prefetch(lb + 1, (lb + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const cpx<T> *buf = sU + (size_t)(lb & 1) * tile;
        if (act) {
            const cpx<T> *A = buf + (size_t)pd.a * NAP;
            const cpx<T> *B = (pd.kind == PK_LAMBDA) ? buf + (size_t)(nimg + pd.b) * NAP : buf + (size_t)pd.b * NAP;
            cpx<T> v[8];
            if (pd.kind == PK_OMEGA2) {  // |U_a|^2 + i |U_b|^2
#pragma unroll
                for (int r2 = 0; r2 < 8; ++r2) {
                    const int r = lane + G * r2;
                    const cpx<T> ua = A[r], ub = B[r];
                    v[r2] = mk(ua.re * ua.re + ua.im * ua.im, ub.re * ub.re + ub.im * ub.im);
                }
            } else {
#pragma unroll
                for (int r2 = 0; r2 < 8; ++r2) {
                    const int r = lane + G * r2;
                    v[r2] = cmulc(A[r], B[r]);
                }
            }
            if (m == 0 && lb == 0 && lane == 0) v[0] = mk((T)0, (T)0);  // DC bin removed
            dft8(v, 1);
#pragma unroll
            for (int s2 = 1; s2 < 8; ++s2) v[s2] = cmul(v[s2], wi[s2]);
            if (G == 8) {
                // transpose through rows of 9 (8 + 1 pad): constant offsets
                // from one base per lane, no bank conflicts for 64-bit words
#pragma unroll
                for (int s2 = 0; s2 < 8; ++s2) tg[s2 * 9 + lane] = v[s2];
            } else {
#pragma unroll
                for (int s2 = 0; s2 < 8; ++s2) tg[s2 * G + lane] = v[s2];
            }
        }
        __syncwarp();
        if (act && NS == 5) {
            // G = 8: this lane's s2 = lane; outputs s1 in {0, 1, 2, 6, 7} with
            // their lags precomputed (they do not depend on lb)
            const cpx<T> *wrow_lb = sW + (size_t)lb * wrow + hmax;
            cpx<T> u[G];
#pragma unroll
            for (int r1 = 0; r1 < G; ++r1) u[r1] = tg[lane * 9 + r1];
            dftG<T, G>(u, 1);
#pragma unroll
            for (int o = 0; o < NS; ++o)
                if (o_ok[o]) part[o] = cfma(part[o], u[o < 3 ? o : o + 3], wrow_lb[o_rho[o]]);
        } else if (act) {
            const cpx<T> *wrow_lb = sW + (size_t)lb * wrow + hmax;
            // lane handles s2 = lane + G*c for c < 8/G; G-point DFT over r1
#pragma unroll
            for (int c = 0; c < 8 / G; ++c) {
                const int s2 = lane + G * c;
                cpx<T> u[G];
#pragma unroll
                for (int r1 = 0; r1 < G; ++r1) u[r1] = (G == 8) ? tg[s2 * 9 + r1] : tg[s2 * G + r1];
                dftG<T, G>(u, 1);
#pragma unroll
                for (int s1 = 0; s1 < G; ++s1) {
                    const int rp = s2 + 8 * s1;  // rho mod NA
                    int rho;
                    if (rp <= h0) rho = rp;
                    else if (rp >= NA - h0) rho = rp - NA;
                    else continue;
                    const int o = out_slot<G, NS>(c, s1);
                    if (o >= 0) part[o] = cfma(part[o], u[s1], wrow_lb[rho]);
                }
            }
        }
        if (act && ((lb & (kFold - 1)) == kFold - 1 || lb == nbk - 1)) {
#pragma unroll
            for (int o = 0; o < NS; ++o) {
                acc[o].add(part[o]);
                part[o] = mk((T)0, (T)0);
            }
        }
        __syncthreads();  // the buffer of this step is refilled two steps later
    }
    cpx<T> z[NS];
#pragma unroll
    for (int o = 0; o < NS; ++o) z[o] = mk((T)acc[o].re.value(), (T)acc[o].im.value());
    // A packed pair holds Z = Q_a + i Q_b with Q_a, Q_b the lag sums of two
    // real sequences, so Q_a(rho) = (Z(rho) + conj Z(-rho)) / 2 and
    // Q_b(rho) = (Z(rho) - conj Z(-rho)) / 2i.  Z(-rho) of this lane's slot o
    // sits in lane (8 - lane) mod 8 of the group, slot map0[o] (lane 0) or
    // map1[o] (others); every lane takes part in the shuffles.
    cpx<T> zn[NS];
    if constexpr (NS == 5) {
        const int wl = threadIdx.x & 31;
        const int src = (wl & ~7) | ((8 - lane) & 7);
        cpx<T> zs[NS];
#pragma unroll
        for (int o = 0; o < NS; ++o) {
            zs[o].re = __shfl_sync(0xffffffffu, z[o].re, src);
            zs[o].im = __shfl_sync(0xffffffffu, z[o].im, src);
        }
        constexpr int map0[5] = {0, 4, 3, 2, 1}, map1[5] = {4, 3, 2, 1, 0};
#pragma unroll
        for (int o = 0; o < NS; ++o) zn[o] = lane == 0 ? zs[map0[o]] : zs[map1[o]];
    }
    if (!act) return;
#pragma unroll
    for (int c = 0; c < 8 / G; ++c) {
        const int s2 = lane + G * c;
#pragma unroll
        for (int s1 = 0; s1 < G; ++s1) {
            const int rp = s2 + 8 * s1;
            int rho;
            if (rp <= h0) rho = rp;
            else if (rp >= NA - h0) rho = rp - NA;
            else continue;
            const int o = out_slot<G, NS>(c, s1);
            if (o < 0) continue;
            if (NS == 5 && pd.kind == PK_OMEGA2) {
                const cpx<T> a = z[o], b = zn[o];
                Q[(size_t)(pd.row0 + rho + h0) * h1c + m] = mk((a.re + b.re) * (T)0.5, (a.im - b.im) * (T)0.5);
                Q[(size_t)(pd.row1 + rho + h0) * h1c + m] = mk((a.im + b.im) * (T)0.5, (b.re - a.re) * (T)0.5);
            } else {
                Q[(size_t)(pd.row0 + rho + h0) * h1c + m] = z[o];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Gather for a column count n0 that is not a power of two: no column FFT; the
// lag sums along x are evaluated directly as circular cross-correlations in
// the (x, frequency-y) domain, only at the needed lags |rho| <= h0:
//     Q(rho, m) = n0 * sum_x conj(Ga(x, m)) Gb(x + rho mod n0, m),
// which equals the frequency-domain sum of k_gather (correlation theorem).
// Ga, Gb are xt^i F_j (image (i, j)), S, or xt^p for Lambda.  The DC bin of
// column m = 0 is removed there by centring both sequences (their means come
// from an FP64 reduction).  Each term is rounded once in FP32; plain FP32
// partials over kXcFold steps are folded into two-sum accumulators.
// Block per column m; per product, Ga and Gb (with a wrapped halo) are staged
// in shared memory; warp w takes kXcLags lags, each lane 4 consecutive x per
// step, so that one step is 4 + 4 + kXcLags - 1 loads for 4 kXcLags products.
constexpr int kXcLags = 5;
constexpr int kXcFold = 4;
constexpr int kXcThreads = 256;

// Element x of a sequence at column m: idx < 0 is image t = -idx - 1 (t = nk
// is S), idx >= 0 the background x-function idx (xt^idx or its table);
// `centre` subtracts its mean.
template <typename T>
__device__ __forceinline__ cpx<T> xc_seq(int idx, const BasisView &bv, const FTab<T> &ft, int m, bool centre, int x,
                                         int h1c, int n0, const cpx<T> *__restrict__ F, const T *xt,
                                         const double *mu_re, const double *mu_im, const double *mu_p) {
    if (idx >= 0) {
        const T w = ft.bx ? ft.bx[(size_t)idx * n0 + x] : ipow(xt[x], idx);
        const T v = w - (centre ? (T)mu_p[idx] : (T)0);
        return mk(v, (T)0);
    }
    const int t = -idx - 1;
    int i = 0, j = bv.nfy;
    if (t < bv.nk) {
        i = bv.ti(t);
        j = bv.tj(t);
    }
    const T wx = (ft.fx && t < bv.nk) ? ft.fx[(size_t)i * n0 + x] : ipow(xt[x], i);
    const cpx<T> v = scale(F[((size_t)j * h1c + m) * n0 + x], wx);
    return centre ? v - mk((T)mu_re[t], (T)mu_im[t]) : v;
}

template <typename T>
__global__ void __launch_bounds__(kXcThreads) k_xcorr(int n0, int n1, BasisView bv, FTab<T> ft, int npairs, int hmax,
                                                      const PairDesc *__restrict__ pairs,
                                                      const cpx<T> *__restrict__ F, cpx<T> *__restrict__ Q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int hB = hmax + 8;                                     // halo of B on each side
    cpx<T> *A = reinterpret_cast<cpx<T> *>(smem_raw);            // n0 + 8
    cpx<T> *B = A + n0 + 8;                                      // n0 + 2 hB + 8
    T *xt = reinterpret_cast<T *>(B + n0 + 2 * hB + 8);          // n0
    __shared__ double mu_re[kMaxKTerms + 1], mu_im[kMaxKTerms + 1], mu_p[kMaxFun];
    __shared__ double red[kXcThreads / 32][2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = blockIdx.x, h1c = n1 / 2 + 1;
    const int nk = bv.nk;
    for (int x = tid; x < n0; x += kXcThreads) xt[x] = coord<T>(x, n0);
    __syncthreads();
    if (m == 0) {
        // means of every sequence at m = 0 (the DC bin is removed there)
        for (int q = 0; q < nk + 1 + bv.nbx; ++q) {
            const int idx = q <= nk ? -q - 1 : q - nk - 1;
            double sr = 0.0, si = 0.0;
            for (int x = tid; x < n0; x += kXcThreads) {
                const cpx<T> v = xc_seq<T>(idx, bv, ft, 0, false, x, h1c, n0, F, xt, mu_re, mu_im, mu_p);
                sr += (double)v.re;
                si += (double)v.im;
            }
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0) {
                red[warp][0] = sr;
                red[warp][1] = si;
            }
            __syncthreads();
            if (tid == 0) {
                double a = 0.0, b = 0.0;
                for (int w = 0; w < kXcThreads / 32; ++w) {
                    a += red[w][0];
                    b += red[w][1];
                }
                if (q <= nk) {
                    mu_re[q] = a / n0;
                    mu_im[q] = b / n0;
                } else {
                    mu_p[q - nk - 1] = a / n0;
                }
            }
            __syncthreads();
        }
    }
    for (int pi = 0; pi < npairs; ++pi) {
        const PairDesc pd = pairs[pi];
        const int h0 = pd.h0;
        const int ia = -pd.a - 1;
        const int ib = pd.kind == PK_LAMBDA ? pd.b : -pd.b - 1;  // Theta: b = nk (S)
        for (int x = tid; x < n0 + 8; x += kXcThreads)
            A[x] = x < n0 ? conj(xc_seq<T>(ia, bv, ft, m, m == 0, x, h1c, n0, F, xt, mu_re, mu_im, mu_p))
                          : mk((T)0, (T)0);
        for (int e = tid; e < n0 + 2 * hB + 8; e += kXcThreads) {
            int x = (e - hB) % n0;
            if (x < 0) x += n0;
            B[e] = xc_seq<T>(ib, bv, ft, m, m == 0, x, h1c, n0, F, xt, mu_re, mu_im, mu_p);
        }
        __syncthreads();
        const int nlag = 2 * h0 + 1;
        for (int c0 = warp * kXcLags; c0 < nlag; c0 += (kXcThreads / 32) * kXcLags) {
            CAcc<T> acc[kXcLags];
            cpx<T> part[kXcLags];
#pragma unroll
            for (int k = 0; k < kXcLags; ++k) {
                acc[k].zero();
                part[k] = mk((T)0, (T)0);
            }
            int step = 0;
            for (int x0 = 4 * lane; x0 < n0; x0 += 128) {
                cpx<T> a[4], bw[4 + kXcLags - 1];
#pragma unroll
                for (int q = 0; q < 4; ++q) a[q] = A[x0 + q];
                const int base = x0 - h0 + c0 + hB;  // B index of x0 + rho_0
#pragma unroll
                for (int e = 0; e < 4 + kXcLags - 1; ++e) bw[e] = B[base + e];
#pragma unroll
                for (int k = 0; k < kXcLags; ++k)
#pragma unroll
                    for (int q = 0; q < 4; ++q) part[k] = cfma(part[k], a[q], bw[q + k]);
                if (++step == kXcFold) {
#pragma unroll
                    for (int k = 0; k < kXcLags; ++k) {
                        acc[k].add(part[k]);
                        part[k] = mk((T)0, (T)0);
                    }
                    step = 0;
                }
            }
#pragma unroll
            for (int k = 0; k < kXcLags; ++k) {
                acc[k].add(part[k]);
                for (int o = 16; o > 0; o >>= 1) {
                    shfl_add(acc[k].re, o);
                    shfl_add(acc[k].im, o);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < kXcLags; ++k)
                    if (c0 + k < nlag)
                        Q[(size_t)(pd.row0 + c0 + k) * h1c + m] =
                            mk((T)((double)n0 * acc[k].re.wide()), (T)((double)n0 * acc[k].im.wide()));
            }
        }
        __syncthreads();  // A and B are refilled for the next product
    }
}

// ---------------------------------------------------------------------------
// Stage 2: sum over m.  One block per stage-1 row.
constexpr int kS2Out = 8;  // lag outputs per warp task in k_stage2
constexpr int kS2Fold = 8;  // frequencies per plain partial sum in k_stage2

template <typename T>
__global__ void k_stage2(int n0, int n1, int w0, int w1, BasisView bv, int npairs,
                         const PairDesc *__restrict__ pairs, const cpx<T> *__restrict__ Q,
                         const cpx<T> *__restrict__ yhat, const cpx<T> *__restrict__ tw1,
                         double *__restrict__ lag, int off_om, int off_la, int off_th) {
    const int row = blockIdx.x;
    // find the pair of this row
    int pi = 0;
    for (int k = 0; k < npairs; ++k)
        if (row >= pairs[k].row0 && row < pairs[k].row0 + 2 * pairs[k].h0 + 1) pi = k;
    const PairDesc pd = pairs[pi];
    const int rho0 = row - pd.row0 - pd.h0;
    const int h1c = n1 / 2 + 1;
    const int nk = bv.nk;
    const int nbt = bv.nb;
    const int h1 = (pd.kind == PK_OMEGA) ? 2 * w1 : w1;
    int nq = 1;
    if (pd.kind == PK_LAMBDA) nq = bv.lamn(pd.b);  // background terms whose x-function is p = b
    const cpx<T> *q = Q + (size_t)row * h1c;
    const double invP = 1.0 / ((double)n0 * (double)n1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // outputs in chunks of up to kS2Out lags rho1 >= 0 of one q index, each
    // with its mirror -rho1 (cpq chunks per q): both come from one twiddle,
    // Re(v e) and Re(v conj e).  Warp w takes chunk w % nchr of the round and
    // every nsp-th slice of the frequencies, nsp = nw / nchr
    __shared__ Acc<T> part[8][2 * kS2Out];
    const int cpq = (h1 + 1 + kS2Out - 1) / kS2Out;
    const int nch = nq * cpq;
    for (int c0 = 0; c0 < nch; c0 += nw) {
        const int nchr = min(nw, nch - c0);  // chunks in this round
        const int nsp = nw / nchr;
        const int ch = c0 + warp % nchr, sp = warp / nchr;
        const bool act = sp < nsp;
        // each lane: plain partial sums over kS2Fold of its frequencies, folded
        // into two-sum accumulators (one rounding per term, compensated sums);
        // [k] lag r0 + k, [kS2Out + k] lag -(r0 + k)
        Acc<T> a[2 * kS2Out];
        T pl[2 * kS2Out];
#pragma unroll
        for (int k = 0; k < 2 * kS2Out; ++k) {
            a[k].zero();
            pl[k] = (T)0;
        }
        const int qi = ch / cpq, r0 = (ch - qi * cpq) * kS2Out;  // first rho1 >= 0 of the chunk
        if (act) {
            int cnt = 0;
            const int mstep = nsp * 32;
            const int dstep = imod(mstep * r0, n1);  // change of (mm r0) mod n1 per step of mm
            int idx0 = imod((sp * 32 + lane) * r0, n1);
            for (int mm = sp * 32 + lane; mm < h1c; mm += mstep) {
                cpx<T> v = q[mm];
                if (pd.kind == PK_LAMBDA) v = cmul(v, yhat[(size_t)bv.lamq(pd.b, qi) * h1c + mm]);
                const T wm = (mm == 0 || (2 * mm == n1)) ? (T)1 : (T)2;
                v = scale(v, wm);
                int idx = idx0;  // (mm rho1) mod n1, stepped by mm over the chunk's lags
                idx0 += dstep;
                if (idx0 >= n1) idx0 -= n1;
#pragma unroll
                for (int k = 0; k < kS2Out; ++k) {
                    if (r0 + k <= h1) {
                        const cpx<T> e = conj(tw1[idx]);
                        pl[k] += v.re * e.re - v.im * e.im;
                        pl[kS2Out + k] += v.re * e.re + v.im * e.im;
                    }
                    idx += mm;
                    if (idx >= n1) idx -= n1;
                }
                if (++cnt == kS2Fold) {
#pragma unroll
                    for (int k = 0; k < 2 * kS2Out; ++k) {
                        a[k].add(pl[k]);
                        pl[k] = (T)0;
                    }
                    cnt = 0;
                }
            }
#pragma unroll
            for (int k = 0; k < 2 * kS2Out; ++k) a[k].add(pl[k]);
        }
#pragma unroll
        for (int k = 0; k < 2 * kS2Out; ++k)
            for (int s = 16; s > 0; s >>= 1) shfl_add(a[k], s);
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 2 * kS2Out; ++k) part[warp][k] = a[k];
        }
        __syncthreads();
        // warps of the same chunk combine their slices in a fixed order
        if (threadIdx.x < nchr * 2 * kS2Out) {
            const int cc = threadIdx.x / (2 * kS2Out), k = threadIdx.x % (2 * kS2Out);
            const int chw = c0 + cc;
            const int qo = chw / cpq, rr = (chw - qo * cpq) * kS2Out + (k % kS2Out);
            Acc<T> t = part[cc][k];
            for (int sp2 = 1; sp2 < nsp; ++sp2) t.add(part[cc + sp2 * nchr][k]);
            if (rr <= h1 && !(k >= kS2Out && rr == 0)) {
                const int rho1 = k < kS2Out ? rr : -rr;
                const double val = t.wide() * invP;
                size_t idx;
                if (pd.kind == PK_OMEGA) {
                    const int ia = pd.a, ib = pd.b;
                    const int pidx = ia * nk - ia * (ia - 1) / 2 + (ib - ia);
                    idx = off_om + ((size_t)pidx * (4 * w0 + 1) + (rho0 + 2 * w0)) * (4 * w1 + 1) + (rho1 + 2 * w1);
                } else if (pd.kind == PK_LAMBDA) {
                    const int s2 = bv.lams(pd.b, qo);  // background term (p, q)
                    idx = off_la + (((size_t)pd.a * nbt + s2) * (2 * w0 + 1) + (rho0 + w0)) * (2 * w1 + 1) + (rho1 + w1);
                } else {
                    idx = off_th + ((size_t)pd.a * (2 * w0 + 1) + (rho0 + w0)) * (2 * w1 + 1) + (rho1 + w1);
                }
                lag[idx] = val;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Assembly of M and rhs (Eq. B5, B7, B9, B11, B13, B15).
struct LagView {
    const double *lag;
    int off_om, off_la, off_th;
    int w0, w1, nk, nbt;
    // FFT-derived Omega_{t u}(rho) (DC removed) for any ordered pair
    __device__ double om(int t, int u, int r0, int r1) const {
        if (t > u) {
            int z = t;
            t = u;
            u = z;
            r0 = -r0;
            r1 = -r1;
        }
        const int pidx = t * nk - t * (t - 1) / 2 + (u - t);
        return lag[off_om + ((size_t)pidx * (4 * w0 + 1) + (r0 + 2 * w0)) * (4 * w1 + 1) + (r1 + 2 * w1)];
    }
    __device__ double la(int t, int s, int r0, int r1) const {
        return lag[off_la + (((size_t)t * nbt + s) * (2 * w0 + 1) + (r0 + w0)) * (2 * w1 + 1) + (r1 + w1)];
    }
    __device__ double th(int t, int r0, int r1) const {
        return lag[off_th + ((size_t)t * (2 * w0 + 1) + (r0 + w0)) * (2 * w1 + 1) + (r1 + w1)];
    }
};

// Zero-lag values z0: Omega_tu(0,0) by pair index (t <= u), then
// Lambda_ts(0,0) [t][s], Theta_t(0,0), E_s; C (Eq. B11) in cmat[s][s'].
// unk[u] = (kernel term?, term, alpha, beta).
__global__ void k_assemble(int n, const int4 *__restrict__ unk, LagView lv, const double *__restrict__ z0,
                           const double *__restrict__ cmat, double *__restrict__ M, double *__restrict__ rhs) {
    const int nk = lv.nk, nb = lv.nbt;
    const int z_la = nk * (nk + 1) / 2, z_th = z_la + nk * nb, z_e = z_th + nk;
    // rows blockIdx.y + k gridDim.y of M (row n: rhs), threads along the columns
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= n) return;
    for (int row = blockIdx.y; row <= n; row += gridDim.y) {
        if (row == n) {  // rhs
            const int4 ur = unk[col];
            double v;
            if (ur.x) {
                if (ur.z == 0 && ur.w == 0) v = z0[z_th + ur.y];  // Theta(0,0)
                else v = lv.th(ur.y, ur.z, ur.w) - lv.th(ur.y, 0, 0);
            } else {
                v = z0[z_e + ur.y];  // E (Eq. B15)
            }
            rhs[col] = v;
            continue;
        }
        const int4 ur = unk[row], uc = unk[col];
        double v;
        if (ur.x && uc.x) {
            const bool rz = (ur.z == 0 && ur.w == 0), cz = (uc.z == 0 && uc.w == 0);
            if (rz && cz) {
                const int t = min(ur.y, uc.y), u = max(ur.y, uc.y);
                v = z0[t * nk - t * (t - 1) / 2 + (u - t)];  // Omega(0,0)
            } else if (rz) {
                v = lv.om(ur.y, uc.y, -uc.z, -uc.w) - lv.om(ur.y, uc.y, 0, 0);
            } else if (cz) {
                v = lv.om(ur.y, uc.y, ur.z, ur.w) - lv.om(ur.y, uc.y, 0, 0);
            } else {
                v = lv.om(ur.y, uc.y, ur.z - uc.z, ur.w - uc.w) - lv.om(ur.y, uc.y, ur.z, ur.w) -
                    lv.om(ur.y, uc.y, -uc.z, -uc.w) + lv.om(ur.y, uc.y, 0, 0);
            }
        } else if (ur.x) {  // B (Eq. B7)
            if (ur.z == 0 && ur.w == 0) v = z0[z_la + ur.y * nb + uc.y];
            else v = lv.la(ur.y, uc.y, ur.z, ur.w) - lv.la(ur.y, uc.y, 0, 0);
        } else if (uc.x) {  // B~ (Eq. B9)
            if (uc.z == 0 && uc.w == 0) v = z0[z_la + uc.y * nb + ur.y];
            else v = lv.la(uc.y, ur.y, uc.z, uc.w) - lv.la(uc.y, ur.y, 0, 0);
        } else {  // C (Eq. B11)
            v = cmat[(size_t)ur.y * nb + uc.y];
        }
        M[(size_t)row * n + col] = v;
    }
}

// ---------------------------------------------------------------------------
// k_rows prefetches into L2 the rows of the block this many waves of one
// block per multiprocessor later
constexpr int kRowsPrefetch = 1;

template <typename T, typename I>
static cudaError_t launch_rows(Plan *p, const void *ref, const void *sci, const uint8_t *mask,
                               bool moments, cudaStream_t s) {
    const int nfft = (p->nfy + 2) / 2;
    const FTab<T> ft = ftab_of<T>(p);
    if (p->gen1) {
        const int G = p->m1 / 16;
        int TR = (sizeof(T) == 4 ? 1024 : 512) / G;
        if (TR < 1) TR = 1;
        if (TR > 16) TR = 16;
        auto smem_of = [&](int tr) { return (size_t)tr * (padded_len(p->m1) + 4) * sizeof(cpx<T>); };
        while (TR > 1 && smem_of(TR) > 200 * 1024) TR /= 2;
        if (p->tune_tr > 0 && p->tune_tr < TR) TR = p->tune_tr;
        const size_t smem = smem_of(TR);
        auto kern = k_rows_blu<T, I>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<((p->n0 + TR - 1) / TR) * nfft, TR * G, smem, s>>>(
            p->n0, p->n1, p->m1, p->nfy, TR, (const I *)ref, (const I *)sci, mask, (cpx<T> *)p->F,
            (const cpx<T> *)p->chirp1, (const cpx<T> *)p->bfilt1, (const cpx<T> *)p->twpm1, ft.fy);
    } else {
    const int G = p->n1 / 16;
    int TR = (sizeof(T) == 4 ? 1024 : 512) / G;
    if (TR > 16) TR = 16;
    if (TR > p->n0) TR = p->n0;
    auto smem_of = [&](int tr) { return (size_t)tr * (padded_len(p->n1) + 4) * sizeof(cpx<T>); };
    while (TR > 1 && smem_of(TR) > 200 * 1024) TR /= 2;
    if (p->tune_tr > 0 && p->tune_tr < TR) TR = p->tune_tr;
    const size_t smem = smem_of(TR);
    auto kern = k_rows<T, I>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // polynomial weights yt^j are computed in the kernel (a multiply per
    // power), cheaper than the table's per-thread strided reads
    kern<<<((p->n0 + TR - 1) / TR) * nfft, TR * G, smem, s>>>(p->n0, p->n1, p->nfy, TR, (const I *)ref,
                                                              (const I *)sci, mask, (cpx<T> *)p->F,
                                                              (const cpx<T> *)p->twp1, p->bspline ? ft.fy : nullptr,
                                                              kRowsPrefetch * p->sms);
    }
    p->launches++;
    if (moments && !p->bspline) {
        auto km = (p->cfg.dk == 2 && p->cfg.db == 2) ? k_row_moments<T, I, 5, 5, 3, 3> : k_row_moments<T, I>;
        km<<<p->n0, 256, 0, s>>>(p->n1, p->cfg.dk, p->cfg.db, (const I *)ref, (const I *)sci, mask, p->rowmom);
        p->launches++;
        if (p->lam_closed) {
            k_boundary<I><<<dim3(2 * p->cfg.w1 + 1, kBndChunks), 256, 0, s>>>(p->n0, p->n1, p->cfg.w0, p->cfg.w1,
                                                            p->cfg.dk + p->cfg.db, (const I *)ref, mask, p->bnd);
            p->launches++;
        }
    } else if (moments) {  // ytab = fy | by
        dim3 grid(p->n0, (p->nmom + kMomChunk - 1) / kMomChunk);
        k_row_moments_tab<T, I><<<grid, 256, 0, s>>>(p->n1, p->nmom, p->d_rdesc, ft.fy, (const I *)ref,
                                                     (const I *)sci, mask, p->rowmom);
        p->launches++;
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_cols(Plan *p, cudaStream_t s) {
    k_zero_lag<<<p->nzm, 256, 0, s>>>(p->n0, p->nmom, p->d_zdesc, p->ftab64, p->rowmom, p->z0);
    p->launches++;
    if (p->gen0) return cudaGetLastError();  // the lag sums along x need no column spectra
    const int G = p->n0 / 16;
    // about 256 threads per block (one 4096-point transform; the twiddles
    // come through L1, so small blocks cost no table copies), at most 4 images
    int GI = 256 / G;
    if (GI < 1) GI = 1;
    if (GI > 4) GI = 4;
    const int nimg = p->nk + 1;
    if (GI > nimg) GI = nimg;
    size_t smem = (size_t)GI * padded_len(p->n0) * sizeof(cpx<T>);
    while (GI > 1 && smem > 110 * 1024) {
        --GI;
        smem = (size_t)GI * padded_len(p->n0) * sizeof(cpx<T>);
    }
    if (p->tune_gi > 0 && p->tune_gi < GI) {
        GI = p->tune_gi;
        smem = (size_t)GI * padded_len(p->n0) * sizeof(cpx<T>);
    }
    auto kern = k_cols<T>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((nimg + GI - 1) / GI, p->h1c);
    kern<<<grid, GI * G, smem, s>>>(p->n0, p->n1, p->bv, p->na, p->nbk, GI, (const cpx<T> *)p->F,
                                    (cpx<T> *)p->U, (const cpx<T> *)p->twp0, ftab_of<T>(p).fx);
    p->launches++;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_gather(Plan *p, cudaStream_t s) {
    if (p->gen0) {
        const int hmax = 2 * p->cfg.w0;
        const size_t smem = (size_t)(2 * p->n0 + 2 * (hmax + 8) + 16) * sizeof(cpx<T>) + (size_t)p->n0 * sizeof(T);
        cudaFuncSetAttribute(k_xcorr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_xcorr<T><<<p->h1c, kXcThreads, smem, s>>>(p->n0, p->n1, p->bv, ftab_of<T>(p), p->npairs, hmax, p->pairs,
                                                    (const cpx<T> *)p->F, (cpx<T> *)p->Q);
        p->launches++;
        return cudaGetLastError();
    }
    const int G = p->na / 8;
    const int nimg = p->nimg, nxp = p->lam_closed ? 0 : p->nbx;
    const int hmax = 2 * p->cfg.w0;
    const bool ns5 = G == 8 && hmax <= 16;
    // one group of G lanes per product, whole warps, at most kGatherThreads
    // threads per block; more products go to further blocks along y
    const int max_groups = (ns5 ? kGatherThreads<T, 5>() : kGatherThreads<T, 8>()) / G;
    const int nchunks = (p->ngpairs + max_groups - 1) / max_groups;
    const int per_chunk = (p->ngpairs + nchunks - 1) / nchunks;
    int nthr = per_chunk * G;
    nthr = ((nthr + 31) / 32) * 32;
    const int ngroups = nthr / G;
    const int nap = p->na + kPad;
    size_t smem = (2 * (size_t)(nimg + nxp) * nap + (size_t)ngroups * nap + (size_t)p->nbk * (2 * hmax + 1)) *
                  sizeof(cpx<T>);
    void (*kern)(int, int, int, int, int, int, int, const PairDesc *, const cpx<T> *, const cpx<T> *,
                 const cpx<T> *, cpx<T> *) = nullptr;
    if (G == 8) kern = ns5 ? k_gather<T, 8, 5> : k_gather<T, 8, 8>;
    if (G == 4) kern = k_gather<T, 4, 8>;
    if (G == 2) kern = k_gather<T, 2, 8>;
    if (!kern) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    dim3 grid(p->h1c, nchunks);
    kern<<<grid, nthr, smem, s>>>(p->n0, p->n1, p->nk, nxp, p->nbk, p->ngpairs, hmax, p->gpairs,
                                  (const cpx<T> *)p->U, (const cpx<T> *)p->xhat, (const cpx<T> *)p->tw0,
                                  (cpx<T> *)p->Q);
    p->launches++;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_lags(Plan *p, double *M, double *rhs, cudaStream_t s) {
    cudaError_t err;
    k_stage2<T><<<p->nrows, 256, 0, s>>>(p->n0, p->n1, p->cfg.w0, p->cfg.w1, p->bv, p->npairs,
                                         p->pairs, (const cpx<T> *)p->Q, (const cpx<T> *)p->yhat,
                                         (const cpx<T> *)p->tw1, p->lag, p->lag_om, p->lag_la, p->lag_th);
    p->launches++;
    if ((err = cudaGetLastError())) return err;
    LagView lv;
    lv.lag = p->lag;
    lv.off_om = p->lag_om;
    lv.off_la = p->lag_la;
    lv.off_th = p->lag_th;
    lv.w0 = p->cfg.w0;
    lv.w1 = p->cfg.w1;
    lv.nk = p->nk;
    lv.nbt = p->nb;
    if (p->lam_closed) {
        const int fR = 2 * p->cfg.dk + 1;  // row moments sum_y Rm yt^v (k_row_moments layout)
        k_lambda_closed<<<p->nk * p->nb, 256, 0, s>>>(p->n0, p->n1, p->cfg.w0, p->cfg.w1, p->cfg.dk + p->cfg.db,
                                                          p->bv, p->rowmom, p->nmom, fR, p->z0 + p->z_mu, p->bnd,
                                                          p->lag + p->lag_la);
        p->launches++;
        if ((err = cudaGetLastError())) return err;
    }
    const dim3 grid((p->n + 255) / 256, p->n + 1 < 65535 ? p->n + 1 : 65535);
    k_assemble<<<grid, 256, 0, s>>>(p->n, p->unk, lv, p->z0, p->cmat, M, rhs);
    p->launches++;
    return cudaGetLastError();
}

cudaError_t build_stage(Plan *p, int stage, double *M, double *rhs, cudaStream_t s) {
    switch (stage) {
        case 1: return p->fp64 ? launch_cols<double>(p, s) : launch_cols<float>(p, s);
        case 2: return p->fp64 ? launch_gather<double>(p, s) : launch_gather<float>(p, s);
        case 3: return p->fp64 ? launch_lags<double>(p, M, rhs, s) : launch_lags<float>(p, M, rhs, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t row_transform(Plan *p, const void *ref, const void *sci, const uint8_t *mask, bool moments,
                          cudaStream_t s) {
    const bool img64 = p->cfg.dtype == SFFT_F64;
    if (p->fp64) {
        return img64 ? launch_rows<double, double>(p, ref, sci, mask, moments, s)
                     : launch_rows<double, float>(p, ref, sci, mask, moments, s);
    }
    return img64 ? launch_rows<float, double>(p, ref, sci, mask, moments, s)
                 : launch_rows<float, float>(p, ref, sci, mask, moments, s);
}

cudaError_t build_system(Plan *p, const void *ref, const void *sci, const uint8_t *mask, double *M,
                         double *rhs, cudaStream_t s) {
    cudaError_t err = row_transform(p, ref, sci, mask, true, s);
    for (int stage = 1; stage <= 3 && err == cudaSuccess; ++stage) err = build_stage(p, stage, M, rhs, s);
    return err;
}

}  // namespace sfft
