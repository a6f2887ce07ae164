// fft16.cuh -- register-based FFTs in shared memory, radix-16 passes.
//
// A transform of length n = 2^e is done by one group of gsize threads on a
// padded shared buffer: element i lives at i + (i >> 4), which keeps the
// strided accesses of every pass free of bank conflicts.  Stockham
// auto-sort passes: an optional first pass of radix 2, 4 or 8 (so that the
// rest is a whole number of radix-16 passes), then radix-16 passes, each
// thread holding one butterfly's 16 values in registers.  Passes are in
// place: all loads of a pass complete (block barrier) before its stores.
// Twiddles come from a pass-ordered table (pass_table_*): the radix-16 pass
// of stride ns > 1 reads exp(-2 pi i r k / (16 ns)) at (r - 1) * ns + k, so
// the lanes of a warp (consecutive k) read consecutive words; the inverse
// uses conjugates.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace sfft {

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 4); }

template <typename T>
__device__ __forceinline__ cpx<T> tw_get(const cpx<T> *tw, int q, int sgn) {
    const cpx<T> w = tw[q];
    return sgn < 0 ? w : mk(w.re, -w.im);
}

// in-place DFT of 2, 4, 8 or 16 values with sign sgn, natural output order
template <typename T>
__device__ __forceinline__ void dft2(cpx<T> &a, cpx<T> &b) {
    const cpx<T> s = a + b, d = a - b;
    a = s;
    b = d;
}

template <typename T>
__device__ __forceinline__ void dft16(cpx<T> (&v)[16], int sgn) {
    // X[k2 + 4 k1] = sum_r1 W4^(r1 k1) W16^(r1 k2) sum_r2 W4^(r2 k2) v[r1 + 4 r2]
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, c2 = (T)0.70710678118654752440;
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) dft4(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12], sgn);
    // now v[r1 + 4 k2] = Y[r1][k2]; twiddle by W16^(r1 k2)
    const T sg = (T)sgn;
    v[1 + 4 * 1] = cmul(v[5], mk(c1, sg * s1));   // r1=1,k2=1: m=1
    v[1 + 4 * 2] = cmul(v[9], mk(c2, sg * c2));   // m=2
    v[1 + 4 * 3] = cmul(v[13], mk(s1, sg * c1));  // m=3
    v[2 + 4 * 1] = cmul(v[6], mk(c2, sg * c2));   // m=2
    v[2 + 4 * 2] = mul_i(v[10], sgn);             // m=4
    v[2 + 4 * 3] = cmul(v[14], mk(-c2, sg * c2)); // m=6
    v[3 + 4 * 1] = cmul(v[7], mk(s1, sg * c1));   // m=3
    v[3 + 4 * 2] = cmul(v[11], mk(-c2, sg * c2)); // m=6
    v[3 + 4 * 3] = cmul(v[15], mk(-c1, -sg * s1));// m=9
    // DFT4 over r1 for each k2, in place: v[4 k2 + k1] = X[k2 + 4 k1]
    // (transposed slot order; see slot16)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) dft4(v[4 * k2], v[4 * k2 + 1], v[4 * k2 + 2], v[4 * k2 + 3], sgn);
}

// register slot of output X[r] after dft16
__device__ __forceinline__ constexpr int slot16(int r) { return (r & 3) * 4 + (r >> 2); }

// Store position of output l: the padded natural layout, or (perm_lnb >= 0)
// the residue-class layout [l mod nb][l / nb], nb = 2^perm_lnb, with rows of
// perm_na + 1 elements.
__device__ __forceinline__ int out_pos(int l, int perm_lnb, int perm_na) {
    return perm_lnb >= 0 ? (l & ((1 << perm_lnb) - 1)) * (perm_na + 1) + (l >> perm_lnb) : pad16(l);
}

// One Stockham pass of radix R on the padded buffer.  All threads of the
// block call it (block barriers inside); gtid/gsize index the group.
template <typename T, int R>
__device__ __forceinline__ void fft_pass(cpx<T> *buf, int n, int ns, int sgn, const cpx<T> *twp, int gtid,
                                         int gsize, int perm_lnb = -1, int perm_na = 0) {
    const int nb = n / R;  // butterflies
    constexpr int kMaxPer = 16 / R;  // butterflies per thread (gsize = n / 16)
    cpx<T> v[kMaxPer][R];
#pragma unroll
    for (int u = 0; u < kMaxPer; ++u) {
        const int j = gtid + u * gsize;
        if (j < nb) {
            const int k = j & (ns - 1);
#pragma unroll
            for (int r = 0; r < R; ++r) v[u][r] = buf[pad16(j + r * nb)];
            if (ns > 1) {  // only radix-16 passes have ns > 1
#pragma unroll
                for (int r = 1; r < R; ++r) v[u][r] = cmul(v[u][r], tw_get(twp, (r - 1) * ns + k, sgn));
            }
            if constexpr (R == 16) dft16(v[u], sgn);
            else if constexpr (R == 8) dft8(v[u], sgn);
            else if constexpr (R == 4) dft4(v[u][0], v[u][1], v[u][2], v[u][3], sgn);
            else dft2(v[u][0], v[u][1]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kMaxPer; ++u) {
        const int j = gtid + u * gsize;
        if (j < nb) {
            const int k = j & (ns - 1);
            const int o = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[out_pos(o + r * ns, perm_lnb, perm_na)] = v[u][(R == 16) ? slot16(r) : r];
        }
    }
    __syncthreads();
}

// Whole transform of length n (power of two, 16 <= n <= 4096) on the padded
// buffer, with the length known only at run time; see group_fft.
template <typename T>
__device__ void group_fft_rt(cpx<T> *buf, int n, int sgn, const cpx<T> *twp, int gtid, int gsize, int perm_lnb = -1,
                             int perm_na = 0) {
    const int e = 31 - __clz(n);
    int ns = 1;
    const bool only_first = (e >> 2) == 0;  // no radix-16 pass follows
    switch (e & 3) {
        case 1:
            fft_pass<T, 2>(buf, n, ns, sgn, twp, gtid, gsize, only_first ? perm_lnb : -1, perm_na);
            ns = 2;
            break;
        case 2:
            fft_pass<T, 4>(buf, n, ns, sgn, twp, gtid, gsize, only_first ? perm_lnb : -1, perm_na);
            ns = 4;
            break;
        case 3:
            fft_pass<T, 8>(buf, n, ns, sgn, twp, gtid, gsize, only_first ? perm_lnb : -1, perm_na);
            ns = 8;
            break;
        default: break;
    }
    int off = 0;  // this pass's entries in the pass-ordered table
    for (; ns < n; ns *= 16) {
        const bool last = ns * 16 >= n;
        fft_pass<T, 16>(buf, n, ns, sgn, twp + off, gtid, gsize, last ? perm_lnb : -1, perm_na);
        if (ns > 1) off += 15 * ns;
    }
}

// ---- the same transform with the length, the sign and the pass strides known
// at compile time (lengths 256..4096).  The arithmetic and its order are those
// of fft_pass / group_fft_rt; what changes is the addressing: with N/R and
// NS constants, every element a thread loads or stores sits at a constant
// offset from one per-thread base, and the twiddles of a pass at constant
// offsets from base + k, so no index is recomputed per element.
//   load  pad16(j + r NB) = pad16(j) + r (NB + NB/16)          (16 | NB)
//   store pad16(o + r NS) = pad16(o) + r NS + ((r NS) >> 4)    (o = 16 NS q + k, k < NS)
//   residue-class store of the last pass (NA = 64, N = NA NBK, NS = N/16 = 4 NBK):
//         out_pos(k + r NS) = out_pos(k) + 4 r
template <typename T, int N, int R, int NS, int SGN, bool PERM>
__device__ __forceinline__ void fft_pass_ct(cpx<T> *buf, const cpx<T> *twp, int gtid) {
    constexpr int NB = N / R;
    constexpr int G = N / 16;
    constexpr int PER = 16 / R;  // butterflies per thread
    static_assert(NB % 16 == 0, "compile-time passes need 16 | N/R");
    constexpr int LDSTEP = NB + NB / 16;
    cpx<T> v[PER][R];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = gtid + u * G;
        const cpx<T> *src = buf + pad16(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[u][r] = src[r * LDSTEP];
        if constexpr (NS > 1) {
            const int k = j & (NS - 1);
            const cpx<T> *tk = twp + k;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const cpx<T> w = tk[(r - 1) * NS];
                v[u][r] = cmul(v[u][r], SGN < 0 ? w : mk(w.re, -w.im));
            }
        }
        if constexpr (R == 16) dft16(v[u], SGN);
        else if constexpr (R == 8) dft8(v[u], SGN);
        else if constexpr (R == 4) dft4(v[u][0], v[u][1], v[u][2], v[u][3], SGN);
        else dft2(v[u][0], v[u][1]);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = gtid + u * G;
        const int k = j & (NS - 1);
        const int o = (j - k) * R + k;
        if constexpr (PERM) {
            // last pass (NS * 16 == N): o = k; bin l = k + r NS goes to
            // (l mod NBK) * (NA + 1) + l / NBK with NBK = N / 64
            static_assert(R == 16 && NS * 16 == N && N >= 64, "residue-class store on the last radix-16 pass");
            constexpr int NBK = N / 64;
            cpx<T> *dst = buf + (k & (NBK - 1)) * 65 + k / NBK;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[4 * r] = v[u][(R == 16) ? slot16(r) : r];
        } else {
            cpx<T> *dst = buf + pad16(o);
#pragma unroll
            for (int r = 0; r < R; ++r) dst[r * NS + ((r * NS) >> 4)] = v[u][(R == 16) ? slot16(r) : r];
        }
    }
    __syncthreads();
}

// Radix-16 passes from stride NS on (twiddle table offset OFF), the last one
// with the residue-class store if PERM.
template <typename T, int N, int NS, int OFF, int SGN, bool PERM>
__device__ __forceinline__ void fft_passes16_ct(cpx<T> *buf, const cpx<T> *twp, int gtid) {
    if constexpr (NS < N) {
        constexpr bool last = NS * 16 >= N;
        fft_pass_ct<T, N, 16, NS, SGN, PERM && last>(buf, twp + OFF, gtid);
        fft_passes16_ct<T, N, NS * 16, (NS > 1 ? OFF + 15 * NS : OFF), SGN, PERM>(buf, twp, gtid);
    }
}

template <typename T, int LOGN, int SGN, bool PERM>
__device__ __forceinline__ void group_fft_ct(cpx<T> *buf, const cpx<T> *twp, int gtid) {
    constexpr int N = 1 << LOGN;
    constexpr int E = LOGN & 3;
    static_assert(LOGN >= 8 && LOGN <= 12, "compile-time lengths 256..4096");
    if constexpr (E == 1) fft_pass_ct<T, N, 2, 1, SGN, false>(buf, twp, gtid);
    if constexpr (E == 2) fft_pass_ct<T, N, 4, 1, SGN, false>(buf, twp, gtid);
    if constexpr (E == 3) fft_pass_ct<T, N, 8, 1, SGN, false>(buf, twp, gtid);
    fft_passes16_ct<T, N, (1 << E), 0, SGN, PERM>(buf, twp, gtid);
}

template <typename T, int SGN>
__device__ __forceinline__ bool group_fft_ct_dispatch(cpx<T> *buf, int n, const cpx<T> *twp, int gtid, bool perm) {
    switch (n) {
        case 4096:
            if (perm) group_fft_ct<T, 12, SGN, true>(buf, twp, gtid);
            else group_fft_ct<T, 12, SGN, false>(buf, twp, gtid);
            return true;
        case 2048:
            if (perm) group_fft_ct<T, 11, SGN, true>(buf, twp, gtid);
            else group_fft_ct<T, 11, SGN, false>(buf, twp, gtid);
            return true;
        case 1024:
            if (perm) group_fft_ct<T, 10, SGN, true>(buf, twp, gtid);
            else group_fft_ct<T, 10, SGN, false>(buf, twp, gtid);
            return true;
        default: return false;
    }
}

// Whole transform of length n (power of two, 16 <= n <= 4096) on the padded
// buffer; the block must call it with the same n in every group, and gsize
// must be n / 16.  With perm_lnb >= 0 the last pass stores in the
// residue-class layout (out_pos).  Lengths 1024, 2048 and 4096 (and the
// residue-class store with NA = 64) take the compile-time passes; the others
// the run-time ones.  Both give the same results.
template <typename T>
__device__ __forceinline__ void group_fft(cpx<T> *buf, int n, int sgn, const cpx<T> *twp, int gtid, int gsize,
                                          int perm_lnb = -1, int perm_na = 0) {
    const bool perm = perm_lnb >= 0;
    if (!perm || perm_na == 64) {
        if (sgn < 0 ? group_fft_ct_dispatch<T, -1>(buf, n, twp, gtid, perm)
                    : group_fft_ct_dispatch<T, 1>(buf, n, twp, gtid, perm))
            return;
    }
    group_fft_rt(buf, n, sgn, twp, gtid, gsize, perm_lnb, perm_na);
}

// Strides ns of the radix-16 passes with twiddles, in execution order, for a
// transform of length n (power of two): ns = 2^(e mod 4) * 16^m, ns > 1.
// The pass-ordered table holds 15 ns entries per pass, fewer than n in all.
__host__ __device__ inline int pass_table_len(int n) {
    int e = 0;
    while ((1 << e) < n) ++e;
    int len = 0;
    for (int ns = 1 << (e & 3); ns < n; ns *= 16)
        if (ns > 1) len += 15 * ns;
    return len;
}

// Bluestein (chirp-z) DFT of any length n through power-of-two FFTs of
// length m >= 2n - 1 (L. Bluestein, 1970): with c_t = exp(-i pi t^2 / n),
// jk = (j^2 + k^2 - (k - j)^2) / 2 gives
//     X_k = sum_j x_j exp(-2 pi i jk / n) = c_k sum_j (x_j c_j) conj(c_(k-j)),
// a convolution of a_j = x_j c_j with b_t = conj(c_t), |t| < n, evaluated by
// FFTs of length m.  The inverse direction (sgn > 0) conjugates the chirps.
//   buf   : padded buffer of m entries; x_j at pad16(j) for j < n on entry,
//           X_k at pad16(k) for k < n on exit (unnormalised);
//   chirp : c_t, t < n;  bfilt : FFT_m of b (forward chirps);
//   twpm  : the pass-ordered twiddles of length m.
// All threads of the block call it (block barriers); gtid/gsize index the
// group of m/16 threads that owns buf.
template <typename T>
__device__ void bluestein(cpx<T> *buf, int n, int m, int sgn, const cpx<T> *__restrict__ chirp,
                          const cpx<T> *__restrict__ bfilt, const cpx<T> *__restrict__ twpm, int gtid, int gsize) {
    for (int j = gtid; j < m; j += gsize) {
        cpx<T> v = mk((T)0, (T)0);
        if (j < n) {
            const cpx<T> c = chirp[j];
            v = cmul(buf[pad16(j)], sgn < 0 ? c : conj(c));
        }
        buf[pad16(j)] = v;
    }
    __syncthreads();
    group_fft(buf, m, -1, twpm, gtid, gsize);
    // the filter of the conjugated chirps is conj(B(-k))
    for (int k = gtid; k < m; k += gsize) {
        const cpx<T> b = sgn < 0 ? bfilt[k] : conj(bfilt[(m - k) & (m - 1)]);
        buf[pad16(k)] = cmul(buf[pad16(k)], b);
    }
    __syncthreads();
    group_fft(buf, m, 1, twpm, gtid, gsize);
    const T inv = (T)1 / (T)m;
    for (int k = gtid; k < n; k += gsize) {
        const cpx<T> c = chirp[k];
        buf[pad16(k)] = scale(cmul(buf[pad16(k)], sgn < 0 ? c : conj(c)), inv);
    }
    __syncthreads();
}

// Bluestein transform length for n: the least power of two >= 2n - 1.
__host__ __device__ inline int bluestein_len(int n) {
    int m = 1;
    while (m < 2 * n - 1) m *= 2;
    return m;
}

// 16 consecutive values of type I from global memory into registers as T,
// with 16-byte vector loads (p must be 16-byte aligned).
template <typename T, typename I>
__device__ __forceinline__ void load16(const I *__restrict__ p, T (&out)[16]) {
    if constexpr (sizeof(I) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
        float4 a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = __ldg(q + k);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            out[4 * k] = (T)a[k].x;
            out[4 * k + 1] = (T)a[k].y;
            out[4 * k + 2] = (T)a[k].z;
            out[4 * k + 3] = (T)a[k].w;
        }
    } else {
        const double2 *q = reinterpret_cast<const double2 *>(p);
        double2 a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = __ldg(q + k);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            out[2 * k] = (T)a[k].x;
            out[2 * k + 1] = (T)a[k].y;
        }
    }
}

}  // namespace sfft
