"""Noise decorrelation of the difference image (App. C, Eq. 21-24), FP64.

Two forms: one pair (below) and the co-added form of Eq. 21-24 in full
(decorrelate_coadd).

TEST INFRASTRUCTURE ONLY (see the package header): imported by the tests.

For one pair with no co-addition (M = N = 1 and G = H = delta in Eq. 21),
Eq. 23-24 give the real decorrelation filter

    Q0(p) = sqrt( sigma_D^2 / (sigma_S^2 + sigma_R^2 |K(p)|^2) ),

where K(p) is the DFT of the matching kernel.  App. C ignores the spatial
variation of the kernel, so K is the kernel of Eq. 6 evaluated at one
normalised position (xt0, yt0).  The filter is normalised to unit kernel
sum (the flux-preserving choice App. C names), i.e. Q(0) = 1, which sets
sigma_D^2 = sigma_S^2 + sigma_R^2 K(0)^2.  The decorrelated image is the
circular convolution D_dc = D (*) Q.  numpy's FFT serves as the DFT primitive.
"""
import numpy as np

from . import bruteforce


def term_weight_at(label, xt0, yt0, spline=None):
    """Weight of a kernel term (label as in bruteforce.kernel_terms) at one
    normalised position: xt0^i yt0^j (Eq. 6), B_i(xt0) B_j(yt0) (Eq. 8), or 1."""
    if label[0] == "one":
        return 1.0
    if label[0] == "spl":
        kdeg, kint = spline[0], spline[1]
        return float(bruteforce.spline_basis(kdeg, kint, [xt0])[label[1], 0] *
                     bruteforce.spline_basis(kdeg, kint, [yt0])[label[2], 0])
    i, j = label
    return xt0 ** i * yt0 ** j


def kernel_image(x, w0, w1, dk, db, const_phot_ratio, xt0, yt0, spline=None):
    """Matching kernel at (xt0, yt0) as an image k[alpha + w0, beta + w1].

    With the delta basis of Eq. 3-4, K_ab = delta(a, b) - delta(0, 0) for
    (a, b) != 0 and K_00 = delta(0, 0), so a coefficient of offset (a, b) != 0
    adds at the offset and subtracts at the centre; Eq. 6 weights the
    coefficients of term (i, j) by xt0^i yt0^j (Eq. 8: by B_i(xt0) B_j(yt0)).
    """
    k = np.zeros((2 * w0 + 1, 2 * w1 + 1))
    for u, unk in enumerate(bruteforce.unknown_list(w0, w1, dk, db, const_phot_ratio, spline)):
        if unk[0] != "k":
            continue
        (a, b) = unk[2]
        c = x[u] * term_weight_at(unk[1], xt0, yt0, spline)
        if (a, b) == (0, 0):
            k[w0, w1] += c
        else:
            k[a + w0, b + w1] += c
            k[w0, w1] -= c
    return k


def filter_spectrum(k, n0, n1, sigma_ref, sigma_sci):
    """Q(l, m) of Eq. 24, normalised to Q(0, 0) = 1, for the kernel image k."""
    w0, w1 = k.shape[0] // 2, k.shape[1] // 2
    full = np.zeros((n0, n1))
    for a in range(-w0, w0 + 1):
        for b in range(-w1, w1 + 1):
            full[a % n0, b % n1] += k[a + w0, b + w1]
    kh = np.fft.fft2(full)
    sd2 = sigma_sci ** 2 + sigma_ref ** 2 * abs(kh[0, 0]) ** 2
    return np.sqrt(sd2 / (sigma_sci ** 2 + sigma_ref ** 2 * np.abs(kh) ** 2))


def decorrelate(D, k, sigma_ref, sigma_sci):
    """D (*) Q, circular, with Q from filter_spectrum."""
    D = np.asarray(D, np.float64)
    q = filter_spectrum(k, D.shape[0], D.shape[1], sigma_ref, sigma_sci)
    return np.real(np.fft.ifft2(np.fft.fft2(D) * q))


def kernel_spectrum(k, n0, n1):
    """2-D DFT of a centred kernel image k (half-widths k.shape // 2) placed
    circularly on the n0 x n1 grid."""
    w0, w1 = k.shape[0] // 2, k.shape[1] // 2
    full = np.zeros((n0, n1))
    for a in range(-w0, w0 + 1):
        for b in range(-w1, w1 + 1):
            full[a % n0, b % n1] += k[a + w0, b + w1]
    return np.fft.fft2(full)


def coadd_filter(k, n0, n1, sigma_sci, G, sigma_ref, H):
    """Q0 of Eq. 24 for D = sum_j S_j (*) G_j - [sum_i R_i (*) H_i] (*) K (Eq. 21):
    sqrt(s_D^2 / (sum_j s_Sj^2 |G^_j|^2 + |K^|^2 sum_i s_Ri^2 |H^_i|^2)),
    with s_D^2 the denominator at frequency 0 (unit kernel sum)."""
    kh = kernel_spectrum(k, n0, n1)
    den = np.zeros((n0, n1))
    for s, g in zip(sigma_sci, G):
        den += s ** 2 * np.abs(kernel_spectrum(g, n0, n1)) ** 2
    dh = np.zeros((n0, n1))
    for s, h in zip(sigma_ref, H):
        dh += s ** 2 * np.abs(kernel_spectrum(h, n0, n1)) ** 2
    den = den + np.abs(kh) ** 2 * dh
    return np.sqrt(den[0, 0] / den)


def decorrelate_coadd(D, k, sigma_sci, G, sigma_ref, H):
    """D (*) Q, circular, with Q from coadd_filter."""
    D = np.asarray(D, np.float64)
    q = coadd_filter(k, D.shape[0], D.shape[1], sigma_sci, G, sigma_ref, H)
    return np.real(np.fft.ifft2(np.fft.fft2(D) * q))
