"""Pins of the decorrelation oracle (App. C, Eq. 21-24) against what the
mathematics fixes, on the CPU."""
import numpy as np
import pytest

from oracle import bruteforce, decorr
from synth import random_field


def test_kernel_image_reproduces_the_model_convolution():
    """For D_K = 0 the kernel part of the model, sum_u x_u C_u (the design
    matrix of Eq. 12), is the circular convolution of R with the kernel image."""
    rng = np.random.default_rng(3)
    n0, n1, w0, w1 = 12, 10, 2, 1
    R = random_field(n0, n1, 5)
    for cpr in (True, False):
        unk = bruteforce.unknown_list(w0, w1, 0, 1, cpr)
        x = rng.standard_normal(len(unk))
        C = bruteforce.design_matrix(R, w0, w1, 0, 1, cpr)
        kcols = [u for u, e in enumerate(unk) if e[0] == "k"]
        model = (C[:, kcols] @ x[kcols]).reshape(n0, n1)
        k = decorr.kernel_image(x, w0, w1, 0, 1, cpr, 0.3, -0.7)
        conv = np.zeros((n0, n1))
        for a in range(-w0, w0 + 1):
            for b in range(-w1, w1 + 1):
                conv += k[a + w0, b + w1] * np.roll(np.roll(R, a, axis=0), b, axis=1)
        assert np.allclose(conv, model, rtol=0, atol=1e-10 * np.abs(model).max())


def test_delta_kernel_leaves_the_image_unchanged():
    k = np.zeros((5, 3))
    k[2, 1] = 1.3  # a scaled delta: |K^| is constant, so Q = 1
    D = random_field(16, 12, 9)
    assert np.allclose(decorr.decorrelate(D, k, 4.0, 6.0), D, rtol=0, atol=1e-10 * np.abs(D).max())


def test_mean_is_preserved():
    rng = np.random.default_rng(1)
    k = rng.standard_normal((5, 5)) * 0.1
    k[2, 2] += 1.0
    D = random_field(20, 24, 2)
    assert np.isclose(decorr.decorrelate(D, k, 5.0, 3.0).mean(), D.mean(), rtol=1e-12)


def test_whitens_the_difference_noise():
    """White noise in R and S (sigma_R, sigma_S) through D = S - K (*) R has
    the power spectrum sigma_S^2 + sigma_R^2 |K^|^2; after decorrelation it is
    flat at sigma_S^2 + sigma_R^2 K^(0)^2.  Averaged over many realisations."""
    rng = np.random.default_rng(7)
    n0, n1, sr, ss = 24, 20, 3.0, 2.0
    k = np.zeros((5, 5))
    k[2, 2], k[1, 2], k[3, 2], k[2, 1], k[2, 3] = 0.6, 0.15, 0.1, 0.1, 0.05  # a blur
    full = np.zeros((n0, n1))
    for a in range(-2, 3):
        for b in range(-2, 3):
            full[a % n0, b % n1] = k[a + 2, b + 2]
    kh = np.fft.fft2(full)
    raw = np.zeros((n0, n1))
    dec = np.zeros((n0, n1))
    trials = 400
    for _ in range(trials):
        R = rng.normal(0, sr, (n0, n1))
        S = rng.normal(0, ss, (n0, n1))
        D = S - np.real(np.fft.ifft2(np.fft.fft2(R) * kh))
        raw += np.abs(np.fft.fft2(D)) ** 2
        dec += np.abs(np.fft.fft2(decorr.decorrelate(D, k, sr, ss))) ** 2
    raw /= trials * n0 * n1
    dec /= trials * n0 * n1
    flat = ss ** 2 + sr ** 2 * kh[0, 0].real ** 2
    assert raw.max() / raw.min() > 2.0  # the difference's noise is correlated
    # each averaged bin has a relative error of about 1/sqrt(trials) = 5 %
    assert np.abs(dec / flat - 1).max() < 0.3
    assert abs(dec.mean() / flat - 1) < 0.02


def _blur(rng, w0, w1, spread=0.1):
    k = np.abs(rng.standard_normal((2 * w0 + 1, 2 * w1 + 1))) * spread
    k[w0, w1] += 1.0
    return k / k.sum()


def test_coadd_form_with_delta_kernels_is_the_pair_form():
    """M = N = 1 and G = H = delta reduce Eq. 21 to D = S - R (*) K."""
    rng = np.random.default_rng(3)
    k = _blur(rng, 2, 2)
    d = np.zeros((3, 3))
    d[1, 1] = 1.0
    D = random_field(20, 16, 4)
    a = decorr.decorrelate_coadd(D, k, [6.0], [d], [4.0], [d])
    b = decorr.decorrelate(D, k, 4.0, 6.0)
    assert np.allclose(a, b, rtol=0, atol=1e-10 * np.abs(D).max())


def test_coadd_filter_whitens_coadded_noise():
    """White noise in M = 3 science and N = 2 reference exposures, homogenised
    by G_j, H_i, co-added (Eq. 21) and subtracted through K: after the filter
    of Eq. 24 the power spectrum is flat (Monte Carlo, 400 realisations)."""
    rng = np.random.default_rng(11)
    n0, n1 = 20, 24
    k = _blur(rng, 2, 2, 0.3)
    G = [_blur(rng, 1, 1, 0.4) / 3 for _ in range(3)]
    H = [_blur(rng, 2, 1, 0.4) / 2 for _ in range(2)]
    ss, sr = [2.0, 3.0, 2.5], [1.5, 4.0]
    kh = decorr.kernel_spectrum(k, n0, n1)
    gh = [decorr.kernel_spectrum(g, n0, n1) for g in G]
    hh = [decorr.kernel_spectrum(h, n0, n1) for h in H]
    raw = np.zeros((n0, n1))
    dec = np.zeros((n0, n1))
    trials = 400
    for _ in range(trials):
        Sf = sum(np.fft.fft2(rng.normal(0, s, (n0, n1))) * g for s, g in zip(ss, gh))
        Rf = sum(np.fft.fft2(rng.normal(0, s, (n0, n1))) * h for s, h in zip(sr, hh))
        D = np.real(np.fft.ifft2(Sf - Rf * kh))
        raw += np.abs(np.fft.fft2(D)) ** 2
        dec += np.abs(np.fft.fft2(decorr.decorrelate_coadd(D, k, ss, G, sr, H))) ** 2
    raw /= trials * n0 * n1
    dec /= trials * n0 * n1
    flat = sum(s ** 2 * abs(g[0, 0]) ** 2 for s, g in zip(ss, gh)) + abs(kh[0, 0]) ** 2 * sum(
        s ** 2 * abs(h[0, 0]) ** 2 for s, h in zip(sr, hh))
    assert raw.max() / raw.min() > 2.0
    assert np.abs(dec / flat - 1).max() < 0.3
    assert abs(dec.mean() / flat - 1) < 0.02


def test_saturation_mask_matches_binary_dilation():
    """The crowded-flavor mask against scipy's binary dilation with a square
    structuring element (a library routine the oracle does not use)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    from oracle import masking
    rng = np.random.default_rng(5)
    for n0, n1, grow in ((17, 23, 0), (32, 32, 2), (20, 13, 4)):
        R = rng.uniform(0, 100, (n0, n1))
        S = rng.uniform(0, 100, (n0, n1))
        sat = (R >= 97.0) | (S >= 98.5)
        want = ~ndimage.binary_dilation(sat, structure=np.ones((2 * grow + 1, 2 * grow + 1), bool)) if grow else ~sat
        got = masking.saturation_mask(R, S, 97.0, 98.5, grow)
        assert np.array_equal(got.astype(bool), want)
        m_in = (rng.random((n0, n1)) > 0.1).astype(np.uint8)
        got2 = masking.saturation_mask(R, S, 97.0, 98.5, grow, m_in)
        assert np.array_equal(got2.astype(bool), want & (m_in != 0))


def test_saturation_mask_edge_cases():
    """Closed expectations: a pixel exactly at its level counts as saturated;
    nothing saturated keeps everything; a window wider than the image masks
    every pixel once anything saturates; a saturated corner pixel masks exactly
    the (grow + 1)^2 pixels of the clipped square at that corner."""
    from oracle import masking
    n0, n1 = 24, 19
    R = np.zeros((n0, n1))
    S = np.zeros((n0, n1))
    assert masking.saturation_mask(R, S, 1.0, 1.0, 3).all()
    R[5, 7] = 1.0                                   # exactly at the level
    m = masking.saturation_mask(R, S, 1.0, 2.0, 0)
    assert m[5, 7] == 0 and m.sum() == n0 * n1 - 1
    assert not masking.saturation_mask(R, S, 1.0, 2.0, 30).any()
    R[5, 7] = 0.0
    S[n0 - 1, 0] = 5.0                              # a saturated corner of S
    for grow in (0, 1, 16):
        m = masking.saturation_mask(R, S, 1.0, 5.0, grow)
        assert (m == 0).sum() == (grow + 1) ** 2
        assert (m[n0 - 1 - grow:, :grow + 1] == 0).all()
