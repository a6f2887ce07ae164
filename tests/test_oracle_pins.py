"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU.  Each test ties one oracle function to something other than itself:
the least-squares definition (brute-force design matrix), closed forms,
invariants, a frequency-domain evaluation of Eq. 19-24 and exact recovery.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import bruteforce, fourier
from synth import random_field

HERE = os.path.dirname(os.path.abspath(__file__))


def cfg(n0, n1, w0, w1, dk, db, cpr):
    return oracle.OracleConfig(n0, n1, w0, w1, dk, db, bool(cpr))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def pair(n0, n1, seed, sigma=5.0):
    R = random_field(n0, n1, seed)
    S = random_field(n0, n1, seed + 1000) * 0.5 + 0.7 * np.roll(R, (1, -1), axis=(0, 1))
    return R, S


CASES = [
    # n0, n1, w0, w1, dk, db, cpr
    (8, 8, 1, 1, 0, 0, 1),
    (12, 12, 2, 2, 1, 1, 0),
    (12, 10, 2, 1, 2, 1, 1),
    (13, 11, 1, 2, 1, 2, 0),
    (24, 22, 3, 3, 2, 2, 1),
    (9, 14, 0, 0, 2, 0, 0),
    (10, 10, 2, 2, 0, 2, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_system_equals_design_matrix(case):
    """M = C^T C and rhs = C^T S with C built column by column from Eq. 3-4, 11-12."""
    n0, n1, w0, w1, dk, db, cpr = case
    R, S = pair(n0, n1, seed=n0 * 7 + n1)
    M, rhs = oracle.build_system(R, S, cfg(*case))
    Mb, rb = bruteforce.normal_equations(R, S, w0, w1, dk, db, cpr)
    assert M.shape == Mb.shape
    assert rel(M, Mb) < 1e-12
    assert rel(rhs, rb) < 1e-12


@pytest.mark.parametrize("case", CASES[:4])
def test_system_with_mask_equals_masked_design_matrix(case):
    """Masked pixels are zero-filled in both images before the build (Sec. 3, zero fill)."""
    n0, n1, w0, w1, dk, db, cpr = case
    R, S = pair(n0, n1, seed=3 * n0 + n1)
    mask = (np.random.default_rng(5).random((n0, n1)) > 0.3).astype(np.uint8)
    M, rhs = oracle.build_system(R, S, cfg(*case), mask=mask)
    Mb, rb = bruteforce.normal_equations(R, S, w0, w1, dk, db, cpr, mask=mask)
    assert rel(M, Mb) < 1e-12 and rel(rhs, rb) < 1e-12


@pytest.mark.parametrize("case", [(8, 8, 1, 1, 1, 1, 1), (10, 12, 2, 1, 1, 1, 0), (9, 9, 1, 1, 2, 2, 1)])
def test_fourier_form_matches_real_space(case):
    """Eq. 19-24 evaluated as frequency sums with the basis spectra of Eq. 14 equal
    the real-space lag-sum system after the rescaling a = N0 N1 a-ring (Eq. 13)."""
    n0, n1, w0, w1, dk, db, cpr = case
    R, S = pair(n0, n1, seed=11)
    Mp, rp = fourier.paper_system(R, S, w0, w1, dk, db, cpr)
    nkern = oracle.num_unknowns(cfg(*case)) - (db + 1) * (db + 2) // 2
    Mr, rr = fourier.to_real_space_units(Mp, rp, n0, n1, nkern)
    M, rhs = oracle.build_system(R, S, cfg(*case))
    assert rel(M, Mr) < 1e-11
    assert rel(rhs, rr) < 1e-11


def test_closed_form_regression_w0():
    """w=0, D_K=D_B=0: S ~ a R + b, the textbook 2x2 normal equations."""
    R, S = pair(20, 24, seed=2)
    c = cfg(20, 24, 0, 0, 0, 0, 1)
    M, rhs = oracle.build_system(R, S, c)
    P = R.size
    assert M.shape == (2, 2)
    np.testing.assert_allclose(M, [[np.sum(R * R), np.sum(R)], [np.sum(R), P]], rtol=1e-13)
    np.testing.assert_allclose(rhs, [np.sum(R * S), np.sum(S)], rtol=1e-13)
    x = oracle.cholesky_solve(M, rhs)
    slope = np.sum((R - R.mean()) * (S - S.mean())) / np.sum((R - R.mean()) ** 2)
    icpt = S.mean() - slope * R.mean()
    np.testing.assert_allclose(x, [slope, icpt], rtol=1e-10)


def test_shift_case_golden():
    """S = R shifted by one pixel along x: delta_10 = K_10 + K_00 (Eq. 3-4), so the
    only non-zero coefficients are a_00 = 1 and a_(1,0) = 1, and D == 0."""
    with open(os.path.join(HERE, "golden", "shift_case.json")) as f:
        g = json.load(f)
    n0, n1, w = g["n0"], g["n1"], g["w"]
    R = random_field(n0, n1, g["seed"])
    S = np.roll(R, tuple(g["shift"]), axis=(0, 1))
    c = cfg(n0, n1, w, w, 0, 0, 1)
    M, rhs = oracle.build_system(R, S, c)
    x = oracle.cholesky_solve(M, rhs)
    expect = np.zeros_like(x)
    for item in g["nonzero"]:
        a, b = item["alpha"], item["beta"]
        expect[(a + w) * (2 * w + 1) + (b + w)] = item["value"]
    np.testing.assert_allclose(x, expect, atol=1e-8)
    D = oracle.subtract(R, S, x, c)
    assert np.max(np.abs(D)) < 1e-7 * np.max(np.abs(S))


@pytest.mark.parametrize("case", [(16, 16, 2, 2, 1, 1, 0), (14, 18, 1, 2, 2, 2, 1), (20, 20, 3, 3, 2, 1, 0)])
def test_exact_recovery(case):
    """Noise-free S built from an injected kernel, scale and background through the
    circular model of Eq. 12: the solve returns the injected coefficients."""
    n0, n1, w0, w1, dk, db, cpr = case
    R = random_field(n0, n1, seed=21)
    unk = bruteforce.unknown_list(w0, w1, dk, db, cpr)
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 0.05, len(unk))
    theta[0] += 1.0
    # S written out from Eq. 12 with np.roll, independently of the oracle code
    S = np.zeros((n0, n1))
    cx, cy = bruteforce.coords(n0), bruteforce.coords(n1)
    for k, u in enumerate(unk):
        if u[0] == "k":
            (i, j), (a, b) = u[1], u[2]
            g = np.outer(cx ** i, cy ** j) * R
            S += theta[k] * (g if (a, b) == (0, 0) else np.roll(g, (a, b), axis=(0, 1)) - g)
        else:
            p, q = u[1]
            S += theta[k] * np.outer(cx ** p, cy ** q)
    c = cfg(*case)
    M, rhs = oracle.build_system(R, S, c)
    x = oracle.cholesky_solve(M, rhs)
    np.testing.assert_allclose(x, theta, atol=1e-7 * max(1.0, np.abs(theta).max()))
    D = oracle.subtract(R, S, x, c)
    assert np.sqrt(np.mean(D ** 2)) < 1e-8 * np.sqrt(np.mean(S ** 2))


@pytest.mark.parametrize("case", CASES[1:5])
def test_invariants(case):
    """Symmetry, PSD, orthogonality of the residual, residual energy and the
    structural zero B[(t, ab != 0), (p,q) = (0,0)] = 0 (difference columns sum to zero)."""
    n0, n1, w0, w1, dk, db, cpr = case
    R, S = pair(n0, n1, seed=9)
    c = cfg(*case)
    M, rhs = oracle.build_system(R, S, c)
    assert np.max(np.abs(M - M.T)) <= 1e-12 * np.max(np.abs(M))
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= -1e-12 * ev.max()
    x = oracle.cholesky_solve(M, rhs)
    D = oracle.subtract(R, S, x, c)
    C = bruteforce.design_matrix(R, w0, w1, dk, db, cpr)
    assert np.max(np.abs(C.T @ D.ravel())) < 1e-8 * np.max(np.abs(rhs))
    np.testing.assert_allclose(np.sum(D * D), np.sum(S * S) - rhs @ x, rtol=1e-7)
    unk = bruteforce.unknown_list(w0, w1, dk, db, cpr)
    b00 = [k for k, u in enumerate(unk) if u[0] == "b" and u[1] == (0, 0)][0]
    for k, u in enumerate(unk):
        if u[0] == "k" and u[2] != (0, 0):
            assert abs(M[k, b00]) <= 1e-12 * np.max(np.abs(M))


def test_plain_delta_gram_is_toeplitz():
    """For D_K = 0, mapping the K basis back to the plain delta basis
    (D_ab = K_ab + K_00, Eq. 3-4) gives a Gram matrix that depends only on
    the offset difference: G(ab_row, ab_col) = Omega(ab_row - ab_col)."""
    w = 2
    R, S = pair(14, 14, seed=31)
    c = cfg(14, 14, w, w, 0, 0, 1)
    M, _ = oracle.build_system(R, S, c)
    L = (2 * w + 1) ** 2
    A = M[:L, :L]
    z = (L - 1) // 2
    G = A + A[:, [z]] + A[[z], :] + A[z, z]
    G[z, :] = A[z, :] + A[z, z]
    G[:, z] = A[:, z] + A[z, z]
    G[z, z] = A[z, z]
    offs = [(a, b) for a in range(-w, w + 1) for b in range(-w, w + 1)]
    for r, (ar, br) in enumerate(offs):
        for k, (ac, bc) in enumerate(offs):
            ref = oracle.lag_sum(R, R, ar - ac, br - bc)
            assert abs(G[r, k] - ref) <= 1e-10 * abs(A[z, z])


def test_lag_sum_against_roll():
    rng = np.random.default_rng(0)
    f = rng.normal(size=(7, 9))
    g = rng.normal(size=(7, 9))
    for r0, r1 in [(0, 0), (1, -2), (-3, 4), (6, 8), (-7, -9)]:
        ref = np.sum(f * np.roll(g, (-r0, -r1), axis=(0, 1)))
        assert abs(oracle.lag_sum(f, g, r0, r1) - ref) < 1e-12
        assert abs(oracle.lag_sum(f, g, r0, r1) - oracle.lag_sum(g, f, -r0, -r1)) < 1e-12


def test_system_entries_match_full_build():
    case = (12, 10, 2, 1, 2, 1, 1)
    R, S = pair(12, 10, seed=17)
    mask = (np.random.default_rng(1).random((12, 10)) > 0.2).astype(np.uint8)
    M, rhs = oracle.build_system(R, S, cfg(*case), mask=mask)
    n = M.shape[0]
    rng = np.random.default_rng(3)
    rows = rng.integers(0, n, 60)
    cols = rng.integers(-1, n, 60)
    out = oracle.system_entries(R, S, cfg(*case), rows, cols, mask=mask)
    ref = np.where(cols >= 0, M[rows, np.maximum(cols, 0)], rhs[rows])
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(M).max())


def test_unknown_order_and_count():
    for (w0, w1, dk, db, cpr) in [(4, 4, 0, 0, 1), (6, 6, 1, 1, 0), (8, 8, 2, 2, 1), (8, 8, 2, 2, 0), (1, 3, 2, 1, 1)]:
        c = cfg(40, 40, w0, w1, dk, db, cpr)
        unk = bruteforce.unknown_list(w0, w1, dk, db, cpr)
        assert oracle.num_unknowns(c) == len(unk)
        for k, u in enumerate(unk):
            is_k, t, a, b = oracle.decode_unknown(c, k)
            if u[0] == "k":
                assert is_k and bruteforce.monomials(dk)[t] == u[1] and (a, b) == u[2]
            else:
                assert (not is_k) and bruteforce.monomials(db)[t] == u[1]
    assert oracle.num_unknowns(cfg(256, 256, 4, 4, 0, 0, 1)) == 82
    assert oracle.num_unknowns(cfg(1024, 1024, 6, 6, 1, 1, 0)) == 510
    assert oracle.num_unknowns(cfg(4096, 4096, 8, 8, 2, 2, 1)) == 1735


def test_cholesky_against_library_and_failure():
    rng = np.random.default_rng(7)
    A = rng.normal(size=(40, 40))
    M = A @ A.T + 40 * np.eye(40)
    b = rng.normal(size=40)
    np.testing.assert_allclose(oracle.cholesky_solve(M, b), np.linalg.solve(M, b), rtol=1e-11)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky_solve(-M, b)
    # a zero reference image makes every kernel column vanish: rank deficient
    R = np.zeros((10, 10))
    S = random_field(10, 10, 1)
    Mz, rz = oracle.build_system(R, S, cfg(10, 10, 1, 1, 0, 0, 1))
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky_solve(Mz, rz)


@pytest.mark.parametrize("case", CASES[:5])
def test_subtract_equals_design_product(case):
    """D = S - C theta (Eq. 12) for an arbitrary coefficient vector, and the
    per-pixel form agrees with the full image."""
    n0, n1, w0, w1, dk, db, cpr = case
    R, S = pair(n0, n1, seed=41)
    theta = np.random.default_rng(2).normal(size=len(bruteforce.unknown_list(w0, w1, dk, db, cpr)))
    D = oracle.subtract(R, S, theta, cfg(*case))
    Db = bruteforce.difference(R, S, theta, w0, w1, dk, db, cpr)
    np.testing.assert_allclose(D, Db, rtol=1e-12, atol=1e-12 * np.abs(Db).max())
    idx = np.array([0, 5, n0 * n1 - 1, n0 * n1 // 2])
    np.testing.assert_allclose(oracle.subtract_pixels(R, S, theta, cfg(*case), idx), D.ravel()[idx], rtol=1e-14)


def test_flux_conservation_physical_psf():
    """Gaussian PSFs (reference FWHM 2.5, science 3.5) and photometric scale
    1.0 -> 1.1 along y: the fitted kernel sum, sum_ij a_ij00 x^i y^j (Eq. 3-6:
    only K_00 carries flux), follows the injected scale."""
    from synth import PAIR1024, make_pair, scaled
    spec = scaled(PAIR1024, 256)
    R, S = make_pair(spec, seed=2)
    R, S = R.astype(np.float64), S.astype(np.float64)
    c = cfg(256, 256, 4, 4, 1, 1, 0)
    M, rhs = oracle.build_system(R, S, c)
    x = oracle.cholesky_solve(M, rhs)
    L = 81
    a00_00, a10_00, a01_00 = x[(L - 1) // 2], x[L + (L - 1) // 2], x[2 * L + (L - 1) // 2]
    # scale(y) = 1.0 + 0.1 (yt + 1) / 2 = 1.05 + 0.05 yt
    assert abs(a00_00 - 1.05) < 0.01
    assert abs(a01_00 - 0.05) < 0.01
    assert abs(a10_00) < 0.01


@pytest.mark.parametrize("n0,n1", [(13, 11), (16, 16)])
def test_lambda_lag_sums_against_moment_closed_form(n0, n1):
    """Lambda_ts(rho) = sum_x g_t(x) T_s((x + rho) mod N) for g_t = x^i y^j R and
    T_s = x^p y^q (App. B, Eq. B8) against its closed form: on rows whose
    shifted index stays inside the image the shifted coordinate is
    x + 2 rho0/(n0-1); on the rows that wrap it moves by a further
    -/+ 2 n0/(n0-1) (likewise along y).  So Lambda is a sum over four
    row/column blocks of binomial expansions in the blocks' 2-D moments
    mu_B(u, v) = sum_B x^u y^v R, with no circular index anywhere."""
    from math import comb
    R = random_field(n0, n1, seed=17)
    xt = bruteforce.coords(n0)
    yt = bruteforce.coords(n1)

    def classes(n, rho):
        """Index sets and coordinate offsets: the rows that stay inside and those that wrap."""
        idx = np.arange(n)
        wraps = (idx + rho >= n) | (idx + rho < 0)
        d = 2.0 * rho / (n - 1)
        dw = d - np.sign(rho) * 2.0 * n / (n - 1)
        return [(idx[~wraps], d), (idx[wraps], dw)]

    for (i, j) in [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1)]:
        g = np.outer(xt ** i, yt ** j) * R
        for (p, q) in [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]:
            T = np.outer(xt ** p, yt ** q)
            for r0 in range(-3, 4):
                for r1 in range(-3, 4):
                    closed = 0.0
                    for rows, d0 in classes(n0, r0):
                        for cols, d1 in classes(n1, r1):
                            if rows.size == 0 or cols.size == 0:
                                continue
                            blk = R[np.ix_(rows, cols)]
                            xs, ys = xt[rows], yt[cols]
                            for a in range(p + 1):
                                for b in range(q + 1):
                                    mu = xs ** (i + a) @ blk @ ys ** (j + b)
                                    closed += comb(p, a) * comb(q, b) * d0 ** (p - a) * d1 ** (q - b) * mu
                    lag = oracle.lag_sum(g, T, r0, r1)
                    assert abs(lag - closed) <= 1e-12 * max(1.0, np.abs(R).sum()), (i, j, p, q, r0, r1)
