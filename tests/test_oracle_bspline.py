"""Pins of the oracle's B-spline bases (Eq. 7-9) against what the mathematics fixes.

No GPU.  The C oracle evaluates the basis by its own Cox-de Boor recursion and
builds the system from lag sums; here it is tied to scipy's B-splines (a
library primitive the oracle does not use), to the brute-force design matrix
built on scipy's values, to partition of unity, to the degree-0 case (the
constant function, which is the polynomial basis of degree 0), and to exact
recovery of an injected spatially varying kernel and background.
"""
import numpy as np
import pytest

import oracle
from oracle import bruteforce
from synth import random_field

pytest.importorskip("scipy")


def cfg(n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint):
    return oracle.OracleConfig(n0, n1, w0, w1, 0, 0, bool(cpr), "bspline", kdeg, kint, bdeg, bint)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def pair(n0, n1, seed):
    R = random_field(n0, n1, seed)
    S = random_field(n0, n1, seed + 1000) * 0.5 + 0.7 * np.roll(R, (1, -1), axis=(0, 1))
    return R, S


@pytest.mark.parametrize("deg,nint", [(0, 0), (0, 3), (1, 0), (1, 2), (2, 3), (3, 0), (3, 4), (5, 2)])
def test_basis_matches_scipy_and_partitions_unity(deg, nint):
    u = np.concatenate([np.linspace(-1.0, 1.0, 201), [-1.0, 1.0, -0.999999, 0.999999]])
    K = deg + nint + 1
    ours = np.array([[oracle.bspline(deg, nint, i, v) for v in u] for i in range(K)])
    ref = bruteforce.spline_basis(deg, nint, u)
    assert np.max(np.abs(ours - ref)) < 1e-13
    assert np.all(ours >= -1e-15)
    assert np.max(np.abs(ours.sum(axis=0) - 1.0)) < 1e-13
    # the knots are where the text puts them: function 0 starts at 1 at the left end
    assert abs(oracle.bspline(deg, nint, 0, -1.0) - 1.0) < 1e-15
    assert abs(oracle.bspline(deg, nint, K - 1, 1.0) - 1.0) < 1e-15


CASES = [
    # n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint
    (10, 12, 1, 1, 1, 1, 0, 1, 0),
    (12, 12, 2, 1, 0, 1, 1, 0, 0),
    (14, 11, 1, 2, 1, 2, 1, 1, 1),
    (16, 16, 2, 2, 1, 3, 0, 2, 0),
    (9, 13, 1, 1, 0, 0, 2, 2, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_system_equals_design_matrix(case):
    """Lag-sum system (C, Cox-de Boor) = C^T C, C^T S of the explicit design matrix (scipy basis)."""
    n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint = case
    R, S = pair(n0, n1, seed=n0 * 7 + n1)
    c = cfg(*case)
    M, rhs = oracle.build_system(R, S, c)
    Mb, rb = bruteforce.normal_equations(R, S, w0, w1, 0, 0, cpr, spline=(kdeg, kint, bdeg, bint))
    assert M.shape == Mb.shape == (oracle.num_unknowns(c),) * 2
    assert rel(M, Mb) < 1e-12
    assert rel(rhs, rb) < 1e-12


def test_masked_system_equals_masked_design_matrix():
    n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint = (14, 12, 1, 1, 1, 2, 1, 1, 1)
    R, S = pair(n0, n1, seed=5)
    mask = (np.random.default_rng(6).random((n0, n1)) > 0.2).astype(np.uint8)
    M, rhs = oracle.build_system(R, S, cfg(n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint), mask=mask)
    Mb, rb = bruteforce.normal_equations(R, S, w0, w1, 0, 0, cpr, mask=mask, spline=(kdeg, kint, bdeg, bint))
    assert rel(M, Mb) < 1e-12
    assert rel(rhs, rb) < 1e-12


@pytest.mark.parametrize("cpr", [0, 1])
def test_degree0_without_interior_knots_is_the_constant_polynomial(cpr):
    """One B-spline of degree 0 on the whole field is the constant 1, so the
    fit equals the polynomial fit with D_K = D_B = 0: same difference image
    (and, without a constant ratio, the same unknowns in the same order)."""
    n0, n1, w0, w1 = 12, 14, 2, 1
    R, S = pair(n0, n1, seed=31)
    cb = cfg(n0, n1, w0, w1, cpr, 0, 0, 0, 0)
    cp = oracle.OracleConfig(n0, n1, w0, w1, 0, 0, bool(cpr))
    assert oracle.num_unknowns(cb) == oracle.num_unknowns(cp)
    xb = oracle.cholesky_solve(*oracle.build_system(R, S, cb))
    xp = oracle.cholesky_solve(*oracle.build_system(R, S, cp))
    Db, Dp = oracle.subtract(R, S, xb, cb), oracle.subtract(R, S, xp, cp)
    assert np.max(np.abs(Db - Dp)) < 1e-9 * np.max(np.abs(S))
    if not cpr:
        assert rel(xb, xp) < 1e-10


@pytest.mark.parametrize("case", [(16, 16, 1, 1, 1, 1, 1, 1, 0), (18, 14, 2, 1, 0, 2, 0, 1, 1),
                                  (20, 20, 1, 2, 1, 3, 1, 2, 1)])
def test_exact_recovery(case):
    """Noise-free S written out from Eq. 12 with a B-spline-varying kernel and
    background (np.roll and scipy's basis): the solve returns the injected
    coefficients and the difference image vanishes."""
    n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint = case
    spline = (kdeg, kint, bdeg, bint)
    R = random_field(n0, n1, seed=21)
    unk = bruteforce.unknown_list(w0, w1, 0, 0, cpr, spline)
    weight = {lab: w for lab, w, _, _ in bruteforce.kernel_terms(n0, n1, 0, cpr, spline)}
    bg = dict(bruteforce.background_terms(n0, n1, 0, spline))
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 0.05, len(unk))
    S = np.zeros((n0, n1))
    for k, u in enumerate(unk):
        if u[0] == "k":
            (a, b) = u[2]
            if (a, b) == (0, 0):
                theta[k] += 1.0
            g = weight[u[1]] * R
            S += theta[k] * (g if (a, b) == (0, 0) else np.roll(g, (a, b), axis=(0, 1)) - g)
        else:
            S += theta[k] * 100.0 * bg[u[1]]
            theta[k] *= 100.0
    c = cfg(*case)
    M, rhs = oracle.build_system(R, S, c)
    x = oracle.cholesky_solve(M, rhs)
    # exact up to the conditioning of the system: |dx|/|x| <~ cond(M) u
    assert rel(x, theta) < 10 * np.linalg.cond(M) * np.finfo(float).eps
    D = oracle.subtract(R, S, x, c)
    assert np.max(np.abs(D)) < 1e-8 * np.max(np.abs(S))


def test_subtract_matches_design_matrix():
    n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint = (15, 13, 2, 1, 1, 2, 1, 1, 2)
    spline = (kdeg, kint, bdeg, bint)
    R, S = pair(n0, n1, seed=44)
    c = cfg(n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint)
    theta = np.random.default_rng(8).normal(0, 0.1, oracle.num_unknowns(c))
    D = oracle.subtract(R, S, theta, c)
    Db = bruteforce.difference(R, S, theta, w0, w1, 0, 0, cpr, spline)
    assert np.max(np.abs(D - Db)) < 1e-11 * np.max(np.abs(S))
    flat = np.array([0, 7, n0 * n1 - 1, 3 * n1 + 5])
    assert np.allclose(oracle.subtract_pixels(R, S, theta, c, flat), Db.ravel()[flat], rtol=0, atol=1e-11 * np.abs(S).max())


def test_constant_ratio_kernel_sum_is_the_constant_term():
    """With a constant photometric ratio the kernel sum at every pixel is the
    coefficient of the weight-1 term (the other offsets' basis vectors sum to
    zero, Eq. 4): the recovered sum equals the injected photometric scale."""
    n0, n1, w0, w1 = 16, 18, 1, 1
    spline = (2, 1, 1, 0)
    R = random_field(n0, n1, seed=3)
    scale = 1.37
    S = scale * np.roll(R, (1, 0), axis=(0, 1)) + 20.0
    c = cfg(n0, n1, w0, w1, 1, *spline)
    x = oracle.cholesky_solve(*oracle.build_system(R, S, c))
    unk = bruteforce.unknown_list(w0, w1, 0, 0, True, spline)
    assert unk[0] == ("k", ("one",), (0, 0))
    assert abs(x[0] - scale) < 1e-8
    D = oracle.subtract(R, S, x, c)
    assert np.max(np.abs(D)) < 1e-8 * np.max(np.abs(S))
