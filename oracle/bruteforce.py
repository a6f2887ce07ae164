"""Brute-force tier of the oracle: the least-squares definition written out.

Test infrastructure only.

The difference image of Eq. 12 is linear in the unknowns:
``D = S - C @ theta`` with one design column per unknown --
``(g_t o K_ab)(x) = g_t(x - ab) - g_t(x)`` for (alpha,beta) != 0 (Eq. 4),
``g_t(x)`` for (alpha,beta) = 0 (Eq. 3), and ``T^pq(x)`` for the background
(Eq. 2) -- where ``g_t = x^i y^j R`` (Eq. 10-11), or B-spline products
``B_i(x) B_j(y) R`` (Eq. 8-9), and every shift is circular.
Minimising sum D^2 gives the normal equations ``C^T C theta = C^T S`` (Eq. 18).
Everything here is built from that statement alone: an explicit P x n matrix,
numpy products and ``numpy.linalg.lstsq``.  Only for tiny images.
"""
from __future__ import annotations

import numpy as np


def coords(n: int) -> np.ndarray:
    """Normalised pixel coordinate in [-1, 1]: (2x - (n-1)) / (n-1)."""
    return (2.0 * np.arange(n) - (n - 1)) / (n - 1)


def monomials(d: int):
    """(i, j) with i + j <= d: by total degree, then descending i."""
    return [(deg - k, k) for deg in range(d + 1) for k in range(deg + 1)]


def clamped_knots(deg: int, nint: int) -> np.ndarray:
    """Clamped uniform knot vector on [-1, 1]: deg+1 end knots, nint interior knots."""
    inner = -1.0 + 2.0 * np.arange(1, nint + 1) / (nint + 1)
    return np.concatenate([np.full(deg + 1, -1.0), inner, np.full(deg + 1, 1.0)])


def spline_basis(deg: int, nint: int, u) -> np.ndarray:
    """[K, len(u)] values of the K = nint + deg + 1 B-spline basis functions at u
    (scipy's BSpline as the evaluation primitive; u = 1 lies in the last span)."""
    from scipy.interpolate import BSpline
    t = clamped_knots(deg, nint)
    K = nint + deg + 1
    u = np.asarray(u, np.float64)
    out = np.zeros((K, u.size))
    for i in range(K):
        c = np.zeros(K)
        c[i] = 1.0
        out[i] = BSpline(t, c, deg, extrapolate=False)(u)
    return np.nan_to_num(out)


def kernel_terms(n0, n1, dk, const_phot_ratio, spline=None):
    """Kernel terms in solve order: (label, weight image, has (0,0) offset, has the others).

    Polynomial (Eq. 6): label (i, j), weight x^i y^j, by total degree; with a
    constant photometric ratio only (0,0) keeps the (0,0) offset.  B-spline
    (Eq. 8), spline = (kdeg, kint, bdeg, bint): label ("spl", i, j), weight
    B_i(x) B_j(y), i outer; with a constant photometric ratio a first term
    ("one",) of weight 1 carries the (0,0) offset alone and the spline terms
    carry the others."""
    cx, cy = coords(n0), coords(n1)
    if spline is None:
        return [(ij, np.outer(cx ** ij[0], cy ** ij[1]), (not const_phot_ratio) or t == 0, True)
                for t, ij in enumerate(monomials(dk))]
    kdeg, kint = spline[0], spline[1]
    bx, by = spline_basis(kdeg, kint, cx), spline_basis(kdeg, kint, cy)
    K = kdeg + kint + 1
    out = []
    if const_phot_ratio:
        out.append((("one",), np.ones((n0, n1)), True, False))
    for i in range(K):
        for j in range(K):
            out.append((("spl", i, j), np.outer(bx[i], by[j]), not const_phot_ratio, True))
    return out


def background_terms(n0, n1, db, spline=None):
    """Background terms in solve order: (label, image), x^p y^q with label (p, q)
    (Eq. 2) or B'_p(x) B'_q(y) with label ("spl", p, q) (Eq. 9)."""
    cx, cy = coords(n0), coords(n1)
    if spline is None:
        return [((p, q), np.outer(cx ** p, cy ** q)) for p, q in monomials(db)]
    bdeg, bint = spline[2], spline[3]
    bx, by = spline_basis(bdeg, bint, cx), spline_basis(bdeg, bint, cy)
    K = bdeg + bint + 1
    return [(("spl", p, q), np.outer(bx[p], by[q])) for p in range(K) for q in range(K)]


def unknown_list(w0, w1, dk, db, const_phot_ratio, spline=None):
    """Every unknown as ('k', term label, (alpha,beta)) or ('b', term label), in solve order."""
    out = []
    for label, _, has00, hasother in kernel_terms(2, 2, dk, const_phot_ratio, spline):
        for a in range(-w0, w0 + 1):
            for b in range(-w1, w1 + 1):
                if (a == 0 and b == 0 and not has00) or ((a != 0 or b != 0) and not hasother):
                    continue
                out.append(("k", label, (a, b)))
    for label, _ in background_terms(2, 2, db, spline):
        out.append(("b", label))
    return out


def design_matrix(R, w0, w1, dk, db, const_phot_ratio, spline=None):
    n0, n1 = R.shape
    weight = {lab: w for lab, w, _, _ in kernel_terms(n0, n1, dk, const_phot_ratio, spline)}
    bg = dict(background_terms(n0, n1, db, spline))
    cols = []
    for u in unknown_list(w0, w1, dk, db, const_phot_ratio, spline):
        if u[0] == "k":
            (a, b) = u[2]
            g = weight[u[1]] * R
            if a == 0 and b == 0:
                cols.append(g.ravel())
            else:
                # (g o K_ab)(x, y) = g(x - a, y - b) - g(x, y), circular
                shifted = np.roll(np.roll(g, a, axis=0), b, axis=1)
                cols.append((shifted - g).ravel())
        else:
            cols.append(bg[u[1]].ravel())
    return np.stack(cols, axis=1)


def normal_equations(R, S, w0, w1, dk, db, const_phot_ratio, mask=None, spline=None):
    if mask is not None:
        keep = (np.asarray(mask) != 0).astype(np.float64)
        R = R * keep
        S = S * keep
    C = design_matrix(np.asarray(R, np.float64), w0, w1, dk, db, const_phot_ratio, spline)
    s = np.asarray(S, np.float64).ravel()
    return C.T @ C, C.T @ s


def least_squares(R, S, w0, w1, dk, db, const_phot_ratio, mask=None, spline=None):
    """Coefficients minimising sum D^2 over the (masked) pair, by lstsq."""
    if mask is not None:
        keep = (np.asarray(mask) != 0).astype(np.float64)
        Rm, Sm = R * keep, S * keep
    else:
        Rm, Sm = R, S
    C = design_matrix(np.asarray(Rm, np.float64), w0, w1, dk, db, const_phot_ratio, spline)
    theta, *_ = np.linalg.lstsq(C, np.asarray(Sm, np.float64).ravel(), rcond=None)
    return theta


def difference(R, S, theta, w0, w1, dk, db, const_phot_ratio, spline=None):
    """D = S - C theta on the unmasked pair (Eq. 12)."""
    C = design_matrix(np.asarray(R, np.float64), w0, w1, dk, db, const_phot_ratio, spline)
    return (np.asarray(S, np.float64).ravel() - C @ theta).reshape(R.shape)
