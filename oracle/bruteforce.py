"""Brute-force tier of the oracle: the least-squares definition written out.

Test infrastructure only.

The difference image of Eq. 12 is linear in the unknowns:
``D = S - C @ theta`` with one design column per unknown --
``(g_t o K_ab)(x) = g_t(x - ab) - g_t(x)`` for (alpha,beta) != 0 (Eq. 4),
``g_t(x)`` for (alpha,beta) = 0 (Eq. 3), and ``T^pq(x)`` for the background
(Eq. 2) -- where ``g_t = x^i y^j R`` (Eq. 10-11) and every shift is circular.
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


def unknown_list(w0, w1, dk, db, const_phot_ratio):
    """Every unknown as ('k', (i,j), (alpha,beta)) or ('b', (p,q)), in solve order."""
    out = []
    for t, ij in enumerate(monomials(dk)):
        for a in range(-w0, w0 + 1):
            for b in range(-w1, w1 + 1):
                if const_phot_ratio and t != 0 and a == 0 and b == 0:
                    continue
                out.append(("k", ij, (a, b)))
    for pq in monomials(db):
        out.append(("b", pq))
    return out


def weighted(R, i, j):
    n0, n1 = R.shape
    return np.outer(coords(n0) ** i, coords(n1) ** j) * R


def design_matrix(R, w0, w1, dk, db, const_phot_ratio):
    n0, n1 = R.shape
    cols = []
    for u in unknown_list(w0, w1, dk, db, const_phot_ratio):
        if u[0] == "k":
            (i, j), (a, b) = u[1], u[2]
            g = weighted(R, i, j)
            if a == 0 and b == 0:
                cols.append(g.ravel())
            else:
                # (g o K_ab)(x, y) = g(x - a, y - b) - g(x, y), circular
                shifted = np.roll(np.roll(g, a, axis=0), b, axis=1)
                cols.append((shifted - g).ravel())
        else:
            p, q = u[1]
            cols.append(np.outer(coords(n0) ** p, coords(n1) ** q).ravel())
    return np.stack(cols, axis=1)


def normal_equations(R, S, w0, w1, dk, db, const_phot_ratio, mask=None):
    if mask is not None:
        keep = (np.asarray(mask) != 0).astype(np.float64)
        R = R * keep
        S = S * keep
    C = design_matrix(np.asarray(R, np.float64), w0, w1, dk, db, const_phot_ratio)
    s = np.asarray(S, np.float64).ravel()
    return C.T @ C, C.T @ s


def least_squares(R, S, w0, w1, dk, db, const_phot_ratio, mask=None):
    """Coefficients minimising sum D^2 over the (masked) pair, by lstsq."""
    if mask is not None:
        keep = (np.asarray(mask) != 0).astype(np.float64)
        Rm, Sm = R * keep, S * keep
    else:
        Rm, Sm = R, S
    C = design_matrix(np.asarray(Rm, np.float64), w0, w1, dk, db, const_phot_ratio)
    theta, *_ = np.linalg.lstsq(C, np.asarray(Sm, np.float64).ravel(), rcond=None)
    return theta


def difference(R, S, theta, w0, w1, dk, db, const_phot_ratio):
    """D = S - C theta on the unmasked pair (Eq. 12)."""
    C = design_matrix(np.asarray(R, np.float64), w0, w1, dk, db, const_phot_ratio)
    return (np.asarray(S, np.float64).ravel() - C @ theta).reshape(R.shape)
