"""Frequency-domain tier of the oracle: Eq. 19-24 evaluated literally.

Test infrastructure only.

Every block entry is the frequency sum of a spectrum product exactly as
printed in Eq. 19-24, with the basis spectra of Eq. 14 (including their
1/(N0 N1) factor) and W = exp(-2 pi i / N).  numpy's FFT is the DFT primitive.
This form shares nothing with the real-space lag sums of ``sfft_oracle.c``,
so agreement between the two (after the uniform rescaling ``a = N0 N1 a-ring``
of Eq. 13) pins the reading of App. B independently.  Tiny images only: it
materialises one full spectrum per unknown.
"""
from __future__ import annotations

import numpy as np

from .bruteforce import coords, monomials, unknown_list


def basis_spectrum(n0, n1, a, b):
    """K-hat_ab(l, m) of Eq. 14."""
    P = n0 * n1
    if a == 0 and b == 0:
        return np.full((n0, n1), 1.0 / P, dtype=np.complex128)
    l = np.arange(n0)[:, None]
    m = np.arange(n1)[None, :]
    Wl = np.exp(-2j * np.pi * l * a / n0)
    Wm = np.exp(-2j * np.pi * m * b / n1)
    return (Wl * Wm - 1.0) / P


def paper_system(R, S, w0, w1, dk, db, const_phot_ratio):
    """[A B; B~ C] and [D; E] of Eq. 18-24, in the paper's units (unknowns a = P a-ring, b)."""
    R = np.asarray(R, np.float64)
    S = np.asarray(S, np.float64)
    n0, n1 = R.shape
    cx, cy = coords(n0), coords(n1)
    Rhat = {ij: np.fft.fft2(np.outer(cx ** ij[0], cy ** ij[1]) * R) for ij in monomials(dk)}
    That = {pq: np.fft.fft2(np.outer(cx ** pq[0], cy ** pq[1])) for pq in monomials(db)}
    Shat = np.fft.fft2(S)
    unk = unknown_list(w0, w1, dk, db, const_phot_ratio)
    X = []
    for u in unk:
        if u[0] == "k":
            X.append(("k", Rhat[u[1]] * basis_spectrum(n0, n1, *u[2])))
        else:
            X.append(("b", That[u[1]]))
    n = len(unk)
    M = np.zeros((n, n))
    rhs = np.zeros(n)
    for r, (kr, xr) in enumerate(X):
        for c, (kc, xc) in enumerate(X):
            # Eq. 19 (A), 20 (B), 21 (B~), 22 (C): sum_lm Re[X_r conj(X_c)]
            M[r, c] = np.sum((xr * np.conj(xc)).real)
        # Eq. 23 (D), 24 (E): sum_lm Re[conj(S-hat) X_r]
        rhs[r] = np.sum((np.conj(Shat) * xr).real)
    return M, rhs


def to_real_space_units(M_paper, rhs_paper, n0, n1, n_kernel):
    """Map the paper's system to real-space units.

    With a = P a-ring (Eq. 13), Parseval gives M_paper = D1 M_real D2 and
    rhs_paper = P D1 rhs_real, where D1 = diag(1/P on kernel rows, 1 on
    background rows) and D2 = diag(1 on kernel columns, P on background
    columns).  Returns (M_real, rhs_real).
    """
    P = float(n0 * n1)
    n = M_paper.shape[0]
    d1 = np.ones(n)
    d1[:n_kernel] = 1.0 / P
    d2 = np.ones(n)
    d2[n_kernel:] = P
    M_real = M_paper / d1[:, None] / d2[None, :]
    rhs_real = rhs_paper / d1 / P
    return M_real, rhs_real
