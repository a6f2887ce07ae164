"""Seeded synthetic image pairs shaped like the paper's workloads.

This module only *draws inputs*: star fields rendered with Gaussian PSFs, sky
levels and noise.  It holds none of the subtraction method's arithmetic, and
both the oracle tests and the GPU tests use it so that the two sides see the
same pixels.

Workloads (the paper's real data -- ZTF, DECam, TMTS -- are not available;
these stand in for them with matching sizes and fit parameters, Sec. 4-5 and
Table A1 defaults):

``pair256``   256 x 256 float64: 200 sources, log-uniform flux 1e2-1e5,
              circular Gaussian PSF FWHM 2.5 (reference) / 3.5 (science),
              sky 100, Gaussian noise sigma 5.  Fit: w=4, D_K=0, D_B=0,
              constant photometric ratio (82 unknowns).
``pair1024``  1024 x 1024 float32: 2000 sources, log-uniform flux; science
              FWHM 3.0 -> 4.0 linear in x, reference 2.5; science sky
              100 + 0.01 x + 0.02 y (pixels), reference sky 100; photometric
              scale 1.0 -> 1.1 linear in y; Poisson (gain 1) + read noise 5.
              Fit: w=6, D_K=1, D_B=1, varying photometric ratio (510 unknowns).
``pair4096``  4096 x 4096 float32 wide field: 20000 sources with cumulative
              counts N(>F) ~ F^-1.5 on [1e2, 1e5]; elliptical Gaussian PSFs,
              reference FWHM 2.5 -> 3.0, science 3.5 -> 4.5, ellipticity
              0 -> 0.2 (position angle 30 deg), all quadratic over the field;
              science sky 100 + 20 xt^2 + 10 yt^2 + 5 xt yt, reference sky 100;
              50 transients (flux 1e3-1e4) on the science image only;
              Poisson + read noise 5.  Fit: w=8, D_K=2, D_B=2, constant
              photometric ratio (1735 unknowns).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from math import log, sqrt

import numpy as np

FWHM_TO_SIGMA = 1.0 / (2.0 * sqrt(2.0 * log(2.0)))


@dataclass(frozen=True)
class FitParams:
    w0: int
    w1: int
    dk: int
    db: int
    const_phot_ratio: bool


@dataclass(frozen=True)
class PairSpec:
    name: str
    n0: int
    n1: int
    dtype: str                      # "float32" | "float64"
    n_src: int
    flux: tuple = (1e2, 1e5)
    flux_law: str = "loguniform"    # "loguniform" | "powerlaw15"
    fwhm_ref: tuple = (2.5, 2.5)    # (centre, edge) -- quadratic in radius, or linear (see vary)
    fwhm_sci: tuple = (3.5, 3.5)
    vary: str = "none"              # "none" | "linear_x" | "quadratic"
    ellip: tuple = (0.0, 0.0)
    pa_deg: float = 30.0
    sky_ref: str = "flat"
    sky_sci: str = "flat"           # "flat" | "plane" | "quadratic"
    scale_y: tuple = (1.0, 1.0)     # photometric scale of S relative to R, linear in y
    noise: str = "gauss"            # "gauss" | "poisson"
    sigma: float = 5.0
    n_transients: int = 0
    fit: FitParams = field(default_factory=lambda: FitParams(4, 4, 0, 0, True))


PAIR256 = PairSpec("pair256", 256, 256, "float64", 200, fit=FitParams(4, 4, 0, 0, True))
PAIR1024 = PairSpec("pair1024", 1024, 1024, "float32", 2000, fwhm_ref=(2.5, 2.5),
                    fwhm_sci=(3.0, 4.0), vary="linear_x", sky_sci="plane", scale_y=(1.0, 1.1),
                    noise="poisson", fit=FitParams(6, 6, 1, 1, False))
PAIR4096 = PairSpec("pair4096", 4096, 4096, "float32", 20000, flux_law="powerlaw15",
                    fwhm_ref=(2.5, 3.0), fwhm_sci=(3.5, 4.5), vary="quadratic",
                    ellip=(0.0, 0.2), sky_sci="quadratic", noise="poisson", n_transients=50,
                    fit=FitParams(8, 8, 2, 2, True))

SPECS = {s.name: s for s in (PAIR256, PAIR1024, PAIR4096)}


def sector(n: int, fit: FitParams, name: str | None = None) -> PairSpec:
    """One sector of the variable-size workloads: an n x n float32 pair with
    the PSF, sky and noise family of the 4096^2 pair, one source per 500 px^2."""
    return replace(PAIR4096, name=name or f"sector{n}", n0=n, n1=n, n_src=max(1, (n * n) // 500),
                   n_transients=max(1, (50 * n * n) // (4096 * 4096)), fit=fit)


def draw_sectors(count: int, seed: int, n_range=(512, 2048)):
    """Sector specs with n uniform over the integers of n_range and w in 4..8,
    D_K and D_B in 0..2 drawn per sector (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        w = int(rng.integers(4, 9))
        fit = FitParams(w, w, int(rng.integers(0, 3)), int(rng.integers(0, 3)), True)
        out.append(sector(n, fit, name=f"sector{k}:{n}"))
    return out


def scaled(spec: PairSpec, n0: int, n1: int | None = None, name: str | None = None) -> PairSpec:
    """Same structure at another size, keeping the source density."""
    n1 = n0 if n1 is None else n1
    dens = spec.n_src / float(spec.n0 * spec.n1)
    return replace(spec, name=name or f"{spec.name}@{n0}x{n1}", n0=n0, n1=n1,
                   n_src=max(1, int(round(dens * n0 * n1))))


def _norm_coord(v, n):
    return (2.0 * v - (n - 1)) / max(n - 1, 1)


def _field_value(rng_pair, xt, yt, vary):
    lo, hi = rng_pair
    if vary == "none":
        return np.full_like(xt, lo)
    if vary == "linear_x":
        return lo + (hi - lo) * (xt + 1.0) / 2.0
    # quadratic: grows with squared radius from the field centre, edge value at |r|=sqrt(2)
    r2 = (xt * xt + yt * yt) / 2.0
    return lo + (hi - lo) * r2


def _draw_flux(rng, n, spec):
    lo, hi = spec.flux
    if spec.flux_law == "powerlaw15":
        # cumulative N(>F) proportional to F^-1.5 on [lo, hi]: inverse-CDF sampling
        u = rng.random(n)
        a = 1.5
        return (lo ** -a - u * (lo ** -a - hi ** -a)) ** (-1.0 / a)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def _render(img, xs, ys, fluxes, fwhm, ellip, pa_deg, half):
    """Add Gaussian sources (3x3 sub-pixel sampling per pixel) into img."""
    n0, n1 = img.shape
    sub = (np.arange(3) - 1.0) / 3.0
    su, sv = np.meshgrid(sub, sub, indexing="ij")
    su, sv = su.ravel(), sv.ravel()
    pa = np.deg2rad(pa_deg)
    ca, sa = np.cos(pa), np.sin(pa)
    off = np.arange(-half, half + 1)
    for k in range(len(xs)):
        x, y, f = xs[k], ys[k], fluxes[k]
        s = fwhm[k] * FWHM_TO_SIGMA
        e = ellip[k]
        sa2 = s * s / (1.0 - e) if e > 0 else s * s
        sb2 = s * s * (1.0 - e) if e > 0 else s * s
        # covariance rotated by the position angle
        cxx = ca * ca * sa2 + sa * sa * sb2
        cyy = sa * sa * sa2 + ca * ca * sb2
        cxy = ca * sa * (sa2 - sb2)
        det = cxx * cyy - cxy * cxy
        ixx, iyy, ixy = cyy / det, cxx / det, -cxy / det
        ix, iy = int(np.floor(x)), int(np.floor(y))
        px = ix + off
        py = iy + off
        vx = px[(px >= 0) & (px < n0)]
        vy = py[(py >= 0) & (py < n1)]
        if len(vx) == 0 or len(vy) == 0:
            continue
        dx = (vx[:, None, None] + su[None, None, :]) - x          # (nx, 1, 9)
        dy = (vy[None, :, None] + sv[None, None, :]) - y          # (1, ny, 9)
        q = ixx * dx * dx + iyy * dy * dy + 2.0 * ixy * dx * dy
        val = np.exp(-0.5 * q).mean(axis=2) / (2.0 * np.pi * np.sqrt(det))
        img[np.ix_(vx, vy)] += f * val


def _sky(kind, n0, n1):
    x = np.arange(n0, dtype=np.float64)[:, None]
    y = np.arange(n1, dtype=np.float64)[None, :]
    if kind == "flat":
        return np.full((n0, n1), 100.0)
    if kind == "plane":
        return 100.0 + 0.01 * x + 0.02 * y
    xt = _norm_coord(x, n0)
    yt = _norm_coord(y, n1)
    return 100.0 + 20.0 * xt * xt + 10.0 * yt * yt + 5.0 * xt * yt


def make_pair(spec: PairSpec, seed: int = 0, return_transients: bool = False):
    """Return (R, S) as C-contiguous arrays of spec.dtype; with
    return_transients also the (x, y) positions of the transients injected
    into S (empty arrays when the spec has none)."""
    rng = np.random.default_rng(seed)
    n0, n1 = spec.n0, spec.n1
    xs = rng.uniform(0, n0, spec.n_src)
    ys = rng.uniform(0, n1, spec.n_src)
    flux = _draw_flux(rng, spec.n_src, spec)
    xt, yt = _norm_coord(xs, n0), _norm_coord(ys, n1)
    fr = _field_value(spec.fwhm_ref, xt, yt, spec.vary)
    fs = _field_value(spec.fwhm_sci, xt, yt, spec.vary)
    el = _field_value(spec.ellip, xt, yt, "none" if spec.vary == "linear_x" else spec.vary)
    if spec.vary == "none":
        el = np.full_like(xt, spec.ellip[0])
    scale = spec.scale_y[0] + (spec.scale_y[1] - spec.scale_y[0]) * ys / max(n1 - 1, 1)
    half = int(np.ceil(3.0 * max(spec.fwhm_ref[1], spec.fwhm_sci[1]))) + 1

    R = _sky(spec.sky_ref, n0, n1)
    S = _sky(spec.sky_sci, n0, n1)
    _render(R, xs, ys, flux, fr, el, spec.pa_deg, half)
    _render(S, xs, ys, flux * scale, fs, el, spec.pa_deg, half)
    tx = ty = np.zeros(0)
    if spec.n_transients:
        tx = rng.uniform(0, n0, spec.n_transients)
        ty = rng.uniform(0, n1, spec.n_transients)
        tf = rng.uniform(1e3, 1e4, spec.n_transients)
        txt, tyt = _norm_coord(tx, n0), _norm_coord(ty, n1)
        _render(S, tx, ty, tf, _field_value(spec.fwhm_sci, txt, tyt, spec.vary),
                _field_value(spec.ellip, txt, tyt, spec.vary), spec.pa_deg, half)
    if spec.noise == "poisson":
        R = rng.poisson(np.clip(R, 0, None)).astype(np.float64) + rng.normal(0, spec.sigma, R.shape)
        S = rng.poisson(np.clip(S, 0, None)).astype(np.float64) + rng.normal(0, spec.sigma, S.shape)
    else:
        R = R + rng.normal(0, spec.sigma, R.shape)
        S = S + rng.normal(0, spec.sigma, S.shape)
    dt = np.dtype(spec.dtype)
    R, S = np.ascontiguousarray(R, dtype=dt), np.ascontiguousarray(S, dtype=dt)
    if return_transients:
        return R, S, (tx, ty)
    return R, S


def transient_mask(shape, positions, half: int):
    """uint8 mask of an image of `shape`: 0 on the square of half-width
    `half` around each (x, y) position (clipped at the edges), 1 elsewhere.
    The masked squares are where a caller hides known variable sources from
    the fit (the build sees zeros there; the subtraction is unmasked)."""
    n0, n1 = shape
    mask = np.ones((n0, n1), dtype=np.uint8)
    for x, y in zip(*positions):
        xi, yi = int(np.floor(x)), int(np.floor(y))
        mask[max(0, xi - half):min(n0, xi + half + 1), max(0, yi - half):min(n1, yi + half + 1)] = 0
    return mask


def random_field(n0, n1, seed, n_src=None, sky=100.0, sigma=5.0, fwhm=2.0):
    """Small well-conditioned reference image: sources on white noise."""
    rng = np.random.default_rng(seed)
    n_src = max(2, (n0 * n1) // 40) if n_src is None else n_src
    img = np.full((n0, n1), sky)
    xs = rng.uniform(0, n0, n_src)
    ys = rng.uniform(0, n1, n_src)
    fl = np.exp(rng.uniform(np.log(1e2), np.log(1e4), n_src))
    _render(img, xs, ys, fl, np.full(n_src, fwhm), np.zeros(n_src), 0.0, int(3 * fwhm) + 1)
    return img + rng.normal(0, sigma, img.shape)


def coefficient_draw(n, seed, scale=0.05):
    """Random coefficient vector (used to inject a known kernel)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, n)
