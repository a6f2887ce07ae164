"""ctypes binding of the plain-C FP64 oracle (``sfft_oracle.c``).

Test infrastructure only.  See the package docstring for what may import it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfft_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def library_path() -> str:
    return _LIB


def compile_oracle(force: bool = False) -> str:
    """Compile ``sfft_oracle.c`` with gcc (OpenMP if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        compile_oracle()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i = ctypes.c_int
        lib.orc_num_unknowns.argtypes = [ip]
        lib.orc_build_system.argtypes = [ip, dp, dp, u8p, dp, dp]
        lib.orc_system_entries.argtypes = [ip, dp, dp, u8p, i, ip, ip, dp]
        lib.orc_cholesky_solve.argtypes = [i, dp, dp, dp]
        lib.orc_subtract.argtypes = [ip, dp, dp, dp, dp]
        lib.orc_subtract_pixels.argtypes = [ip, dp, dp, dp, i, ctypes.POINTER(ctypes.c_longlong), dp]
        lib.orc_lag_sum.argtypes = [i, i, dp, dp, i, i]
        lib.orc_lag_sum.restype = ctypes.c_double
        lib.orc_decode_unknown.argtypes = [ip, i, ip]
        lib.orc_bspline.argtypes = [i, i, i, ctypes.c_double]
        lib.orc_bspline.restype = ctypes.c_double
        lib.orc_threads.argtypes = []
        _lib = lib
    return _lib


@dataclass(frozen=True)
class OracleConfig:
    """Fit parameters of one image pair (Sec. 3.3, Table A1).

    basis "poly": polynomial kernel and background variation of degrees dk,
    db (Eq. 2, 6).  basis "bspline": tensor-product B-splines (Eq. 8-9) of
    degree kdeg with kint interior knots for the kernel and bdeg, bint for
    the background (dk, db unused), on clamped uniform knots over the
    normalised coordinates."""
    n0: int
    n1: int
    w0: int
    w1: int
    dk: int
    db: int
    const_phot_ratio: bool
    basis: str = "poly"
    kdeg: int = 0
    kint: int = 0
    bdeg: int = 0
    bint: int = 0

    def args(self):
        """The 12-int configuration array of sfft_oracle.c."""
        v = (self.n0, self.n1, self.w0, self.w1, self.dk, self.db, int(self.const_phot_ratio),
             {"poly": 0, "bspline": 1}[self.basis], self.kdeg, self.kint, self.bdeg, self.bint)
        a = (ctypes.c_int * 12)(*v)
        return (a,)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _mask_ptr(mask):
    if mask is None:
        return None, ctypes.POINTER(ctypes.c_uint8)()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    return m, _ptr(m, ctypes.c_uint8)


def threads() -> int:
    return int(_load().orc_threads())


def num_unknowns(cfg: OracleConfig) -> int:
    return int(_load().orc_num_unknowns(*cfg.args()))


def bspline(deg: int, nint: int, i: int, u: float) -> float:
    """B-spline basis function i (degree deg, nint interior knots, clamped uniform on [-1, 1]) at u."""
    return float(_load().orc_bspline(deg, nint, i, float(u)))


def decode_unknown(cfg: OracleConfig, u: int):
    out = np.zeros(4, dtype=np.int32)
    rc = _load().orc_decode_unknown(*cfg.args(), u, _ptr(out, ctypes.c_int))
    if rc:
        raise ValueError(f"unknown index {u} out of range")
    return bool(out[0]), int(out[1]), int(out[2]), int(out[3])


def build_system(R, S, cfg: OracleConfig, mask=None):
    """Normal matrix M (n x n) and right-hand side (n) of Eq. 18, real-space units."""
    R, S = _f64(R), _f64(S)
    assert R.shape == (cfg.n0, cfg.n1) and S.shape == R.shape
    n = num_unknowns(cfg)
    M = np.zeros((n, n))
    rhs = np.zeros(n)
    keep, mp = _mask_ptr(mask)
    rc = _load().orc_build_system(*cfg.args(), _ptr(R), _ptr(S), mp, _ptr(M), _ptr(rhs))
    if rc:
        raise RuntimeError(f"oracle build failed: {rc}")
    return M, rhs


def system_entries(R, S, cfg: OracleConfig, rows, cols, mask=None):
    """Selected entries of M (cols >= 0) or of rhs (cols == -1), each by direct lag sums."""
    R, S = _f64(R), _f64(S)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.zeros(len(rows))
    keep, mp = _mask_ptr(mask)
    rc = _load().orc_system_entries(*cfg.args(), _ptr(R), _ptr(S), mp, len(rows),
                                    _ptr(rows, ctypes.c_int), _ptr(cols, ctypes.c_int), _ptr(out))
    if rc:
        raise RuntimeError(f"oracle entries failed: {rc}")
    return out


def cholesky_solve(M, rhs):
    """Solve M x = rhs by Cholesky; raises numpy.linalg.LinAlgError if M is not PD."""
    M, rhs = _f64(M), _f64(rhs)
    n = rhs.shape[0]
    x = np.zeros(n)
    rc = _load().orc_cholesky_solve(n, _ptr(M), _ptr(rhs), _ptr(x))
    if rc == -4:
        raise np.linalg.LinAlgError("matrix is not positive definite")
    if rc:
        raise RuntimeError(f"oracle solve failed: {rc}")
    return x


def subtract(R, S, x, cfg: OracleConfig):
    """Difference image of Eq. 12 (circular), from the unmasked R and S."""
    R, S, x = _f64(R), _f64(S), _f64(x)
    D = np.zeros_like(R)
    rc = _load().orc_subtract(*cfg.args(), _ptr(R), _ptr(S), _ptr(x), _ptr(D))
    if rc:
        raise RuntimeError(f"oracle subtract failed: {rc}")
    return D


def subtract_pixels(R, S, x, cfg: OracleConfig, flat_index):
    R, S, x = _f64(R), _f64(S), _f64(x)
    pix = np.ascontiguousarray(flat_index, dtype=np.int64)
    out = np.zeros(len(pix))
    rc = _load().orc_subtract_pixels(*cfg.args(), _ptr(R), _ptr(S), _ptr(x), len(pix),
                                     _ptr(pix, ctypes.c_longlong), _ptr(out))
    if rc:
        raise RuntimeError(f"oracle subtract failed: {rc}")
    return out


def lag_sum(f, g, r0: int, r1: int) -> float:
    """sum_x f(x) g((x + rho) mod N)."""
    f, g = _f64(f), _f64(g)
    return float(_load().orc_lag_sum(f.shape[0], f.shape[1], _ptr(f), _ptr(g), r0, r1))
