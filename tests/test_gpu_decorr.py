"""Noise decorrelation (App. C, Eq. 21-24) on the GPU against the oracle.

Both sides start from the GPU's coefficients and difference image, so the
check is of the decorrelation alone: the kernel image at (xt0, yt0), the
filter of Eq. 24 normalised to unit sum, and the circular convolution.
Tolerance: RMS deviation <= 1e-10 (FP64 path) or 1e-5 (mixed path) of the
RMS of the difference image.
"""
import ctypes

import numpy as np
import pytest

from oracle import decorr
from synth import random_field

torch = pytest.importorskip("torch")


def test_rejects_bad_arguments():
    from paper_2109_09334_gb300 import binding as B
    from paper_2109_09334_gb300.build import build
    build()
    lib = B.library()
    fake = 4096  # never dereferenced: every call below is rejected first
    assert lib.sfft_decorrelate(None, fake, 0.0, 0.0, 1.0, 1.0, fake, fake, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_decorrelate(fake, fake, 0.0, 0.0, 1.0, 0.0, fake, fake, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_decorrelate(fake, fake, 0.0, 0.0, -1.0, 1.0, fake, fake, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_decorrelate(fake, fake, 1.5, 0.0, 1.0, 1.0, fake, fake, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_decorrelate(fake, None, 0.0, 0.0, 1.0, 1.0, fake, fake, None) == B.SFFT_ERR_INVALID


def test_coadd_rejects_bad_arguments():
    from paper_2109_09334_gb300 import binding as B
    from paper_2109_09334_gb300.build import build
    build()
    lib = B.library()
    fake = 4096  # never dereferenced: every call below is rejected first
    s1 = (ctypes.c_double * 1)(2.0)
    s0 = (ctypes.c_double * 1)(0.0)
    sneg = (ctypes.c_double * 1)(-1.0)
    call = lib.sfft_decorrelate_coadd
    assert call(None, fake, 0.0, 0.0, 1, fake, s1, 1, fake, s1, 1, 1, fake, fake, None) == B.SFFT_ERR_INVALID
    assert call(fake, fake, 0.0, 0.0, 0, fake, s1, 1, fake, s1, 1, 1, fake, fake, None) == B.SFFT_ERR_INVALID
    assert call(fake, fake, 0.0, 0.0, 17, fake, s1, 1, fake, s1, 1, 1, fake, fake, None) == B.SFFT_ERR_INVALID
    assert call(fake, fake, 0.0, 0.0, 1, None, s1, 1, fake, s1, 1, 1, fake, fake, None) == B.SFFT_ERR_INVALID
    assert call(fake, fake, 2.0, 0.0, 1, fake, s1, 1, fake, s1, 1, 1, fake, fake, None) == B.SFFT_ERR_INVALID
    assert call(fake, fake, 0.0, 0.0, 1, fake, None, 1, fake, s1, 1, 1, fake, fake, None) == B.SFFT_ERR_INVALID


CASES = [
    # n0, n1, w0, w1, dk, db, cpr
    (64, 64, 2, 2, 1, 1, 1),
    (48, 40, 2, 2, 1, 1, 0),
    (64, 48, 2, 3, 2, 1, 1),
    (40, 64, 3, 2, 0, 2, 1),
    (128, 96, 4, 4, 2, 2, 1),
]


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_decorrelation_matches_oracle(case, precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan
    n0, n1, w0, w1, dk, db, cpr = case
    R = random_field(n0, n1, n0 + w0)
    S = 0.9 * np.roll(R, (1, -1), axis=(0, 1)) + 0.3 * random_field(n0, n1, n1 + 5)
    dtype = "float64" if precision == "fp64" else "float32"
    tdt = torch.float64 if precision == "fp64" else torch.float32
    plan = SfftPlan(n0, n1, w0, w1, dk, db, cpr, dtype=dtype, precision=precision)
    D, x, info, _, _ = plan.run_pair(torch.from_numpy(R).to("cuda", tdt), torch.from_numpy(S).to("cuda", tdt))
    xt0, yt0, sr, ss = 0.25, -0.4, 5.0, 7.0
    out = plan.decorrelate(x, D, sr, ss, xt0, yt0)
    inplace = D.clone()
    plan.decorrelate(x, inplace, sr, ss, xt0, yt0, out=inplace)
    torch.cuda.synchronize()
    xd, Dd, od = x.cpu().numpy(), D.double().cpu().numpy(), out.double().cpu().numpy()
    k = decorr.kernel_image(xd, w0, w1, dk, db, bool(cpr), xt0, yt0)
    ref = decorr.decorrelate(Dd, k, sr, ss)
    tol = (1e-10 if precision == "fp64" else 1e-5) * np.sqrt(np.mean(Dd ** 2))
    assert np.sqrt(np.mean((od - ref) ** 2)) <= tol
    assert np.array_equal(inplace.cpu().numpy(), out.cpu().numpy())
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("cpr", [0, 1])
def test_bspline_decorrelation_matches_oracle(cpr):
    """The kernel of Eq. 8 at (xt0, yt0) (B-spline weights) in the filter of Eq. 24."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan
    n0, n1, w0, w1 = 64, 48, 2, 2
    spline = (2, 1, 1, 0)
    R = random_field(n0, n1, 77)
    S = 0.9 * np.roll(R, (1, -1), axis=(0, 1)) + 0.3 * random_field(n0, n1, 78)
    plan = SfftPlan(n0, n1, w0, w1, 0, 0, cpr, dtype="float64", precision="fp64", spline=spline)
    D, x, info, _, _ = plan.run_pair(torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda())
    xt0, yt0, sr, ss = -0.3, 0.55, 5.0, 7.0
    out = plan.decorrelate(x, D, sr, ss, xt0, yt0)
    torch.cuda.synchronize()
    xd, Dd, od = x.cpu().numpy(), D.cpu().numpy(), out.cpu().numpy()
    k = decorr.kernel_image(xd, w0, w1, 0, 0, bool(cpr), xt0, yt0, spline=spline)
    ref = decorr.decorrelate(Dd, k, sr, ss)
    assert np.sqrt(np.mean((od - ref) ** 2)) <= 1e-10 * np.sqrt(np.mean(Dd ** 2))
    plan.close()


def _blur(rng, w0, w1, spread):
    k = np.abs(rng.standard_normal((2 * w0 + 1, 2 * w1 + 1))) * spread
    k[w0, w1] += 1.0
    return k / k.sum()


@pytest.mark.gpu
@pytest.mark.parametrize("shape,nsci,nref,g", [((64, 64), 3, 2, (1, 2)), ((48, 40), 1, 4, (2, 1)),
                                               ((40, 64), 2, 2, (0, 0))])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coadd_decorrelation_matches_oracle(shape, nsci, nref, g, precision):
    """Eq. 21-24 in full (co-added science and reference images with their
    homogenisation kernels) against the oracle's filter, same tolerances."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan
    n0, n1 = shape
    w0, w1, dk, db, cpr = 2, 2, 1, 1, 1
    rng = np.random.default_rng(n0 + nsci)
    R = random_field(n0, n1, n0 + 1)
    S = 0.9 * np.roll(R, (1, -1), axis=(0, 1)) + 0.3 * random_field(n0, n1, n1 + 2)
    dtype = "float64" if precision == "fp64" else "float32"
    tdt = torch.float64 if precision == "fp64" else torch.float32
    plan = SfftPlan(n0, n1, w0, w1, dk, db, cpr, dtype=dtype, precision=precision)
    D, x, info, _, _ = plan.run_pair(torch.from_numpy(R).to("cuda", tdt), torch.from_numpy(S).to("cuda", tdt))
    G = [_blur(rng, g[0], g[1], 0.4) / nsci for _ in range(nsci)]
    H = [_blur(rng, g[0], g[1], 0.4) / nref for _ in range(nref)]
    ss = list(rng.uniform(1.0, 4.0, nsci))
    sr = list(rng.uniform(1.0, 4.0, nref))
    xt0, yt0 = 0.1, -0.6
    out = plan.decorrelate_coadd(x, D, torch.from_numpy(np.stack(G)).cuda(), ss, torch.from_numpy(np.stack(H)).cuda(),
                                 sr, xt0, yt0)
    torch.cuda.synchronize()
    xd, Dd, od = x.cpu().numpy(), D.double().cpu().numpy(), out.double().cpu().numpy()
    k = decorr.kernel_image(xd, w0, w1, dk, db, bool(cpr), xt0, yt0)
    ref = decorr.decorrelate_coadd(Dd, k, ss, G, sr, H)
    tol = (1e-10 if precision == "fp64" else 1e-5) * np.sqrt(np.mean(Dd ** 2))
    assert np.sqrt(np.mean((od - ref) ** 2)) <= tol
    plan.close()
