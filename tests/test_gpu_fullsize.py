"""Parity at full sizes, on sampled outputs the oracle computes one by one.

Sizes: the 4096^2 wide-field pair (the bench workload, w = 8, D_K = D_B = 2,
1735 unknowns), and three sizes that are not powers of two, in the range of
the variable-size sector (N in [512, 2048]) and stream (N in [1024, 4096])
workloads.  All on the mixed path with float32 images, as the bench runs.

Checks (float32-rounded inputs on both sides):
  * M: 400 sampled entries (the diagonal included) and rhs: 150 sampled
    entries, each a direct lag sum over the whole image in the oracle.  The
    relative Frobenius error estimated from the sample (RMS of the entry
    errors over RMS of the entries) <= 1e-5; no single entry off by more than
    1e-4 of sqrt(M_ii M_jj) (1e-4 of the RMS rhs entry for rhs);
  * the solver: ||x - solve(M, rhs)|| / ||x|| <= 1e-8 against an FP64 solve of
    the GPU-built system;
  * D at 2000 sampled pixels against the oracle's circular subtraction with
    the GPU's coefficients: RMS deviation <= 1e-3 sigma.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("pair4096", None),
    ("sector1537x1999", (1537, 1999, synth.FitParams(7, 7, 2, 1, True))),
    ("sector3001x2048", (3001, 2048, synth.FitParams(8, 8, 1, 2, False))),
    ("sector2048x1283", (2048, 1283, synth.FitParams(5, 5, 2, 2, True))),
]


def spec_of(name, shape):
    if shape is None:
        return synth.PAIR4096
    n0, n1, fit = shape
    from dataclasses import replace
    return replace(synth.scaled(synth.PAIR4096, n0, n1, name=name), fit=fit)


@pytest.mark.parametrize("name,shape", CASES, ids=[c[0] for c in CASES])
def test_sampled_parity(name, shape):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, info_from_bytes
    from paper_2109_09334_gb300.build import build
    build()
    spec = spec_of(name, shape)
    f = spec.fit
    R, S = synth.make_pair(spec, seed=5)
    R32 = R.astype(np.float32)
    S32 = S.astype(np.float32)
    plan = SfftPlan(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype="float32",
                    precision="mixed")
    D, x, info, M, rhs = plan.run_pair(torch.from_numpy(R32).cuda(), torch.from_numpy(S32).cuda(),
                                       keep_system=True)
    torch.cuda.synchronize()
    M, rhs, x, D = M.cpu().numpy(), rhs.cpu().numpy(), x.cpu().numpy(), D.cpu().numpy().astype(np.float64)
    inf = info_from_bytes(info.cpu().numpy())
    assert inf["status"] == 0, inf
    n = rhs.shape[0]
    c = oracle.OracleConfig(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio)
    rng = np.random.default_rng(11)
    rows = np.concatenate([rng.integers(0, n, 300), np.arange(0, n, max(1, n // 100))[:100]])
    cols = np.concatenate([rng.integers(0, n, 300), np.arange(0, n, max(1, n // 100))[:100]])
    Me = oracle.system_entries(R32, S32, c, rows, cols)
    Mg = M[rows, cols]
    d = np.sqrt(np.abs(np.diag(M)))
    assert np.sqrt(np.mean((Mg - Me) ** 2)) <= 1e-5 * np.sqrt(np.mean(Me ** 2))
    assert np.max(np.abs(Mg - Me) / (d[rows] * d[cols])) <= 1e-4
    rr = rng.integers(0, n, 150)
    re = oracle.system_entries(R32, S32, c, rr, -np.ones_like(rr))
    assert np.sqrt(np.mean((rhs[rr] - re) ** 2)) <= 1e-5 * np.sqrt(np.mean(re ** 2))
    assert np.max(np.abs(rhs[rr] - re)) <= 1e-4 * np.sqrt(np.mean(re ** 2))
    xs = np.linalg.solve(M, rhs)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    pix = rng.integers(0, spec.n0 * spec.n1, 2000)
    De = oracle.subtract_pixels(R32, S32, x, c, pix)
    assert np.sqrt(np.mean((D.ravel()[pix] - De) ** 2)) <= 1e-3 * spec.sigma
    plan.close()


def test_fp64_path_sampled_parity_4096():
    """The plain FP64 GPU path (FP64 FFTs, products, sums and Cholesky) on the
    4096^2 pair: sampled M and rhs within 1e-10 (relative, RMS over the
    sample), the solution within 1e-8 of an FP64 solve of the GPU-built
    system, and D within 1e-6 sigma RMS at sampled pixels."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, info_from_bytes
    from paper_2109_09334_gb300.build import build
    build()
    spec = synth.PAIR4096
    f = spec.fit
    R, S = synth.make_pair(spec, seed=5)
    R32, S32 = R.astype(np.float32), S.astype(np.float32)
    plan = SfftPlan(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype="float32",
                    precision="fp64")
    D, x, info, M, rhs = plan.run_pair(torch.from_numpy(R32).cuda(), torch.from_numpy(S32).cuda(),
                                       keep_system=True)
    torch.cuda.synchronize()
    M, rhs, x, D = M.cpu().numpy(), rhs.cpu().numpy(), x.cpu().numpy(), D.cpu().numpy().astype(np.float64)
    assert info_from_bytes(info.cpu().numpy())["status"] == 0
    n = rhs.shape[0]
    c = oracle.OracleConfig(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio)
    rng = np.random.default_rng(13)
    rows, cols = rng.integers(0, n, 200), rng.integers(0, n, 200)
    Me = oracle.system_entries(R32, S32, c, rows, cols)
    assert np.sqrt(np.mean((M[rows, cols] - Me) ** 2)) <= 1e-10 * np.sqrt(np.mean(Me ** 2))
    rr = rng.integers(0, n, 100)
    re = oracle.system_entries(R32, S32, c, rr, -np.ones_like(rr))
    assert np.sqrt(np.mean((rhs[rr] - re) ** 2)) <= 1e-10 * np.sqrt(np.mean(re ** 2))
    xs = np.linalg.solve(M, rhs)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    pix = rng.integers(0, spec.n0 * spec.n1, 2000)
    De = oracle.subtract_pixels(R32, S32, x, c, pix)
    # D is written as float32 (the image type): compare within its rounding too
    assert np.sqrt(np.mean((D.ravel()[pix] - De) ** 2)) <= 1e-6 * spec.sigma + 1e-7 * np.sqrt(np.mean(De ** 2))
    plan.close()


# The 4096^2 pair with tensor-product B-splines (Eq. 7-9): piecewise-linear
# kernel variation with one interior knot (K = 3), quadratic background with
# one interior knot (K' = 4), w = 8, constant ratio: 2609 unknowns.
BSPLINE_4096 = (1, 1, 2, 1)


def test_bspline_sampled_parity_4096():
    """Mixed path, B-spline basis, 4096^2: the sampled checks of test_sampled_parity."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, info_from_bytes
    from paper_2109_09334_gb300.build import build
    build()
    spec = synth.PAIR4096
    f = spec.fit
    R, S = synth.make_pair(spec, seed=6)
    R32, S32 = R.astype(np.float32), S.astype(np.float32)
    plan = SfftPlan(spec.n0, spec.n1, f.w0, f.w1, 0, 0, True, dtype="float32", precision="mixed",
                    spline=BSPLINE_4096)
    D, x, info, M, rhs = plan.run_pair(torch.from_numpy(R32).cuda(), torch.from_numpy(S32).cuda(),
                                       keep_system=True)
    torch.cuda.synchronize()
    M, rhs, x, D = M.cpu().numpy(), rhs.cpu().numpy(), x.cpu().numpy(), D.cpu().numpy().astype(np.float64)
    inf = info_from_bytes(info.cpu().numpy())
    assert inf["status"] == 0, inf
    n = rhs.shape[0]
    c = oracle.OracleConfig(spec.n0, spec.n1, f.w0, f.w1, 0, 0, True, "bspline", *BSPLINE_4096)
    assert n == oracle.num_unknowns(c) == 2609
    rng = np.random.default_rng(17)
    rows = np.concatenate([rng.integers(0, n, 300), np.arange(0, n, max(1, n // 100))[:100]])
    cols = np.concatenate([rng.integers(0, n, 300), np.arange(0, n, max(1, n // 100))[:100]])
    Me = oracle.system_entries(R32, S32, c, rows, cols)
    Mg = M[rows, cols]
    d = np.sqrt(np.abs(np.diag(M)))
    assert np.sqrt(np.mean((Mg - Me) ** 2)) <= 1e-5 * np.sqrt(np.mean(Me ** 2))
    assert np.max(np.abs(Mg - Me) / (d[rows] * d[cols])) <= 1e-4
    rr = rng.integers(0, n, 150)
    re = oracle.system_entries(R32, S32, c, rr, -np.ones_like(rr))
    assert np.sqrt(np.mean((rhs[rr] - re) ** 2)) <= 1e-5 * np.sqrt(np.mean(re ** 2))
    assert np.max(np.abs(rhs[rr] - re)) <= 1e-4 * np.sqrt(np.mean(re ** 2))
    xs = np.linalg.solve(M, rhs)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    pix = rng.integers(0, spec.n0 * spec.n1, 2000)
    De = oracle.subtract_pixels(R32, S32, x, c, pix)
    assert np.sqrt(np.mean((D.ravel()[pix] - De) ** 2)) <= 1e-3 * spec.sigma
    plan.close()
