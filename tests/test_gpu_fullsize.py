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
  * D at 2000 random pixels plus pixels on the wrap seams (every row and
    column within w of an edge, sampled along it, and the four w x w corner
    blocks in full, where the circular index arithmetic of the stencil and
    of Lambda's wrapping rows and columns lives) against the oracle's
    circular subtraction with the GPU's coefficients: RMS deviation
    <= 1e-3 sigma over each set, and no pixel off by more than 1e-3 sigma.

The transient-masked case runs the two-step process of Sec. 3 at 4096^2:
the system is built on the pair with squares around the 50 injected
transients zeroed (mask argument), the subtraction uses the unmasked pair;
the same request through the serving path gives the same bits.
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


def seam_pixels(n0, n1, w0, w1, rng, per_edge=150):
    """Flat indices of pixels near the wrap seams: rows x < w0 and
    x >= n0 - w0 (random y), columns y < w1 and y >= n1 - w1 (random x), and
    the four corner blocks of w0 x w1 pixels in full."""
    ws0, ws1 = max(w0, 1), max(w1, 1)
    xs = [rng.integers(0, ws0, per_edge), n0 - 1 - rng.integers(0, ws0, per_edge),
          rng.integers(0, n0, per_edge), rng.integers(0, n0, per_edge)]
    ys = [rng.integers(0, n1, per_edge), rng.integers(0, n1, per_edge),
          rng.integers(0, ws1, per_edge), n1 - 1 - rng.integers(0, ws1, per_edge)]
    cx = np.r_[np.arange(ws0), np.arange(n0 - ws0, n0)]
    cy = np.r_[np.arange(ws1), np.arange(n1 - ws1, n1)]
    gx, gy = np.meshgrid(cx, cy, indexing="ij")
    x = np.concatenate(xs + [gx.ravel()])
    y = np.concatenate(ys + [gy.ravel()])
    return x.astype(np.int64) * n1 + y


def check_pixels(D, R32, S32, x, c, pix_sets, sigma, rms_tol, max_tol):
    """RMS and largest deviation of D from the oracle's subtraction, per set."""
    for name, pix in pix_sets.items():
        De = oracle.subtract_pixels(R32, S32, x, c, pix)
        dev = D.ravel()[pix] - De
        rms, mx = float(np.sqrt(np.mean(dev ** 2))), float(np.max(np.abs(dev)))
        print(f"D {name}: rms {rms / sigma:.2e} sigma, max {mx / sigma:.2e} sigma")
        assert rms <= rms_tol * sigma, (name, rms / sigma)
        assert mx <= max_tol * sigma, (name, mx / sigma)


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
    pix = {"random": rng.integers(0, spec.n0 * spec.n1, 2000),
           "seams": seam_pixels(spec.n0, spec.n1, f.w0, f.w1, rng)}
    check_pixels(D, R32, S32, x, c, pix, spec.sigma, 1e-3, 1e-3)
    plan.close()


def test_masked_transients_4096():
    """The 4096^2 pair with its 50 transients masked for the build (squares
    of half-width 14 px, about 3x the largest science FWHM, zeroed), the
    subtraction on the unmasked pair (Sec. 3, two-step process): sampled M
    and rhs against the oracle's masked lag sums, the solver, D at random,
    seam and transient pixels; then the same request through the serving
    path (sfft_submit with the mask) gives the same coefficients and
    difference image bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, SfftServer, info_from_bytes
    from paper_2109_09334_gb300.build import build
    build()
    spec = synth.PAIR4096
    f = spec.fit
    R, S, tpos = synth.make_pair(spec, seed=5, return_transients=True)
    assert len(tpos[0]) == 50
    mask = synth.transient_mask(R.shape, tpos, half=14)
    assert 0 < int((mask == 0).sum()) < 50 * 29 * 29 + 1
    R32, S32 = R.astype(np.float32), S.astype(np.float32)
    plan = SfftPlan(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype="float32",
                    precision="mixed")
    Rt, St = torch.from_numpy(R32).cuda(), torch.from_numpy(S32).cuda()
    mt = torch.from_numpy(mask).cuda()
    D, x, info, M, rhs = plan.run_pair(Rt, St, mask=mt, keep_system=True)
    torch.cuda.synchronize()
    Mn, rn = M.cpu().numpy(), rhs.cpu().numpy()
    xn, Dn = x.cpu().numpy(), D.cpu().numpy().astype(np.float64)
    assert info_from_bytes(info.cpu().numpy())["status"] == 0
    n = rn.shape[0]
    c = oracle.OracleConfig(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio)
    rng = np.random.default_rng(19)
    rows = np.concatenate([rng.integers(0, n, 300), np.arange(0, n, max(1, n // 100))[:100]])
    cols = np.concatenate([rng.integers(0, n, 300), np.arange(0, n, max(1, n // 100))[:100]])
    Me = oracle.system_entries(R32, S32, c, rows, cols, mask=mask)
    Mg = Mn[rows, cols]
    d = np.sqrt(np.abs(np.diag(Mn)))
    assert np.sqrt(np.mean((Mg - Me) ** 2)) <= 1e-5 * np.sqrt(np.mean(Me ** 2))
    assert np.max(np.abs(Mg - Me) / (d[rows] * d[cols])) <= 1e-4
    rr = rng.integers(0, n, 150)
    re = oracle.system_entries(R32, S32, c, rr, -np.ones_like(rr), mask=mask)
    assert np.sqrt(np.mean((rn[rr] - re) ** 2)) <= 1e-5 * np.sqrt(np.mean(re ** 2))
    assert np.max(np.abs(rn[rr] - re)) <= 1e-4 * np.sqrt(np.mean(re ** 2))
    # the mask changes the system: the unmasked diagonal differs
    du = oracle.system_entries(R32, S32, c, np.arange(3), np.arange(3))
    assert np.all(np.abs(du - Mn[np.arange(3), np.arange(3)]) > 1e-6 * np.abs(du))
    xs = np.linalg.solve(Mn, rn)
    assert np.linalg.norm(xn - xs) <= 1e-8 * np.linalg.norm(xs)
    tx = np.clip(np.floor(tpos[0]).astype(np.int64), 0, spec.n0 - 1)
    ty = np.clip(np.floor(tpos[1]).astype(np.int64), 0, spec.n1 - 1)
    pix = {"random": rng.integers(0, spec.n0 * spec.n1, 2000),
           "seams": seam_pixels(spec.n0, spec.n1, f.w0, f.w1, rng),
           "transients": tx * spec.n1 + ty}
    check_pixels(Dn, R32, S32, xn, c, pix, spec.sigma, 1e-3, 1e-3)
    # the transients stand out in D (the subtraction is unmasked)
    assert float(np.median(Dn.ravel()[pix["transients"]])) > 5 * spec.sigma
    # the serving path with the same mask: bit-identical
    srv = SfftServer(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, dtype="float32",
                     precision="mixed", depth=2, batch=2)
    outs = []
    for _ in range(2):  # two requests share one batched solve
        Dk, xk, ik = torch.empty_like(Rt), torch.empty(n, dtype=torch.float64, device="cuda"), \
            torch.zeros(24, dtype=torch.uint8, device="cuda")
        t = srv.submit(Rt, St, mask=mt, diff=Dk, x=xk, info=ik)[0]
        outs.append((Dk, xk, ik, t))
    for Dk, xk, ik, t in outs:
        srv.wait(t)
    torch.cuda.synchronize()
    for Dk, xk, ik, t in outs:
        assert info_from_bytes(ik.cpu().numpy())["status"] == 0
        np.testing.assert_array_equal(xk.cpu().numpy(), xn)
        np.testing.assert_array_equal(Dk.cpu().numpy().astype(np.float64), Dn)
    srv.close()
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
    pix = np.concatenate([rng.integers(0, spec.n0 * spec.n1, 2000), seam_pixels(spec.n0, spec.n1, f.w0, f.w1, rng)])
    De = oracle.subtract_pixels(R32, S32, x, c, pix)
    # D is written as float32 (the image type): compare within its rounding too
    dev = D.ravel()[pix] - De
    assert np.sqrt(np.mean(dev ** 2)) <= 1e-6 * spec.sigma + 1e-7 * np.sqrt(np.mean(De ** 2))
    assert np.all(np.abs(dev) <= 1e-5 * spec.sigma + 1.2e-7 * np.abs(De))
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
    pix = {"random": rng.integers(0, spec.n0 * spec.n1, 2000),
           "seams": seam_pixels(spec.n0, spec.n1, f.w0, f.w1, rng)}
    check_pixels(D, R32, S32, x, c, pix, spec.sigma, 1e-3, 1e-3)
    plan.close()
