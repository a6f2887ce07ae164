"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (stated per result):
  * plain FP64 path: rel. Frobenius error of M and rhs <= 1e-10, coefficient
    rel. error <= 1e-8, difference-image RMS deviation <= 1e-6 sigma;
  * mixed path (FP32 FFTs/products, compensated sums, FP32 Cholesky + FP64
    refinement): rel. error of M and rhs <= 1e-5; the solver is checked
    against an FP64 solve of the same GPU-built system (<= 1e-8); the
    difference image RMS deviation from the oracle's is <= 1e-3 sigma.

Beyond the norms, every small case checks each block of Eq. 18 on its own
(the kernel-kernel block A of Eq. B5, the kernel-background block B of
Eq. B7/B9, the background block C of Eq. B11, the rhs parts D of Eq. B13 and
E of Eq. B15), since C, B and E are orders of magnitude smaller than A and a
wrong one could hide under a norm of the whole matrix:
  * per block, rel. Frobenius error <= the tolerance of the whole matrix;
  * per entry, |dM_ij| <= tol_e * sqrt(M_ii M_jj) (Cauchy-Schwarz bounds
    |M_ij| by that product, so this is a relative error on the scale the
    entry can reach), and |drhs_i| <= tol_e * sqrt(M_ii) * ||S_masked||;
    tol_e = 1e-4 mixed, 1e-9 FP64;
  * D: the largest pixel deviation <= 1e-2 sigma (mixed) or 1e-5 sigma
    (FP64), so that one wrong pixel cannot hide in the RMS.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import random_field

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIGMA = 5.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300.build import build
    build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def gpu_run(R, S, w0, w1, dk, db, cpr, precision, dtype, mask=None, spline=None):
    from paper_2109_09334_gb300 import SfftPlan, info_from_bytes
    n0, n1 = R.shape
    plan = SfftPlan(n0, n1, w0, w1, dk, db, cpr, dtype=dtype, precision=precision, spline=spline)
    tdt = torch.float32 if dtype == "float32" else torch.float64
    Rt = torch.from_numpy(np.ascontiguousarray(R)).to("cuda", tdt)
    St = torch.from_numpy(np.ascontiguousarray(S)).to("cuda", tdt)
    mt = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask, dtype=np.uint8)).cuda()
    D, x, info, M, rhs = plan.run_pair(Rt, St, mask=mt, keep_system=True)
    torch.cuda.synchronize()
    out = dict(D=D.double().cpu().numpy(), x=x.cpu().numpy(), M=M.cpu().numpy(), rhs=rhs.cpu().numpy(),
               info=info_from_bytes(info.cpu().numpy()), plan=plan, R=Rt, S=St)
    return out


def small_pair(n0, n1, seed):
    R = random_field(n0, n1, seed)
    S = 0.8 * np.roll(R, (1, -1), axis=(0, 1)) + 0.3 * random_field(n0, n1, seed + 7)
    return R, S


SMALL = [
    # n0, n1, w0, w1, dk, db, cpr, masked
    (16, 16, 1, 1, 0, 0, 1, False),
    (16, 32, 2, 1, 1, 1, 0, False),
    (32, 16, 1, 2, 2, 1, 1, True),
    (64, 64, 3, 3, 1, 2, 1, False),
    (64, 32, 2, 3, 2, 2, 0, True),
    (128, 64, 4, 2, 3, 3, 1, False),
    (64, 128, 5, 6, 0, 3, 1, True),
    (256, 64, 0, 0, 2, 2, 1, False),
    # sizes that are not powers of two: Bluestein row transforms (n1) and
    # direct lag sums along x (n0)
    (48, 40, 2, 2, 1, 1, 1, False),
    (40, 64, 3, 2, 2, 1, 0, True),
    (64, 48, 2, 3, 1, 2, 1, False),
    (37, 41, 2, 1, 0, 1, 1, True),
    (17, 19, 1, 1, 1, 0, 0, False),
    (100, 96, 4, 4, 2, 2, 1, False),
    # a half-width above 16: Lambda through the gather, not in closed form
    (64, 96, 2, 20, 1, 1, 1, False),
    # the size limits: the largest and smallest axes, power of two or not,
    # and the largest degrees
    (16, 4096, 1, 3, 2, 2, 1, False),
    (4096, 16, 3, 1, 1, 1, 0, True),
    (4093, 17, 2, 2, 1, 1, 1, False),
    (64, 64, 2, 2, 3, 3, 1, False),
]


# B-spline bases (Eq. 7-9): n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint, masked
SPLINE = [
    (32, 32, 2, 2, 1, 1, 0, 1, 0, False),   # linear, no interior knot, constant ratio
    (64, 48, 2, 3, 0, 2, 1, 1, 1, True),    # quadratic, varying ratio, Bluestein rows
    (48, 64, 3, 2, 1, 3, 0, 2, 1, False),   # cubic, direct lag sums along x
    (64, 64, 2, 2, 1, 0, 2, 0, 1, True),    # piecewise constant in three spans
    (128, 64, 3, 2, 1, 2, 2, 2, 0, False),
    (40, 37, 1, 2, 0, 1, 1, 1, 0, False),   # neither axis a power of two
]


def kernel_unknowns(c):
    """Boolean mask over the unknowns: True for kernel coefficients (the
    oracle's own decoding of the unknown order), False for background ones."""
    return np.array([oracle.decode_unknown(c, u)[0] for u in range(oracle.num_unknowns(c))])


def block_errors(Mg, rg, Mo, ro, c, S, mask):
    """Relative Frobenius error of each block of Eq. 18 and the largest
    per-entry errors on the Cauchy-Schwarz scale (module docstring)."""
    k = kernel_unknowns(c)
    b = ~k
    out = {}
    for name, (ri, ci) in {"A": (k, k), "B": (k, b), "C": (b, b)}.items():
        if ri.any() and ci.any():
            out[name] = rel(Mg[np.ix_(ri, ci)], Mo[np.ix_(ri, ci)])
    out["rhs_D"] = rel(rg[k], ro[k])
    out["rhs_E"] = rel(rg[b], ro[b])
    d = np.sqrt(np.abs(np.diag(Mo)))
    out["entry_M"] = float(np.max(np.abs(Mg - Mo) / np.maximum(np.outer(d, d), 1e-300)))
    Sm = S if mask is None else S * (mask != 0)
    out["entry_rhs"] = float(np.max(np.abs(rg - ro) / np.maximum(d * np.linalg.norm(Sm), 1e-300)))
    return out


def check_system(Mg, rg, Mo, ro, c, S, mask, tol, tol_e):
    assert rel(Mg, Mo) <= tol
    assert rel(rg, ro) <= tol
    e = block_errors(Mg, rg, Mo, ro, c, S, mask)
    print("block errors", {k: f"{v:.1e}" for k, v in e.items()})
    for name in ("A", "B", "C", "rhs_D", "rhs_E"):
        if name in e:
            assert e[name] <= tol, (name, e)
    assert e["entry_M"] <= tol_e, e
    assert e["entry_rhs"] <= tol_e, e


def check_against_oracle(R, S, c, precision, mask, g):
    """The tolerances of the module docstring, oracle config c vs GPU result g."""
    Mo, ro = oracle.build_system(R, S, c, mask=mask)
    xo = oracle.cholesky_solve(Mo, ro)
    Do = oracle.subtract(R, S, xo, c)
    assert g["info"]["status"] == 0, g["info"]
    if precision == "fp64":
        check_system(g["M"], g["rhs"], Mo, ro, c, S, mask, 1e-10, 1e-9)
        assert rel(g["x"], xo) <= 1e-8
        assert np.sqrt(np.mean((g["D"] - Do) ** 2)) <= 1e-6 * SIGMA
        assert np.max(np.abs(g["D"] - Do)) <= 1e-5 * SIGMA
    else:
        # inputs rounded to float32 on both sides for the system check
        R32, S32 = R.astype(np.float32).astype(np.float64), S.astype(np.float32).astype(np.float64)
        Mo32, ro32 = oracle.build_system(R32, S32, c, mask=mask)
        check_system(g["M"], g["rhs"], Mo32, ro32, c, S32, mask, 1e-5, 1e-4)
        xs = np.linalg.solve(g["M"], g["rhs"])
        assert rel(g["x"], xs) <= 1e-8
        Do32 = oracle.subtract(R32, S32, oracle.cholesky_solve(Mo32, ro32), c)
        assert np.sqrt(np.mean((g["D"] - Do32) ** 2)) <= 1e-3 * SIGMA
        assert np.max(np.abs(g["D"] - Do32)) <= 1e-2 * SIGMA


@pytest.mark.parametrize("case", SPLINE)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bspline_cases_against_oracle(case, precision):
    n0, n1, w0, w1, cpr, kdeg, kint, bdeg, bint, masked = case
    R, S = small_pair(n0, n1, seed=n0 + 5 * n1 + kdeg)
    mask = None
    if masked:
        mask = (np.random.default_rng(n1).random((n0, n1)) > 0.15).astype(np.uint8)
    c = oracle.OracleConfig(n0, n1, w0, w1, 0, 0, bool(cpr), "bspline", kdeg, kint, bdeg, bint)
    dtype = "float64" if precision == "fp64" else "float32"
    g = gpu_run(R, S, w0, w1, 0, 0, cpr, precision, dtype, mask, spline=(kdeg, kint, bdeg, bint))
    assert g["M"].shape == (oracle.num_unknowns(c),) * 2
    check_against_oracle(R, S, c, precision, mask, g)
    g["plan"].close()


@pytest.mark.parametrize("case", SMALL)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_cases_against_oracle(case, precision):
    n0, n1, w0, w1, dk, db, cpr, masked = case
    R, S = small_pair(n0, n1, seed=n0 + 3 * n1 + w0)
    mask = None
    if masked:
        mask = (np.random.default_rng(n0).random((n0, n1)) > 0.15).astype(np.uint8)
    c = oracle.OracleConfig(n0, n1, w0, w1, dk, db, bool(cpr))
    dtype = "float64" if precision == "fp64" else "float32"
    g = gpu_run(R, S, w0, w1, dk, db, cpr, precision, dtype, mask)
    check_against_oracle(R, S, c, precision, mask, g)
    g["plan"].close()


def test_pair256_fp64_full():
    """256^2 float64 pair, w=4, D_K=D_B=0, constant ratio (82 unknowns), plain FP64 path."""
    spec = synth.PAIR256
    R, S = synth.make_pair(spec, seed=1)
    f = spec.fit
    c = oracle.OracleConfig(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio)
    Mo, ro = oracle.build_system(R, S, c)
    xo = oracle.cholesky_solve(Mo, ro)
    Do = oracle.subtract(R, S, xo, c)
    g = gpu_run(R, S, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, "fp64", "float64")
    assert g["M"].shape == (82, 82)
    assert g["info"]["status"] == 0
    check_system(g["M"], g["rhs"], Mo, ro, c, S, None, 1e-10, 1e-9)
    assert rel(g["x"], xo) <= 1e-8
    assert np.sqrt(np.mean((g["D"] - Do) ** 2)) <= 1e-6 * SIGMA
    assert np.max(np.abs(g["D"] - Do)) <= 1e-5 * SIGMA
    g["plan"].close()


def test_pair1024_mixed_full():
    """1024^2 float32 pair, w=6, D_K=D_B=1, varying ratio (510 unknowns), mixed path."""
    spec = synth.PAIR1024
    R, S = synth.make_pair(spec, seed=2)
    f = spec.fit
    c = oracle.OracleConfig(spec.n0, spec.n1, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio)
    R64, S64 = R.astype(np.float64), S.astype(np.float64)
    Mo, ro = oracle.build_system(R64, S64, c)
    xo = oracle.cholesky_solve(Mo, ro)
    Do = oracle.subtract(R64, S64, xo, c)
    g = gpu_run(R, S, f.w0, f.w1, f.dk, f.db, f.const_phot_ratio, "mixed", "float32")
    assert g["M"].shape == (510, 510)
    assert g["info"]["status"] == 0, g["info"]
    check_system(g["M"], g["rhs"], Mo, ro, c, S64, None, 1e-5, 1e-4)
    assert rel(g["x"], np.linalg.solve(g["M"], g["rhs"])) <= 1e-8
    assert np.sqrt(np.mean((g["D"] - Do) ** 2)) <= 1e-3 * SIGMA
    assert np.max(np.abs(g["D"] - Do)) <= 1e-2 * SIGMA
    g["plan"].close()


def test_singular_reference_reports_status():
    """R == 0 makes every kernel column vanish: the solve reports SINGULAR."""
    R = np.zeros((32, 32))
    S = random_field(32, 32, 5)
    g = gpu_run(R, S, 1, 1, 0, 0, 1, "fp64", "float64")
    assert g["info"]["status"] == -4
    g["plan"].close()


def test_invalid_configs_rejected():
    from paper_2109_09334_gb300 import SfftError, SfftPlan
    with pytest.raises(SfftError):
        SfftPlan(5000, 64, 2, 2, 0, 0, 1)       # beyond the largest supported size
    with pytest.raises(SfftError):
        SfftPlan(64, 64, 16, 2, 0, 0, 1)        # lag range beyond the inner transform
    with pytest.raises(SfftError):
        SfftPlan(64, 64, 2, 2, 4, 0, 1)         # D_K > 3


def test_host_entry_point_matches_device():
    R, S = small_pair(64, 64, 9)
    g = gpu_run(R, S, 2, 2, 1, 1, 1, "mixed", "float32")
    plan = g["plan"]
    Rh = torch.from_numpy(R.astype(np.float32)).pin_memory()
    Sh = torch.from_numpy(S.astype(np.float32)).pin_memory()
    D, x, info = plan.run_pair_host(Rh, Sh)
    assert info["status"] == 0
    np.testing.assert_array_equal(D.double().numpy(), g["D"])
    np.testing.assert_array_equal(x.numpy(), g["x"])
    plan.close()


def test_mask_of_ones_equals_no_mask_and_repeat_is_bitwise():
    R, S = small_pair(64, 64, 12)
    a = gpu_run(R, S, 3, 3, 2, 1, 0, "mixed", "float32")
    b = gpu_run(R, S, 3, 3, 2, 1, 0, "mixed", "float32", mask=np.ones((64, 64), np.uint8))
    c = gpu_run(R, S, 3, 3, 2, 1, 0, "mixed", "float32")
    np.testing.assert_array_equal(a["M"], b["M"])
    np.testing.assert_array_equal(a["D"], b["D"])
    np.testing.assert_array_equal(a["M"], c["M"])
    np.testing.assert_array_equal(a["x"], c["x"])
    for g in (a, b, c):
        g["plan"].close()


@pytest.mark.parametrize("case", [SMALL[3], SMALL[5], SMALL[13]])
def test_tensor_core_solve_against_oracle(case):
    """The FP32 solve with its trailing-update tile products on the tensor
    cores (tcgen05, 3xTF32; launch-shape knob solve_tensor_cores = 2): the
    same tolerances as the CUDA-core path, and the refinement still
    converges in at most 4 iterations."""
    from paper_2109_09334_gb300 import SfftPlan, binding, info_from_bytes
    n0, n1, w0, w1, dk, db, cpr, masked = case
    R, S = small_pair(n0, n1, seed=n0 + 3 * n1 + w0)
    mask = None
    if masked:
        mask = (np.random.default_rng(n0).random((n0, n1)) > 0.15).astype(np.uint8)
    c = oracle.OracleConfig(n0, n1, w0, w1, dk, db, bool(cpr))
    plan = SfftPlan(n0, n1, w0, w1, dk, db, cpr, dtype="float32", precision="mixed")
    shapes = binding.sfft_plan_tuning(plan.handle)
    binding.sfft_plan_set_tuning(plan.handle, dict(shapes, solve_tensor_cores=2))
    try:
        Rt = torch.from_numpy(np.ascontiguousarray(R)).to("cuda", torch.float32)
        St = torch.from_numpy(np.ascontiguousarray(S)).to("cuda", torch.float32)
        mt = None if mask is None else torch.from_numpy(mask).cuda()
        D, x, info, M, rhs = plan.run_pair(Rt, St, mask=mt, keep_system=True)
        torch.cuda.synchronize()
        g = dict(D=D.double().cpu().numpy(), x=x.cpu().numpy(), M=M.cpu().numpy(), rhs=rhs.cpu().numpy(),
                 info=info_from_bytes(info.cpu().numpy()))
        assert g["info"]["iters"] <= 4, g["info"]
        check_against_oracle(R, S, c, "mixed", mask, g)
    finally:
        binding.sfft_plan_set_tuning(plan.handle, dict(shapes, solve_tensor_cores=0))
        plan.close()


@pytest.mark.parametrize("case", SMALL, ids=[f"{c[0]}x{c[1]}w{c[2]}" for c in SMALL])
def test_panel64_solve_against_oracle(case):
    """The FP32 solve with 64-wide Cholesky panels (sfft_plan_set_solve_panel;
    the diagonal 64-block factored as two 32-blocks, L21 = A21 L11^-T and
    W21 = -L22^-1 L21 L11^-1): the same tolerances as the 32-wide default,
    and the refinement still converges in at most 4 iterations."""
    from paper_2109_09334_gb300 import SfftPlan, info_from_bytes
    n0, n1, w0, w1, dk, db, cpr, masked = case
    R, S = small_pair(n0, n1, seed=n0 + 3 * n1 + w0)
    mask = None
    if masked:
        mask = (np.random.default_rng(n0).random((n0, n1)) > 0.15).astype(np.uint8)
    c = oracle.OracleConfig(n0, n1, w0, w1, dk, db, bool(cpr))
    plan = SfftPlan(n0, n1, w0, w1, dk, db, cpr, dtype="float32", precision="mixed")
    plan.solve_panel = 64
    try:
        assert plan.solve_panel == 64
        Rt = torch.from_numpy(np.ascontiguousarray(R)).to("cuda", torch.float32)
        St = torch.from_numpy(np.ascontiguousarray(S)).to("cuda", torch.float32)
        mt = None if mask is None else torch.from_numpy(mask).cuda()
        D, x, info, M, rhs = plan.run_pair(Rt, St, mask=mt, keep_system=True)
        torch.cuda.synchronize()
        g = dict(D=D.double().cpu().numpy(), x=x.cpu().numpy(), M=M.cpu().numpy(), rhs=rhs.cpu().numpy(),
                 info=info_from_bytes(info.cpu().numpy()))
        assert g["info"]["iters"] <= 4, g["info"]
        check_against_oracle(R, S, c, "mixed", mask, g)
    finally:
        plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fully_masked_pair_reports_singular(precision):
    """A mask that hides every pixel leaves the build no data: the kernel
    columns (built from the masked R) and the right-hand side vanish, only
    the background block C (Eq. B11, from the unmasked basis functions)
    remains, and the solve reports SINGULAR instead of coefficients."""
    from paper_2109_09334_gb300 import binding as B
    R, S = small_pair(32, 32, 77)
    dtype = "float64" if precision == "fp64" else "float32"
    c = oracle.OracleConfig(32, 32, 1, 1, 1, 1, True)
    g = gpu_run(R, S, 1, 1, 1, 1, 1, precision, dtype, mask=np.zeros((32, 32), np.uint8))
    assert g["info"]["status"] == B.SFFT_ERR_SINGULAR, g["info"]
    k = kernel_unknowns(c)
    assert not np.any(g["M"][k]) and not np.any(g["rhs"])
    Mo, _ = oracle.build_system(R, S, c, mask=np.zeros((32, 32), np.uint8))
    assert rel(g["M"], Mo) <= 1e-10
    g["plan"].close()
