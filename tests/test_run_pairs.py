"""sfft_run_pairs: several pairs of different sizes and bases, their systems
solved together (up to eight per launch), against sfft_run_pair pair by pair.

The batched solve performs, for each system, the operations of the solve on
its own in the same order, whatever the sizes of the other systems, so every
result must be bitwise equal to sfft_run_pair's.  sfft_run_pair itself is
pinned to the oracle in test_gpu_parity.py.
"""
import ctypes

import numpy as np
import pytest

from synth import random_field

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2109_09334_gb300 import binding
    from paper_2109_09334_gb300.build import build
    build()
    return binding.library()


def test_run_pairs_rejects_bad_arguments(lib):
    """Argument checks that return before any plan is read or any CUDA call."""
    from paper_2109_09334_gb300 import binding as B
    vp = ctypes.c_void_p
    one = (vp * 1)(1)
    assert lib.sfft_run_pairs(None, 1, one, one, None, None, None, one, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_run_pairs(one, 0, one, one, None, None, None, one, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_run_pairs(one, -3, one, one, None, None, None, one, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_run_pairs(one, 1, None, one, None, None, None, one, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_run_pairs(one, 1, one, None, None, None, None, one, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_run_pairs(one, 1, one, one, None, None, None, None, None) == B.SFFT_ERR_INVALID
    nul = (vp * 1)(None)
    assert lib.sfft_run_pairs(nul, 1, one, one, None, None, None, one, None) == B.SFFT_ERR_INVALID


# n0, n1, w, dk, db, cpr: sizes and bases of one mixed batch (non-powers of
# two included); eleven pairs make one full launch of eight and one of three.
MIXED = [
    (256, 256, 4, 2, 2, 1),
    (128, 64, 3, 1, 1, 0),
    (192, 160, 3, 2, 1, 1),
    (64, 64, 2, 0, 0, 1),
    (256, 128, 5, 1, 2, 1),
    (100, 96, 2, 1, 1, 1),
    (128, 128, 4, 2, 0, 0),
    (64, 96, 3, 1, 1, 1),
    (160, 256, 2, 2, 2, 1),
    (96, 64, 4, 0, 1, 0),
    (128, 192, 3, 2, 2, 1),
]


def _pair(n0, n1, k, seed, tdt):
    R = random_field(n0, n1, seed + 10 * k)
    S = 0.9 * np.roll(R, (k % 3 - 1, 1), axis=(0, 1)) + 0.3 * random_field(n0, n1, seed + 10 * k + 5)
    mask = None
    if k % 3 == 1:
        mask = torch.from_numpy((np.random.default_rng(seed + k).random((n0, n1)) > 0.1).astype(np.uint8)).cuda()
    return torch.from_numpy(R).to(tdt).cuda(), torch.from_numpy(S).to(tdt).cuda(), mask


def _expected(plan, R, S, mask):
    from paper_2109_09334_gb300 import info_from_bytes
    D, x, info, _, _ = plan.run_pair(R, S, mask)
    torch.cuda.synchronize()
    return D.cpu().numpy(), x.cpu().numpy(), info_from_bytes(info.cpu().numpy())


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,precision,count", [("float32", "mixed", 11), ("float64", "fp64", 5)])
def test_run_pairs_matches_run_pair(lib, dtype, precision, count):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, info_from_bytes, run_pairs
    tdt = torch.float32 if dtype == "float32" else torch.float64
    plans, inputs, expected = [], [], []
    for k, (n0, n1, w, dk, db, cpr) in enumerate(MIXED[:count]):
        p = SfftPlan(n0, n1, w, w, dk, db, cpr, dtype=dtype, precision=precision)
        R, S, mask = _pair(n0, n1, k, 300, tdt)
        expected.append(_expected(p, R, S, mask))
        plans.append(p)
        inputs.append((R, S, mask))
    out = run_pairs(plans, [i[0] for i in inputs], [i[1] for i in inputs], [i[2] for i in inputs])
    torch.cuda.synchronize()
    for k, (D, x, info) in enumerate(out):
        got = info_from_bytes(info.cpu().numpy())
        assert got["status"] == 0, (k, got)
        assert got == expected[k][2], k
        assert np.array_equal(x.cpu().numpy(), expected[k][1]), k
        assert np.array_equal(D.cpu().numpy(), expected[k][0]), k
    for p in plans:
        p.close()


@pytest.mark.gpu
def test_run_pairs_singular_member(lib):
    """A singular system among pairs of other sizes reports its status; the others are unaffected."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, binding as B, info_from_bytes, run_pairs
    plans, inputs, expected = [], [], []
    for k, (n0, n1, w, dk, db, cpr) in enumerate(MIXED[:4]):
        p = SfftPlan(n0, n1, w, w, dk, db, cpr)
        R, S, _ = _pair(n0, n1, k, 900, torch.float32)
        if k == 2:
            R = torch.zeros_like(R)  # R = 0: every kernel column vanishes, M is singular
        expected.append(_expected(p, R, S, None))
        plans.append(p)
        inputs.append((R, S))
    out = run_pairs(plans, [i[0] for i in inputs], [i[1] for i in inputs])
    torch.cuda.synchronize()
    for k, (D, x, info) in enumerate(out):
        got = info_from_bytes(info.cpu().numpy())
        assert got["status"] == expected[k][2]["status"]
        if k == 2:
            assert got["status"] == B.SFFT_ERR_SINGULAR
        else:
            assert got["status"] == 0
            assert np.array_equal(x.cpu().numpy(), expected[k][1])
            assert np.array_equal(D.cpu().numpy(), expected[k][0])
    for p in plans:
        p.close()


@pytest.mark.gpu
def test_run_pairs_rejects_duplicates_and_mixed_precision(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, binding as B, run_pairs
    a = SfftPlan(64, 64, 2, 2, 1, 1, 1)
    b = SfftPlan(64, 64, 2, 2, 1, 1, 1, dtype="float64", precision="fp64")
    R = torch.randn(64, 64, device="cuda")
    S = torch.randn(64, 64, device="cuda")
    with pytest.raises(B.SfftError) as e:
        run_pairs([a, a], [R, R], [S, S])
    assert e.value.status == B.SFFT_ERR_INVALID
    with pytest.raises(B.SfftError) as e:
        B.sfft_run_pairs([a.handle, b.handle], [R, R.double()], [S, S.double()], None, None, None,
                         [torch.empty_like(R), torch.empty_like(R.double())])
    assert e.value.status == B.SFFT_ERR_INVALID
    a.close()
    b.close()


def test_batch_rejects_bad_arguments(lib):
    """sfft_batch_create checks its arguments before any capture or CUDA call."""
    from paper_2109_09334_gb300 import binding as B
    vp = ctypes.c_void_p
    one = (vp * 1)(1)
    h = vp()
    assert lib.sfft_batch_create(one, 1, one, one, None, None, None, one, 0, None) == B.SFFT_ERR_INVALID
    for group in (-1, 9):
        assert lib.sfft_batch_create(one, 1, one, one, None, None, None, one, group, ctypes.byref(h)) == \
            B.SFFT_ERR_INVALID
    assert lib.sfft_batch_create(None, 1, one, one, None, None, None, one, 0, ctypes.byref(h)) == B.SFFT_ERR_INVALID
    assert lib.sfft_batch_create(one, 0, one, one, None, None, None, one, 0, ctypes.byref(h)) == B.SFFT_ERR_INVALID
    assert h.value is None
    assert lib.sfft_batch_launch(None, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_batch_info(None, None, None, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_batch_destroy(None) == B.SFFT_OK


@pytest.mark.gpu
@pytest.mark.parametrize("solve_group", [0, 3])
def test_batch_graph_matches_run_pair(lib, solve_group):
    """The captured batch (autotuned grouping, or groups of three) replayed
    twice, with new images written into the input buffers in between:
    every pair bitwise equal to sfft_run_pair on the same inputs."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftBatch, SfftPlan, info_from_bytes
    plans, inputs = [], []
    for k, (n0, n1, w, dk, db, cpr) in enumerate(MIXED):
        plans.append(SfftPlan(n0, n1, w, w, dk, db, cpr))
        inputs.append(_pair(n0, n1, k, 500, torch.float32))
    refs = [torch.empty_like(i[0]) for i in inputs]
    scis = [torch.empty_like(i[1]) for i in inputs]
    masks = [i[2] for i in inputs]
    for r, s, i in zip(refs, scis, inputs):
        r.copy_(i[0])
        s.copy_(i[1])
    torch.cuda.synchronize()
    batch = SfftBatch(plans, refs, scis, masks, solve_group=solve_group)
    info = batch.info_dict
    assert info["solve_group"] == (solve_group or info["solve_group"]) and 1 <= info["solve_group"] <= 8
    assert info["launches"] > len(plans)
    for rnd in range(2):
        if rnd == 1:  # new data in the same buffers
            for k, (r, s) in enumerate(zip(refs, scis)):
                r.copy_(torch.roll(inputs[k][0], 1, 0))
                s.copy_(torch.roll(inputs[k][1], 1, 0))
        stream = torch.cuda.current_stream()
        batch.launch(stream)
        torch.cuda.synchronize()
        got = [(D.cpu().numpy(), x.cpu().numpy(), info_from_bytes(i.cpu().numpy()))
               for D, x, i in zip(batch.D, batch.x, batch.info)]
        for k, p in enumerate(plans):
            eD, ex, ei = _expected(p, refs[k], scis[k], masks[k])
            assert ei["status"] == 0
            assert got[k][2] == ei, (rnd, k)
            assert np.array_equal(got[k][1], ex), (rnd, k)
            assert np.array_equal(got[k][0], eD), (rnd, k)
    batch.close()
    for p in plans:
        p.close()


def test_solve_batch_rejects_bad_arguments(lib):
    """sfft_solve_batch checks its arguments before any plan is read or any CUDA call."""
    from paper_2109_09334_gb300 import binding as B
    vp = ctypes.c_void_p
    one = (vp * 1)(1)
    two = (vp * 2)(1, 1)
    assert lib.sfft_solve_batch(None, 1, one, one, one, None, None) == B.SFFT_ERR_INVALID
    for count in (0, -1, 9):
        assert lib.sfft_solve_batch(one, count, one, one, one, None, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_solve_batch(one, 1, None, one, one, None, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_solve_batch(one, 1, one, None, one, None, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_solve_batch(one, 1, one, one, None, None, None) == B.SFFT_ERR_INVALID
    nul = (vp * 1)(None)
    assert lib.sfft_solve_batch(nul, 1, one, one, one, None, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_solve_batch(one, 1, nul, one, one, None, None) == B.SFFT_ERR_INVALID
    # a plan listed twice (rejected before the plans are read)
    assert lib.sfft_solve_batch(two, 2, two, two, two, None, None) == B.SFFT_ERR_INVALID


@pytest.mark.gpu
@pytest.mark.parametrize("panel", [32, 64])
def test_solve_batch_matches_solve(lib, panel):
    """Systems of different sizes built by sfft_build_system, solved together
    by sfft_solve_batch: every solution and status bitwise equal to
    sfft_solve's one at a time (same panel width); a width mismatch is
    rejected."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, binding as B, info_from_bytes
    plans, systems = [], []
    for k, (n0, n1, w, dk, db, cpr) in enumerate(MIXED[:5]):
        p = SfftPlan(n0, n1, w, w, dk, db, cpr)
        p.solve_panel = panel
        R, S, mask = _pair(n0, n1, k, 700, torch.float32)
        _, _, _, M, rhs = p.run_pair(R, S, mask, keep_system=True)
        plans.append(p)
        systems.append((M, rhs))
    stream = torch.cuda.current_stream()
    alone = []
    for p, (M, rhs) in zip(plans, systems):
        x = torch.empty(p.n, dtype=torch.float64, device="cuda")
        info = torch.zeros(24, dtype=torch.uint8, device="cuda")
        B.sfft_solve(p.handle, M, rhs, x, info, stream)
        alone.append((x, info))
    xs = [torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda") for p in plans]
    infos = [torch.zeros(24, dtype=torch.uint8, device="cuda") for _ in plans]
    B.sfft_solve_batch([p.handle for p in plans], [s[0] for s in systems], [s[1] for s in systems], xs, infos,
                       stream)
    torch.cuda.synchronize()
    for k in range(len(plans)):
        assert info_from_bytes(infos[k].cpu().numpy())["status"] == 0
        assert info_from_bytes(infos[k].cpu().numpy()) == info_from_bytes(alone[k][1].cpu().numpy()), k
        assert np.array_equal(xs[k].cpu().numpy(), alone[k][0].cpu().numpy()), k
    plans[1].solve_panel = 96 - panel  # the other width
    with pytest.raises(B.SfftError) as e:
        B.sfft_solve_batch([p.handle for p in plans[:2]], [s[0] for s in systems[:2]],
                           [s[1] for s in systems[:2]], xs[:2], None, stream)
    assert e.value.status == B.SFFT_ERR_INVALID
    for p in plans:
        p.close()
