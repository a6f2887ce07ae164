"""The pool (sfft_pool_*): pairs of several sizes and fit configurations in
flight together under one memory budget.

Each request runs the kernels of sfft_run_pair on its own lane's workspace
and those kernels are deterministic, so every result must equal
sfft_run_pair's bit for bit, alone and in the mix.  Admission: a
configuration whose lane does not fit the budget is refused (SFFT_ERR_BUSY)
unless idle lanes can be released, least recently used first.
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


def test_pool_rejects_bad_arguments(lib):
    from paper_2109_09334_gb300 import binding as B
    h = ctypes.c_void_p()
    assert lib.sfft_pool_create(0, 2, 1, ctypes.byref(h)) == B.SFFT_ERR_INVALID
    assert lib.sfft_pool_create(1 << 30, 0, 1, ctypes.byref(h)) == B.SFFT_ERR_INVALID
    assert lib.sfft_pool_create(1 << 30, 2, 3, ctypes.byref(h)) == B.SFFT_ERR_INVALID
    assert lib.sfft_pool_create(1 << 30, 2, 1, None) == B.SFFT_ERR_INVALID
    t = B.sfft_pool_ticket()
    assert lib.sfft_pool_wait(None, ctypes.byref(t), 0) == B.SFFT_ERR_INVALID
    assert lib.sfft_pool_poll(None, ctypes.byref(t)) == B.SFFT_ERR_INVALID
    assert lib.sfft_pool_destroy(None) == B.SFFT_OK
    # a pool allocates nothing until its first request
    assert lib.sfft_pool_create(1 << 30, 2, 1, ctypes.byref(h)) == B.SFFT_OK
    b, n = ctypes.c_uint64(), ctypes.c_int32()
    assert lib.sfft_pool_usage(h, ctypes.byref(b), ctypes.byref(n)) == B.SFFT_OK
    assert b.value == 0 and n.value == 0
    bad = B.make_config(64, 64, 2, 2, 1, 1, 1)
    assert lib.sfft_pool_wait(h, ctypes.byref(t), 0) == B.SFFT_ERR_INVALID  # no such lane
    assert lib.sfft_pool_destroy(h) == B.SFFT_OK
    del bad


def pair(n0, n1, seed):
    R = random_field(n0, n1, seed)
    S = 0.9 * np.roll(R, (1, -1), axis=(0, 1)) + 0.3 * random_field(n0, n1, seed + 3)
    return R.astype(np.float32), S.astype(np.float32)


# (n0, n1, w, dk, db, cpr)
MIX = [(64, 64, 2, 1, 1, 1), (48, 40, 2, 2, 1, 0), (128, 96, 3, 1, 2, 1), (37, 41, 1, 0, 1, 1)]


@pytest.mark.gpu
def test_mixed_configurations_equal_single_pair_results(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, SfftPool, info_from_bytes
    jobs = []
    for k in range(3):
        for c, (n0, n1, w, dk, db, cpr) in enumerate(MIX):
            jobs.append((c, pair(n0, n1, 10 * k + c)))
    expected = []
    for c, (R, S) in jobs:
        n0, n1, w, dk, db, cpr = MIX[c]
        plan = SfftPlan(n0, n1, w, w, dk, db, cpr)
        D, x, info, _, _ = plan.run_pair(torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda())
        torch.cuda.synchronize()
        expected.append((D.cpu().numpy(), x.cpu().numpy()))
        plan.close()
    pool = SfftPool(64 << 30, depth=2, batch=1)
    handles = []
    for k, (c, (R, S)) in enumerate(jobs):  # all in flight, configurations interleaved
        n0, n1, w, dk, db, cpr = MIX[c]
        if k % 2:
            Rin, Sin = torch.from_numpy(R).pin_memory(), torch.from_numpy(S).pin_memory()
        else:
            Rin, Sin = torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda()
        got = pool.submit(Rin, Sin, w, w, dk, db, cpr)
        assert got is not None
        handles.append(got)
    assert pool.usage[1] == len(MIX)
    for k, (t, D, x, info) in enumerate(handles):
        assert pool.wait(t, timeout_us=60_000_000)
        assert info_from_bytes(info.cpu().numpy())["status"] == 0
        assert np.array_equal(D.cpu().numpy(), expected[k][0]), k
        assert np.array_equal(x.cpu().numpy(), expected[k][1]), k
    pool.close()


@pytest.mark.gpu
def test_admission_by_memory_budget(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPool
    A, B = (2, 2, 1, 1, 1), (2, 2, 1, 1, 1)  # w0, w1, dk, db, const_phot_ratio
    RA, SA = pair(64, 64, 1)
    RB, SB = pair(96, 80, 2)
    # a budget smaller than any lane admits nothing
    tiny = SfftPool(4096)
    assert tiny.submit(torch.from_numpy(RA).cuda(), torch.from_numpy(SA).cuda(), *A) is None
    assert tiny.usage == (0, 0)
    tiny.close()
    # room for lane A only: B is admitted once A is idle, by releasing A
    probe = SfftPool(64 << 30)
    tA = probe.submit(torch.from_numpy(RA).cuda(), torch.from_numpy(SA).cuda(), *A)
    probe.wait(tA[0])
    bytes_a = probe.usage[0]
    probe.close()
    tB_probe = SfftPool(64 << 30)
    t = tB_probe.submit(torch.from_numpy(RB).cuda(), torch.from_numpy(SB).cuda(), *B)
    tB_probe.wait(t[0])
    bytes_b = tB_probe.usage[0]
    tB_probe.close()
    pool = SfftPool(max(bytes_a, bytes_b) + 1024)
    ta = pool.submit(torch.from_numpy(RA).cuda(), torch.from_numpy(SA).cuda(), *A)
    assert ta is not None and pool.usage[1] == 1
    assert pool.wait(ta[0], timeout_us=60_000_000)
    tb = pool.submit(torch.from_numpy(RB).cuda(), torch.from_numpy(SB).cuda(), *B)
    assert tb is not None
    assert pool.usage == (bytes_b, 1)  # lane A was released
    assert pool.wait(ta[0], timeout_us=0)  # a released lane's requests have completed
    assert pool.wait(tb[0], timeout_us=60_000_000)
    pool.close()


@pytest.mark.gpu
def test_pool_mixes_polynomial_and_bspline_configurations(lib):
    """A B-spline configuration is its own lane; results equal sfft_run_pair's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, SfftPool, info_from_bytes
    cases = [(64, 64, 2, 1, 1, 1, None), (64, 64, 2, 0, 0, 1, (2, 1, 1, 0)), (48, 64, 2, 0, 0, 0, (1, 0, 1, 1))]
    expected, inputs = [], []
    for k, (n0, n1, w, dk, db, cpr, spline) in enumerate(cases):
        R, S = pair(n0, n1, 70 + k)
        plan = SfftPlan(n0, n1, w, w, dk, db, cpr, spline=spline)
        D, x, info, _, _ = plan.run_pair(torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda())
        torch.cuda.synchronize()
        expected.append((D.cpu().numpy(), x.cpu().numpy()))
        inputs.append((R, S))
        plan.close()
    pool = SfftPool(64 << 30, depth=2, batch=1)
    handles = []
    for (n0, n1, w, dk, db, cpr, spline), (R, S) in zip(cases, inputs):
        got = pool.submit(torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda(), w, w, dk, db, cpr, spline=spline)
        assert got is not None
        handles.append(got)
    assert pool.usage[1] == len(cases)
    for k, (t, D, x, info) in enumerate(handles):
        assert pool.wait(t, timeout_us=60_000_000)
        assert info_from_bytes(info.cpu().numpy())["status"] == 0
        assert np.array_equal(D.cpu().numpy(), expected[k][0]), k
        assert np.array_equal(x.cpu().numpy(), expected[k][1]), k
    pool.close()
