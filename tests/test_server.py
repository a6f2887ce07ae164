"""The serving path (sfft_submit / sfft_poll / sfft_wait) against the
single-pair path.

Each request runs the kernels of sfft_run_pair on its own slot, and those
kernels are deterministic, so results must be bitwise equal to sfft_run_pair
on the same inputs, alone and in a mix of in-flight requests (device and host
memory, with and without masks).  A server that batches four or more pairs
solves with 64-wide Cholesky panels, so the reference plan is set to the
same width.  The single-pair path itself is pinned to
the oracle in test_gpu_parity.py.
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


def test_server_rejects_bad_arguments(lib):
    """Argument checks that return before any CUDA call."""
    from paper_2109_09334_gb300 import binding as B
    cfg = B.make_config(64, 64, 2, 2, 1, 1, 1)
    h = ctypes.c_void_p()
    for depth, batch in ((0, 1), (9, 1), (-1, 1), (2, 0), (2, 3), (8, 9)):
        assert lib.sfft_server_create(ctypes.byref(cfg), depth, batch, ctypes.byref(h)) == B.SFFT_ERR_INVALID
        assert h.value is None
    bad = B.make_config(64, 64, -1, 2, 1, 1, 1)
    assert lib.sfft_server_create(ctypes.byref(bad), 2, 1, ctypes.byref(h)) == B.SFFT_ERR_INVALID
    big = B.make_config(5000, 64, 2, 2, 1, 1, 1)  # beyond the largest supported size
    assert lib.sfft_server_create(ctypes.byref(big), 2, 1, ctypes.byref(h)) == B.SFFT_ERR_UNSUPPORTED
    assert lib.sfft_server_create(None, 2, 1, ctypes.byref(h)) == B.SFFT_ERR_INVALID
    assert lib.sfft_server_create(ctypes.byref(cfg), 2, 1, None) == B.SFFT_ERR_INVALID
    assert lib.sfft_flush(None) == B.SFFT_ERR_INVALID
    t = B.sfft_ticket()
    req = B.sfft_request()
    assert lib.sfft_submit(None, ctypes.byref(req), ctypes.byref(t)) == B.SFFT_ERR_INVALID
    assert lib.sfft_poll(None, ctypes.byref(t)) == B.SFFT_ERR_INVALID
    assert lib.sfft_wait(None, ctypes.byref(t), 0) == B.SFFT_ERR_INVALID
    assert lib.sfft_server_destroy(None) == B.SFFT_OK


def make_pairs(n0, n1, count, seed):
    out = []
    for k in range(count):
        R = random_field(n0, n1, seed + 10 * k)
        S = 0.9 * np.roll(R, (k % 3 - 1, 1), axis=(0, 1)) + 0.3 * random_field(n0, n1, seed + 10 * k + 5)
        mask = None
        if k % 2 == 1:
            mask = (np.random.default_rng(seed + k).random((n0, n1)) > 0.1).astype(np.uint8)
        out.append((R, S, mask))
    return out


CASES = [
    # n0, n1, w, dk, db, cpr, dtype, precision
    (256, 256, 4, 2, 2, 1, "float32", "mixed"),
    (128, 64, 3, 1, 1, 0, "float64", "fp64"),
]


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("depth,batch", [(2, 1), (3, 1), (2, 2), (4, 3), (6, 6)])
def test_server_matches_run_pair(lib, case, depth, batch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, SfftServer, info_from_bytes
    n0, n1, w, dk, db, cpr, dtype, precision = case
    tdt = torch.float32 if dtype == "float32" else torch.float64
    pairs = make_pairs(n0, n1, 6, seed=n0 + depth)
    plan = SfftPlan(n0, n1, w, w, dk, db, cpr, dtype=dtype, precision=precision)
    plan.solve_panel = 64 if batch >= 4 else 32  # the server's slots batch with 64-wide panels
    expected = []
    dev_inputs = []
    for R, S, mask in pairs:
        Rt = torch.from_numpy(R).to("cuda", tdt)
        St = torch.from_numpy(S).to("cuda", tdt)
        mt = None if mask is None else torch.from_numpy(mask).cuda()
        D, x, info, _, _ = plan.run_pair(Rt, St, mask=mt)
        torch.cuda.synchronize()
        expected.append((D.cpu().numpy(), x.cpu().numpy(), info_from_bytes(info.cpu().numpy())))
        dev_inputs.append((Rt, St, mt))
    plan.close()

    srv = SfftServer(n0, n1, w, w, dk, db, cpr, dtype=dtype, precision=precision, depth=depth, batch=batch)
    assert srv.workspace_bytes > 0
    # all requests in flight before the first wait: even ones device, odd ones host
    jobs = []
    for k, ((R, S, mask), (Rt, St, mt)) in enumerate(zip(pairs, dev_inputs)):
        if k % 2 == 0:
            jobs.append(srv.submit(Rt, St, mask=mt))
        else:
            Rh = torch.from_numpy(R).to(tdt).pin_memory()
            Sh = torch.from_numpy(S).to(tdt).pin_memory()
            mh = None if mask is None else torch.from_numpy(mask).pin_memory()
            jobs.append(srv.submit(Rh, Sh, mask=mh))
    for k, (ticket, D, x, info) in enumerate(jobs):
        assert srv.wait(ticket, timeout_us=60_000_000)
        assert srv.poll(ticket)
        De, xe, ie = expected[k]
        got = info_from_bytes(info.cpu().numpy())
        assert got["status"] == 0 and got["iters"] == ie["iters"], (k, got, ie)
        assert np.array_equal(x.cpu().numpy(), xe), f"request {k}: coefficients differ from sfft_run_pair"
        assert np.array_equal(D.cpu().numpy(), De), f"request {k}: difference image differs from sfft_run_pair"
    srv.close()


@pytest.mark.gpu
def test_wait_timeout_and_unknown_ticket(lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftServer, binding as B
    srv = SfftServer(64, 64, 2, 2, 1, 1, 1)
    R = torch.from_numpy(random_field(64, 64, 3)).float().cuda()
    S = torch.from_numpy(random_field(64, 64, 4)).float().cuda()
    ticket, D, x, info = srv.submit(R, S)
    srv.wait(ticket, timeout_us=0)  # returns at once, done or not
    assert srv.wait(ticket, timeout_us=60_000_000)
    unknown = B.sfft_ticket(ticket.seq + 5)
    with pytest.raises(B.SfftError):
        B.sfft_wait(srv.handle, unknown, 0)
    srv.close()


@pytest.mark.gpu
def test_batch_with_a_singular_system(lib):
    """A singular system in a batch reports its status; the others are unaffected."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, SfftServer, binding as B, info_from_bytes
    n0 = n1 = 64
    pairs = make_pairs(n0, n1, 3, seed=77)
    plan = SfftPlan(n0, n1, 2, 2, 1, 1, 1)
    srv = SfftServer(n0, n1, 2, 2, 1, 1, 1, depth=3, batch=3)
    jobs, expected = [], []
    for k, (R, S, mask) in enumerate(pairs):
        Rt = torch.from_numpy(R).float().cuda()
        if k == 1:
            Rt = torch.zeros_like(Rt)  # R = 0: every kernel column vanishes, M is singular
        St = torch.from_numpy(S).float().cuda()
        D, x, info, _, _ = plan.run_pair(Rt, St)
        torch.cuda.synchronize()
        expected.append((D.cpu().numpy(), x.cpu().numpy(), info_from_bytes(info.cpu().numpy())))
        jobs.append(srv.submit(Rt, St))
    for k, (ticket, D, x, info) in enumerate(jobs):
        assert srv.wait(ticket, timeout_us=60_000_000)
        got = info_from_bytes(info.cpu().numpy())
        assert got["status"] == expected[k][2]["status"]
        if k == 1:
            assert got["status"] == B.SFFT_ERR_SINGULAR
        else:
            assert got["status"] == 0
            assert np.array_equal(x.cpu().numpy(), expected[k][1])
            assert np.array_equal(D.cpu().numpy(), expected[k][0])
    srv.close()
    plan.close()


@pytest.mark.gpu
def test_failed_completion_query_ends_wait_with_error(lib):
    """A completion query that reports a CUDA error ends sfft_wait with
    SFFT_ERR_CUDA instead of spinning (timeout -1 included), and the error
    is sticky for poll, wait and submit.  The failure is made on the host by
    the server's testing hook: no fault on the GPU, and the enqueued work
    runs to completion (destroy waits for it)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import threading
    from paper_2109_09334_gb300 import SfftServer, binding as B
    n0 = n1 = 64
    R, S, _ = make_pairs(n0, n1, 1, seed=41)[0]
    srv = SfftServer(n0, n1, 2, 2, 1, 1, 1, dtype="float32", precision="mixed", depth=2, batch=2)
    Rt = torch.from_numpy(R.astype(np.float32)).cuda()
    St = torch.from_numpy(S.astype(np.float32)).cuda()
    t0 = srv.submit(Rt, St)[0]
    t1 = srv.submit(Rt, St)[0]
    assert srv.wait(t0)  # the server works before the hook is set
    B.sfft_server_debug_fail_queries(srv.handle, True)
    rc = {}

    def waiter():
        rc["wait"] = lib.sfft_wait(srv.handle, ctypes.byref(t1), -1)

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    th.join(timeout=30)
    assert not th.is_alive(), "sfft_wait kept spinning after a failed completion query"
    assert rc["wait"] == B.SFFT_ERR_CUDA
    assert lib.sfft_poll(srv.handle, ctypes.byref(t1)) == B.SFFT_ERR_CUDA
    assert lib.sfft_wait(srv.handle, ctypes.byref(t1), 1000) == B.SFFT_ERR_CUDA
    req = B.make_request(Rt, St, torch.empty_like(Rt))
    t = B.sfft_ticket()
    assert lib.sfft_submit(srv.handle, ctypes.byref(req), ctypes.byref(t)) == B.SFFT_ERR_CUDA
    with pytest.raises(B.SfftError):
        srv.wait(t1)
    # the hook only fakes the queries: the device finished the work
    B.sfft_server_debug_fail_queries(srv.handle, False)
    torch.cuda.synchronize()
    srv.close()
    assert lib.sfft_server_debug_fail_queries(None, 1) == B.SFFT_ERR_INVALID


@pytest.mark.gpu
def test_eager_flush_solves_incomplete_batch_without_wait(lib):
    """With eager flushing, a lone request in a batch of four is solved and
    subtracted as soon as it is submitted to an idle server: after a device
    synchronisation (no poll, wait or flush) its outputs equal sfft_run_pair's
    bit for bit.  Without it the batch waits: the outputs are untouched."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09334_gb300 import SfftPlan, SfftServer
    n0 = n1 = 64
    R, S, _ = make_pairs(n0, n1, 1, seed=51)[0]
    Rt = torch.from_numpy(R.astype(np.float32)).cuda()
    St = torch.from_numpy(S.astype(np.float32)).cuda()
    plan = SfftPlan(n0, n1, 2, 2, 1, 1, 1, dtype="float32", precision="mixed")
    plan.solve_panel = 64  # as the batching server's slots
    De, xe, _, _, _ = plan.run_pair(Rt, St)
    torch.cuda.synchronize()
    for eager in (True, False):
        srv = SfftServer(n0, n1, 2, 2, 1, 1, 1, dtype="float32", precision="mixed", depth=4, batch=4, eager=eager)
        D = torch.full_like(Rt, float("nan"))
        t, _, x, _ = srv.submit(Rt, St, diff=D)
        torch.cuda.synchronize()
        if eager:
            np.testing.assert_array_equal(D.cpu().numpy(), De.cpu().numpy())
            np.testing.assert_array_equal(x.cpu().numpy(), xe.cpu().numpy())
        else:
            assert torch.isnan(D).all()
        assert srv.wait(t)
        np.testing.assert_array_equal(D.cpu().numpy(), De.cpu().numpy())
        srv.close()
    plan.close()
