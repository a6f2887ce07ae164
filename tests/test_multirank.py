"""The replicated (multi-GPU) bench path on CPU: two `gloo` ranks.

Pairs are independent, so N GPUs run N replicas with no collective on the
data path; the only cross-rank operation is the maximum of the timings, and
the job's throughput is all ranks' pairs over the slowest rank's time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    # rank r took (10 + r) ms for its steps and 3 - r s on the host
    t = bench.max_over_ranks([10.0 + r, 3.0 - r], w)
    v = bench.pairs_per_second(w, 4, t[0])
    torch.distributed.destroy_process_group()
    q.put((r, w, t, v))


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, t, v in out:
        assert w == world
        assert t == [11.0, 3.0]  # the maximum over ranks of each entry
        assert abs(v - world * 4 / 0.011) < 1e-9


def test_single_rank_is_a_no_op():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.pairs_per_second(1, 10, 1000.0) == 10.0
