"""The N > 1 path of bench.py on CPU: two ranks over gloo (127.0.0.1) agree on
the slowest rank's time, the whole-job value counts every replica, and the
reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        tmax = bench.max_over_ranks(10.0 + 7.5 * rank, dist, torch.device("cpu"))
        value = bench.whole_job_value(w, 1.0e6, 10, 2, tmax)
        ref = bench.run_reference(None, r, w) if r != 0 else "rank0"
        dist.barrier()
        q.put((r, w, local, tmax, value, ref))
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_max_time_and_whole_job_value():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    # both ranks see the slowest rank's 17.5 ms; the value counts 2 replicas
    assert all(o[3] == pytest.approx(17.5) for o in out)
    assert all(o[4] == pytest.approx(2 * 1.0e6 * 10 * 2 / 17.5e-3 / 1e6) for o in out)
    # the reference arm does its work on rank 0 only
    assert out[1][5] is None


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.25, None, None) == 3.25
    assert bench.whole_job_value(1, 8.0, 5, 3, 2.0) == pytest.approx(8 * 5 * 3 / 2e-3 / 1e6)
