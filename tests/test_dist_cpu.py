"""The benchmark's multi-process path on CPU: two ranks over gloo on
127.0.0.1 (one process per GPU on a GPU machine; replicas, no collective on the
data path).  The job's time is the slowest rank's (max over ranks), the
whole-job rate counts every rank's units (weak scaling), and the reference
arm's extra ranks exit without work."""
import os
import socket
import types

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        import bench
        import synthetic as S
        r, w, dist = bench.dist_init(world)
        t = bench.max_over_ranks(1.5 + r, dist, "cpu")
        extra = None
        if r != 0:      # the reference arm: only rank 0 runs the oracle
            args = types.SimpleNamespace(gpus=world, steps=1, warmup=0)
            extra = bench.run_reference(args, S.DISK_2D_Q2)
        q.put((r, w, t, bench.job_rate(w, 100, t), extra))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:      # report, do not leave the parent waiting
        q.put((rank, -1, repr(e), None, None))


def test_two_ranks_max_time_and_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted((q.get(timeout=60) for _ in procs), key=lambda o: o[0])
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
    assert all(o[1] == 2 for o in out), out
    assert all(p.exitcode == 0 for p in procs)
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == pytest.approx(2.5) for o in out)          # the slower rank's time
    assert all(o[3] == pytest.approx(2 * 100 / 2.5) for o in out)
    assert out[1][4] is None


def test_single_process_needs_no_group():
    import bench
    assert bench.dist_init(1) == (0, 1, None)
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.job_rate(1, 10, 2.0) == 5.0
