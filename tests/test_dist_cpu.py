"""Multi-process replica path of the benchmark on CPU (gloo, world size 2):
the barrier around the timed region, the maximum of the ranks' times, and
the whole-job throughput (units every rank processed over the slowest rank's
time).  The path has no exchange step, so this is all that runs across
ranks; on GPUs the same code runs over NCCL."""
import multiprocessing
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    try:
        rep = bench.Replicas(world, None)
        rep.barrier()
        slowest = rep.max(10.0 + 3.0 * rank)  # rank 1 is the slower replica
        rate = bench.aggregate_rate(500, world, slowest)
        rep.barrier()
        rep.close()
        q.put((rank, slowest, rate, None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, None, repr(e)))


def test_replicas_gloo_two_ranks():
    pytest.importorskip("torch.distributed")
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, err in out:
        assert err is None, err
        assert slowest == 13.0
        assert rate == pytest.approx(2 * 500 / 0.013)


def test_single_process_has_no_group():
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas(1, None)
    rep.barrier()
    assert rep.max(7.5) == 7.5
    assert bench.aggregate_rate(100, 1, 50.0) == pytest.approx(2000.0)
    rep.close()


def test_reference_arm_other_ranks_do_no_work():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, cpu_sample_gates = 1, 0, 1
    assert bench.run_reference(A(), 1, 2) == 0
