"""The N > 1 path of bench.py (one replica per GPU, no data-path collective)
on CPU: two gloo ranks.  The job time is the slowest rank's, the rate counts
the units of all ranks, and the reference arm runs on rank 0 only."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    b = load_bench()
    r, w, lr, dist = b.init_replicas("gloo")
    local_ms = [3.0, 5.0][r]          # rank 1 is the slow replica
    ms = b.replica_max(local_ms, dist)
    out.put((r, w, ms, b.job_rate(192, w, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r, w, ms, rate in res:
        assert w == 2 and ms == 5.0
        assert rate == pytest.approx(2 * 192 * 1e3 / 5.0)


def test_single_process_needs_no_process_group():
    b = load_bench()
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    r, w, lr, dist = b.init_replicas("gloo")
    assert (r, w, lr, dist) == (0, 1, 0, None)
    assert b.replica_max(7.5, None) == 7.5
    assert b.job_rate(1, 1, 250.0) == 4.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    b = load_bench()

    class A:
        steps, warmup, gpus = 1, 3, 2

    assert b.run_reference(A(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""
