"""The multi-rank path of bench.py on CPU: two gloo ranks (the launcher's environment variables,
127.0.0.1 rendezvous) agree on the slowest rank's time, run distinct replicas, report the
whole-job aggregate, and only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    slowest = bench.max_over_ranks(1.5 + rank, dist, device="cpu")
    seed = bench.replica_config({"seed": 0, "noise": False}, rank)["seed"]
    q.put((rank, slowest, bench.dist_env(), seed))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
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
    assert [o[1] for o in out] == [2.5, 2.5]
    assert [o[2] for o in out] == [(2, 0, 0), (2, 1, 1)]
    assert out[0][3] != out[1][3]


def test_whole_job_value_and_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_value(2, 100, 0.5) == 400.0
    assert bench.max_over_ranks(0.25, None) == 0.25
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup = 1, 0

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
