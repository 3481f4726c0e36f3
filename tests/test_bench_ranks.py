"""bench.py's multi-process logic on the CPU (two `gloo` ranks, no GPU): each rank
decodes its own instance (weak scaling, no data-path exchange), the job's time is the
slowest rank's (max over ranks), and the whole-job value counts every rank's units.
The reference arm runs on rank 0 alone."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="env://")
    try:
        t = bench.max_over_ranks(0.25 + 0.5 * rank, ws, "cpu")     # rank 1 is the slow one
        q.put((rank, bench.dist_env(), t, bench.job_throughput(1000.0, ws, t), bench.rank_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [(2, 0, 0), (2, 1, 1)]
    for rank, _, t, value, seed in out:
        assert t == 0.75                                            # max over the ranks
        assert value == pytest.approx(2 * 1000.0 / 0.75)            # both ranks' units over that time
    assert out[0][4] != out[1][4]                                   # each rank its own instance


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(0.5, 1, "cpu") == 0.5
    assert bench.job_throughput(10.0, 1, 0.5) == 20.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 3, 2
    assert bench.run_reference(Args(), bench.workload()) == 0
    assert capsys.readouterr().out == ""
