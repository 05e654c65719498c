"""The benchmark's multi-rank host logic on CPU, with two gloo ranks.

Under torchrun each rank solves its own instance of the workload (the path shards
only as independent problems, so there is no data-path exchange): every rank reads
its place from the environment, the step time reported is the slowest rank's (a
max all-reduce), and the whole-job rate counts the units of all ranks.  The
reference arm runs on rank 0 alone.  These are the parts of bench.py that need no
GPU; here they run as two CPU processes over gloo at 127.0.0.1."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        env = bench._dist_env()
        step_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        slowest = bench._max_over_ranks(step_ms, world, "cpu")
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"env": list(env), "slowest": slowest,
                       "rate": bench._job_rate(0.25, slowest, world)}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_step(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["env"] == [world, r, r]
        assert x["slowest"] == 15.0  # every rank reports the slowest rank's time
        # 2 ranks x 0.25 units per step, over 15 ms
        assert x["rate"] == pytest.approx(2 * 0.25 / 0.015, rel=1e-12)


def test_one_rank_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist_env() == (1, 0, 0)
    assert bench._max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench._job_rate(0.262144, 1.82, 1) == pytest.approx(0.262144 / 0.00182, rel=1e-12)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    # the other ranks return at once, before reading the arguments or starting any
    # oracle work, and print nothing
    assert bench.run_reference(None) is None
    assert capsys.readouterr().out == ""
