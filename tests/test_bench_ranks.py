"""Multi-rank bench logic on CPU (gloo, world size 2): each rank solves its
own instances (replicas, weak scaling); the job time is the slowest rank's
and the rate counts every rank's solves."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        per_rank_ms = [1000.0, 2500.0][rank]
        total = bench.max_over_ranks(per_rank_ms, world)
        out[rank] = (total, bench.whole_job_rate(5, world, total))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in range(2):
        total, rate = out[rank]
        assert total == 2500.0
        assert rate == pytest.approx(2 * 5 / 2.5)


def test_single_rank_identity():
    assert bench.max_over_ranks(123.0, 1) == 123.0
    assert bench.whole_job_rate(4, 1, 2000.0) == pytest.approx(2.0)


def test_reference_arm_line_contract(monkeypatch):
    """The reference arm (the oracle on the host cores) prints the contract's
    keys; its config is the GPU arm's physics and solver settings on the
    smaller mesh it actually timed (named as a sample of the GPU arm's
    workload), with its own cpu_baseline and a copy-free e2e."""
    import sys
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1",
                                      "--warmup", "0"])
    args = bench.parse()
    line = bench.run_reference(args)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    cfg = dict(line["config"])
    head = bench.headline_config(args)
    assert cfg["sample_of"] == head["workload"]
    assert (cfg["nx"], cfg["ny"]) == (bench.ORACLE_SIZES[0],) * 2
    assert 1000.0 / line["ms_per_step"] == pytest.approx(line["value"])
    for key in ("k", "n_hlevels", "rtol", "inner_rtol", "inner_norm", "inner_krylov", "precision"):
        assert cfg[key] == head[key], key
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
