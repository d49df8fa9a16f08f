"""The N > 1 bench path on CPU: replicas with gloo (world size 2), the
max-over-ranks timing and the whole-job rate, and the reference arm's ranks
other than 0 exiting without work."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = 10.0 + 5.0 * rank              # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, ws, device="cpu")
        out[rank] = (ms_max, bench.whole_job_mlups(1e6, ws, ms_max))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo_two_ranks():
    ws, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a threaded process
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    # 2 ranks x 1e6 updates in 15 ms = 133.3 M updates/s
    assert abs(res[0][1] - 2e6 / 15e-3 / 1e6) < 1e-9 and res[0][1] == res[1][1]


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_mlups(2e6, 1, 4.0) == 2e6 / 4e-3 / 1e6


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup = 1, 1

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_rank0_prints_one_contract_line(monkeypatch, capsys):
    import json
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("LOCAL_RANK", "0")

    class Args:
        steps, warmup = 1, 1

    assert bench.run_reference(Args()) == 0
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_clamp_count_classifies_nodes():
    import numpy as np

    class Lat:
        def __init__(self, rho, gd):
            self.rho, self.gd = rho, gd

        def fields(self):
            return self.rho, None, self.gd

    class Prob:
        K, n = 0.01, 0.5

    rho = np.ones(5)
    # nu = K / rho * gd^(n - 1): gd = 0 -> inf (nu_max), 4e4 -> 5e-5 (below nu_min),
    # 1 -> 1e-2 (free), 1e-5 -> 3.2 (free), 1e-7 -> 31.6 (above nu_max)
    gd = np.array([0.0, 4e4, 1.0, 1e-5, 1e-7])
    got = bench._clamp_active_nodes([Lat(rho, gd)], [Prob()])
    assert got == {"at_nu_min": 1, "at_nu_max": 2}
