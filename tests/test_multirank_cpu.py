"""The multi-rank logic of bench.py on the CPU, without a GPU.

The path shards by replicas only: every rank runs the same step on its own GPU
with no data-path collective, and the ranks meet only to time the job.  Two
gloo ranks on 127.0.0.1 (world size 2) check that the timed duration is the
maximum over the ranks and that the reported value is the whole job's units
per second of the slowest rank; the reference arm runs on rank 0 alone."""
import argparse
import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 3.0 * rank            # the ranks' own timed durations differ
        dist.barrier()
        total_ms = bench.max_over_ranks(local_ms, dist, "cpu")
        rate = bench.whole_job_rate(4 * 5, world, total_ms / 1e3)   # 4 maps x 5 steps per rank
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{total_ms!r} {rate!r}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_the_whole_job_rate(tmp_path):
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        total_ms, rate = map(float, (tmp_path / f"rank{r}.txt").read_text().split())
        assert total_ms == 13.0
        assert rate == pytest.approx(4 * 5 * 2 / 0.013, rel=1e-12)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.whole_job_rate(20, 1, 0.5) == 40.0


def _reference_args():
    return argparse.Namespace(warmup=3, steps=2, gpus=2, precision="mixed", inner_cycles=6, adaptive_inner=True,
                              refine_fp64=False, sequential=False)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    calls = []

    class FakeStep:
        workers = 3

        def __init__(self):
            calls.append("init")

        def run(self):
            calls.append("run")
            return {"wall_s": 0.25, "solve_wall_s": 0.2, "ff_wall_s": 0.05, "scaled_s": 2.0, "single_thread_s": 4.0,
                    "solve_s": [0.1] * 4, "cycles": [10] * 4}

        def close(self):
            calls.append("close")

    monkeypatch.setattr(bench, "OracleStep", FakeStep)
    bench.run_reference(_reference_args(), rank=1, world=2)
    assert calls == [] and capsys.readouterr().out == ""
    bench.run_reference(_reference_args(), rank=0, world=2)
    assert calls.count("run") == 3 + 2 and calls[-1] == "close"      # warm-up and timed steps
    line = json.loads(capsys.readouterr().out.strip())
    assert line["impl"] == "reference" and line["value"] == pytest.approx(4 / 2.0)
    assert line["ms_per_step"] == pytest.approx(250.0)                # measured wall time per step
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 3
    assert line["cpu_baseline"]["single_thread"]["value"] == pytest.approx(1.0)
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"] == bench._config(_reference_args())       # the same config as the GPU arm


def test_reference_arm_end_to_end_on_the_host():
    """`bench.py --impl reference` (the oracle on the host cores, one bounded
    sample of the workload) prints one JSON line with the contract's keys."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], check=True, capture_output=True, text=True, timeout=600).stdout
    line = json.loads(out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "maps/s"
    assert line["config"]["workload"].startswith("2D 1025x1025")
