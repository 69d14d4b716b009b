"""The benchmark's multi-rank host logic on CPU, with two gloo ranks.

Under torchrun every rank solves its own replica of the workload (independent
problems, no data exchange: weak scaling); the only collectives are the
barrier around the timed region and the maximum of the timed durations over
the ranks, and the whole-job value counts the unknowns of every replica.  The
reference arm runs on rank 0 alone; the other ranks exit without work.  The
clock record's throttle reasons are parsed from nvidia-smi's CSV.
"""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    ms = bench.max_over_ranks(10.0 + 5.0 * r, w)      # rank 1 is the slower one
    e2e = bench.max_over_ranks(3.0 * (r + 1), w)
    dist.barrier()
    q.put((r, w, ms, e2e, bench.job_value(w, 1000, 4, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_replica():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rr, w, ms, e2e, val) in enumerate(out):
        assert rr == r and w == world
        assert ms == 15.0 and e2e == 6.0
        assert val == pytest.approx(world * 1000 * 4 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_value(1, 2_000_000, 5, 100.0) == pytest.approx(1e8)


def _reference(monkeypatch, rank, world, extra=()):
    calls = []

    def fake_oracle(expr, reps):
        calls.append((expr, reps))
        return {"ndof": 59280, "runs": [[0.5 + 0.1 * i, 14, 5e-9] for i in range(reps)]}

    monkeypatch.setattr(bench, "run_oracle", fake_oracle)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "3", "--warmup", "1",
                                      "--gpus", str(world), *extra])
    monkeypatch.setenv("RANK", str(rank))
    monkeypatch.setenv("WORLD_SIZE", str(world))
    bench.reference_arm(bench.parse())
    return calls


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    assert _reference(monkeypatch, 1, 2) == [] and capsys.readouterr().out == ""
    calls = _reference(monkeypatch, 0, 2)
    # warm-up + timed solves of the bounded sample: the 2D layout at 64/96 intervals, p = 2
    assert calls == [("W.sipg_3x3(2, scale=1, smoother='hybrid')", 4)]
    line = json.loads(capsys.readouterr().out.strip())
    times = [0.6, 0.7, 0.8]  # the three timed runs after the warm-up one
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 3
    assert line["value"] == pytest.approx(59280 * 3 / sum(times))
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "DoF/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_clock_record_reasons_and_median():
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2050, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 1980, 2070, 1399.0, 0x8, Active, Not Active, Not Active, Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2050.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unavailable"]


def test_reference_arm_of_the_cube_times_a_cube_sample(monkeypatch, capsys):
    calls = _reference(monkeypatch, 0, 1, ("--workload", "cube-sipg"))
    assert calls == [("W.cube_2x2x2(3, 'sipg', n=12)", 4)]
    line = json.loads(capsys.readouterr().out.strip())
    assert "2x2x2" in line["metric"] and "cube_2x2x2" in line["config"]["workload"]


def test_workload_defaults():
    for name, (degrees, expr, desc) in bench.WORKLOADS.items():
        assert name in bench.METRIC_OF and degrees and expr.startswith("W.")
    assert bench.METRIC_OF["sipg3x3"] == bench.METRIC
