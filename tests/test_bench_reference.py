"""The benchmark's reference arm (the CPU oracle, timed on the host) prints
one JSON line with the keys of the benchmark contract, for every workload;
the oracle timing itself is replaced here by a fixed rate so that the test
stays fast."""
import argparse
import json

import pytest

import bench


@pytest.mark.parametrize("workload", ["c2", "c3", "c5"])
def test_reference_line_keys(workload, monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_steps_per_s", lambda n_warm, n_steps, sc=None: (0.5, 2.0))
    if workload != "c2":
        # skip the full scene generation: the name only needs the env count
        monkeypatch.setattr(bench, "build_scene", lambda args, rank=0, world=1: argparse.Namespace(
            n_envs=args.envs, tets=[], affines=[argparse.Namespace(mode=0, F=[0])]))
    args = argparse.Namespace(workload=workload, envs=256, warmup=20, steps=30, gpus=1, c5_tets=60000, cpu_steps=2)
    bench.run_reference(args, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] == 0.5 and line["higher_is_better"] is True
    assert line["unit"] == ("env-steps/s" if workload == "c3" else "steps/s")
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == 0.5
    assert line["config"]["workload"]
    if workload == "c2":
        assert (line["warmup"], line["steps"]) == (20, 3)  # the GPU arm's window start, up to 3 steps


def test_reference_arm_is_silent_off_rank_zero(capsys):
    args = argparse.Namespace(workload="c2", envs=256, warmup=20, steps=30, gpus=2, c5_tets=60000, cpu_steps=2)
    bench.run_reference(args, 1)
    assert capsys.readouterr().out == ""
