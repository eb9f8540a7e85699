"""The benchmark's reference arm (the CPU oracle, timed on the host) prints
one JSON line with the keys of the benchmark contract, for every workload;
the oracle timing itself is replaced here by a fixed rate so that the test
stays fast.  The timed window starts at the contact step whatever the
warm-up, and the plain sequential sample strides over the batch."""
import argparse
import json
import os

import pytest

import bench


def fake_scene(args, rank=0, world=1):
    return argparse.Namespace(n_envs=args.envs, tets=[], affines=[argparse.Namespace(mode=0, F=[0])])


@pytest.mark.parametrize("workload", ["c2", "c3", "c5"])
def test_reference_line_keys(workload, monkeypatch, capsys):
    monkeypatch.setattr(bench, "oracle_rate", lambda args, sc, n, threads: (0.5, 2.0, "fixed sample"))
    monkeypatch.setattr(bench, "build_scene", fake_scene)
    args = argparse.Namespace(workload=workload, envs=256, warmup=5, steps=20, gpus=1, c5_tets=60000, cpu_steps=2)
    bench.run_reference(args, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] == 0.5 and line["higher_is_better"] is True
    assert line["unit"] == ("env-steps/s" if workload == "c3" else "steps/s")
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == 0.5
    assert line["config"]["workload"]
    assert line["steps"] == 3  # up to 3 oracle steps of the window
    if workload != "c5":
        assert line["warmup"] == 20  # the GPU arm's window start


def test_reference_arm_is_silent_off_rank_zero(capsys):
    args = argparse.Namespace(workload="c2", envs=256, warmup=20, steps=30, gpus=2, c5_tets=60000, cpu_steps=2)
    bench.run_reference(args, 1)
    assert capsys.readouterr().out == ""


def test_window_starts_at_contact_and_sample_strides():
    args = argparse.Namespace(workload="c3", warmup=5, steps=20, envs=256, seq_envs=16)
    assert bench.window(args) == 20
    args.warmup = 30
    assert bench.window(args) == 30
    ids = bench.sequential_sample(args, argparse.Namespace(n_envs=256))
    assert ids == list(range(0, 256, 16))
    args.seq_envs = 400
    assert bench.sequential_sample(args, argparse.Namespace(n_envs=256)) == list(range(256))


def test_clock_record_parsing(tmp_path):
    # the clocks line summarises nvidia-smi's samples: median SM clock under
    # load, the maximum, and every throttle reason seen active at least once
    rows = [
        "0, 2032, 2032, 700.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2032, 1090.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2032, 1050.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, [N/A], 2032, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
        "0, 2032",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.Clocks(0)
    c.proc, c.path = Done(), str(path)
    out = c.stop()
    assert out == {"sm_mhz": 2010.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()
    # a throttle that a run must be rejected for is reported by name
    path.write_text("0, 1500, 2032, 900.0, 0x48, Not Active, Active, Not Active, Not Active\n")
    c.proc, c.path = Done(), str(path)
    assert c.stop()["reasons"] == ["hw_thermal_slowdown"]
    # no sampler, or no usable sample: no clocks line
    assert bench.Clocks(0).stop() is None
    path.write_text("")
    c.proc, c.path = Done(), str(path)
    assert c.stop() is None
