#!/usr/bin/env python3
"""Benchmark: IPC time steps per second of the soft-rigid coupled IPC stepper.

Default workload: the batched parallel-jaw grasp, 256 environments per GPU in
one scene (seeded synthetic stand-ins for the paper's grasp objects: soft
ellipsoids, tori and boxes of 2k-20k tets, log-uniform, E log-uniform in
[1e4, 1e6] Pa, mu in [0.3, 1.0], nu = 0.45), each squeezed by two kinematic
affine box fingers (972 triangles each) on a fixed floor, dt = 0.005 s,
Newton tolerance 1e-3 x bbox diagonal x dt.  A "step" is one full time step
of the method over every environment (predictor, lagged friction, warm
start, projected Newton with broad phase, distances, PSD Hessians, assembly,
PCG, ACCD line search, velocity update); the unit is env-steps/s.

Timed window: steps [S0, S0 + K) of the grasp script with S0 = max(20, W):
the fingers start 0.5 cm off the object and close at 0.25 mm per step, so
from step 20 on both fingers and the floor are in contact.  The first S0
steps run untimed (the last W of them are the warm-up); the state at S0 is
checkpointed and every form below is timed from that same state:

  headline   mixed precision, all envs batched, learned warm start
  cv         mixed precision, all envs batched, constant-velocity warm start
  plain      plain FP64, all envs batched, constant-velocity warm start
  sequential plain FP64 with the envs stepped one at a time (a strided
             sample of the batch, each env positioned by itself)

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload c3|c2|c5] [--envs E]

--workload c2 times the single-env grasp (steps/s), --workload c5 the dense
soft-rigid pile (8 soft bodies of ~60k tets, 20 affine spheres and tori, a
fixed bin; one scene).  One JSON line on rank 0.  Under torchrun each rank
steps its own batch of E envs (seeds 1000 + E r + i: weak scaling, no
collective in the step); the slowest rank's time is used.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IPC time steps/sec at fixed Newton tol, batched+warm-start vs plain, one B300"
C2_WORKLOAD = "parallel-jaw grasp, 1 env: soft ellipsoid 9600 tets + 2 kinematic affine fingers (972 tris each) + fixed floor"
# the grid-wide solve of the scenes too large for one cluster
ROOFLINE_KERNEL_BY_WORKLOAD = {"c2": "k_pcg_cluster", "c3": "k_pcg_cluster", "c5": "k_pcg_persistent"}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# roofline kernel, from an ncu capture of the kernel as it stands; None where
# no capture was taken since the kernel last changed.  c3: the mean over the
# 7 solves of grasp step 20 at 256 envs (a size-binned solve, one launch per
# cluster size, counts as one launch here as in the live timing).
ROOFLINE_TRAFFIC = {"c2": None, "c3": 330e6, "c5": None}
# first step of the grasp script with both fingers on the object
CONTACT_STEP = {"c2": 20, "c3": 20, "c5": 13}
WEIGHTS = os.path.join(ROOT, "paper_2311_05945_b300", "weights")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def window(args):
    """First timed step of the grasp script: the contact window's start, or
    later when more warm-up steps are asked for."""
    return max(CONTACT_STEP[args.workload], args.warmup)


def build_scene(args, rank=0, world=1):
    """The rank's scene: the single-env grasp, the pile, or the rank's batch
    of args.envs grasp envs (seeds 1000 + args.envs * rank + i)."""
    from paper_2311_05945_b300 import scenes
    n_steps = window(args) + args.steps + 1
    if args.workload == "c2":
        return scenes.scene_c2(n_steps=n_steps)
    if args.workload == "c5":
        return scenes.scene_c5(n_steps=n_steps, tets_per_body=args.c5_tets)
    return scenes.scene_c3(n_envs=args.envs, n_steps=n_steps, seed0=1000 + args.envs * rank)


def env_tets(sc):
    w = [0] * sc.n_envs
    for b in sc.tets:
        w[b.env] += len(b.tets)
    return w


def workload_name(args, sc):
    """The config's workload string (the same for both arms)."""
    if args.workload == "c2":
        return C2_WORKLOAD
    if args.workload == "c5":
        return (f"dense soft-rigid pile: {sum(len(b.tets) for b in sc.tets)} tets in {len(sc.tets)} soft bodies "
                f"+ {sum(1 for a in sc.affines if a.mode == 0)} affine spheres/tori "
                f"({max(len(a.F) for a in sc.affines)} tris max) in a fixed 5-box bin, one scene")
    return (f"batched parallel-jaw grasp, {args.envs} envs per GPU (ellipsoid/torus/box, 2k-20k tets log-uniform, "
            f"{sum(env_tets(sc))} tets on rank 0, E 1e4-1e6, mu 0.3-1.0), all envs in one launch per kernel")


def unit_of(args):
    return "env-steps/s" if args.workload == "c3" else "steps/s"


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_scene(args, sc):
    """(scene, description) of the oracle's sample: for the batched grasp the
    env of the batch whose tet count is closest to the batch mean, on its
    own; the single-env grasp itself; for the pile the same generator at 300
    tets per body (the oracle's all-pairs search cannot step the full pile
    in bounded time)."""
    from paper_2311_05945_b300 import scenes
    n_steps = window(args) + args.steps + 1
    if args.workload == "c3":
        w = env_tets(sc)
        mean = sum(w) / len(w)
        k = min(range(len(w)), key=lambda i: abs(w[i] - mean))
        return (scenes.scene_c3(n_envs=1, n_steps=n_steps, seed0=1000 + k),
                f"env {k} of the batch (seed {1000 + k}, {w[k]} tets, the batch mean is {mean:.0f})")
    if args.workload == "c5":
        return (scenes.scene_c5(n_steps=4, tets_per_body=300, n_seg=8, bin_subdiv=1),
                "the same pile generator at 300 tets per body, 8 x 8 affine meshes, unsplit bin faces")
    return scenes.scene_c2(n_steps=n_steps), "the grasp itself"


def oracle_rate(args, sc, n_time, threads):
    """The CPU oracle, as it stands, on the window of the GPU arm: positioned
    untimed to the window's first step (all host threads; the OpenMP build
    is bit-identical to the serial one), then n_time steps timed with
    `threads` threads.  Returns (rate in the workload's unit, seconds,
    sample description)."""
    from oracle import oracle as O
    osc, desc = oracle_scene(args, sc)
    s0 = 0 if args.workload == "c5" else window(args)
    nproc = os.cpu_count() or 1
    O.set_threads(nproc)
    o = O.Oracle(osc)
    if s0:
        o.step(s0)
    O.set_threads(threads)
    t0 = time.perf_counter()
    o.step(n_time)
    dt = time.perf_counter() - t0
    O.set_threads(1)
    where = "its first steps" if args.workload == "c5" else f"steps [{s0}, {s0 + n_time})"
    return n_time / dt, dt, f"{desc}: {where} of the same script on the CPU oracle, {threads} thread(s) ({dt:.1f} s)"


def run_reference(args, rank):
    if rank != 0:
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    n_time = max(1, min(args.steps, 3))
    sc = build_scene(args, 0, world)
    cores = os.cpu_count() or 1
    v, dt, sample = oracle_rate(args, sc, n_time, cores)
    unit = unit_of(args)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": unit, "n_gpus": args.gpus,
        "steps": n_time, "warmup": window(args) if args.workload != "c5" else 0,
        "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded generators)",
        "config": {"workload": workload_name(args, sc),
                   "form": "CPU oracle: FP64, brute-force pairs, direct/CG solve, OpenMP over independent loops "
                           "(bit-identical to serial)"},
        "cpu_baseline": {"value": v, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def state_bytes(sc):
    return sum(8 * 6 * len(b.X) for b in sc.tets) + 8 * 24 * len(sc.affines)


def load_weights(g):
    """Load every trained warm-start network that applies to the scene."""
    from paper_2311_05945_b300 import zema as Z
    n = 0
    for name in ("warmstart.bin", "warmstart_affine.bin"):
        path = os.path.join(WEIGHTS, name)
        if os.path.exists(path):
            dims, theta = Z.read_warmstart_blob(open(path, "rb").read())
            g.load_warmstart(dims, theta)
            n += 1
    return n


class Form:
    """The statistics and time of one timed form."""

    def __init__(self, name, ms, stats, units, steps):
        self.name, self.ms, self.stats = name, ms, stats
        self.value = units * steps / (ms / 1e3)

    def summary(self):
        agg = {k: sum(s[k] for s in self.stats) for k in ("newton_iters", "pcg_iters", "ls_halvings", "al_rounds",
                                                           "pcg_refines", "warm_accepted", "warm_learned",
                                                           "warm_fallback")}
        return {"value": self.value, "ms_per_step": self.ms / len(self.stats), **agg}


def timed_steps(g, k, flush, dist=None, profile_kernel=None, profile_region=False):
    """k steps with CUDA events on the library's stream, the L2 flushed before
    each; returns (total ms, per-step stats, launches, profile)."""
    import torch

    from paper_2311_05945_b300 import zema as Z
    from paper_2311_05945_b300.sharding import max_over_ranks
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if profile_region:
        torch.cuda.profiler.start()
    if profile_kernel:
        Z.profile_kernel(profile_kernel)
    l0 = Z.launch_count()
    for i in range(k):
        flush.zero_()
        ev[i][0].record(st)
        stats.append(g.step(1))
        ev[i][1].record(st)
    torch.cuda.synchronize()
    if profile_region:
        torch.cuda.profiler.stop()
    launches = Z.launch_count() - l0
    prof = Z.profile_read() if profile_kernel else None
    Z.profile_kernel(None)
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, "cuda")
    return total_ms, stats, launches, prof


def sequential_sample(args, sc):
    """Env ids of the plain sequential form: a stride over the batch."""
    n = sc.n_envs
    m = max(1, min(n, args.seq_envs))
    return [int(i * n / m) for i in range(m)]


def run_ours(args, rank, world):
    import torch

    from paper_2311_05945_b300 import scenes
    from paper_2311_05945_b300 import zema as Z
    from paper_2311_05945_b300.sharding import max_over_ranks

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    K, S0 = args.steps, window(args)
    sc = build_scene(args, rank, world)
    units = sc.n_envs if args.workload == "c3" else 1
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device="cuda")  # 512 MB > L2
    # untimed positioning to the window's first step in the mixed form (the
    # last W steps are the warm-up; the solve's autotuner runs on the last)
    g = Z.Scene(sc, precision=1, warm_start=1)
    for k in range(S0):
        if k == S0 - 1:
            g.autotune()
        g.step(1)
    torch.cuda.synchronize()
    ck = g.save_checkpoint()
    forms = {}
    # mixed + constant-velocity warm start (no network loaded yet)
    ms, stats, _, _ = timed_steps(g, K, flush, dist)
    forms["cv"] = Form("cv", ms, stats, units, K)
    # headline: mixed + learned warm start; clocks and the roofline kernel
    # sampled while it runs
    g.load_checkpoint(ck)
    n_nets = load_weights(g)
    clocks = Clocks(local)
    clocks.start()
    kname = ROOFLINE_KERNEL_BY_WORKLOAD[args.workload]
    ms, stats, launches, prof = timed_steps(g, K, flush, dist, kname, args.profile_region)
    clk = clocks.stop()
    head = Form("headline", ms, stats, units, K)
    tuned = g.tuning()
    # end to end through the C ABI with a pinned host buffer, same window,
    # same form: every step uploads every body's state (one copy), steps,
    # and reads them all back (one copy)
    g.load_checkpoint(ck)
    host = torch.from_numpy(g.get_scene_state()).pin_memory()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        g.set_scene_state_ptr(host.data_ptr(), host.numel())
        g.step(1)
        g.get_scene_state_ptr(host.data_ptr(), host.numel())
    torch.cuda.synchronize()
    e2e_val = units * K / max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    g.close()
    # plain FP64, batched, from the same checkpoint (one untimed step for its
    # own autotuning first)
    gp = Z.Scene(sc, precision=0)
    gp.load_checkpoint(ck)
    gp.autotune()
    gp.step(1)
    gp.load_checkpoint(ck)
    ms, stats, _, _ = timed_steps(gp, K, flush, dist)
    forms["plain"] = Form("plain", ms, stats, units, K)
    gp.close()
    # plain FP64, envs stepped one at a time (strided sample, each env
    # positioned by itself in FP64)
    if args.workload == "c3" and args.seq_envs > 0:
        ids = sequential_sample(args, sc)
        seq_ms, seq_stats = 0.0, []
        for i in ids:
            one = scenes.scene_c3(n_envs=1, n_steps=S0 + K + 1, seed0=1000 + args.envs * rank + i)
            gs = Z.Scene(one, precision=0)
            for k in range(S0):
                if k == S0 - 1:
                    gs.autotune()
                gs.step(1)
            ms, stats, _, _ = timed_steps(gs, K, flush)
            seq_ms += ms
            seq_stats += stats
            gs.close()
        seq_ms = max_over_ranks(seq_ms, dist, "cuda")
        seq = Form("sequential", seq_ms, seq_stats, len(ids), K)
        forms["sequential"] = seq
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    peak_gbs = peaks["hbm_gbs"] if peaks else 6400.0
    roof = None
    k_ms, k_launches, k_bytes = prof
    if k_launches:
        per_launch_bytes = k_bytes / k_launches
        achieved = per_launch_bytes / (k_ms / k_launches / 1e3) / 1e9
        roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved / peak_gbs, "traffic": ROOFLINE_TRAFFIC.get(args.workload),
                "peak_source": "measured" if peaks else "fallback",
                "alg_bytes_per_launch": per_launch_bytes, "avg_launch_us": 1e3 * k_ms / k_launches,
                "launches": k_launches, "share_of_step_time": k_ms / head.ms if world == 1 else None}
    unit = unit_of(args)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        v, _, sample = oracle_rate(args, sc, args.cpu_steps, cores)
        v1, _, sample1 = oracle_rate(args, sc, 1, 1) if args.cpu_serial else (None, None, None)
        cpu = {"value": v, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample}
        if v1 is not None:
            cpu["serial_1_core"] = {"value": v1, "sample": sample1}
    phase = {k: sum(s["ms_phase"][k] for s in head.stats) for k in head.stats[0]["ms_phase"]}
    cfg = {
        "workload": workload_name(args, sc),
        "timed_steps": [S0, S0 + K],
        "form": ("mixed precision (FP32 Hessians, matrices and PCG with FP64 residual refinement; FP64 gradients, "
                 "energies, distances, CCD and convergence) + learned warm start (trained networks: "
                 f"{n_nets}; CCD-filtered, energy-checked, plain-Newton fallback)"
                 + ("; all envs batched" if args.workload == "c3" else "")),
        "headline": head.summary(),
        "mixed_cv_warm_start": forms["cv"].summary(),
        "plain_fp64_batched" if args.workload == "c3" else "plain_fp64": forms["plain"].summary(),
        "speedup_vs_plain": head.value / forms["plain"].value,
        "parallelism": (f"weak: {args.envs} envs per rank on {world} ranks" if args.workload == "c3"
                        else f"replicas x{world}") if world > 1 else "single GPU",
        "l2": "flushed between timed steps (512 MB write)",
        "state": f"every form starts from the same checkpoint at step {S0}",
        "pcg_autotune": {"ctas_per_env": tuned[0], "solve_ms_by_ctas": {str(k): round(v, 4)
                                                                         for k, v in tuned[1].items()}},
        "host_phase_ms": {k: round(v, 2) for k, v in phase.items()},
    }
    if "sequential" in forms:
        seq = forms["sequential"]
        cfg["plain_fp64_sequential"] = {**seq.summary(), "envs_sampled": sequential_sample(args, sc),
                                        "how": "each sampled env alone in its own scene, positioned to the "
                                               "window in FP64, timed over the same steps; env-steps/s over "
                                               "the sample"}
        cfg["speedup_vs_plain_sequential"] = head.value / seq.value
    line = {
        "metric": METRIC, "value": head.value, "unit": unit, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": head.ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed f32/f64", "data": "synthetic (seeded generators)",
        "config": cfg,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": unit, "h2d_bytes_per_step": state_bytes(sc),
                "d2h_bytes_per_step": state_bytes(sc)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c2", "c3", "c5"],
                    help="c3: the batched grasp (headline, env-steps/s); c2: the single-env grasp; "
                         "c5: the dense soft-rigid pile")
    ap.add_argument("--c5-tets", type=int, default=60000, help="tets per soft body of the pile (c5)")
    ap.add_argument("--envs", type=int, default=256, help="envs per GPU of the batched grasp (c3)")
    ap.add_argument("--seq-envs", type=int, default=16,
                    help="envs of the batch sampled for the plain sequential form (c3; 0 skips it)")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--cpu-serial", action="store_true", help="also time one oracle step on 1 thread")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the headline form's timed steps with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
