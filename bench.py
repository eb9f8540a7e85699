#!/usr/bin/env python3
"""Benchmark: IPC time steps per second of the soft-rigid coupled IPC stepper.

Workload: the parallel-jaw grasp scene (seeded synthetic stand-in for the
paper's grasp objects): a jittered Kuhn-lattice soft ellipsoid (semi-axes
4/2/3 cm, 9,600 tets, Neo-Hookean E = 5e4 Pa, nu = 0.45) on a fixed floor,
squeezed and lifted by two kinematic affine box fingers (972 triangles each),
mu = 0.8, dt = 0.005 s, Newton tolerance 1e-3 x bbox diagonal x dt.  A "step"
is one full time step of the method (predictor, lagged friction, warm start,
projected Newton with broad phase, distances, PSD Hessians, assembly, PCG,
ACCD line search, velocity update).  Timed steps are steps [W, W + K) of the
grasp script after W warm-up steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload c2|c3|c5]

--workload c3 times the batched grasp (env-steps/s); --workload c5 the dense
soft-rigid pile (8 soft bodies of ~60k tets, 20 affine spheres and tori, a
fixed bin), one scene too large for a cluster solve.

One JSON line on rank 0.  Under torchrun each rank steps its own replica of
the workload (environments are independent: weak scaling, no collective in
the step); the slowest rank's time is used.
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
UNIT = "steps/s"
WORKLOAD = "parallel-jaw grasp, 1 env: soft ellipsoid 9600 tets + 2 kinematic affine fingers (972 tris each) + fixed floor"
ROOFLINE_KERNEL = "k_pcg_cluster"
# the grid-wide solve of the scenes too large for one cluster
ROOFLINE_KERNEL_BY_WORKLOAD = {"c2": "k_pcg_cluster", "c3": "k_pcg_cluster", "c5": "k_pcg_persistent"}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# ROOFLINE_KERNEL per workload, from an ncu capture: c2, the first solve of
# grasp step 20 (751.9 us, near the bench's 705 us average launch); None where
# no capture was taken or once the kernel changes.
ROOFLINE_TRAFFIC = {"c2": 1384448 + 8448, "c3": None, "c5": None}


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


def build_scene(args=None, rank=0, world=1):
    """The rank's scene: the single-env grasp, or its share of the batched
    grasp (contiguous env range balanced by tet count; env i keeps seed
    1000 + i whatever the sharding)."""
    from paper_2311_05945_b300 import scenes
    if args is None or args.workload == "c2":
        return scenes.scene_c2()
    if args.workload == "c5":
        # one scene: every rank steps its own replica
        return scenes.scene_c5(n_steps=args.warmup + args.steps, tets_per_body=args.c5_tets)
    from paper_2311_05945_b300.sharding import shard_envs
    full = scenes.scene_c3(n_envs=args.envs, n_steps=args.warmup + args.steps)
    w = [0] * args.envs
    for b in full.tets:
        w[b.env] += len(b.tets)
    a, b = shard_envs(w, world)[rank]
    return scenes.scene_c3(n_envs=b - a, n_steps=args.warmup + args.steps, seed0=1000 + a)


def oracle_steps_per_s(n_warm, n_steps, sc=None):
    """The CPU oracle, as it stands, on the same workload (single core)."""
    from oracle.oracle import Oracle
    sc = build_scene() if sc is None else sc
    o = Oracle(sc)
    if n_warm:
        o.step(n_warm)
    t0 = time.perf_counter()
    o.step(n_steps)
    dt = time.perf_counter() - t0
    return n_steps / dt, dt


def workload_name(args, sc, envs_per_rank):
    """The config's workload string (the same for both arms)."""
    if args.workload == "c2":
        return WORKLOAD
    if args.workload == "c5":
        return (f"dense soft-rigid pile: {sum(len(b.tets) for b in sc.tets)} tets in {len(sc.tets)} soft bodies "
                f"+ {sum(1 for a in sc.affines if a.mode == 0)} affine spheres/tori "
                f"({max(len(a.F) for a in sc.affines)} tris max) in a fixed 5-box bin, one scene")
    return (f"batched parallel-jaw grasp, {args.envs} envs (ellipsoid/torus/box, 2k-20k tets log-uniform, "
            f"E 1e4-1e6, mu 0.3-1.0), one launch per phase over all envs; {envs_per_rank} envs per rank")


def oracle_sample(args, n_warm, n_steps):
    """Time the CPU oracle, as it stands, on a bounded sample of the workload:
    returns (value in the workload's unit, seconds, description)."""
    from paper_2311_05945_b300 import scenes
    if args.workload == "c5":
        # the oracle's brute-force pair search is quadratic in the surface
        # size: one step of the full pile does not fit the sample bound, so
        # the sample is the same pile generator at 300 tets per body
        small = scenes.scene_c5(n_steps=2, tets_per_body=300, n_seg=8, bin_subdiv=1)
        v, dt = oracle_steps_per_s(0, 1, small)
        return v, dt, (f"step 0 of the same pile generator at 300 tets per body, 8 x 8 affine meshes, unsplit "
                       f"bin faces, on the CPU oracle ({dt:.1f} s)")
    if args.workload == "c3":
        v, dt = oracle_steps_per_s(0, 1, scenes.scene_c3(n_envs=1, n_steps=2))
        return v, dt, f"env 0 of the batch (seed 1000), step 0, on the CPU oracle ({dt:.1f} s)"
    v, dt = oracle_steps_per_s(n_warm, n_steps)
    return v, dt, (f"grasp steps [{n_warm}, {n_warm + n_steps}) of the same script on the CPU oracle "
                   f"({dt:.1f} s)")


def run_reference(args, rank):
    if rank != 0:
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    # the GPU arm times steps [W, W + K) of the grasp script: step the oracle
    # untimed to W (capped so that the run stays within a few minutes), then
    # time up to 3 steps of the same window
    n_warm = min(args.warmup, 40)
    n_steps = max(1, min(args.steps, 3))
    unit = "env-steps/s" if args.workload == "c3" else UNIT
    sc = None if args.workload == "c2" else build_scene(args, 0, world)
    name = workload_name(args, sc, sc.n_envs if sc is not None else 1)
    v, dt, sample = oracle_sample(args, n_warm, n_steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": unit, "n_gpus": args.gpus,
        "steps": n_steps if args.workload == "c2" else 1, "warmup": n_warm if args.workload == "c2" else 0,
        "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded generators)",
        "config": {"workload": name, "form": "CPU oracle: serial FP64, brute-force pairs, direct/CG solve"},
        "cpu_baseline": {"value": v, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def state_bytes(sc):
    return sum(8 * 6 * len(b.X) for b in sc.tets) + 8 * 24 * len(sc.affines)


def time_form(args, world, dist, precision, profile_kernel=None):
    """W warm-up steps, then K timed steps of the grasp script in one form."""
    import torch

    from paper_2311_05945_b300 import zema as Z

    rank = int(os.environ.get("RANK", "0"))
    sc = build_scene(args, rank, world)
    gpu = Z.Scene(sc, precision=precision)
    st = torch.cuda.current_stream()
    for k in range(args.warmup):
        if k == args.warmup - 1:
            gpu.autotune()  # the solve's CTAs per env, timed on a warm-up system
        gpu.step(1)
    torch.cuda.synchronize()
    # L2 flush buffer: 512 MB, written between timed steps (L2 is 126 MB)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if args.profile_region and profile_kernel:
        torch.cuda.profiler.start()
    if profile_kernel:
        Z.profile_kernel(profile_kernel)
    l0 = Z.launch_count()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(st)
        stats.append(gpu.step(1))
        ev[k][1].record(st)
    torch.cuda.synchronize()
    if args.profile_region and profile_kernel:
        torch.cuda.profiler.stop()
    launches = Z.launch_count() - l0
    prof = Z.profile_read() if profile_kernel else None
    Z.profile_kernel(None)
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    from paper_2311_05945_b300.sharding import max_over_ranks
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    gpu.tuned = gpu.tuning()
    return sc, gpu, total_ms, stats, launches, prof


def run_ours(args, rank, world):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # plain FP64 stepper over the same steps (the comparison form)
    _, _, plain_ms, plain_stats, _, _ = time_form(args, world, dist, 0)
    # headline: mixed precision + warm start; clocks sampled while it runs
    clocks = Clocks(local)
    clocks.start()
    sc, gpu, total_ms, stats, launches, prof = time_form(args, world, dist, 1,
                                                         ROOFLINE_KERNEL_BY_WORKLOAD[args.workload])
    clk = clocks.stop()
    from paper_2311_05945_b300.sharding import max_over_ranks
    envs_per_rank = sc.n_envs
    units = world * envs_per_rank if args.workload == "c3" else world
    value = units * args.steps / (total_ms / 1e3)
    plain_value = units * args.steps / (plain_ms / 1e3)
    # end to end through the C ABI with pinned host buffers, over the same
    # step window [W, W + K) of a fresh scene: every timed step uploads the
    # bodies' states from pinned host memory, steps, and reads them back
    from paper_2311_05945_b300 import zema as Z
    e2e_steps = args.steps if args.e2e_steps is None else max(1, min(args.steps, args.e2e_steps))
    g2 = Z.Scene(sc, precision=1)
    for _ in range(args.warmup):
        g2.step(1)
    bodies = list(range(len(sc.body_order())))
    host = [torch.from_numpy(g2.get_state(b)).pin_memory() for b in bodies]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for b in bodies:
            g2.set_state_ptr(b, host[b].data_ptr(), host[b].numel())
        g2.step(1)
        for b in bodies:
            g2.get_state_ptr(b, host[b].data_ptr(), host[b].numel())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = units * e2e_steps / max_over_ranks(e2e_s, dist, "cuda")
    g2.close()
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
        roof = {"kernel": ROOFLINE_KERNEL_BY_WORKLOAD[args.workload], "bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved / peak_gbs, "traffic": ROOFLINE_TRAFFIC.get(args.workload),
                "peak_source": "measured" if peaks else "fallback",
                "alg_bytes_per_launch": per_launch_bytes, "avg_launch_us": 1e3 * k_ms / k_launches,
                "launches": k_launches, "share_of_step_time": k_ms / total_ms if world == 1 else None}
    unit = "env-steps/s" if args.workload == "c3" else UNIT
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, dt, sample = oracle_sample(args, 0, args.cpu_steps)
        cpu = {"value": v, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample}
    agg = {k: sum(s[k] for s in stats) for k in ("newton_iters", "pcg_iters", "ls_halvings", "al_rounds", "pcg_refines")}
    phase = {k: sum(s["ms_phase"][k] for s in stats) for k in stats[0]["ms_phase"]}
    line = {
        "metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed f32/f64", "data": "synthetic (seeded generators)",
        "config": {"workload": workload_name(args, sc, envs_per_rank),
                   "timed_steps": [args.warmup, args.warmup + args.steps],
                   "form": "mixed precision (FP32 Hessians, matrices and PCG with FP64 residual refinement; FP64 "
                           "gradients/energies/distances/CCD/convergence) + CCD-filtered constant-velocity warm "
                           "start" + ("; all envs batched" if args.workload == "c3" else "; 1 env so no batching"),
                   "plain_fp64": {"value": plain_value, "ms_per_step": plain_ms / args.steps,
                                  "newton_iters": sum(s["newton_iters"] for s in plain_stats),
                                  "pcg_iters": sum(s["pcg_iters"] for s in plain_stats)},
                   "speedup_vs_plain": value / plain_value,
                   "parallelism": (f"envs sharded over {world} ranks" if args.workload == "c3" else f"replicas x{world}")
                   if world > 1 else "single GPU",
                   "l2": "flushed between timed steps (512 MB write)",
                   "newton_iters": agg["newton_iters"], "pcg_iters": agg["pcg_iters"],
                   "ls_halvings": agg["ls_halvings"], "al_rounds": agg["al_rounds"],
                   "pcg_fp64_refinements": agg["pcg_refines"],
                   "pcg_autotune": {"ctas_per_env": gpu.tuned[0],
                                    "solve_ms_by_ctas": {str(k): round(v, 4) for k, v in gpu.tuned[1].items()}},
                   "host_phase_ms": {k: round(v, 2) for k, v in phase.items()}},
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
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c5"],
                    help="c2: the single-env grasp (headline); c3: the batched grasp, env-steps/s; "
                         "c5: the dense soft-rigid pile")
    ap.add_argument("--c5-tets", type=int, default=60000, help="tets per soft body of the pile (c5)")
    ap.add_argument("--envs", type=int, default=256, help="envs of the batched grasp (c3)")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end steps (default: the timed steps, same window)")
    ap.add_argument("--cpu-steps", type=int, default=2)
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
