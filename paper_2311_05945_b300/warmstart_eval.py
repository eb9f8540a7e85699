"""Evaluate the learned Newton warm start on held-out environments.

Steps the batched grasp scene with held-out seeds (from 100000) twice, with
the constant-velocity proposal and with the learned one, at the same Newton
tolerance, and reports Newton and PCG iterations, accepted proposals and
time.  Both runs converge every step to the same tolerance; only the start
of Newton differs.

    python -m paper_2311_05945_b300.warmstart_eval --weights weights/warmstart.bin
"""
import argparse
import json
import time


def run(scene, steps, warm_start, blob):
    import torch

    from . import zema as Z
    g = Z.Scene(scene, warm_start=warm_start)
    if warm_start:
        dims, theta = Z.read_warmstart_blob(blob)
        g.load_warmstart(dims, theta)
    tot = {"newton_iters": 0, "pcg_iters": 0, "warm_accepted": 0, "warm_learned": 0, "warm_fallback": 0,
           "ls_halvings": 0}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        st = g.step(1)
        for k in tot:
            tot[k] += st[k]
    torch.cuda.synchronize()
    tot["seconds"] = time.perf_counter() - t0
    tot["steps_per_s"] = steps / tot["seconds"]
    pos = [g.tet_positions(i).copy() for i in range(len(scene.tets))]
    g.close()
    return tot, pos


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--weights", required=True)
    ap.add_argument("--envs", type=int, default=64)
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--seed0", type=int, default=100000)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import numpy as np

    from . import scenes as S
    blob = open(args.weights, "rb").read()
    sc = S.scene_c3(n_envs=args.envs, n_steps=args.steps, seed0=args.seed0)
    base, p0 = run(sc, args.steps, 0, blob)
    learned, p1 = run(sc, args.steps, 1, blob)
    diff = max(float(np.abs(a - b).max()) for a, b in zip(p0, p1))
    rep = {"envs": args.envs, "steps": args.steps, "seed0": args.seed0, "constant_velocity": base,
           "learned": learned, "newton_ratio": learned["newton_iters"] / max(1, base["newton_iters"]),
           "max_position_difference_m": diff}
    print(json.dumps(rep))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
