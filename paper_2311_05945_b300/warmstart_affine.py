"""Train and evaluate the per-body learned warm start of the affine bodies.

Data: small seeded piles from the dense-pile generator (soft lattice bodies
of ~2k tets, 16 x 16 UV spheres and tori as dynamic affine bodies, the fixed
bin), stepped with the default constant-velocity warm start; every step
records each dynamic affine body's 40 features at the step's start and its
change of q beyond h qdot^t (zema_record_warmstart_affine).  Training: the
library's tensor-core MLP (40 -> 128 -> 128 -> 128 -> 12), mean squared
error, AdamW with cosine learning-rate decay.  Evaluation: held-out piles
(seeds from 100000) stepped with the constant-velocity start and with the
learned one at the same Newton tolerance.

    python -m paper_2311_05945_b300.warmstart_affine --out weights/warmstart_affine.bin
"""
import argparse
import json
import math
import os
import time

import numpy as np

DIMS = [40, 128, 128, 128, 12]


def pile(seed, steps):
    from . import scenes as S
    return S.scene_c5(n_steps=steps, tets_per_body=2000, n_soft=4, n_convex=6, n_nonconvex=6, n_seg=16,
                      seed=seed, bin_subdiv=2)


def n_dynamic_affine(scene):
    return sum(1 for a in scene.affines if a.mode == 0)


def collect(scene, steps, log):
    import torch

    from . import zema as Z
    g = Z.Scene(scene)
    rows = n_dynamic_affine(scene)
    fb = torch.empty((rows, 40), dtype=torch.float32, device="cuda")
    tb = torch.empty((rows, 12), dtype=torch.float32, device="cuda")
    g.record_warmstart_affine(fb, tb)
    feats, targs = [], []
    newton = 0
    for _ in range(steps):
        st = g.step(1)
        newton += st["newton_iters"]
        feats.append(fb.clone())
        targs.append(tb.clone())
    g.record_warmstart_affine(None)
    g.close()
    log(f"  seed {scene.name}: {steps} steps x {rows} bodies, {newton} Newton iterations")
    return torch.cat(feats), torch.cat(targs)


def run(scene, steps, blob):
    """Step with the constant-velocity start (blob None) or the learned one."""
    import torch

    from . import zema as Z
    g = Z.Scene(scene, warm_start=1 if blob is not None else 0)
    if blob is not None:
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
    g.close()
    return tot


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--piles", type=int, default=40, help="training piles (seeds 1000...)")
    ap.add_argument("--steps", type=int, default=80)
    ap.add_argument("--iters", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--wd", type=float, default=1e-4, help="AdamW weight decay")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--eval-piles", type=int, default=3, help="held-out piles (seeds 100000...)")
    ap.add_argument("--eval-steps", type=int, default=60)
    args = ap.parse_args()
    import torch

    from . import zema as Z
    t0 = time.time()
    report = {"dims": DIMS, "args": vars(args)}

    def log(m):
        print(m, flush=True)

    log("collecting trajectories")
    parts = [collect(pile(1000 + i, args.steps), args.steps, log) for i in range(args.piles)]
    X = torch.cat([p[0] for p in parts]).contiguous()
    Y = torch.cat([p[1] for p in parts]).contiguous()
    ok = torch.isfinite(X).all(1) & torch.isfinite(Y).all(1)
    X, Y = X[ok].contiguous(), Y[ok].contiguous()
    n = X.shape[0]
    report["rows"] = int(n)
    report["collect_s"] = time.time() - t0
    log(f"{n} rows in {report['collect_s']:.1f} s")
    net = Z.Mlp(DIMS, seed=args.seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed)
    losses = []
    t1 = time.time()
    for it in range(args.iters):
        idx = torch.randint(0, n, (min(args.batch, n),), device="cuda", generator=gen)
        lr = args.lr * 0.5 * (1.0 + math.cos(math.pi * it / args.iters))
        losses.append(net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr=lr, weight_decay=args.wd))
        if it % 250 == 0 or it == args.iters - 1:
            log(f"  iter {it}: loss {losses[-1]:.5f}")
    report["train_s"] = time.time() - t1
    report["loss_first"], report["loss_last"] = losses[0], float(np.mean(losses[-50:]))
    report["loss_constant_velocity"] = float((Y ** 2).mean())
    theta = net.get_params()
    blob = Z.warmstart_blob(DIMS, theta)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    blob.tofile(args.out)
    # held-out piles: constant velocity vs learned, same tolerance
    ev = []
    for i in range(args.eval_piles):
        sc = pile(100000 + i, args.eval_steps)
        Xe, Ye = collect(pile(100000 + i, args.eval_steps), args.eval_steps, log)
        pred = net.forward(Xe.contiguous())
        base = run(sc, args.eval_steps, None)
        learned = run(sc, args.eval_steps, blob.tobytes())
        ev.append({"seed": 100000 + i, "mse_learned": float(((pred - Ye) ** 2).mean()),
                   "mse_constant_velocity": float((Ye ** 2).mean()), "constant_velocity": base, "learned": learned,
                   "newton_ratio": learned["newton_iters"] / max(1, base["newton_iters"])})
        log(json.dumps(ev[-1]))
    report["eval"] = ev
    if ev:
        report["eval_newton_ratio"] = (sum(e["learned"]["newton_iters"] for e in ev) /
                                       max(1, sum(e["constant_velocity"]["newton_iters"] for e in ev)))
        report["eval_mse_ratio"] = (sum(e["mse_learned"] for e in ev) /
                                    max(1e-30, sum(e["mse_constant_velocity"] for e in ev)))
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(report, f, indent=1)
    log(json.dumps({k: v for k, v in report.items() if k not in ("args", "eval")}))


if __name__ == "__main__":
    main()
