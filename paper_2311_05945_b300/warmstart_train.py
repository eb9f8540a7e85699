"""Train the learned Newton warm start on trajectories the stepper generates.

Data: the batched grasp scene (training seeds 1000-1255 by default: 256 envs
x 200 steps, the 50k env-steps of the learned-warm-start configuration) and
the single-env grasp, stepped with the default constant-velocity warm start;
every step
records each soft vertex's 13 features at the step's start and its
displacement over the step beyond h v^t (both scaled by h^2 |g|).  Training: the
library's tensor-core MLP (13 -> 128 -> 128 -> 128 -> 3), mean squared error,
AdamW with cosine learning-rate decay, minibatches drawn with a seeded
generator.  Writes the warm-start blob read by zema_load_warmstart and a
JSON report next to it.

    python -m paper_2311_05945_b300.warmstart_train --out weights/warmstart.bin
"""
import argparse
import json
import math
import os
import time

import numpy as np

DIMS = [13, 128, 128, 128, 3]


def collect(scene, steps, log):
    """Step `scene` for `steps` steps recording features and targets."""
    import torch

    from . import zema as Z
    g = Z.Scene(scene)
    rows = g.counts()["n_verts"]
    fb = torch.empty((rows, 13), dtype=torch.float32, device="cuda")
    tb = torch.empty((rows, 3), dtype=torch.float32, device="cuda")
    g.record_warmstart(fb, tb)
    feats, targs = [], []
    newton = 0
    for k in range(steps):
        st = g.step(1)
        newton += st["newton_iters"]
        feats.append(fb.clone())
        targs.append(tb.clone())
    g.record_warmstart(None)
    g.close()
    log(f"  {scene.name}: {steps} steps x {rows} soft vertices, {newton} Newton iterations")
    return torch.cat(feats), torch.cat(targs)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--envs", type=int, default=256, help="training envs of the batched grasp (seeds 1000...)")
    ap.add_argument("--steps", type=int, default=200, help="recorded steps per scene")
    ap.add_argument("--c2-steps", type=int, default=300)
    ap.add_argument("--iters", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=7)
    args = ap.parse_args()
    import torch

    from . import scenes as S
    from . import zema as Z
    t0 = time.time()
    report = {"dims": DIMS, "args": vars(args)}

    def log(m):
        print(m, flush=True)

    log("collecting trajectories")
    c3 = S.scene_c3(n_envs=args.envs, n_steps=args.steps)
    # a few of the 256 envs need more than 100 Newton iterations in some
    # lift step (stiff objects held by friction alone); the cap of the dense
    # pile applies
    c3.params.max_newton = 1000
    parts = [collect(c3, args.steps, log)]
    if args.c2_steps:
        parts.append(collect(S.scene_c2(n_steps=args.c2_steps), args.c2_steps, log))
    report["env_steps"] = args.envs * args.steps + args.c2_steps
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
        loss = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr=lr, weight_decay=1e-5)
        losses.append(loss)
        if it % 250 == 0 or it == args.iters - 1:
            log(f"  iter {it}: loss {loss:.5f}")
    report["train_s"] = time.time() - t1
    report["loss_first"], report["loss_last"] = losses[0], float(np.mean(losses[-50:]))
    # baseline: the constant-velocity proposal (a zero residual)
    with torch.no_grad():
        cv = float((Y ** 2).mean())
    report["loss_constant_velocity"] = cv
    theta = net.get_params()
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    Z.warmstart_blob(DIMS, theta).tofile(args.out)
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(report, f, indent=1)
    log(json.dumps({k: v for k, v in report.items() if k != "args"}))


if __name__ == "__main__":
    main()
