"""Runtime of the stepper over rigid-mesh resolution (the paper's Table IV
experiment, with seeded synthetic remeshings): the same scene (an affine
sphere dropped on a soft box on a fixed floor) with the sphere's UV mesh at
652 ... 77,564 vertices.  The system's DOF are the same at every resolution
(the sphere is one affine body, 12 DOF); only the contact primitives grow.

    python -m paper_2311_05945_b300.resolution [--steps 60] [--out file.json]
"""
import argparse
import json
import time


def run(n_seg, steps, precision):
    import torch

    from . import scenes as S
    from . import zema as Z
    sc = S.scene_resolution(n_seg, n_steps=steps, precision=precision)
    g = Z.Scene(sc, precision=precision)
    c = g.counts()
    tot = {"newton_iters": 0, "pcg_iters": 0, "max_active": 0}
    dmin = float("inf")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        st = g.step(1)
        tot["newton_iters"] += st["newton_iters"]
        tot["pcg_iters"] += st["pcg_iters"]
        tot["max_active"] = max(tot["max_active"], st["max_active"])
        dmin = min(dmin, st["dmin"])
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    V, F = sc.affines[1].V, sc.affines[1].F
    dof = 3 * len(sc.tets[0].X) + 12
    g.close()
    return {"n_seg": n_seg, "sphere_vertices": len(V), "sphere_triangles": len(F), "dof": dof,
            "surface_triangles": c.get("n_tris"), "steps": steps, "seconds": secs, "ms_per_step": 1e3 * secs / steps,
            "min_distance": dmin, **tot}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from . import scenes as S
    rows = [run(n, args.steps, args.precision) for n in S.RESOLUTION_SEGMENTS]
    for r in rows:
        print(json.dumps(r), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
