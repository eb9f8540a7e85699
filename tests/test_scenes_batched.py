"""The batched grasp generator (C3) against its recipe, on the CPU: per env a
seeded object kind, a tet count log-uniform in [2k, 20k], E log-uniform in
[1e4, 1e6] Pa, mu uniform in [0.3, 1], nu = 0.45, two kinematic fingers of
972 triangles and a fixed floor, envs 0.5 m apart and spatially disjoint.
A range of envs built on its own (seed and slot advanced together) is the
same, array for array and target for target, as that range of the whole
batch: this is what lets ranks step disjoint env ranges of one batch."""
import math

import numpy as np

from paper_2311_05945_b300 import scenes as S


def _env_bodies(sc, e):
    tets = [b for b in sc.tets if b.env == e]
    affs = [a for a in sc.affines if a.env == e]
    return tets, affs


def _bbox(sc, e):
    tets, affs = _env_bodies(sc, e)
    pts = [b.X if b.x0 is None else b.x0 for b in tets]
    for a in affs:
        A = a.q0[3:].reshape(3, 3)
        pts.append(a.V @ A.T + a.q0[:3])
    P = np.vstack(pts)
    return P.min(0), P.max(0)


def test_c3_recipe_over_64_envs():
    n = 64
    sc = S.scene_c3(n_envs=n, n_steps=4)
    assert sc.n_envs == n and sc.params.dt == 0.005 and sc.params.newton_tol_rel == 1e-3
    nt, kinds = [], set()
    for e in range(n):
        tets, affs = _env_bodies(sc, e)
        assert len(tets) == 1
        b = tets[0]
        nt.append(len(b.tets))
        kinds.add(b.name.rstrip("0123456789"))
        assert 1e4 <= b.E <= 1e6 and 0.3 <= b.mu <= 1.0 and b.nu == 0.45
        modes = sorted((a.mode, len(a.F)) for a in affs)
        assert modes == [(1, 12), (2, 972), (2, 972)], modes
    assert kinds == {"ellipsoid", "torus", "box"}
    nt = np.array(nt)
    # the lattice realises the drawn count to within a few per cent
    assert nt.min() >= 0.9 * 2000 and nt.max() <= 1.05 * 20000
    # log-uniform: the mean of log(count) near the interval's midpoint, and
    # every quarter of the log interval populated
    lo, hi = math.log(2000), math.log(20000)
    z = (np.log(nt) - lo) / (hi - lo)
    assert abs(z.mean() - 0.5) < 0.12
    assert all(np.any((z >= q / 4) & (z < (q + 1) / 4)) for q in range(4))
    # envs 0.5 m apart along x and spatially disjoint (gap well above dhat)
    boxes = [_bbox(sc, e) for e in range(n)]
    for e in range(n - 1):
        assert boxes[e + 1][0][0] - boxes[e][1][0] > 0.1


def test_c3_env_range_equals_that_range_of_the_whole_batch():
    kw = dict(n_steps=60, min_tets=300, max_tets=600)
    full = S.scene_c3(n_envs=6, seed0=1000, **kw)
    part = S.scene_c3(n_envs=2, seed0=1003, slot0=3, **kw)
    for i in range(2):
        (tf,), af = _env_bodies(full, 3 + i)
        (tp,), ap = _env_bodies(part, i)
        for k in ("X", "tets", "x0", "v0"):
            assert np.array_equal(getattr(tf, k), getattr(tp, k)), k
        assert (tf.E, tf.nu, tf.rho, tf.mu) == (tp.E, tp.nu, tp.rho, tp.mu)
        assert tf.name.rstrip("0123456789") == tp.name.rstrip("0123456789")
        assert len(af) == len(ap)
        for a, b in zip(af, ap):
            for k in ("V", "F", "q0", "qdot0"):
                assert np.array_equal(getattr(a, k), getattr(b, k)), k
            assert (a.mode, a.rho, a.stiffness, a.mu) == (b.mode, b.rho, b.stiffness, b.mu)
    # the kinematic script moves the range's fingers exactly as in the batch
    aff_of_env_full = {e: [j for j, a in enumerate(full.affines) if a.env == e] for e in range(6)}
    aff_of_env_part = {e: [j for j, a in enumerate(part.affines) if a.env == e] for e in range(2)}
    for step in (0, 10, 39, 40, 59):
        idx_f, Q_f = full.script.arrays(step)
        idx_p, Q_p = part.script.arrays(step)
        tf = {int(j): q for j, q in zip(idx_f, Q_f)}
        tp = {int(j): q for j, q in zip(idx_p, Q_p)}
        for i in range(2):
            for jf, jp in zip(aff_of_env_full[3 + i], aff_of_env_part[i]):
                assert (jf in tf) == (jp in tp)
                if jf in tf:
                    assert np.array_equal(tf[jf], tp[jp]), (step, i)
