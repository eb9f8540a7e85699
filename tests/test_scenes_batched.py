"""The grasp generators on the CPU.

The batched grasp (C3) against its recipe: per env a seeded object kind, a
tet count log-uniform in [2k, 20k], E log-uniform in [1e4, 1e6] Pa, mu
uniform in [0.3, 1], nu = 0.45, two kinematic fingers of 972 triangles and a
fixed floor, envs 0.5 m apart and spatially disjoint.  A range of envs built
on its own (seed and slot advanced together) is the same, array for array
and target for target, as that range of the whole batch: this is what lets
ranks step disjoint env ranges of one batch.

The single-env grasp (C2) against its recipe and its finger script, which
brings both fingers to the object at the 20th step."""
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


def test_c2_grasp_recipe_and_script():
    # one env: a 4 / 2 / 3 cm ellipsoid lattice of 9,600 tets (E = 5e4, nu =
    # 0.45) 0.5 dhat above a fixed floor, two kinematic 6 x 3 x 1 cm fingers
    # of 972 triangles 0.5 cm off its z extremes; mu = 0.8, h = 5 ms
    sc = S.scene_c2(n_steps=300)
    p = sc.params
    assert (p.dt, p.dhat) == (0.005, 1e-3)
    (b,) = sc.tets
    assert len(b.tets) == 9600 and (b.E, b.nu, b.mu) == (5e4, 0.45, 0.8)
    ext = b.X.max(0) - b.X.min(0)
    assert np.all(np.abs(ext - (0.08, 0.04, 0.06)) <= 2 * 0.004), ext
    floor = [a for a in sc.affines if a.mode == 1]
    fingers = [a for a in sc.affines if a.mode == 2]
    assert len(floor) == 1 and len(fingers) == 2
    top = floor[0].q0[1] + floor[0].V[:, 1].max()
    assert abs(b.X[:, 1].min() - top - 0.5 * p.dhat) < 1e-15
    zmax, zmin = b.X[:, 2].max(), b.X[:, 2].min()
    for a in fingers:
        assert len(a.F) == 972 and a.mu == 0.8
        fe = a.V.max(0) - a.V.min(0)
        assert np.allclose(fe, (0.06, 0.03, 0.01))
        inner = a.q0[2] + (a.V[:, 2].min() if a.q0[2] > 0 else a.V[:, 2].max())
        assert abs(abs(inner - (zmax if a.q0[2] > 0 else zmin)) - 0.005) < 1e-12
    # script: close at 5 cm/s for 40 steps, hold 60, lift 5 cm over 200;
    # arrays(n) are the targets of the state after step n
    idx, Q0 = sc.script.arrays(-1)
    fing = {i: sign for i, sign, _ in sc.fingers}
    for n, closed, lifted in ((0, 0.00025, 0.0), (19, 0.005, 0.0), (39, 0.01, 0.0), (99, 0.01, 0.0),
                              (199, 0.01, 0.025), (299, 0.01, 0.05)):
        _, Q = sc.script.arrays(n)
        for j, i in enumerate(idx):
            assert abs(-(Q[j, 2] - Q0[j, 2]) * fing[int(i)] - closed) < 1e-15, (n, closed)
            assert abs(Q[j, 1] - Q0[j, 1] - lifted) < 1e-15
    # both fingers reach the object's extremes at the 20th step: the start of
    # the contact window the benchmark times
    _, Q = sc.script.arrays(19)
    for j, i in enumerate(idx):
        a = sc.affines[int(i)]
        inner = Q[j, 2] + (a.V[:, 2].min() if fing[int(i)] > 0 else a.V[:, 2].max())
        assert abs(inner - (zmax if fing[int(i)] > 0 else zmin)) < 1e-12
