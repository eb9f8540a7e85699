"""Host checks of the dense soft-rigid pile generator: closed, outward
meshes whose enclosed volumes match the closed forms of an ellipsoid and a
torus (up to the polyhedral error), the triangle counts of 32 x 32 meshes,
positively oriented tets, and bodies that start in disjoint slots inside the
bin."""
import math
from collections import Counter

import numpy as np

from paper_2311_05945_b300 import scenes as S


def signed_volume(V, F):
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def closed_and_consistent(F):
    # every directed edge appears once and its reverse once
    e = Counter()
    for t in F:
        for i in range(3):
            e[(int(t[i]), int(t[(i + 1) % 3]))] += 1
    return all(c == 1 and e[(b, a)] == 1 for (a, b), c in e.items())


def test_uv_sphere_mesh():
    V, F = S.uv_sphere_surface((0.1, 0.08, 0.06), 32, 32)
    assert len(F) == 1984 and len(V) == 994
    assert closed_and_consistent(F)
    vol = signed_volume(V, F)
    exact = 4.0 / 3.0 * math.pi * 0.1 * 0.08 * 0.06
    assert 0.98 * exact < vol < exact  # inscribed polyhedron: positive (outward) and slightly smaller


def test_torus_mesh():
    V, F = S.torus_surface(0.07, 0.025, 32, 32)
    assert len(F) == 2048 and len(V) == 1024
    assert closed_and_consistent(F)
    vol = signed_volume(V, F)
    exact = 2.0 * math.pi ** 2 * 0.07 * 0.025 ** 2
    assert 0.97 * exact < vol < exact


def test_rotation_from_uniforms():
    for u in ((0.1, 0.2, 0.3), (0.9, 0.5, 0.01), (0.5, 0.5, 0.5)):
        R = S.rotation_from_uniforms(*u)
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(R) - 1.0) < 1e-14


def test_pile_layout_small():
    sc = S.scene_c5(n_steps=2, tets_per_body=300, n_soft=3, n_convex=2, n_nonconvex=2, n_seg=8)
    assert len(sc.tets) == 3 and len(sc.affines) == 5 + 4
    assert sum(a.mode == 1 for a in sc.affines) == 5  # the bin
    boxes = []
    for b in sc.tets:
        a, b1, c, d = (b.X[b.tets[:, k]] for k in range(4))
        J = np.einsum("ij,ij->i", np.cross(b1 - a, c - a), d - a)
        assert (J > 0).all()
        boxes.append((b.X.min(0), b.X.max(0)))
    for a in sc.affines[5:]:
        A = a.q0[3:].reshape(3, 3)
        assert np.abs(A @ A.T - np.eye(3)).max() < 1e-12
        X = a.V @ A.T + a.q0[:3]
        boxes.append((X.min(0), X.max(0)))
    for lo, hi in boxes:
        # inside the bin's inner walls and above its floor (top at y = 0)
        assert lo[0] > -0.5 and hi[0] < 0.5 and lo[2] > -0.5 and hi[2] < 0.5 and lo[1] > 0.0
    for i in range(len(boxes)):
        for j in range(i + 1, len(boxes)):
            (l1, h1), (l2, h2) = boxes[i], boxes[j]
            assert (h1 < l2).any() or (h2 < l1).any(), (i, j)


def test_pile_full_size_counts():
    # the generator's sizes at the full configuration, without building meshes
    # of the soft bodies: lattice spacing solved for ~60k tets per body
    for kind in ("ellipsoid", "torus", "box"):
        sp = S._spacing_for_count(kind, 60000, 2.5, hi=0.1)
        m, _ = S._solid(kind, 2.5, sp)
        assert 0.95 * 60000 < 6 * int(m.sum()) < 1.05 * 60000


def test_grasp_script_arrays_match_per_finger_targets():
    """The grasp script's all-fingers form gives the per-finger targets bit
    for bit at every phase (closing, holding, lifting)."""
    import numpy as np

    from paper_2311_05945_b300 import scenes as S
    sc = S.scene_c3(n_envs=3, n_steps=8, min_tets=300, max_tets=400)
    for step in (0, 5, 39, 40, 99, 100, 150, 299, 400):
        d = sc.script(step)
        idx, Q = sc.script.arrays(step)
        assert list(idx) == list(d.keys())
        assert np.array_equal(Q, np.array([d[i] for i in idx]))
