"""Spatial-hash broad phase: candidate sets bit-exact against the oracle's
brute force over all pairs (static and swept boxes, several envs, oversize
primitives, empty input)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def raw_surface(seed, n_soft=3, n_aff=2, jitter=0.003, envs=1):
    """Surface of a random multi-body scene with seeded perturbations."""
    s = S.random_state_scene(seed, n_soft, n_aff)
    o = __import__("oracle.oracle", fromlist=["Oracle"]).Oracle(s)
    sv, e, t = o.surface()
    soft = np.concatenate([o.tet_positions(i) for i in range(len(s.tets))])
    P = np.zeros((len(sv), 3))
    for i, (b, aff, idx) in enumerate(sv):
        kind, k = s.body_order()[b]
        if kind == "tet":
            P[i] = soft[idx]
        else:
            q = o.get_state(b)[:12]
            P[i] = q[3:].reshape(3, 3) @ s.affines[k].V[idx] + q[:3]
    P += jitter * np.random.default_rng(seed).standard_normal(P.shape)
    order = s.body_order()
    bclass = np.array([0 if k == "tet" else 1 for k, i in order], dtype=np.int32)
    benv = (np.arange(len(order)) % envs).astype(np.int32)
    return P, sv[:, 0].copy(), bclass, benv, e, t


def as_sets(pt, ee, tris, edges):
    return set(map(tuple, pt)), set(map(tuple, ee))


def oracle_sets(P, svb, bc, be, e, t, infl, P1=None):
    pt, ee = O.brute_pairs(P, svb, bc, be, e, t, infl, pos1=P1)
    tri_index = {tuple(x): i for i, x in enumerate(t)}
    edge_index = {tuple(x): i for i, x in enumerate(e)}
    spt = set((int(a[0]), tri_index[tuple(a[1:])]) for a in pt)
    see = set((edge_index[(a[0], a[1])], edge_index[(a[2], a[3])]) for a in ee)
    return spt, see


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("infl", [0.0005, 0.02, 0.08])
def test_static_candidates_bit_exact(seed, infl):
    from paper_2311_05945_b300 import zema as Z
    P, svb, bc, be, e, t = raw_surface(seed)
    pt, ee = Z.candidates_raw(P, svb, bc, be, e, t, infl)
    spt, see = oracle_sets(P, svb, bc, be, e, t, infl)
    assert set(map(tuple, pt)) == spt and len(pt) == len(spt)
    assert set(map(tuple, ee)) == see and len(ee) == len(see)
    assert len(spt) > 0


@pytest.mark.parametrize("seed", [4, 5])
def test_swept_candidates_bit_exact(seed):
    from paper_2311_05945_b300 import zema as Z
    P, svb, bc, be, e, t = raw_surface(seed)
    rng = np.random.default_rng(seed + 100)
    P1 = P + 0.03 * rng.standard_normal(P.shape)
    # a few long moves make oversize swept boxes
    P1[::37] += 0.5 * rng.standard_normal(P1[::37].shape)
    pt, ee = Z.candidates_raw(P, svb, bc, be, e, t, 0.0005, pos1=P1)
    spt, see = oracle_sets(P, svb, bc, be, e, t, 0.0005, P1=P1)
    assert set(map(tuple, pt)) == spt and len(pt) == len(spt)
    assert set(map(tuple, ee)) == see and len(ee) == len(see)


def test_env_and_class_filters():
    from paper_2311_05945_b300 import zema as Z
    P, svb, bc, be, e, t = raw_surface(6, envs=2)
    bc = bc.copy()
    bc[-1] = 2  # fixed
    bc[-2] = 3  # kinematic
    pt, ee = Z.candidates_raw(P, svb, bc, be, e, t, 0.05)
    spt, see = oracle_sets(P, svb, bc, be, e, t, 0.05)
    assert set(map(tuple, pt)) == spt and set(map(tuple, ee)) == see


def test_small_cell_size_many_cells():
    from paper_2311_05945_b300 import zema as Z
    P, svb, bc, be, e, t = raw_surface(7)
    # tiny cells: most triangles become oversize and go through the direct list
    pt, ee = Z.candidates_raw(P, svb, bc, be, e, t, 0.01, cell_size=0.002)
    spt, see = oracle_sets(P, svb, bc, be, e, t, 0.01)
    assert set(map(tuple, pt)) == spt and set(map(tuple, ee)) == see


def test_empty_and_deterministic():
    from paper_2311_05945_b300 import zema as Z
    P, svb, bc, be, e, t = raw_surface(8)
    far = P.copy()
    far[: len(P) // 2] += 100.0
    a = Z.candidates_raw(P, svb, bc, be, e, t, 0.01)
    b = Z.candidates_raw(P, svb, bc, be, e, t, 0.01)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])  # same order, run to run
    pt, ee = Z.candidates_raw(P[:0], svb[:0], bc, be, e[:0], t[:0], 0.01)
    assert len(pt) == 0 and len(ee) == 0


def scene_surface(s):
    """Surface positions and connectivity of a scene's initial state."""
    o = __import__("oracle.oracle", fromlist=["Oracle"]).Oracle(s)
    sv, e, t = o.surface()
    soft = np.concatenate([o.tet_positions(i) for i in range(len(s.tets))])
    P = np.zeros((len(sv), 3))
    for i, (b, aff, idx) in enumerate(sv):
        kind, k = s.body_order()[b]
        if kind == "tet":
            P[i] = soft[idx]
        else:
            q = o.get_state(b)[:12]
            P[i] = q[3:].reshape(3, 3) @ s.affines[k].V[idx] + q[:3]
    order = s.body_order()
    bclass = np.array([0 if k == "tet" else 1 + s.affines[i].mode for k, i in order], dtype=np.int32)
    benv = np.array([s.tets[i].env if k == "tet" else s.affines[i].env for k, i in order], dtype=np.int32)
    return P, sv[:, 0].copy(), bclass, benv, e, t


@pytest.mark.parametrize("name", ["c2", "c3x4", "mixed_scale"])
def test_large_surfaces_bit_exact(name):
    # ~10k primitives (the grasp: counts and flags scanned by the single-CTA
    # scan), ~40k (four batched envs: the multi-block scan), and a 1 cm soft
    # box under a finely meshed sphere, where the grid cell follows the
    # sphere's 1.5 mm edges and the box's edges become oversize queries that
    # walk the grid cells
    from paper_2311_05945_b300 import zema as Z
    if name == "c2":
        s = S.scene_c2()
    elif name == "c3x4":
        s = S.scene_c3(n_envs=4, n_steps=1)
    else:
        s = S.scene_resolution(105, n_steps=1)
    P, svb, bc, be, e, t = scene_surface(s)
    n_prims = len(t) + len(e)
    assert (4096 < n_prims <= 32768) if name == "c2" else n_prims > 32768
    for infl in (1e-3, 4e-3):
        pt, ee = Z.candidates_raw(P, svb, bc, be, e, t, infl)
        spt, see = oracle_sets(P, svb, bc, be, e, t, infl)
        assert set(map(tuple, pt)) == spt and len(pt) == len(spt)
        assert set(map(tuple, ee)) == see and len(ee) == len(see)
    assert len(spt) > 0
