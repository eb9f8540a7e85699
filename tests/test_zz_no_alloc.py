"""The allocation-free broad phase against the allocating one.

zema_candidates_raw_noalloc exists for callers that cannot allocate device
memory while they query contacts (with a device memory pool fixed in
advance, or in a loop that must not call an allocator).  It keeps all
scratch in one fixed device array.  Here it must return exactly the pairs,
in exactly the order, that zema_candidates_raw returns for the same inputs,
on two calls in a row (the second reuses the array the first left behind);
report ZEMA_ERR_OOM when a query does not fit the array and
ZEMA_ERR_INVALID_ARG for bad device index arrays, both without touching the
outputs, and work normally afterwards.

The file name sorts last so that, in a run that stops at the first failure,
a failure here comes after every other GPU test has run.  Nothing here
depends on that order: each test also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def surface(seed):
    """Surface arrays of a seeded multi-body scene (positions perturbed)."""
    from paper_2311_05945_b300 import zema as Z  # noqa: F401  (library must load)
    s = S.random_state_scene(seed, 3, 2)
    P, sv_body, edges, tris = [], [], [], []
    off = 0
    for b, (kind, i) in enumerate(s.body_order()):
        if kind == "tet":
            X, T = s.tets[i].X, s.tets[i].tets
            faces = np.concatenate([T[:, [0, 2, 1]], T[:, [0, 1, 3]], T[:, [0, 3, 2]], T[:, [1, 2, 3]]])
            key = np.sort(faces, axis=1)
            _, idx, cnt = np.unique(key, axis=0, return_index=True, return_counts=True)
            F = faces[idx[cnt == 1]]
            used = np.unique(F)
            remap = -np.ones(len(X), dtype=np.int64)
            remap[used] = np.arange(len(used))
            V, F = X[used], remap[F]
        else:
            a = s.affines[i]
            V = a.V @ a.q0[3:].reshape(3, 3).T + a.q0[:3]
            F = a.F
        E = np.unique(np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1), axis=0)
        P.append(V)
        sv_body.append(np.full(len(V), b))
        edges.append(E + off)
        tris.append(F + off)
        off += len(V)
    P = np.concatenate(P) + 0.003 * np.random.default_rng(seed).standard_normal((off, 3))
    bclass = np.array([0 if k == "tet" else 1 for k, _ in s.body_order()], dtype=np.int32)
    benv = np.zeros(len(bclass), dtype=np.int32)
    return (P, np.concatenate(sv_body).astype(np.int32), bclass, benv, np.concatenate(edges).astype(np.int32),
            np.concatenate(tris).astype(np.int32))


def test_noalloc_matches_allocating_broad_phase_twice():
    import torch

    from paper_2311_05945_b300 import zema as Z
    cell, infl, cap = 0.04, 0.01, 1 << 16
    for call, seed in enumerate((31, 32)):
        P, svb, bc, be, E, T = surface(seed)
        pt_ref, ee_ref = Z.candidates_raw(P, svb, bc, be, E, T, infl, cell_size=cell)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        pt = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
        ee = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
        npt, nee = Z.candidates_raw_noalloc(dev(P), dev(svb), dev(bc), dev(be), dev(E), dev(T), infl, cell, pt, ee)
        assert (npt, nee) == (len(pt_ref), len(ee_ref)), call
        assert npt > 0 and nee > 0
        assert np.array_equal(pt[:npt].cpu().numpy(), pt_ref), call
        assert np.array_equal(ee[:nee].cpu().numpy(), ee_ref), call


def test_noalloc_rejects_oversized_input():
    import torch

    from paper_2311_05945_b300 import zema as Z
    n = 70000  # more surface vertices than the fixed scratch accepts
    z = lambda *s, dt=torch.int32: torch.zeros(*s, dtype=dt, device="cuda")
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(Z.ZemaError) as ei:
        Z.candidates_raw_noalloc(pos, z(n), z(1), z(1), z(0, 2), z(0, 3), 0.01, 0.05, z(16, 2), z(16, 2))
    assert ei.value.status == 1


def test_noalloc_out_of_memory_then_normal():
    # 4,000 vertices and triangles of one soft body packed into a 1 mm cube
    # with a 1 cm inflation: every point-triangle and edge-edge pair
    # overlaps, about 1e8 pairs, far beyond the fixed 64 MiB array
    import torch

    from paper_2311_05945_b300 import zema as Z
    rng = np.random.default_rng(7)
    n = 4000
    P = 1e-3 * rng.random((n, 3))
    T = np.stack([rng.permutation(n)[:3] for _ in range(n)]).astype(np.int32)
    E = np.unique(np.sort(np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]]), axis=1), axis=0)
    E = E[:20000].astype(np.int32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    svb = np.zeros(n, dtype=np.int32)
    bc, be = np.zeros(1, dtype=np.int32), np.zeros(1, dtype=np.int32)
    cap = 1 << 10
    pt = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    ee = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(Z.ZemaError) as ei:
        Z.candidates_raw_noalloc(dev(P), dev(svb), dev(bc), dev(be), dev(E), dev(T), 0.01, 0.05, pt, ee)
    assert ei.value.status == 2
    assert bool((pt == -1).all()) and bool((ee == -1).all())
    # the array is usable again at once
    cell, infl, cap = 0.04, 0.01, 1 << 16
    P, svb, bc, be, E, T = surface(33)
    pt_ref, ee_ref = Z.candidates_raw(P, svb, bc, be, E, T, infl, cell_size=cell)
    pt = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    ee = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
    npt, nee = Z.candidates_raw_noalloc(dev(P), dev(svb), dev(bc), dev(be), dev(E), dev(T), infl, cell, pt, ee)
    assert (npt, nee) == (len(pt_ref), len(ee_ref))
    assert np.array_equal(pt[:npt].cpu().numpy(), pt_ref)
    assert np.array_equal(ee[:nee].cpu().numpy(), ee_ref)


@pytest.mark.parametrize("field", ["body", "edge", "tri", "class"])
def test_noalloc_rejects_bad_device_indices(field):
    import torch

    from paper_2311_05945_b300 import zema as Z
    P, svb, bc, be, E, T = surface(34)
    svb, E, T, bc = svb.copy(), E.copy(), T.copy(), bc.copy()
    if field == "body":
        svb[5] = len(bc)          # one past the last body
    elif field == "edge":
        E[3, 1] = len(P)          # one past the last vertex
    elif field == "tri":
        T[2, 0] = -1
    else:
        bc[0] = 4
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pt = torch.full((64, 2), -1, dtype=torch.int32, device="cuda")
    ee = torch.full((64, 2), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(Z.ZemaError) as ei:
        Z.candidates_raw_noalloc(dev(P), dev(svb), dev(bc), dev(be), dev(E), dev(T), 0.01, 0.04, pt, ee)
    assert ei.value.status == 1
    assert bool((pt == -1).all()) and bool((ee == -1).all())
