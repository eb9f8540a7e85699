"""The dense soft-rigid pile on the GPU: a small pile against the oracle
(both linear-solve forms, so the grid-wide solve with its per-affine-body
tiles is covered), and the full-size pile (484k tets, 96k nodes): d_min > 0
every step, and the mixed-precision form following the FP64 form while the
bodies fall and first touch the bin."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def small_pile():
    # two soft bodies (~100 tets), a 6 x 6 UV sphere and a 6 x 6 torus, all
    # resting 0.5 dhat above the bin floor
    return S.scene_c5(n_steps=12, tets_per_body=100, n_soft=2, n_convex=1, n_nonconvex=1, n_seg=6,
                      bin_subdiv=1, gap=0.5e-3, precision=0)


def mesh_positions(obj, sc):
    out = [obj.tet_positions(i).ravel() for i in range(len(sc.tets))]
    for i, a in enumerate(sc.affines):
        q = obj.affine_q(i)
        out.append((a.V @ q[3:].reshape(3, 3).T + q[:3]).ravel())
    return np.concatenate(out)


@pytest.mark.parametrize("pcg_kind", [0, 1])
def test_small_pile_trajectory_matches_oracle(pcg_kind):
    from paper_2311_05945_b300.zema import Scene
    sc = small_pile()
    orc = Oracle(sc, tol_scale=1e-2)
    gpu = Scene(sc, tol_scale=1e-2, pcg_kind=pcg_kind)
    diag = orc.diag()
    for k in range(10):
        orc.step(1)
        st = gpu.step(1)
        err = np.abs(mesh_positions(orc, sc) - mesh_positions(gpu, sc)).max()
        print("small pile step", k, "err/diag", err / diag, "active", st["max_active"])
        assert err < 1e-5 * diag, (k, err / diag)
        assert st["dmin"] > 0
    assert st["max_active"] > 0  # in contact with the floor


def test_full_pile_mixed_follows_fp64():
    from paper_2311_05945_b300.zema import Scene
    sc = S.scene_c5(n_steps=6)
    assert sum(len(b.tets) for b in sc.tets) > 450000
    g64 = Scene(sc, precision=0)
    g32 = Scene(sc, precision=1)
    diag = None
    for k in range(6):
        s64 = g64.step(1)
        s32 = g32.step(1)
        assert s64["dmin"] > 0 and s32["dmin"] > 0
        p64, p32 = mesh_positions(g64, sc), mesh_positions(g32, sc)
        if diag is None:
            diag = float(np.linalg.norm(p64.reshape(-1, 3).max(0) - p64.reshape(-1, 3).min(0)))
        # both forms stop Newton at 1e-3 x diag x dt; they must land within
        # that step tolerance of each other
        err = np.abs(p64 - p32).max()
        print("pile step", k, "mixed - fp64", err, "tol", 1e-3 * diag * sc.params.dt)
        assert err < 1e-3 * diag * sc.params.dt, k
    assert s32["max_active"] > 0  # the lowest layer reached the floor
    g64.close()
    g32.close()
