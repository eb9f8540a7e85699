"""Prismatic joints on the GPU against the oracle: free fall along the axis
is exact, a horizontal joint holds its slider against gravity, and a moving
dynamic base drags the slider across the axis with the pair's linear
momentum conserved (both precisions)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def test_free_fall_along_the_axis_gpu():
    from paper_2311_05945_b300.zema import Scene
    sc = S.scene_joint(axis=(0.0, 1.0, 0.0), fixed_base=True)
    sc.params.pcg_rel_tol = 1e-12
    g = Scene(sc, tol_scale=1e-3, precision=0)
    q0 = g.affine_q(1).copy()
    g.step(5)
    h, gy, n = sc.params.dt, sc.params.gravity[1], 5
    q = g.affine_q(1)
    assert abs(q[1] - q0[1] - h * h * gy * n * (n + 1) / 2) < 1e-9
    assert np.abs(np.delete(q - q0, 1)).max() < 1e-9
    g.close()


@pytest.mark.parametrize("case,precision", [("hold", 0), ("hold", 1), ("drag", 0), ("drag", 1)])
def test_joint_trajectory_matches_oracle(case, precision):
    from paper_2311_05945_b300.zema import Scene
    if case == "hold":
        sc = S.scene_joint(axis=(1.0, 0.0, 0.0), fixed_base=True)
    else:
        sc = S.scene_joint(axis=(1.0, 0.0, 0.0), fixed_base=False, gravity=(0.0, 0.0, 0.0),
                           base_velocity=(0.0, 0.3, -0.4))
    orc = Oracle(sc, tol_scale=1e-2)
    gpu = Scene(sc, tol_scale=1e-2, precision=precision)
    diag = orc.diag()
    for k in range(10):
        orc.step(1)
        st = gpu.step(1)
        for b in (0, 1):
            qa, qb = orc.affine_q(b), gpu.affine_q(b)
            # positions of the box corners (A by rows, p)
            V = sc.affines[b].V
            xa = V @ qa[3:].reshape(3, 3).T + qa[:3]
            xb = V @ qb[3:].reshape(3, 3).T + qb[:3]
            assert np.abs(xa - xb).max() < 1e-5 * diag, (k, b)
    if case == "drag":
        # the joint force is internal: the pair's linear momentum (equal
        # masses, boxes centred at their centre of mass, so p' = p) stays the
        # base's initial one, while the slider is dragged across the axis
        # (the pair translates and spins as one rigid body)
        pd = gpu.get_state(0)[12:15] + gpu.get_state(1)[12:15]
        assert np.abs(pd - np.array([0.0, 0.3, -0.4])).max() < 1e-6
        assert abs(gpu.affine_q(1)[2]) > 1e-3
    gpu.close()
