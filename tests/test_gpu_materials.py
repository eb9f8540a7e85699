"""St. Venant-Kirchhoff and fixed-corotated soft bodies and spring constraints on the GPU,
against the oracle: the incremental potential and its gradient at the same
state, and short trajectories at tight tolerance (with contact and with
springs moved between steps)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def spring_scene(model=1):
    p = S.Params(dt=0.01)
    s = S.Scene("springs", p)
    X, T = S.soft_cube(3, 0.2, (0.0, 1.0, 0.0))
    s.tets.append(S.TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=0.3, model=model))
    verts = np.array([0, 4, 13, 26], dtype=np.int32)
    s.springs.append((0, verts, X[verts] + np.array([0.01, -0.01, 0.005]), 2.0e3))
    return s


def contact_scene(model=1):
    s = S.scene_tiny_contact(mu=0.5)
    s.tets[0].model = model
    return s


@pytest.mark.parametrize("which", ["springs", "contact", "contact_fcr"])
def test_energy_and_gradient_match_oracle(which):
    from paper_2311_05945_b300.zema import Scene
    sc = spring_scene() if which == "springs" else contact_scene(2 if which == "contact_fcr" else 1)
    orc = Oracle(sc)
    orc.step(6)
    orc.prepare(0, friction=True)
    E_o, g_o, _, _ = orc.eval(orc.dofs(), grad=True)
    gpu = Scene(sc)
    for b in range(len(sc.body_order())):
        gpu.set_state(b, orc.get_state(b))
    gpu.set_kappa(0, orc.kappa(0), orc.kappa_min(0))
    E, g = gpu.eval_energy_grad(apply_predictor=True)
    assert abs(E[0] - E_o) <= 1e-9 * abs(E_o), (E[0], E_o)
    parts, off = [], 0
    for kind, i in sc.body_order():
        n = 3 * len(sc.tets[i].X) if kind == "tet" else 12
        if not (kind == "affine" and sc.affines[i].mode == 1):
            parts.append(g[off:off + n])
        off += n
    gg = np.concatenate(parts)
    assert np.abs(gg - g_o).max() <= 1e-8 * np.abs(g_o).max()
    gpu.close()


@pytest.mark.parametrize("which,precision", [("springs", 0), ("contact", 0), ("contact", 1), ("contact_fcr", 0),
                                             ("contact_fcr", 1)])
def test_trajectory_matches_oracle(which, precision):
    from paper_2311_05945_b300.zema import Scene
    sc = spring_scene() if which == "springs" else contact_scene(2 if which == "contact_fcr" else 1)
    orc = Oracle(sc, tol_scale=1e-2)
    gpu = Scene(sc, tol_scale=1e-2, precision=precision)
    diag = orc.diag()
    for k in range(12):
        if which == "springs" and k == 6:
            # move the springs' targets between steps
            verts = np.array([2, 8, 20], dtype=np.int32)
            t = sc.tets[0].X[verts] + np.array([-0.02, 0.0, 0.01])
            orc.set_springs(0, verts, t, 5.0e3)
            gpu.set_springs(0, verts, t, 5.0e3)
        orc.step(1)
        st = gpu.step(1)
        err = np.abs(orc.tet_positions(0) - gpu.tet_positions(0)).max()
        assert err < 1e-5 * diag, (k, err / diag)
        assert st["dmin"] > 0
    gpu.close()
