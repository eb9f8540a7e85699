"""Contact force sensing and the force-controlled grasp on the GPU.

Pins of the sensed forces (the barrier gradient summed over a body's
vertices, over h^2):
- Third law: every pair's barrier gradient sums to zero over its four
  vertices, so the sensed forces of all bodies add up to zero.
- Momentum: at a converged step, the vertical momentum balance of each
  dynamic body has only inertia and contact terms.  Elastic forces cancel
  inside a body, and friction is tangential on horizontal contacts.  So
  sum_v m_v (y_v^{t+1} - yhat_v) / h^2 + F_y = 0, with the lumped masses the
  oracle computes from the paper's mass matrix.
- At rest on the floor the sensed force is the body's weight.

The controller: closing with force feedback stops near the desired finger
force, and the lift then carries the object off the floor."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def test_sensed_forces_balance_momentum():
    from paper_2311_05945_b300.zema import Scene
    sc = S.scene_tiny_contact(mu=0.5)
    h, gy = sc.params.dt, sc.params.gravity[1]
    m_soft = Oracle(sc).lumped_mass()[: len(sc.tets[0].X)]
    m_cube = 1000.0 * 0.1 ** 3  # the affine cube: 0.1 m box, rho = 1000, centred at its COM
    g = Scene(sc, tol_scale=1e-4)
    st = g.step(1)
    checked = 0
    for k in range(30):
        x0, v0 = g.tet_positions(0).copy(), g.get_state(0)[3 * len(sc.tets[0].X):].reshape(-1, 3).copy()
        q0 = g.get_state(2)
        kap0 = st["kappa"]
        st = g.step(1)
        if st["kappa"] != kap0 or st["max_active"] == 0:
            continue  # the barrier stiffness changed at the end of this step
        F = g.contact_forces()
        assert np.abs(F.sum(0)).max() <= 1e-9 * np.abs(F).max()
        x1 = g.tet_positions(0)
        yhat = x0[:, 1] + h * v0[:, 1] + h * h * gy
        inertia_soft = float(np.dot(m_soft, x1[:, 1] - yhat)) / (h * h)
        q1 = g.get_state(2)
        phat = q0[1] + h * q0[13] + h * h * gy
        inertia_cube = m_cube * (q1[1] - phat) / (h * h)
        w = (m_soft.sum() + m_cube) * abs(gy)
        assert abs(inertia_soft + F[0, 1]) < 2e-3 * w, (k, inertia_soft, F[0, 1])
        assert abs(inertia_cube + F[2, 1]) < 2e-3 * w, (k, inertia_cube, F[2, 1])
        checked += 1
    assert checked >= 10
    # settled: the floor carries both bodies' weight
    assert abs(F[1, 1] - w) < 0.05 * w


def test_force_controlled_grasp_lifts_the_object():
    from paper_2311_05945_b300.grasp import AutoGrasp
    from paper_2311_05945_b300.zema import Scene
    sc = S.scene_c2(precision=1)
    g = Scene(sc)
    # gentler decay than the paper's k = 20 1/N so that closing reaches 1 N
    # within a few hundred steps at a 5 cm/s increment
    ag = AutoGrasp(g, sc, k=4.0, f_star=1.0, lift_steps=40, lift_height=0.01)
    y0 = g.tet_positions(0)[:, 1].min()
    lift_at = None
    for n in range(600):
        ag.step()
        if lift_at is None and ag.lift_done[0] is not None:
            lift_at = n
            f = ag.history[-1]["forces"]
            assert min(f.values()) >= 0.95, f  # closing ended by reaching the force
        if lift_at is not None and n >= lift_at + 60:
            break
    assert lift_at is not None
    forces = g.contact_forces()
    floor = sc.affines.index(next(a for a in sc.affines if a.mode == 1))
    assert abs(forces[g.affine_body_id(floor)]).max() < 1e-9  # off the floor
    assert g.tet_positions(0)[:, 1].min() > y0 + 0.005
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_sensed_forces_match_the_oracle(precision):
    # the library's force sensing against the oracle's (its barrier gradient
    # by dual numbers over brute-force pairs) at the same in-contact states:
    # the tiny scene and C1, with the oracle's states and stiffness
    from paper_2311_05945_b300.zema import Scene
    for sc, steps in ((S.scene_tiny_contact(mu=0.5), 6), (S.scene_c1(n_steps=14), 12)):
        orc = Oracle(sc)
        orc.step(steps)
        g = Scene(sc, precision=precision)
        for b in range(len(sc.body_order())):
            g.set_state(b, orc.get_state(b))
        g.set_kappa(0, orc.kappa(), orc.kappa_min())
        Fo, Fg = orc.contact_forces(), g.contact_forces()
        scale = np.abs(Fo).max()
        assert scale > 0
        assert np.abs(Fg - Fo).max() <= 1e-9 * scale, (np.abs(Fg - Fo).max(), scale)
        g.close()
