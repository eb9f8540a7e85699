"""Scene-level parity of the CUDA stepper against the oracle: analytic free
fall, total incremental potential and gradient at the same state, one-step
parity from identical states, short trajectories, determinism and d_min > 0."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def gpu_scene(sc, **kw):
    from paper_2311_05945_b300.zema import Scene
    return Scene(sc, **kw)


def transplant(orc, gpu, sc):
    """Copy the oracle's body states and kappa into the GPU scene."""
    for b in range(len(sc.body_order())):
        gpu.set_state(b, orc.get_state(b))
    for e in range(sc.n_envs):
        gpu.set_kappa(e, orc.kappa(e), orc.kappa_min(e))


def positions(obj, sc):
    out = [obj.tet_positions(i).ravel() for i in range(len(sc.tets))]
    out += [obj.affine_q(i) for i in range(len(sc.affines))]
    return np.concatenate(out)


def affine_vertex_positions(obj, sc):
    out = []
    for i, a in enumerate(sc.affines):
        q = obj.affine_q(i)
        out.append((a.V @ q[3:].reshape(3, 3).T + q[:3]).ravel())
    return np.concatenate(out) if out else np.zeros(0)


def test_free_fall_analytic_gpu():
    sc = S.scene_free_fall(n_steps=4)
    g = gpu_scene(sc)
    x0 = g.tet_positions(0).copy()
    q0 = g.affine_q(0).copy()
    g.step(4)
    h, gy, n = sc.params.dt, sc.params.gravity[1], 4
    dy = h * h * gy * n * (n + 1) / 2
    x = g.tet_positions(0)
    assert np.abs(x[:, 1] - x0[:, 1] - dy).max() < 1e-12
    assert np.abs(x[:, [0, 2]] - x0[:, [0, 2]]).max() < 1e-12
    q = g.affine_q(0)
    assert abs(q[1] - q0[1] - dy) < 1e-12


@pytest.mark.parametrize("steps", [0, 5])
def test_energy_and_gradient_match_oracle(steps):
    sc = S.scene_tiny_contact(mu=0.5)
    orc = Oracle(sc)
    orc.step(steps)
    orc.prepare(0, friction=True)
    E_o, g_o, _, na = orc.eval(orc.dofs(), grad=True)
    gpu = gpu_scene(sc)
    transplant(orc, gpu, sc)
    # the oracle's prepare already applied the predictor from the same state
    E, g = gpu.eval_energy_grad(apply_predictor=True)
    assert abs(E[0] - E_o) <= 1e-9 * abs(E_o), (E[0], E_o)
    # GPU gradient: per body in order (fixed bodies as 12 zeros); oracle: env DOFs
    parts = []
    off = 0
    for kind, i in sc.body_order():
        n = 3 * len(sc.tets[i].X) if kind == "tet" else 12
        if not (kind == "affine" and sc.affines[i].mode == 1):
            parts.append(g[off:off + n])
        off += n
    gg = np.concatenate(parts)
    assert np.abs(gg - g_o).max() <= 1e-8 * np.abs(g_o).max()


def test_one_step_parity_c1_tight():
    sc = S.scene_c1()
    orc = Oracle(sc, tol_scale=1e-2)
    orc.step(12)  # in contact
    gpu = gpu_scene(sc, tol_scale=1e-2)
    transplant(orc, gpu, sc)
    orc.step(1)
    gpu.step(1)
    diag = orc.diag()
    po, pg = positions(orc, sc), positions(gpu, sc)
    err = np.abs(po - pg).max()
    assert err < 1e-5 * diag, err
    err_a = np.abs(affine_vertex_positions(orc, sc) - affine_vertex_positions(gpu, sc)).max()
    assert err_a < 1e-5 * diag, err_a


def test_trajectory_parity_tiny_contact():
    sc = S.scene_tiny_contact(mu=0.5)
    orc = Oracle(sc)
    gpu = gpu_scene(sc)
    diag = orc.diag()
    for k in range(15):
        so = orc.step(1)
        st = gpu.step(1)
        err = max(np.abs(orc.tet_positions(0) - gpu.tet_positions(0)).max(),
                  np.abs(affine_vertex_positions(orc, sc) - affine_vertex_positions(gpu, sc)).max())
        assert err < 1e-5 * diag, (k, err)
        assert st["dmin"] > 0


def test_trajectory_parity_c1():
    sc = S.scene_c1()
    orc = Oracle(sc)
    gpu = gpu_scene(sc)
    diag = orc.diag()
    worst = 0.0
    for k in range(25):
        orc.step(1)
        st = gpu.step(1)
        err = max(np.abs(orc.tet_positions(0) - gpu.tet_positions(0)).max(),
                  np.abs(affine_vertex_positions(orc, sc) - affine_vertex_positions(gpu, sc)).max())
        worst = max(worst, err)
        assert st["dmin"] > 0
    assert worst < 1e-5 * diag, worst


def test_deterministic_rerun():
    sc = S.scene_tiny_contact(mu=0.5)
    a = gpu_scene(sc)
    b = gpu_scene(sc)
    a.step(6)
    b.step(6)
    assert np.array_equal(positions(a, sc), positions(b, sc))
