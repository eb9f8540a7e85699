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
    # exact minimiser of Eq. 1 / Eq. 2 without contact; the PCG tolerance is
    # tightened so that the linear solve is exact to round-off
    sc = S.scene_free_fall(n_steps=4)
    sc.params.pcg_rel_tol = 1e-13
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
    st0 = [orc.get_state(b) for b in range(len(sc.body_order()))]
    kap, kmin = orc.kappa(), orc.kappa_min()
    orc.step(1)
    gpu.step(1)
    diag = orc.diag()
    po, pg = positions(orc, sc), positions(gpu, sc)
    err = np.abs(po - pg).max()
    assert err < 1e-5 * diag, err
    err_a = np.abs(affine_vertex_positions(orc, sc) - affine_vertex_positions(gpu, sc)).max()
    assert err_a < 1e-5 * diag, err_a
    # total incremental potential of both results under the step's potential
    # (evaluated by the oracle) within 1e-7 relative
    ev = Oracle(sc, tol_scale=1e-2)
    for b, x in enumerate(st0):
        ev.set_state(b, x)
    ev.set_kappa(0, kap, kmin)
    ev.prepare(0)
    for b in range(len(st0)):
        ev.set_state(b, orc.get_state(b))
    Eo = ev.eval(ev.dofs())[0]
    for b in range(len(st0)):
        ev.set_state(b, gpu.get_state(b))
    Eg = ev.eval(ev.dofs())[0]
    assert abs(Eg - Eo) <= 1e-7 * abs(Eo), (Eg, Eo)


@pytest.mark.parametrize("name,n_steps", [("tiny", 15), ("c1", 25)])
def test_trajectory_parity_tight(name, n_steps):
    # free-running trajectories at 1e-2 x the Newton tolerance: positions of
    # soft vertices and affine mesh vertices within 1e-5 bbox diagonal per step
    sc = S.scene_tiny_contact(mu=0.5) if name == "tiny" else S.scene_c1()
    orc = Oracle(sc, tol_scale=1e-2)
    gpu = gpu_scene(sc, tol_scale=1e-2)
    diag = orc.diag()
    for k in range(n_steps):
        orc.step(1)
        st = gpu.step(1)
        err = max(np.abs(orc.tet_positions(0) - gpu.tet_positions(0)).max(),
                  np.abs(affine_vertex_positions(orc, sc) - affine_vertex_positions(gpu, sc)).max())
        assert err < 1e-5 * diag, (k, err / diag)
        assert st["dmin"] > 0


def test_one_step_parity_along_trajectory_c1():
    # default tolerance: from the oracle's state at step k, one GPU step lands
    # within 1e-5 bbox diagonal of the oracle's step k+1
    sc = S.scene_c1()
    orc = Oracle(sc)
    ev = Oracle(sc)
    gpu = gpu_scene(sc)
    diag = orc.diag()
    for k in range(30):
        if k % 3 == 0 and k >= 6:
            st0 = [orc.get_state(b) for b in range(len(sc.body_order()))]
            kap, kmin = orc.kappa(), orc.kappa_min()
            for b, x in enumerate(st0):
                gpu.set_state(b, x)
            gpu.set_kappa(0, kap, kmin)
            orc.step(1)
            gpu.step(1)
            err = max(np.abs(orc.tet_positions(0) - gpu.tet_positions(0)).max(),
                      np.abs(affine_vertex_positions(orc, sc) - affine_vertex_positions(gpu, sc)).max())
            assert err < 1e-5 * diag, (k, err / diag)
        else:
            orc.step(1)


def test_deterministic_rerun():
    sc = S.scene_tiny_contact(mu=0.5)
    a = gpu_scene(sc)
    b = gpu_scene(sc)
    a.step(6)
    b.step(6)
    assert np.array_equal(positions(a, sc), positions(b, sc))


# ---------------------------------------------------------------------------
# Mixed precision (FP32 Hessians, stored matrices and preconditioner; FP64
# gradients, energies, distances, barrier log term, ACCD and convergence):
# the minimiser is still defined by the FP64 gradient, so the same bounds
# against the FP64 oracle apply.
# ---------------------------------------------------------------------------
def test_mixed_one_step_parity_c1_tight():
    sc = S.scene_c1()
    orc = Oracle(sc, tol_scale=1e-2)
    orc.step(12)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=1)
    transplant(orc, gpu, sc)
    orc.step(1)
    gpu.step(1)
    diag = orc.diag()
    err = max(np.abs(positions(orc, sc) - positions(gpu, sc)).max(),
              np.abs(affine_vertex_positions(orc, sc) - affine_vertex_positions(gpu, sc)).max())
    assert err < 1e-5 * diag, err / diag


@pytest.mark.parametrize("name,n_steps", [("tiny", 15), ("c1", 25)])
def test_mixed_trajectory_parity_tight(name, n_steps):
    sc = S.scene_tiny_contact(mu=0.5) if name == "tiny" else S.scene_c1()
    orc = Oracle(sc, tol_scale=1e-2)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=1)
    diag = orc.diag()
    worst = 0.0
    for k in range(n_steps):
        orc.step(1)
        st = gpu.step(1)
        err = max(np.abs(orc.tet_positions(0) - gpu.tet_positions(0)).max(),
                  np.abs(affine_vertex_positions(orc, sc) - affine_vertex_positions(gpu, sc)).max())
        worst = max(worst, err)
        assert err < 1e-5 * diag, (k, err / diag)
        assert st["dmin"] > 0
    print(f"mixed precision {name}: worst position error vs FP64 oracle {worst / diag:.2e} x bbox diagonal")


def test_mixed_deterministic_rerun():
    sc = S.scene_tiny_contact(mu=0.5)
    a = gpu_scene(sc, precision=1)
    b = gpu_scene(sc, precision=1)
    a.step(6)
    b.step(6)
    assert np.array_equal(positions(a, sc), positions(b, sc))
