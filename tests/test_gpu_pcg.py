"""The two linear-solver launch forms (one thread-block cluster per
environment; one grid-wide cooperative launch) against the oracle, in both
precision modes, and the batched form: several environments stepped in one
scene, each checked against the oracle's step of the same environment."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def gpu_scene(sc, **kw):
    from paper_2311_05945_b300.zema import Scene
    return Scene(sc, **kw)


def transplant(orc, gpu, sc):
    for b in range(len(sc.body_order())):
        gpu.set_state(b, orc.get_state(b))
    for e in range(sc.n_envs):
        gpu.set_kappa(e, orc.kappa(e), orc.kappa_min(e))
    gpu.step_index = orc.step_index


def env_positions(obj, sc, env):
    """Soft vertex positions and affine mesh-vertex positions of one env."""
    out = [obj.tet_positions(i).ravel() for i, b in enumerate(sc.tets) if b.env == env]
    for i, a in enumerate(sc.affines):
        if a.env != env:
            continue
        q = obj.affine_q(i)
        out.append((a.V @ q[3:].reshape(3, 3).T + q[:3]).ravel())
    return np.concatenate(out)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("pcg_kind", [1, 2])
def test_solver_forms_one_step_parity_c1(precision, pcg_kind):
    sc = S.scene_c1()
    orc = Oracle(sc, tol_scale=1e-2)
    orc.step(12)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=precision, pcg_kind=pcg_kind)
    transplant(orc, gpu, sc)
    orc.step(1)
    st = gpu.step(1)
    assert st["pcg_iters"] > 0
    diag = orc.diag()
    err = np.abs(env_positions(orc, sc, 0) - env_positions(gpu, sc, 0)).max()
    assert err < 1e-5 * diag, err / diag


@pytest.mark.parametrize("pcg_kind", [1, 2])
def test_fp64_refinement_of_fp32_solves(pcg_kind):
    # at a linear tolerance FP32 iterations cannot meet, every mixed solve
    # is refined against FP64 residuals (inside the cluster launch, or from
    # the host for the grid-wide form) and the step follows the oracle
    sc = S.scene_c1()
    sc.params.pcg_rel_tol = 1e-9
    orc = Oracle(sc, tol_scale=1e-2)
    orc.step(12)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=1, pcg_kind=pcg_kind)
    transplant(orc, gpu, sc)
    orc.step(1)
    st = gpu.step(1)
    assert st["pcg_refines"] > 0
    diag = orc.diag()
    err = np.abs(env_positions(orc, sc, 0) - env_positions(gpu, sc, 0)).max()
    assert err < 1e-5 * diag, err / diag


def test_solver_forms_free_fall_exact():
    # no contact: the minimiser is the analytic free fall; both forms solve the
    # linear system to round-off at a tight tolerance
    for kind in (1, 2):
        sc = S.scene_free_fall(n_steps=3)
        sc.params.pcg_rel_tol = 1e-13
        g = gpu_scene(sc, pcg_kind=kind)
        x0 = g.tet_positions(0).copy()
        g.step(3)
        h, gy, n = sc.params.dt, sc.params.gravity[1], 3
        dy = h * h * gy * n * (n + 1) / 2
        assert np.abs(g.tet_positions(0)[:, 1] - x0[:, 1] - dy).max() < 1e-12


def small_batched(n_envs=3):
    # the batched grasp generator at test size: coarse objects, coarse fingers
    return S.scene_c3(n_envs=n_envs, n_steps=30, min_tets=200, max_tets=700, finger_subdiv=3, precision=0)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_envs_trajectory_parity(precision):
    sc = small_batched()
    orc = Oracle(sc, tol_scale=1e-2)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=precision)
    diags = [orc.diag(e) for e in range(sc.n_envs)]
    for k in range(4):
        orc.step(1)
        st = gpu.step(1)
        assert st["dmin"] > 0
        for e in range(sc.n_envs):
            err = np.abs(env_positions(orc, sc, e) - env_positions(gpu, sc, e)).max()
            assert err < 1e-5 * diags[e], (k, e, err / diags[e])


def test_batched_envs_one_step_parity_in_contact():
    # start from the oracle's state after the fingers have closed on the
    # objects (contact with the floor and both fingers)
    sc = small_batched()
    orc = Oracle(sc, tol_scale=1e-2)
    orc.step(24)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=1)
    transplant(orc, gpu, sc)
    orc.step(1)
    st = gpu.step(1)
    for e in range(sc.n_envs):
        d = orc.diag(e)
        err = np.abs(env_positions(orc, sc, e) - env_positions(gpu, sc, e)).max()
        assert err < 1e-5 * d, (e, err / d)
    # at most 3 refinement rounds per env and solve (an env solves once per
    # Newton iteration, the converged one included, in every AL round)
    solves = st["newton_iters"] + sc.n_envs * (1 + st["al_rounds"])
    assert 0 <= st["pcg_refines"] <= 3 * solves, (st["pcg_refines"], solves)


def test_batched_deterministic_and_kinds_agree():
    sc = small_batched()
    a = gpu_scene(sc, precision=1, tol_scale=1e-2)
    b = gpu_scene(sc, precision=1, tol_scale=1e-2)
    c = gpu_scene(sc, precision=1, tol_scale=1e-2, pcg_kind=1)
    a.step(5)
    b.step(5)
    c.step(5)
    a_diag = [Oracle(sc).diag(e) for e in range(sc.n_envs)]
    for e in range(sc.n_envs):
        pa, pb, pc = env_positions(a, sc, e), env_positions(b, sc, e), env_positions(c, sc, e)
        assert np.array_equal(pa, pb)
        # the two solver forms differ in summation order and vector precision:
        # equal to within the (tightened) Newton tolerance
        assert np.abs(pa - pc).max() < 1e-5 * a_diag[e]


def test_c2_mixed_follows_fp64_through_first_contact():
    # the full-size grasp: fine meshes put nearly parallel edge pairs in
    # contact, whose Hessian factors leave FP32's range unless normalised;
    # the mixed mode must take real Newton steps and follow the FP64 run
    sc = S.scene_c2()
    a = gpu_scene(sc, precision=0)
    b = gpu_scene(sc, precision=1)
    diag = Oracle(sc).diag()
    for k in range(20):
        sa = a.step(1)
        sb = b.step(1)
        assert sb["al_rounds"] < sc.params.max_al_rounds, (k, sb)
        if sa["newton_iters"] > 0:
            assert sb["newton_iters"] > 0 and sb["pcg_iters"] > 0, (k, sa, sb)
    err = np.abs(env_positions(a, sc, 0) - env_positions(b, sc, 0)).max()
    assert err < 1e-4 * diag, err / diag


def test_autotuned_cluster_solve_keeps_parity():
    # the autotuner times every valid cluster size on one system, keeps the
    # fastest, and the tuned solve still matches the oracle's step
    sc = S.scene_c1()
    orc = Oracle(sc, tol_scale=1e-2)
    orc.step(12)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=1)
    transplant(orc, gpu, sc)
    gpu.autotune()
    orc.step(1)
    gpu.step(1)
    cs, measured = gpu.tuning()
    assert cs in measured and len(measured) >= 2
    assert measured[cs] == min(measured.values())
    diag = orc.diag()
    err = np.abs(env_positions(orc, sc, 0) - env_positions(gpu, sc, 0)).max()
    assert err < 1e-5 * diag, err / diag


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("schedule", [2, 102, 104, 1001, 1102])
def test_cluster_schedules_keep_parity(precision, schedule):
    # both residency variants of the cluster solve (one CTA per SM with the
    # matrix slice staged in shared memory; two per SM, matrix through L1/L2)
    # at pinned cluster sizes, and the size-binned schedules (one launch per
    # cluster size): one tight step from the oracle's in-contact C1 state
    # lands on the oracle's step
    sc = S.scene_c1()
    orc = Oracle(sc, tol_scale=1e-2)
    orc.step(12)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=precision, pcg_cluster_size=schedule)
    transplant(orc, gpu, sc)
    orc.step(1)
    gpu.step(1)
    assert gpu.tuning()[0] == schedule
    diag = orc.diag()
    err = np.abs(env_positions(orc, sc, 0) - env_positions(gpu, sc, 0)).max()
    assert err < 1e-5 * diag, err / diag


@pytest.mark.parametrize("schedule", [8, 1001, 1102])
def test_binned_schedule_on_a_batch_of_uneven_envs(schedule):
    # envs of 2k-12k tets fall into several cluster-size groups; every env of
    # the batch stays within the parity bound of the same batch solved with
    # one uniform schedule (both mixed, tight tolerance)
    sc = S.scene_c3(n_envs=6, n_steps=24, min_tets=2000, max_tets=12000)
    ref = gpu_scene(sc, tol_scale=1e-2, precision=1, pcg_cluster_size=16)
    g = gpu_scene(sc, tol_scale=1e-2, precision=1, pcg_cluster_size=schedule)
    ref.step(22)
    g.step(22)
    assert g.tuning()[0] == schedule
    for e in range(sc.n_envs):
        pr, pg = env_positions(ref, sc, e), env_positions(g, sc, e)
        ext = pr.reshape(-1, 3)
        diag = float(np.linalg.norm(ext.max(0) - ext.min(0)))
        assert np.abs(pr - pg).max() < 1e-5 * diag, (e, np.abs(pr - pg).max() / diag)
