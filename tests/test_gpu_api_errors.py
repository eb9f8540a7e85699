"""Error paths of the C-ABI entry points for springs, materials, joints and
force sensing: invalid arguments and calls in the wrong state return their
documented status and leave the scene usable."""
import ctypes as C

import numpy as np
import pytest

from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu

INVALID_ARG, STATE = 1, 11


def test_spring_and_material_errors():
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_tiny_contact()
    g = Z.Scene(sc)
    L, h = Z.lib(), g.h
    soft, floor = g.tet_body_id(0), g.affine_body_id(0)
    v = np.array([0, 1], dtype=np.int32)
    t = np.zeros((2, 3))
    ip = v.ctypes.data_as(C.POINTER(C.c_int32))
    dp = t.ctypes.data_as(C.POINTER(C.c_double))
    assert L.zema_set_springs(h, floor, ip, 2, dp, 1.0) == INVALID_ARG      # not a tet body
    assert L.zema_set_springs(h, soft, ip, 2, dp, -1.0) == INVALID_ARG      # negative stiffness
    bad = np.array([0, 10 ** 6], dtype=np.int32)
    assert L.zema_set_springs(h, soft, bad.ctypes.data_as(C.POINTER(C.c_int32)), 2, dp, 1.0) == INVALID_ARG
    t_nan = np.full((2, 3), np.nan)
    assert L.zema_set_springs(h, soft, ip, 2, t_nan.ctypes.data_as(C.POINTER(C.c_double)), 1.0) == INVALID_ARG
    # after finalize the material is fixed
    assert L.zema_set_material(h, soft, 1) == INVALID_ARG
    assert L.zema_set_material(h, floor, 0) == INVALID_ARG
    # springs are allowed between steps, and the scene still steps
    assert L.zema_set_springs(h, soft, ip, 2, dp, 10.0) == 0
    assert g.step(1)["dmin"] > 0
    g.close()


def test_joint_and_force_errors():
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_joint(axis=(1.0, 0.0, 0.0), fixed_base=True)
    g = Z.Scene(sc)
    L, h = Z.lib(), g.h
    ax = np.array([1.0, 0.0, 0.0])
    dp = ax.ctypes.data_as(C.POINTER(C.c_double))
    # joints only before the scene is finalized
    assert L.zema_add_prismatic_joint(h, g.affine_body_id(0), g.affine_body_id(1), dp, 0.0, None) == STATE
    # force sensing needs room for 3 values per body
    out = np.zeros(3)
    assert L.zema_contact_forces(h, out.ctypes.data_as(C.POINTER(C.c_double)), 3) == INVALID_ARG
    F = g.contact_forces()
    assert F.shape == (2, 3) and np.all(F == 0.0)  # the boxes touch nothing
    g.close()


def test_joint_argument_checks_before_finalize():
    from paper_2311_05945_b300 import zema as Z
    L = Z.lib()
    P = Z.Params()
    P.dt, P.dhat, P.kappa, P.eps_v, P.newton_tol_rel = 0.01, 1e-3, 0.0, 1e-3, 1e-3
    P.gravity[:] = (0.0, -9.81, 0.0)
    P.pcg_rel_tol, P.max_newton, P.max_pcg, P.max_al_rounds, P.n_envs = 1e-4, 100, 10000, 10, 2
    h = C.c_void_p()
    assert L.zema_create_scene(C.byref(P), C.byref(h)) == 0
    V, F = S.box_surface((0.1, 0.1, 0.1), 1)
    V, F = np.ascontiguousarray(V), np.ascontiguousarray(F, dtype=np.int32)
    ids = []
    for env, mode, x in ((0, 0, 0.0), (0, 1, 0.3), (1, 0, 0.6), (0, 1, 0.9)):
        q = S.q_identity((x, 1.0, 0.0))
        bid = C.c_int32()
        r = L.zema_add_affine_body(h, env, V.ctypes.data_as(C.POINTER(C.c_double)), len(V),
                                   F.ctypes.data_as(C.POINTER(C.c_int32)), len(F),
                                   q.ctypes.data_as(C.POINTER(C.c_double)), None, 1000.0, 1e8, 0.5, mode,
                                   C.byref(bid))
        assert r == 0
        ids.append(bid.value)
    ax = np.array([0.0, 1.0, 0.0])
    dp = ax.ctypes.data_as(C.POINTER(C.c_double))
    zero = np.zeros(3)
    assert L.zema_add_prismatic_joint(h, ids[0], ids[0], dp, 0.0, None) == INVALID_ARG   # same body
    assert L.zema_add_prismatic_joint(h, ids[0], ids[2], dp, 0.0, None) == INVALID_ARG   # other env
    assert L.zema_add_prismatic_joint(h, ids[1], ids[3], dp, 0.0, None) == INVALID_ARG   # both fixed
    assert L.zema_add_prismatic_joint(h, ids[0], ids[1], zero.ctypes.data_as(C.POINTER(C.c_double)), 0.0,
                                      None) == INVALID_ARG                               # zero axis
    jid = C.c_int32(-1)
    assert L.zema_add_prismatic_joint(h, ids[0], ids[1], dp, 0.0, C.byref(jid)) == 0 and jid.value == 0
    L.zema_destroy_scene(h)


def test_batched_kinematic_targets():
    """zema_set_kinematic_targets sets every listed body's target in one call:
    a 3-env grasp batch stepped through it follows the per-body calls bit for
    bit; repeated ids, non-affine ids and NULL arrays are rejected."""
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_c3(n_envs=3, n_steps=8, min_tets=800, max_tets=1200)
    a = Z.Scene(sc)
    b = Z.Scene(sc)
    L = Z.lib()
    script = sc.script
    for step in range(6):
        a.step(1)  # batched call (the script's arrays)
        for idx, q in script(b.step_index).items():
            b.set_kinematic_target(idx, q)
        b.step(1, script=False)
    for i in range(len(sc.tets)):
        assert np.array_equal(a.tet_positions(i), b.tet_positions(i))
    for i in range(len(sc.affines)):
        assert np.array_equal(a.affine_q(i), b.affine_q(i))
    h = a.h
    q = np.zeros((2, 12))
    dp = q.ctypes.data_as(C.POINTER(C.c_double))
    fid = a.affine_body_id(script.arrays(0)[0][0])
    rep = np.array([fid, fid], dtype=np.int32)
    assert L.zema_set_kinematic_targets(h, 2, rep.ctypes.data_as(C.POINTER(C.c_int32)), dp) == INVALID_ARG
    soft = np.array([a.tet_body_id(0), fid], dtype=np.int32)
    assert L.zema_set_kinematic_targets(h, 2, soft.ctypes.data_as(C.POINTER(C.c_int32)), dp) == INVALID_ARG
    assert L.zema_set_kinematic_targets(h, 2, None, dp) == INVALID_ARG
    assert L.zema_set_kinematic_targets(h, -1, None, None) == INVALID_ARG
    assert L.zema_set_kinematic_targets(h, 0, None, None) == 0
    a.close()
    b.close()


def test_whole_scene_state():
    """zema_get/set_scene_state: every body's state in one flat array (the
    per-body layouts back to back in order of addition); a step after setting
    it equals a step after setting each body, bit for bit; size mismatches
    are rejected with nothing changed."""
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_c3(n_envs=2, n_steps=12, min_tets=300, max_tets=600, finger_subdiv=3)
    a, b = Z.Scene(sc, precision=1), Z.Scene(sc, precision=1)
    a.step(6)
    flat = a.get_scene_state()
    per = [a.get_state(i) for i in range(len(sc.body_order()))]
    assert np.array_equal(flat, np.concatenate(per))
    # the same state into two fresh scenes, once through the flat call and
    # once per body (the multipliers stay at their fresh values in both)
    b.set_scene_state(flat)
    assert np.array_equal(b.get_scene_state(), flat)
    c = Z.Scene(sc, precision=1)
    for i, x in enumerate(per):
        c.set_state(i, x)
    for g in (b, c):
        g.step_index = a.step_index
    b.step(2)
    c.step(2)
    assert np.array_equal(b.get_scene_state(), c.get_scene_state())
    L, h = Z.lib(), b.h
    keep = b.get_scene_state()
    short = np.zeros(len(flat) - 1)
    assert L.zema_set_scene_state(h, short.ctypes.data_as(C.c_void_p), len(short)) == INVALID_ARG
    assert L.zema_get_scene_state(h, short.ctypes.data_as(C.c_void_p), len(short), None) == INVALID_ARG
    assert np.array_equal(b.get_scene_state(), keep)
    for g in (a, b, c):
        g.close()
