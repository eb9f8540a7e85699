"""Failure paths of zema_step and the whole-scene checkpoint.

Every non-OK status of a step must leave the scene at the last completed
time step (the boundary's convention), bit for bit.  Failures are made on
the host: a Newton or PCG iteration cap too small for a contact step, or a
one-shot fault armed with zema_inject_fault (a kernel reading a host-set
flag and reporting through the real status words, or a line search whose
trial points are all rejected).  Nothing faults, traps or hangs the GPU.
The checkpoint must resume a trajectory bit for bit.
"""
import numpy as np
import pytest

from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu

NEWTON_MAXITER, LINESEARCH, PCG_MAXITER, NONFINITE, FAULT_INJECTED = 6, 7, 8, 9, 10
FAULT_STATUS, FAULT_SOLVE_NONFINITE, FAULT_NO_DECREASE = 1, 2, 3


def snapshot(g, sc):
    st = [g.get_state(b) for b in range(len(sc.body_order()))]
    return np.concatenate(st), np.array([g.kappa(e) for e in range(sc.n_envs)])


def assert_same(a, b):
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


def failing_step(g):
    from paper_2311_05945_b300 import zema as Z
    with pytest.raises(Z.ZemaError) as ei:
        g.step(1)
    return ei.value.status


def test_newton_cap_leaves_state_at_last_step():
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_tiny_contact()
    sc.params.max_newton = 1  # no contact step converges in one iteration
    g = Z.Scene(sc)
    before = snapshot(g, sc)
    assert failing_step(g) == NEWTON_MAXITER
    assert_same(snapshot(g, sc), before)
    assert "max_newton" in Z.lib().zema_last_error(g.h).decode()
    g.close()


@pytest.mark.parametrize("precision,pcg_kind", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_pcg_cap_leaves_state_at_last_step(precision, pcg_kind):
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_tiny_contact()
    sc.params.max_pcg = 2
    sc.params.pcg_rel_tol = 1e-12
    g = Z.Scene(sc, precision=precision, pcg_kind=pcg_kind)
    before = snapshot(g, sc)
    assert failing_step(g) == PCG_MAXITER
    assert_same(snapshot(g, sc), before)
    g.close()


@pytest.mark.parametrize("kind,status", [(FAULT_STATUS, FAULT_INJECTED), (FAULT_SOLVE_NONFINITE, NONFINITE),
                                         (FAULT_NO_DECREASE, LINESEARCH)])
@pytest.mark.parametrize("precision,pcg_kind", [(0, 0), (1, 0), (1, 1)])
def test_injected_fault_then_clean_resume(kind, status, precision, pcg_kind):
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_tiny_contact(n_steps=6)
    g = Z.Scene(sc, precision=precision, pcg_kind=pcg_kind)
    ref = Z.Scene(sc, precision=precision, pcg_kind=pcg_kind)
    g.step(2)
    ref.step(2)
    before = snapshot(g, sc)
    assert_same(before, snapshot(ref, sc))
    g.inject_fault(kind, 0)  # the first Newton iteration of the next call
    assert failing_step(g) == status
    assert_same(snapshot(g, sc), before)
    # the fault fired once: the same step now completes, identical to a run
    # that never saw it
    g.step(2)
    ref.step(2)
    assert_same(snapshot(g, sc), snapshot(ref, sc))
    g.close()
    ref.close()


def test_disarmed_fault_does_nothing():
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_tiny_contact(n_steps=4)
    g, ref = Z.Scene(sc), Z.Scene(sc)
    g.inject_fault(FAULT_NO_DECREASE, 0)
    g.inject_fault(0, 0)
    g.step(2)
    ref.step(2)
    assert_same(snapshot(g, sc), snapshot(ref, sc))
    with pytest.raises(Z.ZemaError):
        g.inject_fault(7, 0)
    with pytest.raises(Z.ZemaError):
        g.inject_fault(FAULT_STATUS, -1)


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_is_bit_identical(precision):
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_c1(n_steps=12)
    a = Z.Scene(sc, precision=precision)
    a.step(5)
    ck = a.save_checkpoint()
    a.step(4)
    b = Z.Scene(sc, precision=precision)
    b.load_checkpoint(ck)
    assert b.step_index == 5
    b.step(4)
    assert_same(snapshot(a, sc), snapshot(b, sc))
    a.close()
    b.close()


def test_checkpoint_across_precisions_and_mismatch():
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_tiny_contact(n_steps=6)
    a = Z.Scene(sc, precision=0)
    a.step(3)
    ck = a.save_checkpoint()
    m = Z.Scene(sc, precision=1)
    m.load_checkpoint(ck)
    assert_same(snapshot(m, sc), snapshot(a, sc))
    assert m.step(1)["dmin"] > 0
    # a checkpoint of another scene is refused and changes nothing
    other = Z.Scene(S.scene_c1(n_steps=2))
    keep = snapshot(other, S.scene_c1(n_steps=2))
    with pytest.raises(Z.ZemaError) as ei:
        other.load_checkpoint(ck)
    assert ei.value.status == 1
    assert_same(snapshot(other, S.scene_c1(n_steps=2)), keep)
    bad = (ck[0][:-8], ck[1])
    with pytest.raises(Z.ZemaError):
        a.load_checkpoint(bad)
    for g in (a, m, other):
        g.close()


def small_grasp():
    # two grasp envs at test size; the fingers close on the objects by step 20
    return S.scene_c3(n_envs=2, n_steps=40, min_tets=300, max_tets=600, finger_subdiv=3)


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_with_kinematic_multipliers(precision):
    # the fingers' multipliers and the previous step's (the extrapolation's
    # second point) are part of the checkpoint: resuming in contact is bit
    # for bit
    from paper_2311_05945_b300 import zema as Z
    sc = small_grasp()
    a = Z.Scene(sc, precision=precision)
    a.step(24)
    ck = a.save_checkpoint()
    a.step(4)
    b = Z.Scene(sc, precision=precision)
    b.load_checkpoint(ck)
    b.step(4)
    assert_same(snapshot(a, sc), snapshot(b, sc))
    a.close()
    b.close()


def test_fault_on_a_grasp_step_restores_the_multipliers():
    # a failed contact step puts the multipliers and their history back: the
    # trajectory then equals one that never saw the fault
    from paper_2311_05945_b300 import zema as Z
    sc = small_grasp()
    g, ref = Z.Scene(sc, precision=1), Z.Scene(sc, precision=1)
    g.step(24)
    ref.step(24)
    before = snapshot(g, sc)
    g.inject_fault(FAULT_STATUS, 0)
    assert failing_step(g) == FAULT_INJECTED
    assert_same(snapshot(g, sc), before)
    g.step(3)
    ref.step(3)
    assert_same(snapshot(g, sc), snapshot(ref, sc))
    g.close()
    ref.close()
