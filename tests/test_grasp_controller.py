"""The force-feedback closing factor phi of the grasp controller against its
closed form: 1 at zero force, 0 at and above the desired force f*, strictly
decreasing in between, and the paper's example values (k = 20 1/N,
f* = 0.5 N).  Then the controller's host logic (closing by phi, the stop and
stall rules, the per-env lift, one batch of targets per step) on a stand-in
scene with prescribed forces."""
import math
import types

import numpy as np

from paper_2311_05945_b300.grasp import AutoGrasp, phi


def test_phi_end_points_and_cutoff():
    for k, fs in ((20.0, 0.5), (20.0, 1.0), (4.0, 1.0)):
        assert abs(phi(0.0, fs, k) - 1.0) < 1e-15
        assert phi(fs, fs, k) == 0.0
        assert phi(2.0 * fs, fs, k) == 0.0
    assert phi(0.3, 0.0, 20.0) == 0.0


def test_phi_closed_form_and_monotone():
    k, fs = 20.0, 0.5
    f = 0.25
    expect = (math.exp(-5.0) - math.exp(-10.0)) / (1.0 - math.exp(-10.0))
    assert abs(phi(f, fs, k) - expect) < 1e-15
    vals = [phi(0.01 * i, fs, k) for i in range(51)]
    assert all(vals[i] > vals[i + 1] for i in range(50))


def test_phi_small_force_decay():
    # far below f* the factor decays like exp(-k f)
    k, fs = 20.0, 1.0
    for f in (0.05, 0.1, 0.2):
        assert abs(phi(f, fs, k) - math.exp(-k * f)) < 1e-8


# ---------------------------------------------------------------------------
# The controller's host logic on a stand-in scene: forces are prescribed per
# step, and the targets the controller hands over are recorded.


class _RecordingScene:
    """Stands in for a zema Scene: returns prescribed per-finger forces and
    records every batch of kinematic targets and every step."""

    def __init__(self, finger_ids, force_of_step):
        self.body_of = {idx: 10 + j for j, idx in enumerate(finger_ids)}
        self.force_of_step = force_of_step
        self.steps = 0
        self.calls = []

    def affine_body_id(self, idx):
        return self.body_of[idx]

    def contact_forces(self):
        F = np.zeros((10 + len(self.body_of), 3))
        for idx, b in self.body_of.items():
            F[b] = (0.0, self.force_of_step(self.steps, idx), 0.0)
        return F

    def set_kinematic_targets(self, idx, Q):
        self.calls.append((list(idx), np.array(Q, dtype=np.float64)))

    def step(self, n, script=True):
        assert n == 1 and not script
        self.steps += 1
        return {"newton_iters": 1}


def _two_env_scene(dt=0.01):
    # fingers 3, 4 close on env 0 and fingers 7, 8 on env 1, from either side
    fingers = []
    for idx, sign, env in ((3, 1.0, 0), (4, -1.0, 0), (7, 1.0, 1), (8, -1.0, 1)):
        q0 = np.zeros(12)
        q0[0], q0[2] = float(env), 0.1 * sign
        q0[3], q0[7], q0[11] = 1.0, 1.0, 1.0
        fingers.append((idx, sign, q0))
    affines = {idx: types.SimpleNamespace(env=env) for idx, env in ((3, 0), (4, 0), (7, 1), (8, 1))}
    return types.SimpleNamespace(fingers=fingers, affines=affines, params=types.SimpleNamespace(dt=dt))


def test_autograsp_closes_by_phi_then_lifts_each_env_on_its_own():
    sc = _two_env_scene()
    f_star, k, v, H, L = 1.0, 20.0, 0.05, 0.05, 4
    # env 0 touches at step 3 and reaches the stop force at step 6; env 1 never touches
    def force(step, idx):
        if idx in (3, 4):
            return 0.0 if step < 3 else (0.3 if step < 6 else 0.97)
        return 0.0
    gpu = _RecordingScene([3, 4, 7, 8], force)
    ctl = AutoGrasp(gpu, sc, close_speed=v, f_star=f_star, k=k, lift_height=H, lift_steps=L)
    q0 = {idx: q.copy() for idx, _, q in sc.fingers}
    sign = {idx: s for idx, s, _ in sc.fingers}
    expect = {idx: q.copy() for idx, q in q0.items()}
    for step in range(12):
        ctl.step()
        idx, Q = gpu.calls[-1]
        assert len(gpu.calls) == step + 1 and sorted(idx) == [3, 4, 7, 8] and Q.shape == (4, 12)
        for j, i in enumerate(idx):
            f = force(step, i)
            if i in (3, 4) and step >= 6:
                # lifting: the closing coordinate holds, the height rises L times
                if step - 6 < L:
                    expect[i][1] += H / L
            else:
                expect[i][2] -= sign[i] * phi(f, f_star, k) * v * sc.params.dt
            assert np.array_equal(Q[j], expect[i]), (step, i)
    assert gpu.steps == 12
    # env 0 lifted by exactly H and stopped closing; env 1 kept closing at full speed
    for i in (3, 4):
        assert abs(expect[i][1] - H) < 1e-15
        assert np.array_equal(expect[i][[0, 3, 4, 5, 6, 7, 8, 9, 10, 11]], q0[i][[0, 3, 4, 5, 6, 7, 8, 9, 10, 11]])
    for i in (7, 8):
        assert abs(expect[i][2] - (q0[i][2] - 12 * sign[i] * v * sc.params.dt)) < 1e-15
    assert [h["lifting"] for h in ctl.history][5:7] == [{0: False, 1: False}, {0: True, 1: False}]


def test_autograsp_lifts_when_closing_stalls_below_the_stop_force():
    # 0.6 N with k = 20 1/N gives phi = (e^-12 - e^-20)/(1 - e^-20) < 1e-4: stalled
    sc = _two_env_scene()
    gpu = _RecordingScene([3, 4, 7, 8], lambda step, idx: 0.6)
    ctl = AutoGrasp(gpu, sc, lift_steps=2)
    assert phi(0.6, ctl.f_star, ctl.k) <= ctl.phi_stall
    ctl.step()
    assert ctl.lift_done == {0: 1, 1: 1}
    ctl.step()
    ctl.step()
    assert ctl.lift_done == {0: 2, 1: 2}
    # the fingers rose by lift_height and never closed
    idx, Q = gpu.calls[-1]
    for j, i in enumerate(idx):
        q0 = dict((f[0], f[2]) for f in sc.fingers)[i]
        assert Q[j][2] == q0[2] and abs(Q[j][1] - ctl.lift_height) < 1e-15
