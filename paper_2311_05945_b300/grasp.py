"""Force-controlled parallel-jaw grasp: the paper's kinematic controller with
force feedback and its AutoGrasp / lift procedure (Sec. Controller, Contact
Force Sensing, Simulation Procedure).

Each step every finger measures its contact force magnitude f (the resultant
barrier gradient over the finger's vertices, zema_contact_forces) and its
kinematic target advances by phi(f) times the closing increment, where phi
decays exponentially from 1 at f = 0 to 0 at the desired force f* (and
stays 0 above it), with rate k.  When every finger of an environment has
reached f* (phi = 0) the grasp of that environment is established and its
fingers lift by lift_height over lift_steps while holding their closing
position.

Readings of the paper:
- The controller's example desired force (0.5 N) and the AutoGrasp stop
  force (1 N per finger) differ; here f* is the stop force (default 1 N), so
  the controller comes to rest where AutoGrasp stops.
- The joint increment is not given; it is close_speed x h per step here.
  Because phi only reaches 0 at f* itself, the force approaches f*
  asymptotically.  Closing therefore ends when every finger of the env has
  reached stop_ratio x f*, or when closing has stalled (phi <= phi_stall for
  every finger: with the paper's k = 20 1/N and a few-cm/s increment that
  happens near 0.35 N), or after max_close_steps.
"""
import math

import numpy as np

K_PHI = 20.0     # 1/N, the paper's decay rate
F_STOP = 1.0     # N, AutoGrasp stops closing when every finger reaches it


def phi(f, f_star=F_STOP, k=K_PHI):
    """Closing-speed factor: (exp(-k f) - exp(-k f*)) / (1 - exp(-k f*)) for
    0 <= f < f*, 0 for f >= f* (and for f* <= 0)."""
    if f_star <= 0.0 or f >= f_star:
        return 0.0
    f = max(f, 0.0)
    ef = math.exp(-k * f_star)
    return (math.exp(-k * f) - ef) / (1.0 - ef)


class AutoGrasp:
    """Drives the fingers of a grasp scene (scene.fingers) on a zema Scene."""

    def __init__(self, gpu, scene, close_speed=0.05, f_star=F_STOP, k=K_PHI, lift_height=0.05,
                 lift_steps=200, stop_ratio=0.95, phi_stall=1e-4, max_close_steps=1000):
        self.gpu, self.scene = gpu, scene
        self.close_speed, self.f_star, self.k = close_speed, f_star, k
        self.stop_ratio, self.phi_stall, self.max_close_steps = stop_ratio, phi_stall, max_close_steps
        self.close_steps = 0
        self.lift_height, self.lift_steps = lift_height, lift_steps
        self.dt = scene.params.dt
        # per finger: current target, and its env
        self.q = {idx: q0.copy() for idx, _, q0 in scene.fingers}
        self.sign = {idx: sign for idx, sign, _ in scene.fingers}
        self.env = {idx: scene.affines[idx].env for idx, _, _ in scene.fingers}
        self.lift_done = {e: None for e in self.env.values()}  # env -> lift steps taken, None while closing
        self.history = []

    def finger_forces(self):
        F = self.gpu.contact_forces()
        return {idx: float(np.linalg.norm(F[self.gpu.affine_body_id(idx)])) for idx in self.q}

    def step(self):
        """Measure, set the fingers' targets for the next state, step once."""
        f = self.finger_forces()
        for e in self.lift_done:
            if self.lift_done[e] is not None:
                continue
            mine = [i for i in self.q if self.env[i] == e]
            reached = all(f[i] >= self.stop_ratio * self.f_star for i in mine)
            stalled = all(phi(f[i], self.f_star, self.k) <= self.phi_stall for i in mine)
            if reached or stalled or self.close_steps >= self.max_close_steps:
                self.lift_done[e] = 0
        self.close_steps += 1
        for idx in self.q:
            e = self.env[idx]
            if self.lift_done[e] is None:
                self.q[idx][2] -= self.sign[idx] * phi(f[idx], self.f_star, self.k) * self.close_speed * self.dt
            elif self.lift_done[e] < self.lift_steps:
                self.q[idx][1] += self.lift_height / self.lift_steps
        if self.q:
            idx = list(self.q)
            self.gpu.set_kinematic_targets(idx, np.array([self.q[i] for i in idx], dtype=np.float64))
        for e in self.lift_done:
            if self.lift_done[e] is not None and self.lift_done[e] < self.lift_steps:
                self.lift_done[e] += 1
        st = self.gpu.step(1, script=False)
        self.history.append({"forces": f, "lifting": {e: v is not None for e, v in self.lift_done.items()}})
        return st
