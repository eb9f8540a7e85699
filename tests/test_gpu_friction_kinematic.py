"""Closed forms of friction and of the kinematic augmented Lagrangian on the
CUDA stepper, in both precisions, next to the oracle: a block sliding down a
slope at g (sin theta - mu cos theta) (Eq. 9-10 with the barrier's normal
force, Eq. 4), a block held by static friction below the friction angle, and a
kinematic body on its scripted target after every step (Eq. 13)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def gpu_scene(sc, **kw):
    from paper_2311_05945_b300.zema import Scene
    return Scene(sc, **kw)


def vertices(obj, sc, i):
    q = obj.affine_q(i)
    return sc.affines[i].V @ q[3:].reshape(3, 3).T + q[:3]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mu", [0.1, 0.2])
def test_gpu_sliding_down_a_slope(mu, precision):
    theta = 0.3
    sc = S.scene_slope(theta, mu)
    orc = Oracle(sc, tol_scale=1e-2)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=precision)
    diag = orc.diag()
    down = -np.array([np.cos(theta), np.sin(theta), 0.0])
    vs = []
    for k in range(24):
        orc.step(1)
        st = gpu.step(1)
        assert st["dmin"] > 0
        err = np.abs(vertices(orc, sc, 1) - vertices(gpu, sc, 1)).max()
        assert err < 1e-5 * diag, (k, err / diag)
        vs.append(gpu.get_state(gpu.affine_body_id(1))[12:15] @ down)
    a = (vs[23] - vs[11]) / (12 * sc.params.dt)
    a_ref = 9.81 * (np.sin(theta) - mu * np.cos(theta))
    assert abs(a - a_ref) < 0.02 * a_ref, (a, a_ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_block_sticks_below_the_friction_angle(precision):
    sc = S.scene_slope(0.3, 0.5, n_steps=30)
    gpu = gpu_scene(sc, tol_scale=1e-3, precision=precision)
    speeds = []
    for k in range(30):
        st = gpu.step(1)
        assert st["dmin"] > 0
        speeds.append(np.linalg.norm(gpu.get_state(gpu.affine_body_id(1))[12:15]))
    assert max(speeds[10:]) < sc.params.eps_v, speeds


@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_kinematic_body_tracks_its_target(precision):
    sc = S.scene_kinematic_track(10)
    orc = Oracle(sc)
    gpu = gpu_scene(sc, precision=precision)
    tol = sc.params.newton_tol_rel * orc.diag() * sc.params.dt
    rounds = 0
    for n in range(6):
        st = gpu.step(1)
        rounds += st["al_rounds"]
        q = gpu.affine_q(0)
        assert np.abs(q - S.kinematic_track_target(n)).max() <= tol, (n, q - S.kinematic_track_target(n))
    assert rounds > 0
