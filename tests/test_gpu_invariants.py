"""Invariants of the CUDA stepper's trajectories, checked independently of
the oracle's arithmetic: no triangle of one body crosses a triangle of another
at any step (an FP64 segment-triangle test written here), in both precisions;
and, with no gravity and no fixed or kinematic bodies, total linear momentum
is conserved (every term of the incremental potential except inertia is
translation invariant, Eq. 1-2), up to the linear solve's residual."""
import numpy as np
import pytest

from geometry import tri_tri_intersect
from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def gpu_scene(sc, **kw):
    from paper_2311_05945_b300.zema import Scene
    return Scene(sc, **kw)


def surface_positions(gpu, sc, sv):
    """World positions of the surface vertices (body, affine flag, index) from
    the GPU scene's states: soft vertices by global index, affine A x0 + p."""
    soft = np.concatenate([gpu.tet_positions(i) for i in range(len(sc.tets))]) if sc.tets else np.zeros((0, 3))
    order = sc.body_order()
    P = np.zeros((len(sv), 3))
    for i, (b, _, idx) in enumerate(sv):
        kind, k = order[b]
        if kind == "tet":
            P[i] = soft[idx]
        else:
            q = gpu.affine_q(k)
            P[i] = q[3:].reshape(3, 3) @ sc.affines[k].V[idx] + q[:3]
    return P


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,n_steps", [("tiny", 15), ("c1", 25)])
def test_gpu_trajectory_has_no_intersections(name, n_steps, precision):
    sc = S.scene_tiny_contact(mu=0.5) if name == "tiny" else S.scene_c1()
    sv, _, t = Oracle(sc).surface()  # surface topology only
    body = sv[t[:, 0], 0]
    i, j = np.triu_indices(len(t), 1)
    m = body[i] != body[j]
    ii, jj = i[m], j[m]
    gpu = gpu_scene(sc, precision=precision)
    touched = False
    for k in range(n_steps):
        st = gpu.step(1)
        assert st["dmin"] > 0
        touched |= st["max_active"] > 0
        P = surface_positions(gpu, sc, sv)
        assert not tri_tri_intersect(P, t[ii], t[jj]).any(), k
    assert touched


def test_gpu_momentum_conservation_zero_gravity():
    # a soft cube at 2 m/s hits a free box; FP64 solve with a tight linear
    # tolerance, so that the Newton steps conserve momentum to round-off
    p = S.Params(dt=0.01, gravity=(0.0, 0.0, 0.0), pcg_rel_tol=1e-10)
    sc = S.Scene("momentum", p)
    X, T = S.soft_cube(3, 0.2, (0.0, 0.0, 0.0))
    v0 = np.zeros_like(X)
    v0[:, 0] = 2.0
    sc.tets.append(S.TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=0.3, v0=v0))
    V, F = S.box_surface((0.15, 0.15, 0.15), 2)
    sc.affines.append(S.AffineBody(V, F, S.q_identity((0.2 + 0.0755 + 0.01, 0.1, 0.08)), rho=1000.0,
                                   stiffness=1e8, mu=0.3))
    orc = Oracle(sc)
    m = orc.lumped_mass()
    M, mb, _ = orc.affine_mass(0)  # mass matrix of Eq. 2 (scene data, not a result)
    gpu = gpu_scene(sc, tol_scale=1e-2, precision=0)

    def momentum():
        st = gpu.get_state(gpu.tet_body_id(0))
        n = len(st) // 6
        v = st[3 * n:].reshape(n, 3)
        qd = gpu.get_state(gpu.affine_body_id(0))[12:]
        return (m[:, None] * v).sum(0) + mb * qd[:3] + qd[3:].reshape(3, 3) @ M[0, 3:6]

    P0 = momentum()
    touched = False
    for k in range(12):
        st = gpu.step(1)
        touched |= st["max_active"] > 0
    assert touched
    err = np.abs(momentum() - P0).max() / np.abs(P0).max()
    print(f"momentum drift over 12 contact steps: {err:.3e} relative")
    assert err < 1e-8, err
