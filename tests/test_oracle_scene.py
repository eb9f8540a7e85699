"""Scene-level pins of the oracle: analytic free fall, closed-form mass
properties, finite differences of the complete incremental potential,
monotone Newton energies, intersection-free trajectories (independent
triangle-triangle tests), momentum conservation, Coulomb sliding on flat
ground and down a slope, static friction below the friction angle, kinematic
target tracking by the augmented Lagrangian, the barrier-stiffness floor and
the initial gradient-balance stiffness (clamped and unclamped) and its
doubling rule."""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

from geometry import tri_tri_intersect


def test_free_fall_analytic():
    # Eq. 1 / Eq. 2 with no contact: the minimiser of the IP is the predictor,
    # x_n = x_0 + h^2 g n (n+1) / 2 from rest, reached in one Newton step.
    s = S.scene_free_fall(n_steps=4)
    o = Oracle(s)
    x0 = o.tet_positions().copy()
    q0 = o.affine_q(0).copy()
    st = o.step(4)
    h, g, n = s.params.dt, s.params.gravity[1], 4
    dy = h * h * g * n * (n + 1) / 2
    x = o.tet_positions()
    assert np.abs(x[:, 1] - x0[:, 1] - dy).max() < 1e-12
    assert np.abs(x[:, [0, 2]] - x0[:, [0, 2]]).max() < 1e-12
    q = o.affine_q(0)
    assert abs(q[1] - q0[1] - dy) < 1e-12
    assert np.abs(np.delete(q - q0, 1)).max() < 1e-12
    assert np.all(st[:, 0, 0] == 1)


def test_surface_and_lumped_mass_c1():
    s = S.scene_c1()
    o = Oracle(s)
    c = o.counts()
    # soft cube surface: 98 verts, 192 tris, 288 edges; plus two boxes (8, 12, 18 each)
    assert c["n_sv"] == 98 + 16 and c["n_tris"] == 192 + 24 and c["n_edges"] == 288 + 36
    sv, e, t = o.surface()
    soft_t = t[:192]
    P = np.array([s.tets[0].X[sv[i, 2]] for i in range(98)])
    v = P[soft_t]
    vol = np.einsum("ij,ij->i", v[:, 0], np.cross(v[:, 1], v[:, 2])).sum() / 6.0
    assert abs(vol - 1.0) < 1e-12  # closed and outward: encloses the unit cube
    # every surface edge borders exactly two triangles
    from collections import Counter
    cnt = Counter()
    for tri in soft_t:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            cnt[tuple(sorted((tri[a], tri[b])))] += 1
    assert set(cnt.values()) == {2}
    m = o.lumped_mass()
    assert abs(m.sum() - 1000.0) < 1e-9


@pytest.mark.parametrize("ext,center", [((0.3, 0.5, 0.7), (0, 0, 0)), ((0.2, 0.1, 0.4), (0.3, -0.2, 0.1))])
def test_affine_mass_box(ext, center):
    # M_b = integral rho J^T J (Eq. 2) for a box: m = rho a b c, p-block m I,
    # a_i-blocks S = integral rho x0 x0^T = m (diag(a^2, b^2, c^2)/12 + c c^T),
    # p-a_i coupling m c (zero when centred).
    V, F = S.box_surface(ext, 3)
    V = V + np.array(center)
    s = S.Scene("box", S.Params())
    s.affines.append(S.AffineBody(V, F, S.q_identity((0, 0, 0)), rho=700.0, stiffness=1e8, mu=0.5))
    o = Oracle(s)
    M, m, vol = o.affine_mass(0)
    a, b, c = ext
    assert abs(vol - a * b * c) < 1e-14
    assert abs(m - 700.0 * a * b * c) < 1e-11
    cc = np.array(center, dtype=float)
    Sref = m * (np.diag([a * a, b * b, c * c]) / 12.0 + np.outer(cc, cc))
    assert np.allclose(M[:3, :3], m * np.eye(3), atol=1e-12)
    for i in range(3):
        blk = M[3 + 3 * i:6 + 3 * i, 3 + 3 * i:6 + 3 * i]
        assert np.allclose(blk, Sref, atol=1e-12)
        cpl = M[i, 3 + 3 * i:6 + 3 * i]
        assert np.allclose(cpl, m * cc, atol=1e-12)
        for j in range(3):
            if j != i:
                assert np.abs(M[3 + 3 * i:6 + 3 * i, 3 + 3 * j:6 + 3 * j]).max() < 1e-15


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_affine_mass_tetrahedron(seed):
    # M_b (Eq. 2) of a single tetrahedron, skewed and off the origin, against
    # the closed form of its moments: m = rho V, integral rho x0 = m c with c
    # the vertex mean, integral rho x0 x0^T = rho V / 20 (sum v v^T + s s^T)
    # with s the vertex sum.  Unlike an axis-aligned box, every entry of the
    # second moment is nonzero, so a transposed or misplaced term shows.
    rng = np.random.default_rng(40 + seed)
    v = rng.standard_normal((4, 3)) * 0.3 + rng.standard_normal(3)
    if np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], 1)) < 0:
        v[[1, 2]] = v[[2, 1]]
    F = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], dtype=np.int32)
    vol = np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], 1)) / 6.0
    tri = v[F]
    assert abs(np.einsum("ij,ij->i", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum() / 6.0 - vol) < 1e-12
    rho = 900.0
    s = S.Scene("tet", S.Params())
    s.affines.append(S.AffineBody(v, F, S.q_identity((0, 0, 0)), rho=rho, stiffness=1e8, mu=0.5))
    o = Oracle(s)
    M, m, V = o.affine_mass(0)
    assert abs(V - vol) <= 1e-12 * vol and abs(m - rho * vol) <= 1e-12 * rho * vol
    c = v.mean(0)
    sv = v.sum(0)
    Sref = rho * vol / 20.0 * (v.T @ v + np.outer(sv, sv))
    scale = np.abs(Sref).max()
    for i in range(3):
        assert abs(M[i, i] - m) <= 1e-12 * m
        assert np.allclose(M[i, 3 + 3 * i:6 + 3 * i], m * c, rtol=0, atol=1e-12 * m * np.abs(c).max())
        assert np.allclose(M[3 + 3 * i:6 + 3 * i, 3 + 3 * i:6 + 3 * i], Sref, rtol=0, atol=1e-12 * scale)


def _advance(o, n):
    for _ in range(n):
        o.step(1)


def test_full_energy_gradient_fd():
    # Complete B_t + D (Eq. 4, Eq. 11) with inertia, elasticity, orthogonality,
    # barrier and lagged friction active: gradient against central differences.
    s = S.scene_tiny_contact(mu=0.5)
    o = Oracle(s)
    _advance(o, 6)
    o.prepare(0, friction=True)
    y0 = o.dofs()
    rng = np.random.default_rng(3)
    y = y0 + 2e-5 * rng.standard_normal(len(y0)) * (np.abs(y0) > -1)
    E, g, H, na = o.eval(y, grad=True, hess=True)
    assert na > 0 and np.isfinite(E)
    eps = 1e-8
    fd = np.zeros_like(y)
    for i in range(len(y)):
        e = np.zeros_like(y)
        e[i] = eps
        fd[i] = (o.eval(y + e)[0] - o.eval(y - e)[0]) / (2 * eps)
    err = np.abs(fd - g).max() / np.abs(g).max()
    assert err < 1e-5, err
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert ev.min() > 0  # projected Hessian plus mass terms: SPD


def surface_world(o, s):
    """World positions of the oracle's surface vertices, computed here from
    the body states (soft: global vertex index; affine: A x0 + p)."""
    sv, e, t = o.surface()
    soft = np.concatenate([o.tet_positions(i) for i in range(len(s.tets))]) if s.tets else np.zeros((0, 3))
    P = np.zeros((len(sv), 3))
    for i, (b, aff, idx) in enumerate(sv):
        kind, k = s.body_order()[b]
        if kind == "tet":
            P[i] = soft[idx]
        else:
            q = o.get_state(b)[:12]
            A = q[3:].reshape(3, 3)
            P[i] = A @ s.affines[k].V[idx] + q[:3]
    return sv, t, P


def test_monotone_energy_no_intersection_tiny():
    s = S.scene_tiny_contact(mu=0.5)
    o = Oracle(s)
    for step in range(12):
        st = o.step(1)
        log = o.energy_log()
        assert np.all(np.diff(log) <= 1e-12 * np.abs(log).max()), log
        assert st[0, 0, 4] > 0  # d_min > 0
        sv, t, P = surface_world(o, s)
        body = sv[t[:, 0], 0]
        i, j = np.triu_indices(len(t), 1)
        m = body[i] != body[j]
        shared = np.array([len(set(t[a]) & set(t[b])) > 0 for a, b in zip(i[m], j[m])])
        ii, jj = i[m][~shared], j[m][~shared]
        assert not tri_tri_intersect(P, t[ii], t[jj]).any()


def test_momentum_conservation_zero_gravity():
    # no gravity, no fixed or kinematic bodies: total linear momentum
    # sum m_i v_i + sum (m_b pdot_b + Adot_b integral rho x0) is conserved
    p = S.Params(dt=0.01, gravity=(0.0, 0.0, 0.0))
    s = S.Scene("momentum", p)
    X, T = S.soft_cube(3, 0.2, (0.0, 0.0, 0.0))
    v0 = np.zeros_like(X)
    v0[:, 0] = 2.0
    s.tets.append(S.TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=0.3, v0=v0))
    V, F = S.box_surface((0.15, 0.15, 0.15), 2)
    s.affines.append(S.AffineBody(V, F, S.q_identity((0.2 + 0.0755 + 0.01, 0.1, 0.08)), rho=1000.0,
                                  stiffness=1e8, mu=0.3))
    o = Oracle(s, tol_scale=1e-3)
    m = o.lumped_mass()
    M, mb, _ = o.affine_mass(0)

    def momentum():
        st = o.get_state(0)
        n = len(st) // 6
        v = st[3 * n:].reshape(n, 3)
        qs = o.get_state(1)
        qd = qs[12:]
        c = M[0, 3:6] / mb * mb  # integral rho x0
        Ad = qd[3:].reshape(3, 3)
        return (m[:, None] * v).sum(0) + mb * qd[:3] + Ad @ c

    P0 = momentum()
    touched = False
    for k in range(12):
        st = o.step(1)
        touched |= st[0, 0, 3] > 0
    assert touched
    P1 = momentum()
    assert np.abs(P1 - P0).max() < 1e-6 * np.abs(P0).max()


def test_coulomb_sliding_deceleration():
    # A flat affine block sliding on a fixed floor decelerates at mu g (Eq. 9):
    # once settled, the lagged normal force balances gravity and the kinetic
    # friction force is mu N.  The block first settles at rest, then gets 1 m/s.
    p = S.Params(dt=0.01)
    s = S.Scene("slide", p)
    Vf, Ff = S.box_surface((4.0, 0.1, 4.0), 1)
    s.affines.append(S.AffineBody(Vf, Ff, S.q_identity((0, -0.05, 0)), rho=1000.0, stiffness=1e8,
                                  mu=0.5, mode=1))
    V, F = S.box_surface((0.2, 0.04, 0.2), 1)
    s.affines.append(S.AffineBody(V, F, S.q_identity((0.3, 0.02 + 0.002, 0.1)), rho=1000.0,
                                  stiffness=1e8, mu=0.5))
    o = Oracle(s)
    for _ in range(40):
        o.step(1)
    st = o.get_state(1)
    st[12:] = 0.0
    st[12] = 1.0
    o.set_state(1, st)
    vs = []
    for k in range(16):
        o.step(1)
        vs.append(o.get_state(1)[12])
    vs = np.array(vs)
    dec = -(vs[14] - vs[4]) / (10 * p.dt)
    assert abs(dec - 0.5 * 9.81) < 0.02 * 0.5 * 9.81, (dec, vs)


def test_brute_candidates_match_numpy_definition():
    s = S.random_state_scene(7)
    o = Oracle(s)
    sv, e, t = o.surface()
    _, _, P = surface_world(o, s)
    P = P + 0.003 * np.random.default_rng(7).standard_normal(P.shape)
    order = s.body_order()
    bclass = np.array([0 if k == "tet" else (1 + (s.affines[i].mode == 1) + 2 * (s.affines[i].mode == 2))
                       for k, i in order], dtype=np.int32)
    benv = np.zeros(len(order), dtype=np.int32)
    infl = 0.05
    pt, ee = O.brute_pairs(P, sv[:, 0], bclass, benv, e, t, infl)
    # numpy all-pairs definition
    lo = lambda ids: P[ids].min(1) - infl
    hi = lambda ids: P[ids].max(1) + infl
    plo, phi = P - infl, P + infl
    tlo, thi = lo(t), hi(t)
    ov = np.all((plo[:, None] <= thi[None]) & (tlo[None] <= phi[:, None]), -1)
    share = (t[None, :, :] == np.arange(len(P))[:, None, None]).any(-1)
    svb = sv[:, 0]
    same_aff = (svb[:, None] == svb[t[:, 0]][None]) & (bclass[svb][:, None] != 0)
    ref_pt = set(map(tuple, np.argwhere(ov & ~share & ~same_aff)))
    got_pt = set((a, b) for a, b in zip(pt[:, 0], [tuple(x) for x in pt[:, 1:]]))
    tri_index = {tuple(x): i for i, x in enumerate(t)}
    got_pt = set((a, tri_index[b]) for a, b in got_pt)
    assert got_pt == ref_pt and len(ref_pt) > 0
    elo, ehi = lo(e), hi(e)
    ov = np.all((elo[:, None] <= ehi[None]) & (elo[None] <= ehi[:, None]), -1)
    share = (e[:, None, :, None] == e[None, :, None, :]).any((-1, -2))
    same_aff = (svb[e[:, 0]][:, None] == svb[e[:, 0]][None]) & (bclass[svb[e[:, 0]]][:, None] != 0)
    iu = np.triu(np.ones_like(ov), 1)
    ref_ee = set(map(tuple, np.argwhere(ov & ~share & ~same_aff & iu)))
    edge_index = {tuple(x): i for i, x in enumerate(e)}
    got_ee = set((edge_index[(a, b)], edge_index[(c, d)]) for a, b, c, d in ee)
    assert got_ee == ref_ee and len(ref_ee) > 0


def spring_scene(model=0):
    """A 3x3x3-vertex soft cube in free fall with springs pulling four of its
    vertices towards targets 1 cm off their rest positions."""
    p = S.Params(dt=0.01)
    s = S.Scene("springs", p)
    X, T = S.soft_cube(3, 0.2, (0.0, 1.0, 0.0))
    s.tets.append(S.TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=0.3, model=model))
    verts = np.array([0, 4, 13, 26], dtype=np.int32)
    targets = X[verts] + np.array([0.01, -0.01, 0.005])
    s.springs.append((0, verts, targets, 2.0e3))
    return s, verts, targets


@pytest.mark.parametrize("model", [0, 1, 2])
def test_spring_forces_balance_momentum(model):
    # springs are a potential h^2 k |x - t|^2: at a converged step the soft
    # body's momentum balance has only inertia, gravity and springs (elastic
    # forces cancel inside the body): sum_v m_v (x_v - xhat_v) / h^2 +
    # sum_springs 2 k (x_v - t_v) = 0
    s, verts, targets = spring_scene(model)
    o = Oracle(s, tol_scale=1e-4)
    m = o.lumped_mass()
    h = s.params.dt
    g = np.array(s.params.gravity)
    for _ in range(3):
        st0 = o.get_state(0)
        n = len(s.tets[0].X)
        x0, v0 = st0[:3 * n].reshape(-1, 3), st0[3 * n:].reshape(-1, 3)
        o.step(1)
        x1 = o.tet_positions()
        xhat = x0 + h * v0 + h * h * g
        inertia = (m[:, None] * (x1 - xhat)).sum(0) / (h * h)
        spring = (2.0 * 2.0e3 * (x1[verts] - targets)).sum(0)
        scale = np.abs(spring).max() + np.abs(inertia).max()
        assert np.abs(inertia + spring).max() < 1e-6 * scale


def test_joint_constraint_zero_along_axis_only():
    # the constraint vanishes at the initial state and when body 2 moves
    # along the axis; a sideways move d of body 2 gives |slide part| = |d|
    # (r = -d, axis unit), and a relative rotation gives a nonzero rotation part
    s = S.scene_joint(axis=(1.0, 0.0, 0.0), fixed_base=False, gravity=(0.0, 0.0, 0.0))
    o = Oracle(s)
    assert np.abs(o.joint_constraint(0)).max() < 1e-15
    st = o.get_state(1)
    for d, along in (((0.05, 0.0, 0.0), True), ((0.0, 0.03, 0.0), False), ((0.0, 0.0, -0.02), False)):
        x = st.copy()
        x[0:3] += d
        o.set_state(1, x)
        c = o.joint_constraint(0)
        assert np.abs(c[:9]).max() < 1e-15
        if along:
            assert np.abs(c[9:]).max() < 1e-15
        else:
            assert abs(np.linalg.norm(c[9:]) - np.linalg.norm(d)) < 1e-15
    x = st.copy()
    th = 0.01
    x[3:12] = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]]).ravel()
    o.set_state(1, x)
    assert np.abs(o.joint_constraint(0)[:9]).max() > 0.5 * th


def test_joint_along_gravity_is_free_fall():
    # fixed base, axis along gravity: the slider's free fall keeps c = 0, so
    # the joint exerts no force and the motion is the exact free fall
    s = S.scene_joint(axis=(0.0, 1.0, 0.0), fixed_base=True)
    o = Oracle(s, tol_scale=1e-3)
    q0 = o.affine_q(1).copy()
    o.step(5)
    h, g, n = s.params.dt, s.params.gravity[1], 5
    q = o.affine_q(1)
    assert abs(q[1] - q0[1] - h * h * g * n * (n + 1) / 2) < 1e-9
    assert np.abs(np.delete(q - q0, 1)).max() < 1e-9


def test_joint_across_gravity_holds_the_slider():
    # fixed base, axis horizontal: gravity acts across the axis, and after
    # the augmented-Lagrangian rounds the slide part of c (the slider's drop)
    # stays within the Newton step tolerance
    s = S.scene_joint(axis=(1.0, 0.0, 0.0), fixed_base=True)
    o = Oracle(s)
    tol = s.params.newton_tol_rel * o.diag() * s.params.dt
    for _ in range(5):
        o.step(1)
        c = o.joint_constraint(0)
        assert np.abs(c[9:]).max() <= tol
        assert np.abs(c[:9]).max() <= s.params.newton_tol_rel * s.params.dt
    assert abs(o.affine_q(1)[1] - 1.0) < 5 * tol


@pytest.mark.parametrize("mu", [0.1, 0.2])
def test_sliding_down_a_slope(mu):
    # Eq. 9-10 with the normal force of the barrier (Eq. 4): on a slope of
    # angle theta with mu < tan(theta) the block slides with the closed-form
    # acceleration g (sin(theta) - mu cos(theta)) along the downhill direction
    # -(cos(theta), sin(theta), 0).  A wrong normal-force scale, a friction
    # term that ignores the slope's normal, or a sign error changes it.
    theta = 0.3
    s = S.scene_slope(theta, mu)
    o = Oracle(s, tol_scale=1e-2)
    down = -np.array([np.cos(theta), np.sin(theta), 0.0])
    vs = []
    touched = 0
    for k in range(24):
        st = o.step(1)
        touched += st[0, 0, 3] > 0
        vs.append(o.get_state(1)[12:15] @ down)
    assert touched >= 20
    a = (vs[23] - vs[11]) / (12 * s.params.dt)
    a_ref = 9.81 * (np.sin(theta) - mu * np.cos(theta))
    assert abs(a - a_ref) < 0.02 * a_ref, (a, a_ref, vs)


def test_block_sticks_on_a_slope_below_the_friction_angle():
    # mu > tan(theta): static friction holds the block.  The smoothed friction
    # of Eq. 10 lets it creep, but only below eps_v (the speed at which f1
    # saturates), since the force needed is below mu N.
    theta = 0.3
    s = S.scene_slope(theta, 0.5, n_steps=30)
    o = Oracle(s, tol_scale=1e-3)
    speeds = []
    for k in range(30):
        st = o.step(1)
        assert st[0, 0, 3] > 0 or k < 3
        speeds.append(np.linalg.norm(o.get_state(1)[12:15]))
    assert max(speeds[10:]) < s.params.eps_v, speeds


def test_kinematic_body_tracks_its_target():
    # Eq. 13: the augmented Lagrangian drives a kinematic body onto its
    # scripted target.  The penalty kappa_A = 1e3 m alone leaves the body
    # behind by about 1e-3 of the gap between the inertial prediction and the
    # target (5 cm on the first step, above the Newton tolerance); the
    # multiplier update removes that lag, so after every step max |q - q~| is
    # within the tolerance, translation and A block alike.  A sign error in the
    # update doubles the lag instead.
    s, target = S.scene_kinematic_track(10), S.kinematic_track_target
    o = Oracle(s)
    tol = s.params.newton_tol_rel * o.diag() * s.params.dt
    rounds = 0
    for n in range(6):
        st = o.step(1)
        rounds += st[0, 0, 2]
        q = o.affine_q(0)
        assert np.abs(q - target(n)).max() <= tol, (n, q - target(n))
    assert rounds > 0

    # the same scene with the multiplier switched off misses the first target
    s0 = S.scene_kinematic_track(0)
    o0 = Oracle(s0)
    o0.step(1)
    assert np.abs(o0.affine_q(0) - target(0)).max() > tol


def test_kinematic_multiplier_extrapolation():
    # Each step's augmented-Lagrangian iteration starts from 2 lambda^t -
    # lambda^(t-1), and a step ends with one more multiplier update from its
    # accepted state.  The body stays on its target at every step either way;
    # once the start-up transient has passed, the extrapolated multipliers
    # need no further round, where the unextrapolated ones (lagging by one
    # step's change) would.  Without the end-of-step update the tolerance's
    # slack compounds through the extrapolation until the rounds fail to
    # converge (measured on this scene: a deviation of 8 x tol at step 8).
    target = S.kinematic_track_target
    rounds = {}
    for ex in (0, 1):
        s = S.scene_kinematic_track(10, n_steps=14)
        s.params.al_extrapolate = ex
        o = Oracle(s)
        tol = s.params.newton_tol_rel * o.diag() * s.params.dt
        r = []
        for n in range(14):
            st = o.step(1)
            r.append(int(st[0, 0, 2]))
            assert np.abs(o.affine_q(0) - target(n)).max() <= tol, (ex, n)
        rounds[ex] = r
    assert sum(rounds[1][4:]) == 0, rounds


def test_kinematic_multiplier_extrapolation_is_exact_for_a_linearly_growing_force():
    # A kinematic box driven along x with constant jerk j needs a force that
    # grows linearly in time.  The unextrapolated multipliers start every step
    # one step's change behind and leave the body a constant lag (under the
    # tolerance here, so no round runs); the extrapolated ones, 2 lambda^t -
    # lambda^(t-1) after the end-of-step update, are exact for a linear
    # history, so the body lands on its target.  A wrong extrapolation weight
    # or a missing end-of-step update leaves a lag of the unextrapolated size.
    def target(n, dt, j=1000.0):
        t = (n + 1) * dt
        q = np.zeros(12)
        q[:3] = (j * t ** 3 / 6.0, 0.5, 0.0)
        q[3] = q[7] = q[11] = 1.0
        return q

    last = {}
    for ex in (0, 1):
        s = S.scene_kinematic_track(10, n_steps=14)
        s.params.al_extrapolate = ex
        dt = s.params.dt
        s.script = lambda n, dt=dt: {0: target(n, dt)}
        o = Oracle(s)
        tol = s.params.newton_tol_rel * o.diag() * dt
        for n in range(14):
            o.step(1)
        last[ex] = np.abs(o.affine_q(0) - target(13, dt)).max() / tol
    assert last[0] > 0.5, last
    assert last[1] < 0.01, last


def test_kappa_min_is_a_thousand_mean_lumped_masses():
    # the adaptive barrier stiffness floor: 1e3 x the mean lumped soft-vertex mass
    s = S.scene_c1()
    o = Oracle(s)
    m = o.lumped_mass()
    o.step(1)  # kappa is set at the first step
    assert abs(o.kappa_min() - 1e3 * m.mean()) < 1e-12 * o.kappa_min()
    k = o.kappa()
    assert o.kappa_min() <= k <= 100 * o.kappa_min()


@pytest.mark.parametrize("name", ["tiny", "c1"])
def test_initial_kappa_balances_gradients(name):
    # reading c2: at the first step kappa = clamp(-gE . gB / |gB|^2, kappa_min,
    # 100 kappa_min), gE the gradient of the potential without the barrier and
    # gB the barrier gradient at unit stiffness, both at x^t.  Here both come
    # from the full potential's gradient at two stiffnesses (it is affine in
    # kappa without friction): gB = g(2) - g(1), gE = g(1) - gB.
    s = S.scene_tiny_contact(mu=0.5) if name == "tiny" else S.scene_c1()
    if name == "c1":
        o0 = Oracle(s)
        o0.step(12)  # in contact
        states = [o0.get_state(b) for b in range(len(s.body_order()))]
    o = Oracle(s)
    if name == "c1":
        for b, x in enumerate(states):
            o.set_state(b, x)
    o.prepare(0, friction=False)  # predictor, then the stiffness rule
    k0, kmin = o.kappa(), o.kappa_min()
    y = o.dofs()
    grads = []
    for k in (1.0, 2.0):
        o.set_kappa(0, k, kmin)
        grads.append(o.eval(y, grad=True)[1])
    gB = grads[1] - grads[0]
    gE = grads[0] - gB
    assert np.linalg.norm(gB) > 0
    ref = min(max(-(gE @ gB) / (gB @ gB), kmin), 100 * kmin)
    assert abs(k0 - ref) <= 1e-9 * ref, (k0, ref, kmin)


@pytest.mark.parametrize("kmin", [0.05, 7.5e-6])
def test_kappa_doubles_when_contact_closes_below_a_tenth_of_dhat(kmin):
    # reading c2, after each step: kappa <- min(2 kappa, 1e4 kappa_min) when
    # the step's d_min is below 0.1 dhat and below the previous step's d_min,
    # else unchanged.  A deliberately weak barrier (kappa = 0.05) lets the
    # contact close below 0.1 dhat; with kappa_min = 7.5e-6 the cap 1e4
    # kappa_min = 0.075 binds on the first doubling.
    s = S.scene_tiny_contact(mu=0.5)
    o = Oracle(s)
    o.set_kappa(0, 0.05, kmin)
    st = o.step(12)
    d, k = st[:, 0, 4], st[:, 0, 6]
    dhat = s.params.dhat
    d_prev, k_prev, doubled = np.inf, 0.05, 0
    for dk, kk in zip(d, k):
        if dk < 0.1 * dhat and dk < d_prev:
            expect = min(2 * k_prev, 1e4 * kmin)
            doubled += 1
        else:
            expect = k_prev
        assert kk == expect, (dk / dhat, kk, expect)
        d_prev, k_prev = dk, kk
    assert doubled >= 1


@pytest.mark.parametrize("model", [0, 1, 2])
@pytest.mark.parametrize("scale", [0.9, 1.15])
def test_uniformly_scaled_cube_elastic_energy(scale, model):
    # the scene-level elastic term h^2 sum_e V_e Psi(F_e) (Eq. 1) of a soft
    # cube scaled uniformly by s about the origin, at rest and with no
    # gravity: every F_e = s I, so the whole potential is h^2 V Psi(s I), with
    # mu = E / (2 (1 + nu)) and lam = E nu / ((1 + nu)(1 - 2 nu)) and, per
    # material (reading c9 and the two optional models):
    #   Neo-Hookean         3 mu/2 (s^2 - 1) - 3 mu ln s + 9 lam/2 (ln s)^2,
    #   St. Venant-Kirchhoff 3 mu e^2 + 9 lam/2 e^2 with e = (s^2 - 1)/2,
    #   fixed corotated     3 mu (s - 1)^2 + lam/2 (s^3 - 1)^2.
    # This pins the rest shapes, the volumes, the Lame parameters, the h^2 and
    # the per-body material switch.
    p = S.Params(dt=0.01, gravity=(0.0, 0.0, 0.0))
    s = S.Scene("scaled", p)
    X, T = S.soft_cube(4, 0.3, (-0.15, -0.15, -0.15))
    Ey, nu = 2e5, 0.35
    s.tets.append(S.TetBody(X, T, E=Ey, nu=nu, rho=1000.0, mu=0.5, model=model))
    o = Oracle(s)
    st = o.get_state(0)
    n = len(X)
    st[:3 * n] = (scale * X).ravel()
    st[3 * n:] = 0.0
    o.set_state(0, st)
    o.prepare(0)
    E = o.eval(o.dofs())[0]
    mu = Ey / (2 * (1 + nu))
    lam = Ey * nu / ((1 + nu) * (1 - 2 * nu))
    ls, e = np.log(scale), 0.5 * (scale ** 2 - 1)
    psi = (1.5 * mu * (scale ** 2 - 1) - 3 * mu * ls + 4.5 * lam * ls ** 2,
           3 * mu * e ** 2 + 4.5 * lam * e ** 2,
           3 * mu * (scale - 1) ** 2 + 0.5 * lam * (scale ** 3 - 1) ** 2)[model]
    ref = p.dt ** 2 * 0.3 ** 3 * psi
    assert abs(E - ref) <= 1e-10 * abs(ref), (E, ref)


@pytest.mark.parametrize("scale", [0.98, 1.03])
def test_scaled_affine_body_orthogonality_energy(scale):
    # the affine term h^2 lambda V |A A^T - I|_F^2 (Eq. 2) of a box at rest
    # with A = s R (R a rotation) and no gravity: A A^T = s^2 I, so the whole
    # potential is h^2 lambda V 3 (s^2 - 1)^2.  This pins the body volume, the
    # stiffness and the h^2 of the affine term.
    p = S.Params(dt=0.01, gravity=(0.0, 0.0, 0.0))
    s = S.Scene("scaled_affine", p)
    ext = (0.2, 0.3, 0.5)
    V, F = S.box_surface(ext, 2)
    lam = 1e8
    s.affines.append(S.AffineBody(V, F, S.q_identity((0.1, 0.2, 0.3)), rho=800.0, stiffness=lam, mu=0.5))
    o = Oracle(s)
    R = S.rotation_from_uniforms(0.3, 0.6, 0.9)
    st = o.get_state(0)
    st[3:12] = (scale * R).reshape(-1)
    st[12:] = 0.0
    o.set_state(0, st)
    o.prepare(0)
    E = o.eval(o.dofs())[0]
    ref = p.dt ** 2 * lam * np.prod(ext) * 3 * (scale ** 2 - 1) ** 2
    assert abs(E - ref) <= 1e-9 * abs(ref), (E, ref)


def test_kinematic_penalty_energy():
    # reading c13 of Eq. 13 before any multiplier update (lambda_A = 0): a
    # kinematic body at rest with no gravity, its target offset by delta,
    # carries exactly kappa_A / 2 |q - q~|^2 with kappa_A = 1e3 m.
    p = S.Params(dt=0.01, gravity=(0.0, 0.0, 0.0))
    s = S.Scene("kin_penalty", p)
    V, F = S.box_surface((0.1, 0.2, 0.3), 1)
    q0 = S.q_identity((0.0, 0.5, 0.0))
    s.affines.append(S.AffineBody(V, F, q0, rho=1000.0, stiffness=1e8, mu=0.0, mode=2))
    delta = np.array([0.01, -0.02, 0.005, 0.001, 0.0, -0.002, 0.0, 0.003, 0.0, 0.001, 0.0, 0.0])
    s.script = lambda n: {0: q0 + delta}
    o = Oracle(s)
    o.prepare(0)
    E = o.eval(o.dofs())[0]
    m = 1000.0 * 0.1 * 0.2 * 0.3
    ref = 0.5 * 1e3 * m * delta @ delta
    assert abs(E - ref) <= 1e-10 * ref, (E, ref)


def test_inertia_at_the_start_of_a_step():
    # Eq. 1-3 at x = x^t, no deformation: only inertia remains,
    # 1/2 sum m |x^t - x^hat|^2 = 1/2 M |h v + h^2 g|^2 for a soft cube and an
    # affine box (far apart) translating with the same velocity v, M their
    # total mass.  This pins the predictor and both mass models.
    p = S.Params(dt=0.01)
    s = S.Scene("inertia", p)
    X, T = S.soft_cube(3, 0.2, (0.0, 0.0, 0.0))
    v = np.array([0.3, -0.7, 1.1])
    s.tets.append(S.TetBody(X, T, E=1e5, nu=0.4, rho=1200.0, mu=0.5, v0=np.tile(v, (len(X), 1))))
    Vb, Fb = S.box_surface((0.1, 0.2, 0.3), 1)
    qd = np.zeros(12)
    qd[:3] = v
    s.affines.append(S.AffineBody(Vb, Fb, S.q_identity((2.0, 0.0, 0.0)), rho=800.0, stiffness=1e8, mu=0.5,
                                  qdot0=qd))
    o = Oracle(s)
    o.prepare(0)
    E = o.eval(o.dofs())[0]
    M = 1200.0 * 0.2 ** 3 + 800.0 * 0.1 * 0.2 * 0.3
    w = p.dt * v + p.dt ** 2 * np.array(p.gravity)
    ref = 0.5 * M * w @ w
    assert abs(E - ref) <= 1e-10 * ref, (E, ref)


def _tet_surface(v):
    """A tetrahedron as a closed, outward triangle mesh."""
    F = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], dtype=np.int32)
    if np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], 1)) < 0:
        F = F[:, ::-1].copy()
    return np.asarray(v, dtype=float), F


@pytest.mark.parametrize("gap", [0.2e-3, 0.5e-3, 0.9e-3])
def test_single_contact_barrier_and_friction_energy(gap):
    # one active pair at the scene level: the tip of a small affine tetrahedron
    # at height gap < dhat over the interior of a fixed tetrahedron's top face,
    # every other feature far beyond dhat; at rest, no gravity.  Without
    # friction the potential is kappa b(gap) (Eq. 4-5, no mollifier for a
    # point-triangle pair); with friction lagged at this state it adds
    # mu lambda f0(0) = mu kappa |b'(gap)| eps_v h / 3 (Eq. 9-10, readings c3
    # and c4), with mu the smaller of the two bodies' coefficients.
    p = S.Params(dt=0.01, gravity=(0.0, 0.0, 0.0))
    s = S.Scene("one_pair", p)
    Vf, Ff = _tet_surface(np.array([[-1.0, 0, -1], [1.0, 0, -1], [0, 0, 1.5], [0, -1.0, 0]]))
    s.affines.append(S.AffineBody(Vf, Ff, S.q_identity((0, 0, 0)), rho=1000.0, stiffness=1e8, mu=0.7, mode=1))
    tip = np.array([0.1, gap, 0.1])
    Vt, Ft = _tet_surface(np.array([tip, tip + [-0.05, 0.1, -0.05], tip + [0.05, 0.1, -0.05],
                                    tip + [0.0, 0.1, 0.06]]))
    s.affines.append(S.AffineBody(Vt, Ft, S.q_identity((0, 0, 0)), rho=1000.0, stiffness=1e8, mu=0.4))
    dh = p.dhat
    b = -(gap - dh) ** 2 * np.log(gap / dh)
    b1 = -2 * (gap - dh) * np.log(gap / dh) - (gap - dh) ** 2 / gap
    o = Oracle(s)
    o.prepare(0, friction=False)
    kappa = o.kappa()
    E, _, _, na = o.eval(o.dofs(), grad=True)
    assert na == 1
    assert abs(E - kappa * b) <= 1e-12 * kappa * b, (E, kappa * b)
    # sensed contact force: the barrier gradient with respect to the tip is
    # kappa b'(gap) along the face normal (+y), over h^2; the fixed body gets
    # its negative (the third law)
    F = o.contact_forces()
    ref_f = kappa * b1 / p.dt ** 2
    assert abs(F[1, 1] - ref_f) <= 1e-9 * abs(ref_f), (F[1], ref_f)
    assert np.abs(F[1, [0, 2]]).max() <= 1e-9 * abs(ref_f)
    assert np.abs(F[0] + F[1]).max() <= 1e-9 * abs(ref_f)
    o.prepare(0, friction=True)
    E = o.eval(o.dofs())[0]
    ref = kappa * b + 0.4 * kappa * abs(b1) * p.eps_v * p.dt / 3
    assert abs(E - ref) <= 1e-12 * ref, (E, ref)


@pytest.mark.parametrize("phi", [0.5, 0.02])
def test_single_edge_edge_contact_energy(phi):
    # one active edge-edge pair at the scene level: the top edge of a fixed
    # tetrahedron along x and the bottom edge of a free one at height gap,
    # turned by phi about y, crossing at their midpoints; all other features
    # stay beyond dhat.  The potential is kappa e(c) b(gap) with IPC's
    # mollifier (reading c6): c = |ea x eb|^2 = 0.04^2 sin^2(phi) against
    # eps_x = 1e-3 |ea|^2 |eb|^2 = 1.6e-6 at rest, so e = 1 at phi = 0.5 and
    # e = r (2 - r), r = c / eps_x, at phi = 0.02.  Lagged friction adds
    # mu kappa e |b'(gap)| eps_v h / 3.
    gap = 0.5e-3
    p = S.Params(dt=0.01, gravity=(0.0, 0.0, 0.0))
    s = S.Scene("one_ee_pair", p)
    Va, Fa = _tet_surface(np.array([[-0.1, 0, 0], [0.1, 0, 0], [0, -0.1, -0.1], [0, -0.1, 0.1]]))
    s.affines.append(S.AffineBody(Va, Fa, S.q_identity((0, 0, 0)), rho=1000.0, stiffness=1e8, mu=0.6, mode=1))
    d = np.array([np.cos(phi), 0.0, np.sin(phi)])
    nrm = np.array([-np.sin(phi), 0.0, np.cos(phi)])
    top = np.array([0.0, gap + 0.1, 0.0])
    Vb, Fb = _tet_surface(np.array([[0, gap, 0] - 0.1 * d, [0, gap, 0] + 0.1 * d, top - 0.1 * nrm, top + 0.1 * nrm]))
    s.affines.append(S.AffineBody(Vb, Fb, S.q_identity((0, 0, 0)), rho=1000.0, stiffness=1e8, mu=0.3))
    dh = p.dhat
    c = 0.04 ** 2 * np.sin(phi) ** 2
    r = c / 1.6e-6
    e = r * (2 - r) if r < 1 else 1.0
    b = -(gap - dh) ** 2 * np.log(gap / dh)
    b1 = -2 * (gap - dh) * np.log(gap / dh) - (gap - dh) ** 2 / gap
    o = Oracle(s)
    o.prepare(0, friction=False)
    kappa = o.kappa()
    E, _, _, na = o.eval(o.dofs(), grad=True)
    assert na == 1
    assert abs(E - kappa * e * b) <= 1e-9 * kappa * e * b, (E, kappa * e * b, e)
    o.prepare(0, friction=True)
    E = o.eval(o.dofs())[0]
    ref = kappa * e * b + 0.3 * kappa * e * abs(b1) * p.eps_v * p.dt / 3
    assert abs(E - ref) <= 1e-9 * ref, (E, ref)


def test_spring_energy_and_force_at_rest():
    # spring constraints h^2 k |x - target|^2 on body-local vertices of the
    # second soft body (its local indices must map to its own vertices): at
    # the rest shape, at rest, with no gravity, the potential is
    # h^2 k sum |delta|^2 and the gradient 2 h^2 k delta on those vertices only
    p = S.Params(dt=0.01, gravity=(0.0, 0.0, 0.0))
    s = S.Scene("springs_at_rest", p)
    X0, T0 = S.soft_cube(3, 0.2, (0.0, 0.0, 0.0))
    X1, T1 = S.soft_cube(3, 0.2, (1.0, 0.0, 0.0))
    s.tets.append(S.TetBody(X0, T0, E=1e5, nu=0.4, rho=1000.0, mu=0.3))
    s.tets.append(S.TetBody(X1, T1, E=1e5, nu=0.4, rho=1000.0, mu=0.3))
    verts = np.array([2, 11, 20], dtype=np.int32)
    delta = np.array([[0.01, 0.0, 0.0], [0.0, -0.02, 0.0], [0.003, 0.004, 0.0]])
    k = 3.0e3
    s.springs.append((1, verts, X1[verts] - delta, k))
    o = Oracle(s)
    o.prepare(0)
    E, g, _, _ = o.eval(o.dofs(), grad=True)
    h2 = p.dt ** 2
    assert abs(E - h2 * k * (delta ** 2).sum()) <= 1e-12 * h2 * k * (delta ** 2).sum()
    G = g[:3 * (len(X0) + len(X1))].reshape(-1, 3)
    ref = np.zeros_like(G)
    ref[len(X0) + verts] = 2 * h2 * k * delta
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()
