"""Seeded synthetic scene generators (inputs only).

Every scene the library, the tests and the benchmark use is built here from a
seed: tetrahedral soft bodies from a lattice (Kuhn / Freudenthal split of each
kept cube cell into 6 tetrahedra along its main diagonal), closed triangle
meshes for affine bodies, initial states and the kinematic script of the
grasp scenes.  Nothing here evaluates an energy, a distance or any other part
of the time step: this module only produces the arrays that a caller hands to
``zema_add_tet_body`` / ``zema_add_affine_body`` (and the CPU oracle receives
the very same arrays).

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), written here
from its published definition.

Units: metres, kilograms, seconds.  Gravity points along -y.
Affine state q = (p, a1, a2, a3) with A = (a1, a2, a3)^T stored by rows, so a
rest vertex x0 maps to x = A x0 + p (the affine-body map of the paper's
affine IP energy, Eq. 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np

# ----------------------------------------------------------------------------
# SplitMix64
# ----------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of SplitMix64 started from `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ----------------------------------------------------------------------------
# Mesh builders
# ----------------------------------------------------------------------------
# The 6 Kuhn tetrahedra of a unit cube: each is the path v000 -> +e_a -> +e_a+e_b
# -> v111 for a permutation (a, b, c) of the axes.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _corner(i, j, k, d):
    return (i + d[0], j + d[1], k + d[2])


def lattice_tets(mask: np.ndarray, spacing: float, origin) -> tuple:
    """Kuhn-split every kept cell of a boolean cell mask (nx, ny, nz).

    Returns (X, tets): vertex positions (nv, 3) float64 of the vertices used by
    kept cells, and int32 tets (nt, 4), each positively oriented
    (det[x1-x0, x2-x0, x3-x0] > 0)."""
    nx, ny, nz = mask.shape
    vid = -np.ones((nx + 1, ny + 1, nz + 1), dtype=np.int64)
    cells = np.argwhere(mask)
    tets = []
    for (i, j, k) in cells:
        for perm in _PERMS:
            d0 = [0, 0, 0]
            d1 = [0, 0, 0]
            d1[perm[0]] = 1
            d2 = list(d1)
            d2[perm[1]] = 1
            d3 = [1, 1, 1]
            tets.append([_corner(i, j, k, d) for d in (d0, d1, d2, d3)])
    tets = np.array(tets, dtype=np.int64)  # (nt, 4, 3) lattice coords
    flat = tets.reshape(-1, 3)
    uniq, inv = np.unique(flat[:, 0] * (ny + 1) * (nz + 1) + flat[:, 1] * (nz + 1) + flat[:, 2],
                          return_inverse=True)
    li = uniq // ((ny + 1) * (nz + 1))
    lj = (uniq // (nz + 1)) % (ny + 1)
    lk = uniq % (nz + 1)
    X = np.stack([li, lj, lk], axis=1).astype(np.float64) * spacing + np.asarray(origin, dtype=np.float64)
    T = inv.reshape(-1, 4).astype(np.int32)
    # orient positively
    a = X[T[:, 1]] - X[T[:, 0]]
    b = X[T[:, 2]] - X[T[:, 0]]
    c = X[T[:, 3]] - X[T[:, 0]]
    det = np.einsum("ij,ij->i", a, np.cross(b, c))
    neg = det < 0
    T[neg, 1], T[neg, 2] = T[neg, 2].copy(), T[neg, 1].copy()
    return X, T


def boundary_vertex_mask(X: np.ndarray, T: np.ndarray) -> np.ndarray:
    """True for vertices on a face that belongs to exactly one tet (mesh topology only)."""
    faces = np.concatenate([T[:, [0, 2, 1]], T[:, [0, 1, 3]], T[:, [0, 3, 2]], T[:, [1, 2, 3]]])
    key = np.sort(faces, axis=1)
    u, c = np.unique(key, axis=0, return_counts=True)
    onb = np.zeros(len(X), dtype=bool)
    onb[u[c == 1].ravel()] = True
    return onb


def _tet_volumes(X, T):
    a = X[T[:, 1]] - X[T[:, 0]]
    b = X[T[:, 2]] - X[T[:, 0]]
    c = X[T[:, 3]] - X[T[:, 0]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0


def jitter_interior(X, T, spacing, frac, seed, min_ratio=0.2):
    """Move interior vertices by up to frac*spacing per axis (SplitMix64 stream
    `seed`).  A vertex whose move leaves any incident tet with a volume ratio
    (jittered / lattice) below min_ratio keeps its lattice position."""
    X = X.copy()
    vol0 = _tet_volumes(X, T)
    interior = ~boundary_vertex_mask(X, T)
    ids = np.nonzero(interior)[0]
    u = uniform01(seed, 3 * len(ids)).reshape(-1, 3)
    disp = (2.0 * u - 1.0) * frac * spacing
    # vertex -> incident tets
    inc: Dict[int, list] = {}
    for t, row in enumerate(T):
        for v in row:
            inc.setdefault(int(v), []).append(t)
    for n, v in enumerate(ids):
        old = X[v].copy()
        X[v] = old + disp[n]
        ts = np.array(inc[int(v)])
        r = _tet_volumes(X, T[ts]) / vol0[ts]
        if np.any(r < min_ratio):
            X[v] = old
    return X


def box_surface(ext, subdiv: int = 1):
    """Closed, outward-oriented triangle mesh of an axis-aligned box of extents
    ext=(ex, ey, ez) centred at the origin, each face split into subdiv x subdiv
    squares of two triangles.  Returns (V (nv,3) f64, F (nf,3) int32)."""
    ex, ey, ez = [0.5 * float(e) for e in ext]
    n = int(subdiv)
    verts: Dict[tuple, int] = {}
    V = []
    F = []

    def vid(p):
        key = tuple(int(round(c)) for c in p)
        if key not in verts:
            verts[key] = len(V)
            V.append(key)
        return verts[key]

    # integer lattice coords in [0, n] on each axis
    for axis in range(3):
        for side in (0, n):
            u_ax, v_ax = [a for a in range(3) if a != axis]
            for i in range(n):
                for j in range(n):
                    quad = []
                    for (di, dj) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        p = [0, 0, 0]
                        p[axis] = side
                        p[u_ax] = i + di
                        p[v_ax] = j + dj
                        quad.append(vid(p))
                    a, b, c, d = quad
                    # orientation: normal of (u x v) points along +axis when
                    # (axis, u, v) is a cyclic order
                    cyc = (u_ax - axis) % 3 == 1
                    outward_pos = (side == n)
                    if cyc == outward_pos:
                        F.append([a, b, c])
                        F.append([a, c, d])
                    else:
                        F.append([a, c, b])
                        F.append([a, d, c])
    V = np.array(V, dtype=np.float64) / n
    V = V * np.array([2 * ex, 2 * ey, 2 * ez]) - np.array([ex, ey, ez])
    return V, np.array(F, dtype=np.int32)


# ----------------------------------------------------------------------------
# Scene containers
# ----------------------------------------------------------------------------
@dataclass
class Params:
    dt: float = 0.01
    dhat: float = 1e-3
    kappa: float = 0.0          # <= 0: adaptive barrier stiffness
    eps_v: float = 1e-3         # m/s
    newton_tol_rel: float = 1e-3  # x bbox diagonal x dt
    gravity: tuple = (0.0, -9.81, 0.0)
    max_newton: int = 100
    max_pcg: int = 10000
    pcg_rel_tol: float = 1e-4
    precision: int = 0          # 0: FP64, 1: mixed FP32/FP64
    max_al_rounds: int = 10
    al_extrapolate: int = 1     # kinematic multipliers start at 2 lambda^t - lambda^(t-1)


@dataclass
class TetBody:
    X: np.ndarray
    tets: np.ndarray
    E: float
    nu: float
    rho: float
    mu: float
    env: int = 0
    x0: Optional[np.ndarray] = None
    v0: Optional[np.ndarray] = None
    name: str = "soft"
    model: int = 0              # 0 Neo-Hookean, 1 St. Venant-Kirchhoff


@dataclass
class AffineBody:
    V: np.ndarray
    F: np.ndarray
    q0: np.ndarray
    rho: float
    stiffness: float
    mu: float
    mode: int = 0               # 0 dynamic, 1 fixed, 2 kinematic
    env: int = 0
    qdot0: Optional[np.ndarray] = None
    name: str = "rigid"


@dataclass
class Scene:
    name: str
    params: Params
    tets: List[TetBody] = field(default_factory=list)
    affines: List[AffineBody] = field(default_factory=list)
    n_envs: int = 1
    n_steps: int = 1
    # script(step) -> {affine index: q_target (12,)} for the state at step+1
    script: Optional[Callable[[int], Dict[int, np.ndarray]]] = None
    # grasp scenes: (affine index, closing sign along z, q0) of every finger
    fingers: list = field(default_factory=list)
    # spring constraints: (tet body index, body-local vertices, targets (n, 3), k [N/m])
    springs: list = field(default_factory=list)
    # prismatic joints: (affine index 1, affine index 2, world axis at t = 0, kappa; <= 0: default)
    joints: list = field(default_factory=list)

    def body_order(self):
        """(kind, index) in the order bodies are added: tets first, then affines."""
        return [("tet", i) for i in range(len(self.tets))] + [("affine", i) for i in range(len(self.affines))]


def q_identity(p) -> np.ndarray:
    """q = (p, a1, a2, a3) with A = I."""
    q = np.zeros(12)
    q[0:3] = p
    q[3] = 1.0
    q[7] = 1.0
    q[11] = 1.0
    return q


# ----------------------------------------------------------------------------
# Concrete scenes
# ----------------------------------------------------------------------------
def soft_cube(n_vert: int, size: float, origin) -> tuple:
    m = np.ones((n_vert - 1,) * 3, dtype=bool)
    return lattice_tets(m, size / (n_vert - 1), origin)


# Horizontal offsets of the stacked bodies.  With every body centred, resting
# vertices sit exactly above a triangle edge of the surface below (the floor's
# and the cube faces' diagonals).  There the per-triangle barrier sum has an
# unstable symmetric equilibrium, so round-off alone decides on which side a
# vertex settles.  These offsets keep every resting vertex at least ~10 dhat
# away from the edges below it.
C1_SOFT_OFFSET = (0.1, 0.037)
C1_RIGID_OFFSET = (0.043, -0.061)


def scene_c1(n_steps: int = 100) -> Scene:
    """Tiny scene: a 1 m soft cube (5x5x5 vertex grid, 384 tets) whose bottom is
    0.05 m above a fixed affine floor box (3 x 0.2 x 3 m, top at y = 0), with a
    0.3 m affine cube resting on the soft top at a gap of 0.5 dhat."""
    p = Params(dt=0.01, dhat=1e-3, kappa=0.0, eps_v=1e-3, newton_tol_rel=1e-3)
    ox, oz = C1_SOFT_OFFSET
    X, T = soft_cube(5, 1.0, (-0.5 + ox, 0.05, -0.5 + oz))
    s = Scene("c1_soft_cube_drop", p, n_steps=n_steps)
    s.tets.append(TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=0.5, name="soft_cube"))
    Vf, Ff = box_surface((3.0, 0.2, 3.0), 1)
    s.affines.append(AffineBody(Vf, Ff, q_identity((0.0, -0.1, 0.0)), rho=1000.0,
                                stiffness=1e8, mu=0.5, mode=1, name="floor"))
    Vc, Fc = box_surface((0.3, 0.3, 0.3), 1)
    top = 1.05 + 0.5 * p.dhat + 0.15
    rx, rz = C1_RIGID_OFFSET
    s.affines.append(AffineBody(Vc, Fc, q_identity((ox + rx, top, oz + rz)), rho=1000.0,
                                stiffness=1e8, mu=0.5, mode=0, name="rigid_cube"))
    return s


def ellipsoid_mask(semi, spacing):
    a, b, c = semi
    nx, ny, nz = [int(math.ceil(2 * s / spacing)) + 2 for s in semi]
    org = np.array([-(nx * spacing) / 2, -(ny * spacing) / 2, -(nz * spacing) / 2])
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cx = org[0] + (ii + 0.5) * spacing
    cy = org[1] + (jj + 0.5) * spacing
    cz = org[2] + (kk + 0.5) * spacing
    m = (cx / a) ** 2 + (cy / b) ** 2 + (cz / c) ** 2 < 1.0
    return m, org


def torus_mask(R, r, spacing, flat_scale=1.0):
    n = int(math.ceil(2 * (R + r) / spacing)) + 2
    ny = int(math.ceil(2 * r * flat_scale / spacing)) + 2
    org = np.array([-(n * spacing) / 2, -(ny * spacing) / 2, -(n * spacing) / 2])
    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(ny), np.arange(n), indexing="ij")
    cx = org[0] + (ii + 0.5) * spacing
    cy = org[1] + (jj + 0.5) * spacing
    cz = org[2] + (kk + 0.5) * spacing
    rho = np.sqrt(cx ** 2 + cz ** 2)
    m = (rho - R) ** 2 + (cy / flat_scale) ** 2 < r ** 2
    return m, org


def box_mask(ext, spacing):
    n = [max(1, int(round(e / spacing))) for e in ext]
    org = np.array([-(n[0] * spacing) / 2, -(n[1] * spacing) / 2, -(n[2] * spacing) / 2])
    return np.ones(n, dtype=bool), org


def _solid(kind, size_scale, spacing):
    if kind == "ellipsoid":
        return ellipsoid_mask((0.04 * size_scale, 0.02 * size_scale, 0.03 * size_scale), spacing)
    if kind == "torus":
        return torus_mask(0.026 * size_scale, 0.012 * size_scale, spacing, flat_scale=1.0)
    if kind == "box":
        return box_mask((0.07 * size_scale, 0.035 * size_scale, 0.05 * size_scale), spacing)
    raise ValueError(kind)


def _spacing_for_count(kind, target_tets, size_scale=1.0, hi=2e-2):
    """Lattice spacing whose kept-cell count x 6 is closest to target_tets
    (bisection over [5e-4, hi])."""
    lo = 5e-4
    for _ in range(40):
        mid = math.sqrt(lo * hi)
        m, _ = _solid(kind, size_scale, mid)
        n = 6 * int(m.sum())
        if n > target_tets:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def grasp_env(s: Scene, env: int, kind: str, spacing: float, seed: int, E: float, nu: float,
              mu: float, offset, finger_subdiv: int = 9, size_scale: float = 1.0):
    """One parallel-jaw grasp environment: a soft lattice object resting on a
    fixed floor at a gap of 0.5 dhat, and two kinematic box fingers (thickness
    1 cm along z, 6 x 3 cm in x, y) 0.5 cm off the object's +-z extremes."""
    p = s.params
    m, org = _solid(kind, size_scale, spacing)
    X, T = lattice_tets(m, spacing, org)
    X = jitter_interior(X, T, spacing, 0.1, seed)
    ymin = X[:, 1].min()
    shift = np.array(offset, dtype=np.float64) + np.array([0.0, -ymin + 0.5 * p.dhat, 0.0])
    X = X + shift
    s.tets.append(TetBody(X, T, E=E, nu=nu, rho=1000.0, mu=mu, env=env, name=f"{kind}{env}"))
    ext = X.max(0) - X.min(0)
    cx, cy, cz = 0.5 * (X.max(0) + X.min(0))
    fl = max(ext[0], ext[2]) * 2.5
    Vf, Ff = box_surface((fl, 0.02, fl), 1)
    s.affines.append(AffineBody(Vf, Ff, q_identity((cx, offset[1] - 0.01, cz)), rho=1000.0,
                                stiffness=1e8, mu=mu, mode=1, env=env, name=f"floor{env}"))
    fw = (0.06 * size_scale, min(0.03 * size_scale, 0.9 * ext[1]), 0.01)
    Vg, Fg = box_surface(fw, finger_subdiv)
    fy = cy
    zmax = X[:, 2].max()
    zmin = X[:, 2].min()
    gap = 0.005
    fingers = []
    for sign, zface in ((+1, zmax), (-1, zmin)):
        zc = zface + sign * (gap + 0.5 * fw[2])
        q0 = q_identity((cx, fy, zc))
        qd = np.zeros(12)
        qd[2] = -sign * 0.05
        s.affines.append(AffineBody(Vg, Fg, q0, rho=1000.0, stiffness=1e8, mu=mu, mode=2,
                                    env=env, qdot0=qd, name=f"finger{'+' if sign > 0 else '-'}{env}"))
        fingers.append((len(s.affines) - 1, sign, q0.copy()))
    return fingers


def grasp_script(fingers_all, dt, close_steps=40, hold_steps=60, lift_steps=200,
                 close_speed=0.05, lift_height=0.05):
    """Kinematic finger targets: close along -+z at close_speed, hold, lift by
    lift_height along +y over lift_steps.  script(n) gives the targets of the
    state at step n+1."""

    def pose(q0, sign, n):
        q = q0.copy()
        c = min(n, close_steps)
        q[2] -= sign * close_speed * dt * c
        l = min(max(n - close_steps - hold_steps, 0), lift_steps)
        q[1] += lift_height * l / lift_steps
        return q

    def script(step):
        out = {}
        for (idx, sign, q0) in fingers_all:
            out[idx] = pose(q0, sign, step + 1)
        return out

    # the same targets for all fingers at once: (affine indices, (n, 12))
    idx_all = np.array([f[0] for f in fingers_all], dtype=np.int64)
    sign_all = np.array([f[1] for f in fingers_all], dtype=np.float64)
    q0_all = np.array([f[2] for f in fingers_all], dtype=np.float64).reshape(len(fingers_all), 12)

    def arrays(step):
        n = step + 1
        Q = q0_all.copy()
        Q[:, 2] -= sign_all * close_speed * dt * min(n, close_steps)
        Q[:, 1] += lift_height * min(max(n - close_steps - hold_steps, 0), lift_steps) / lift_steps
        return idx_all, Q

    script.arrays = arrays
    return script


def scene_c2(n_steps: int = 300, finger_subdiv: int = 9, precision: int = 0) -> Scene:
    """Parallel-jaw grasp, one environment: jittered Kuhn lattice ellipsoid of
    semi-axes 4 (x) / 2 (y) / 3 (z) cm at 0.4 cm spacing (~10k tets), E=5e4,
    nu=0.45, two kinematic box fingers of 972 triangles each, fixed floor;
    mu=0.8, dt=0.005."""
    p = Params(dt=0.005, dhat=1e-3, kappa=0.0, eps_v=1e-3, newton_tol_rel=1e-3, precision=precision)
    s = Scene("c2_grasp_ellipsoid", p, n_steps=n_steps)
    fingers = grasp_env(s, 0, "ellipsoid", 0.004, seed=2, E=5e4, nu=0.45, mu=0.8,
                        offset=(0.0, 0.0, 0.0), finger_subdiv=finger_subdiv)
    s.script = grasp_script(fingers, p.dt)
    s.fingers = fingers
    return s


def scene_c3(n_envs: int = 256, n_steps: int = 200, min_tets=2000, max_tets=20000,
             finger_subdiv: int = 9, precision: int = 1, seed0: int = 1000, slot0: int = 0) -> Scene:
    """Batched grasping: env i (seed seed0+i) draws its object kind (ellipsoid,
    torus, box), tet count log-uniform in [min_tets, max_tets], E log-uniform in
    [1e4, 1e6], mu uniform in [0.3, 1.0]; nu = 0.45.  Envs are placed 0.5 m
    apart along x (env i at slot slot0 + i) so they are spatially disjoint; a
    range of a larger batch built with seed0 and slot0 advanced together has
    the same coordinates as in the whole batch.  Training envs use seeds from
    1000, held-out evaluation envs from 100000."""
    p = Params(dt=0.005, dhat=1e-3, kappa=0.0, eps_v=1e-3, newton_tol_rel=1e-3, precision=precision)
    s = Scene("c3_batched_grasp", p, n_envs=n_envs, n_steps=n_steps)
    kinds = ["ellipsoid", "torus", "box"]
    allf = []
    for i in range(n_envs):
        u = uniform01(seed0 + i, 4)
        kind = kinds[min(2, int(u[0] * 3))]
        nt = math.exp(math.log(min_tets) + u[1] * (math.log(max_tets) - math.log(min_tets)))
        E = math.exp(math.log(1e4) + u[2] * (math.log(1e6) - math.log(1e4)))
        mu = 0.3 + 0.7 * u[3]
        sp = _spacing_for_count(kind, nt)
        allf += grasp_env(s, i, kind, sp, seed=seed0 + i, E=E, nu=0.45, mu=mu,
                          offset=(0.5 * (slot0 + i), 0.0, 0.0), finger_subdiv=finger_subdiv)
    s.script = grasp_script(allf, p.dt)
    s.fingers = allf
    return s


# ----------------------------------------------------------------------------
# Small scenes for tests
# ----------------------------------------------------------------------------
def scene_free_fall(n_steps: int = 5, gravity=(0.0, -9.81, 0.0)) -> Scene:
    """A soft cube (3x3x3 vertices) and an affine cube, far apart, no floor."""
    p = Params(dt=0.01, gravity=gravity)
    X, T = soft_cube(3, 0.2, (0.0, 1.0, 0.0))
    s = Scene("free_fall", p, n_steps=n_steps)
    s.tets.append(TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=0.5))
    V, F = box_surface((0.2, 0.2, 0.2), 1)
    s.affines.append(AffineBody(V, F, q_identity((1.0, 1.0, 0.0)), rho=1000.0, stiffness=1e8, mu=0.5))
    return s


def scene_tiny_contact(n_steps: int = 10, mu: float = 0.5) -> Scene:
    """A 3x3x3-vertex soft cube dropped onto a fixed floor with an affine cube
    on top: every pair kind (soft-fixed, soft-affine) in a few hundred DOF."""
    p = Params(dt=0.01)
    X, T = soft_cube(3, 0.2, (-0.1 + 0.013, 0.01, -0.1 - 0.029))
    s = Scene("tiny_contact", p, n_steps=n_steps)
    s.tets.append(TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=mu))
    Vf, Ff = box_surface((1.0, 0.1, 1.0), 1)
    s.affines.append(AffineBody(Vf, Ff, q_identity((0.0, -0.05, 0.0)), rho=1000.0, stiffness=1e8,
                                mu=mu, mode=1, name="floor"))
    Vc, Fc = box_surface((0.1, 0.1, 0.1), 2)
    s.affines.append(AffineBody(Vc, Fc, q_identity((0.031, 0.21 + 0.0005 + 0.05, 0.016)), rho=1000.0,
                                stiffness=1e8, mu=mu, mode=0, name="cube"))
    return s


def random_state_scene(seed: int, n_soft: int = 3, n_aff: int = 2) -> Scene:
    """Several small soft cubes and affine boxes at seeded positions in a
    0.6 m box with seeded initial velocities; used for broad-phase and
    distance parity.  Bodies are placed on a coarse lattice of slots so that
    they never overlap at rest."""
    p = Params(dt=0.01)
    s = Scene(f"random{seed}", p)
    u = uniform01(seed, 64)
    k = 0
    slots = [(i, j, l) for i in range(3) for j in range(2) for l in range(2)]
    for b in range(n_soft + n_aff):
        sl = slots[b]
        base = np.array(sl, dtype=np.float64) * 0.2 + (u[k:k + 3] * 0.02)
        k += 3
        if b < n_soft:
            X, T = soft_cube(3, 0.15, base)
            s.tets.append(TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=0.5))
        else:
            V, F = box_surface((0.15, 0.15, 0.15), 2)
            s.affines.append(AffineBody(V, F, q_identity(base + 0.075), rho=1000.0, stiffness=1e8,
                                        mu=0.5, mode=0))
    return s


# ----------------------------------------------------------------------------
# Dense soft-rigid pile
# ----------------------------------------------------------------------------
def uv_sphere_surface(radii, n_seg: int = 32, n_ring: int = 32):
    """Closed, outward-oriented UV sphere (ellipsoid of semi-axes radii): two
    poles on +-y and n_ring - 1 rings of n_seg vertices; 2 n_seg (n_ring - 1)
    triangles (1984 for 32 x 32)."""
    a, b, c = [float(r) for r in radii]
    V = [(0.0, b, 0.0)]
    for i in range(1, n_ring):
        th = math.pi * i / n_ring
        for j in range(n_seg):
            ph = 2.0 * math.pi * j / n_seg
            V.append((a * math.sin(th) * math.cos(ph), b * math.cos(th), c * math.sin(th) * math.sin(ph)))
    V.append((0.0, -b, 0.0))
    south = len(V) - 1

    def ring(i, j):
        return 1 + (i - 1) * n_seg + (j % n_seg)

    F = []
    for j in range(n_seg):
        F.append((0, ring(1, j + 1), ring(1, j)))
    for i in range(1, n_ring - 1):
        for j in range(n_seg):
            p, q, r, s = ring(i, j), ring(i, j + 1), ring(i + 1, j + 1), ring(i + 1, j)
            F.append((p, q, r))
            F.append((p, r, s))
    for j in range(n_seg):
        F.append((south, ring(n_ring - 1, j), ring(n_ring - 1, j + 1)))
    return np.array(V, dtype=np.float64), np.array(F, dtype=np.int32)


def torus_surface(R: float, r: float, n_u: int = 32, n_v: int = 32):
    """Closed, outward-oriented torus about the y axis (major radius R, tube
    radius r): n_u x n_v vertices, 2 n_u n_v triangles (2048 for 32 x 32)."""
    V = []
    for i in range(n_u):
        u = 2.0 * math.pi * i / n_u
        for j in range(n_v):
            v = 2.0 * math.pi * j / n_v
            rho = R + r * math.cos(v)
            V.append((rho * math.cos(u), r * math.sin(v), rho * math.sin(u)))

    def vid(i, j):
        return (i % n_u) * n_v + (j % n_v)

    F = []
    for i in range(n_u):
        for j in range(n_v):
            p, q, s, t = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            F.append((p, s, q))
            F.append((p, t, s))
    return np.array(V, dtype=np.float64), np.array(F, dtype=np.int32)


def rotation_from_uniforms(u1: float, u2: float, u3: float) -> np.ndarray:
    """Uniformly distributed rotation matrix from three uniforms in [0, 1)
    (Shoemake's unit-quaternion construction)."""
    s1, s2 = math.sqrt(1.0 - u1), math.sqrt(u1)
    w, x, y, z = (s2 * math.cos(2 * math.pi * u3), s1 * math.sin(2 * math.pi * u2),
                  s1 * math.cos(2 * math.pi * u2), s2 * math.sin(2 * math.pi * u3))
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _yaw(theta: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def scene_c5(n_steps: int = 200, tets_per_body: int = 60000, n_soft: int = 8, n_convex: int = 10,
             n_nonconvex: int = 10, n_seg: int = 32, seed: int = 5, precision: int = 1,
             bin_subdiv: int = 4, gap: float = 0.01) -> Scene:
    """Dense soft-rigid pile: an open-top 1 m rigid bin of 5 fixed 2 cm thick
    boxes, n_soft soft lattice bodies (ellipsoid, torus or box, ~0.2 m,
    tets_per_body tets each, E = 1e5, nu = 0.4), n_convex affine UV spheres
    (n_seg x n_seg, seeded anisotropic radii in [0.06, 0.1] m and rotation) and
    n_nonconvex affine tori (n_seg x n_seg, R = 0.07 m, r = 0.025 m, seeded
    rotation), all rho = 1000 and stiffness 1e8.  The bodies start at rest in
    seeded distinct slots of a 3 x 3 x L lattice (0.333 m cells across the
    bin, layers 0.25 m apart, the lowest `gap` above the floor) and drop.
    mu = 0.5, dt = 0.01.  Each bin box face is split bin_subdiv x bin_subdiv.

    Newton is capped at 1000 iterations here instead of 100: when kilogram
    rigid bodies land on soft meshes of 0.1 g vertices, single steps take up
    to ~80 projected-Newton iterations (most of them line-search limited),
    whatever the linear-solve tolerance or precision."""
    p = Params(dt=0.01, dhat=1e-3, kappa=0.0, eps_v=1e-3, newton_tol_rel=1e-3, precision=precision,
               max_newton=1000)
    s = Scene("c5_dense_pile", p, n_steps=n_steps)
    wall_t, H = 0.02, 1.0
    # bin: floor (top at y = 0) and four walls standing 1 mm above it; the
    # x-walls span the floor's depth, the z-walls fit between them
    Vb, Fb = box_surface((1.0 + 2 * wall_t, wall_t, 1.0 + 2 * wall_t), bin_subdiv)
    s.affines.append(AffineBody(Vb, Fb, q_identity((0.0, -0.5 * wall_t, 0.0)), rho=1000.0, stiffness=1e8,
                                mu=0.5, mode=1, name="bin_floor"))
    for sx in (-1, 1):
        V, F = box_surface((wall_t, H, 1.0 + 2 * wall_t), bin_subdiv)
        s.affines.append(AffineBody(V, F, q_identity((sx * (0.5 + 0.5 * wall_t), 0.001 + 0.5 * H, 0.0)),
                                    rho=1000.0, stiffness=1e8, mu=0.5, mode=1, name=f"bin_wall_x{sx:+d}"))
    for sz in (-1, 1):
        V, F = box_surface((1.0 - 0.002, H, wall_t), bin_subdiv)
        s.affines.append(AffineBody(V, F, q_identity((0.0, 0.001 + 0.5 * H, sz * (0.5 + 0.5 * wall_t))),
                                    rho=1000.0, stiffness=1e8, mu=0.5, mode=1, name=f"bin_wall_z{sz:+d}"))
    n_bodies = n_soft + n_convex + n_nonconvex
    layers = max(1, (n_bodies + 8) // 9)
    slots = [(l, i, k) for l in range(layers) for i in range(3) for k in range(3)]
    u = uniform01(seed, 8 * n_bodies + len(slots) + n_bodies)
    # the lowest n_bodies slots (seeded order within a layer), dealt to the
    # bodies in a seeded permutation so that kinds mix across layers
    lowest = sorted(range(len(slots)), key=lambda t: (slots[t][0], u[t]))[:n_bodies]
    perm = np.argsort(u[len(slots):len(slots) + n_bodies], kind="stable")
    order = [lowest[int(perm[b])] for b in range(n_bodies)]
    u = u[len(slots) + n_bodies:]
    cell, pitch, base0 = 1.0 / 3.0, 0.25, gap

    def place(Xw, slot):
        l, i, k = slots[slot]
        lo, hi = Xw.min(0), Xw.max(0)
        target = np.array([(i - 1) * cell, base0 + l * pitch, (k - 1) * cell])
        centre = np.array([0.5 * (lo[0] + hi[0]), lo[1], 0.5 * (lo[2] + hi[2])])
        return target - centre

    kinds = ["ellipsoid", "torus", "box"]
    for b in range(n_bodies):
        ub = u[8 * b:8 * b + 8]
        slot = order[b]
        if b < n_soft:
            kind = kinds[min(2, int(ub[0] * 3))]
            sp = _spacing_for_count(kind, tets_per_body, 2.5, hi=0.1)
            m, org = _solid(kind, 2.5, sp)
            X, T = lattice_tets(m, sp, org)
            X = jitter_interior(X, T, sp, 0.1, seed * 1000 + b)
            X = X @ _yaw(2 * math.pi * ub[1]).T
            X = X + place(X, slot)
            s.tets.append(TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=0.5, name=f"soft_{kind}{b}"))
            continue
        if b < n_soft + n_convex:
            V, F = uv_sphere_surface(0.06 + 0.04 * ub[2:5], n_seg, n_seg)
            name = f"sphere{b}"
        else:
            V, F = torus_surface(0.07, 0.025, n_seg, n_seg)
            name = f"torus{b}"
        Rm = rotation_from_uniforms(ub[5], ub[6], ub[7])
        Xw = V @ Rm.T
        q = np.zeros(12)
        q[0:3] = place(Xw, slot)
        q[3:12] = Rm.reshape(-1)
        s.affines.append(AffineBody(V, F, q, rho=1000.0, stiffness=1e8, mu=0.5, mode=0, name=name))
    return s


# ----------------------------------------------------------------------------
# Runtime over rigid-mesh resolution
# ----------------------------------------------------------------------------
RESOLUTION_SEGMENTS = (26, 46, 105, 138, 279)  # UV spheres of 652 ... 77,564 vertices


def scene_resolution(n_seg: int, n_steps: int = 60, precision: int = 1, spacing: float = 0.01) -> Scene:
    """An affine sphere (radius 5 cm, n_seg x n_seg UV mesh: n_seg (n_seg - 1)
    + 2 vertices, 2 n_seg (n_seg - 1) triangles) dropped from 2 mm onto a soft
    box (12 x 4 x 12 cm lattice of the given spacing, E = 1e5, nu = 0.4)
    resting on a fixed floor; mu = 0.5, dt = 0.01.  The system's DOF do not
    depend on n_seg: the sphere is 12 of them at every resolution."""
    p = Params(dt=0.01, dhat=1e-3, kappa=0.0, eps_v=1e-3, newton_tol_rel=1e-3, precision=precision)
    s = Scene(f"resolution_{n_seg}", p, n_steps=n_steps)
    m, org = box_mask((0.12, 0.04, 0.12), spacing)
    X, T = lattice_tets(m, spacing, org)
    X = X - np.array([0.0, X[:, 1].min() - 0.5 * p.dhat, 0.0])
    s.tets.append(TetBody(X, T, E=1e5, nu=0.4, rho=1000.0, mu=0.5, name="soft_box"))
    Vf, Ff = box_surface((0.4, 0.02, 0.4), 1)
    s.affines.append(AffineBody(Vf, Ff, q_identity((0.0, -0.01, 0.0)), rho=1000.0, stiffness=1e8, mu=0.5,
                                mode=1, name="floor"))
    V, F = uv_sphere_surface((0.05, 0.05, 0.05), n_seg, n_seg)
    top = X[:, 1].max() + 0.002 + 0.05
    # offset so that no sphere vertex sits exactly above a lattice vertex
    s.affines.append(AffineBody(V, F, q_identity((0.0131, top, -0.0077)), rho=1000.0, stiffness=1e8, mu=0.5,
                                mode=0, name="sphere"))
    return s


def scene_joint(axis=(0.0, 1.0, 0.0), fixed_base: bool = True, gravity=(0.0, -9.81, 0.0), n_steps: int = 10,
                base_velocity=(0.0, 0.0, 0.0)) -> Scene:
    """Two 0.1 m affine boxes 0.1 m apart along x (no contact), joined by a
    prismatic joint along `axis`: body 1 (the base) fixed or dynamic with an
    initial velocity, body 2 dynamic and at rest."""
    p = Params(dt=0.01, gravity=gravity)
    s = Scene("joint", p, n_steps=n_steps)
    V, F = box_surface((0.1, 0.1, 0.1), 1)
    qd = np.zeros(12)
    qd[0:3] = base_velocity
    s.affines.append(AffineBody(V, F, q_identity((0.0, 1.0, 0.0)), rho=1000.0, stiffness=1e8, mu=0.5,
                                mode=1 if fixed_base else 0, qdot0=qd, name="base"))
    s.affines.append(AffineBody(V, F, q_identity((0.2, 1.0, 0.0)), rho=1000.0, stiffness=1e8, mu=0.5, mode=0,
                                name="slider"))
    s.joints.append((0, 1, np.array(axis, dtype=np.float64), 0.0))
    return s


def rotation_z(theta: float) -> np.ndarray:
    """Rotation by theta (rad) about +z."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def scene_slope(theta: float = 0.3, mu: float = 0.1, n_steps: int = 24, precision: int = 0) -> Scene:
    """A fixed 4 m slab rotated by theta about z and a 0.2 x 0.04 x 0.2 m
    block (1000 kg/m^3) resting on its top face, 2 mm above it along the slope
    normal; both bodies have friction coefficient mu.  The downhill direction
    is -(cos theta, sin theta, 0)."""
    p = Params(dt=0.01, precision=precision)
    s = Scene("slope", p, n_steps=n_steps)
    R = rotation_z(theta)
    Vf, Ff = box_surface((4.0, 0.1, 4.0), 1)
    qf = np.zeros(12)
    qf[3:] = R.reshape(-1)
    s.affines.append(AffineBody(Vf, Ff, qf, rho=1000.0, stiffness=1e8, mu=mu, mode=1, name="slope"))
    V, F = box_surface((0.2, 0.04, 0.2), 1)
    qb = np.zeros(12)
    qb[:3] = R @ np.array([0.3, 0.05 + 0.02 + 0.002, 0.1])
    qb[3:] = R.reshape(-1)
    s.affines.append(AffineBody(V, F, qb, rho=1000.0, stiffness=1e8, mu=mu, name="block"))
    return s


def kinematic_track_target(n: int, dt: float = 0.01, speed: float = 5.0, omega: float = 2.0) -> np.ndarray:
    """Target q at the end of step n of `scene_kinematic_track`: from (0, 0.5,
    0) along +x at `speed` m/s, turning about z at `omega` rad/s."""
    q = np.zeros(12)
    t = (n + 1) * dt
    q[:3] = (speed * t, 0.5, 0.0)
    q[3:] = rotation_z(omega * t).reshape(-1)
    return q


def scene_kinematic_track(max_al_rounds: int = 10, n_steps: int = 6, precision: int = 0) -> Scene:
    """A kinematic 0.1 m box, at rest at (0, 0.5, 0), scripted onto
    `kinematic_track_target`, plus a fixed slab 0.45 m below it (no contact)."""
    p = Params(dt=0.01, max_al_rounds=max_al_rounds, precision=precision)
    s = Scene("kinematic_track", p, n_steps=n_steps)
    V, F = box_surface((0.1, 0.1, 0.1), 1)
    s.affines.append(AffineBody(V, F, q_identity((0.0, 0.5, 0.0)), rho=1000.0, stiffness=1e8, mu=0.0, mode=2,
                                name="kinematic"))
    Vf, Ff = box_surface((1.0, 0.1, 1.0), 1)
    s.affines.append(AffineBody(Vf, Ff, q_identity((0.0, -0.05, 0.0)), rho=1000.0, stiffness=1e8, mu=0.0,
                                mode=1, name="slab"))
    s.script = lambda n: {0: kinematic_track_target(n, p.dt)}
    return s
