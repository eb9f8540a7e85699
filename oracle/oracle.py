"""ctypes wrapper of the CPU oracle (test infrastructure only).

``Oracle(scene)`` loads a scene produced by the seeded generators and exposes
stepping, state access and the local functions the pin tests call.
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        L = _lib
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        lp = C.POINTER(C.c_long)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [dp, ip]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_add_tet_body.argtypes = [C.c_void_p, C.c_int, dp, C.c_long, ip, C.c_long, dp, dp,
                                       C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_add_affine_body.argtypes = [C.c_void_p, C.c_int, dp, C.c_long, ip, C.c_long, dp, dp,
                                          C.c_double, C.c_double, C.c_double, C.c_int]
        L.orc_finalize.argtypes = [C.c_void_p]
        L.orc_set_material.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_add_prismatic_joint.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.c_double]
        L.orc_joint_constraint.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_set_springs.argtypes = [C.c_void_p, C.c_int, ip, C.c_long, dp, C.c_double]
        L.orc_set_kinematic_target.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_get_state.restype = C.c_long
        L.orc_get_state.argtypes = [C.c_void_p, C.c_int, dp, C.c_long]
        L.orc_set_state.argtypes = [C.c_void_p, C.c_int, dp, C.c_long]
        L.orc_kappa.restype = C.c_double
        L.orc_kappa.argtypes = [C.c_void_p, C.c_int]
        L.orc_kappa_min.restype = C.c_double
        L.orc_kappa_min.argtypes = [C.c_void_p, C.c_int]
        L.orc_diag.restype = C.c_double
        L.orc_diag.argtypes = [C.c_void_p, C.c_int]
        L.orc_energy_log.restype = C.c_long
        L.orc_energy_log.argtypes = [C.c_void_p, dp, C.c_long]
        L.orc_set_kappa.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
        L.orc_counts.argtypes = [C.c_void_p, lp]
        L.orc_surface.argtypes = [C.c_void_p, ip, ip, ip]
        L.orc_lumped_mass.argtypes = [C.c_void_p, dp]
        L.orc_affine_mass.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.orc_env_ndof.argtypes = [C.c_void_p, C.c_int]
        L.orc_env_dofs.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_prepare.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_env_eval.restype = C.c_double
        L.orc_env_eval.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, ip]
        L.orc_newton_system_solve.argtypes = [C.c_void_p, C.c_int, dp, C.c_int, dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_contact_forces.argtypes = [C.c_void_p, dp]
        L.orc_stencil_d2.restype = C.c_double
        L.orc_stencil_d2.argtypes = [dp, C.c_int, ip, dp, dp, dp]
        L.orc_pair_barrier.restype = C.c_double
        L.orc_pair_barrier.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_int, dp, dp]
        for f in ("orc_barrier_scalar", "orc_f0", "orc_f1"):
            getattr(L, f).restype = C.c_double
            getattr(L, f).argtypes = [C.c_double, C.c_double]
        L.orc_nh.restype = C.c_double
        L.orc_nh.argtypes = [dp, C.c_double, C.c_double, C.c_int, dp, dp]
        L.orc_fcr.restype = C.c_double
        L.orc_fcr.argtypes = [dp, C.c_double, C.c_double, C.c_int, dp, dp]
        L.orc_stvk.restype = C.c_double
        L.orc_stvk.argtypes = [dp, C.c_double, C.c_double, C.c_int, dp, dp]
        L.orc_ortho.restype = C.c_double
        L.orc_ortho.argtypes = [dp, dp, dp]
        L.orc_accd.restype = C.c_double
        L.orc_accd.argtypes = [dp, dp, C.c_int, C.c_double, C.c_double, ip]
        L.orc_eigvals.argtypes = [C.c_int, dp, dp]
        L.orc_brute_pairs.argtypes = [C.c_long, dp, dp, ip, C.c_long, ip, ip, C.c_long, ip, C.c_long, ip,
                                      C.c_double, C.c_long, ip, ip, lp]
    return _lib


def _d(a):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int))


class OracleError(RuntimeError):
    pass


class Oracle:
    """A scene in the CPU oracle.  Bodies are added in scene.body_order()."""

    def __init__(self, scene, tol_scale: float = 1.0):
        L = lib()
        p = scene.params
        self.scene = scene
        dpar = np.array([p.dt, p.dhat, p.kappa, p.eps_v, p.newton_tol_rel * tol_scale,
                         p.gravity[0], p.gravity[1], p.gravity[2], p.pcg_rel_tol], dtype=np.float64)
        ipar = np.array([p.max_newton, p.max_al_rounds, scene.n_envs, getattr(p, "al_extrapolate", 1)],
                        dtype=np.int32)
        self.h = L.orc_create(_dp(dpar), _ip(ipar))
        self.body_ids = []
        for kind, i in scene.body_order():
            if kind == "tet":
                b = scene.tets[i]
                X = _d(b.X)
                T = np.ascontiguousarray(b.tets, dtype=np.int32)
                x0 = _d(b.x0)
                v0 = _d(b.v0)
                r = L.orc_add_tet_body(self.h, b.env, _dp(X), len(X), _ip(T), len(T), _dp(x0), _dp(v0),
                                       b.E, b.nu, b.rho, b.mu)
            else:
                b = scene.affines[i]
                V = _d(b.V)
                F = np.ascontiguousarray(b.F, dtype=np.int32)
                q0 = _d(b.q0)
                qd = _d(b.qdot0)
                r = L.orc_add_affine_body(self.h, b.env, _dp(V), len(V), _ip(F), len(F), _dp(q0), _dp(qd),
                                          b.rho, b.stiffness, b.mu, b.mode)
            if r < 0:
                raise OracleError(f"add body failed: {r}")
            self.body_ids.append(r)
        for i, b in enumerate(scene.tets):
            if b.model and L.orc_set_material(self.h, self.body_ids[i], int(b.model)) != 0:
                raise OracleError("set material failed")
        for (i, verts, targets, k) in scene.springs:
            self.set_springs(i, verts, targets, k)
        for (a1, a2, axis, kappa) in scene.joints:
            ax = _d(axis)
            if L.orc_add_prismatic_joint(self.h, self.affine_body_id(a1), self.affine_body_id(a2), _dp(ax),
                                         float(kappa)) < 0:
                raise OracleError("add joint failed")
        if L.orc_finalize(self.h) != 0:
            raise OracleError("finalize failed")
        self.n_tet = len(scene.tets)
        self.step_index = 0

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def set_springs(self, tet_index, verts, targets, k):
        """Springs h^2 k |x - target|^2 on body-local vertices of a soft body
        (replacing its springs)."""
        v = np.ascontiguousarray(verts, dtype=np.int32)
        t = _d(targets)
        if lib().orc_set_springs(self.h, self.body_ids[tet_index], _ip(v), len(v), _dp(t), float(k)) != 0:
            raise OracleError("set springs failed")

    def affine_body_id(self, i):
        return self.body_ids[len(self.scene.tets) + i]

    def joint_constraint(self, j):
        """The 12 constraint values of prismatic joint j at the current state."""
        c = np.zeros(12)
        if lib().orc_joint_constraint(self.h, j, _dp(c)) != 0:
            raise OracleError("no such joint")
        return c

    def tet_body_id(self, i):
        return self.body_ids[i]

    def apply_script(self):
        if self.scene.script is None:
            return
        for idx, q in self.scene.script(self.step_index).items():
            qq = _d(q)
            lib().orc_set_kinematic_target(self.h, self.affine_body_id(idx), _dp(qq))

    def step(self, n: int = 1):
        """Advance n steps (applying the scene script before each); returns
        per-step stats (n, n_envs, 8): newton iters, LS halvings, AL rounds,
        n_active, dmin, energy, kappa, status."""
        stats = np.zeros((n, self.scene.n_envs, 8))
        for k in range(n):
            self.apply_script()
            r = lib().orc_step(self.h, 1, _dp(stats[k]))
            if r != 0:
                raise OracleError(f"oracle step failed with status {-r} at step {self.step_index}")
            self.step_index += 1
        return stats

    def get_state(self, body):
        out = np.zeros(1 << 22)
        n = lib().orc_get_state(self.h, body, _dp(out), len(out))
        if n < 0:
            raise OracleError("get_state failed")
        return out[:n].copy()

    def set_state(self, body, arr):
        a = _d(arr)
        if lib().orc_set_state(self.h, body, _dp(a), len(a)) != 0:
            raise OracleError("set_state failed")

    def tet_positions(self, i=0):
        st = self.get_state(self.tet_body_id(i))
        n = len(st) // 6
        return st[:3 * n].reshape(n, 3)

    def affine_q(self, i):
        return self.get_state(self.affine_body_id(i))[:12]

    def kappa(self, env=0):
        return lib().orc_kappa(self.h, env)

    def kappa_min(self, env=0):
        return lib().orc_kappa_min(self.h, env)

    def diag(self, env=0):
        return lib().orc_diag(self.h, env)

    def energy_log(self):
        out = np.zeros(100000)
        n = lib().orc_energy_log(self.h, _dp(out), len(out))
        return out[:min(n, len(out))].copy()

    def set_kappa(self, env, k, kmin):
        lib().orc_set_kappa(self.h, env, k, kmin)

    def counts(self):
        out = np.zeros(5, dtype=np.int64)
        lib().orc_counts(self.h, out.ctypes.data_as(C.POINTER(C.c_long)))
        return dict(n_sv=int(out[0]), n_edges=int(out[1]), n_tris=int(out[2]), n_verts=int(out[3]),
                    n_tets=int(out[4]))

    def surface(self):
        c = self.counts()
        sv = np.zeros((c["n_sv"], 3), dtype=np.int32)
        e = np.zeros((c["n_edges"], 2), dtype=np.int32)
        t = np.zeros((c["n_tris"], 3), dtype=np.int32)
        lib().orc_surface(self.h, _ip(sv), _ip(e), _ip(t))
        return sv, e, t

    def lumped_mass(self):
        m = np.zeros(self.counts()["n_verts"])
        lib().orc_lumped_mass(self.h, _dp(m))
        return m

    def affine_mass(self, i):
        M = np.zeros(144)
        mv = np.zeros(2)
        lib().orc_affine_mass(self.h, self.affine_body_id(i), _dp(M), _dp(mv))
        return M.reshape(12, 12), mv[0], mv[1]

    # env-level evaluation -------------------------------------------------
    def ndof(self, env=0):
        return lib().orc_env_ndof(self.h, env)

    def dofs(self, env=0):
        y = np.zeros(self.ndof(env))
        lib().orc_env_dofs(self.h, env, _dp(y))
        return y

    def prepare(self, env=0, friction=True):
        self.apply_script()
        lib().orc_prepare(self.h, env, 1 if friction else 0)

    def eval(self, y, env=0, grad=False, hess=False):
        y = _d(y)
        n = len(y)
        g = np.zeros(n) if grad else None
        H = np.zeros((n, n)) if hess else None
        na = np.zeros(1, dtype=np.int32)
        E = lib().orc_env_eval(self.h, env, _dp(y), _dp(g), _dp(H), _ip(na))
        return E, g, H, int(na[0])

    def contact_forces(self):
        """(n_bodies, 3) resultant barrier contact force of every body at the
        current state, in newtons (dB/dx summed over the body's surface
        vertices, over h^2; the force on the body is the negative)."""
        out = np.zeros(3 * len(self.body_ids))
        lib().orc_contact_forces(self.h, _dp(out))
        return out.reshape(-1, 3)

    def newton_direction(self, y, env=0, which=0):
        """p = -H^-1 g of the Newton system at DOF vector y, solved as the
        stepper does (which 0: dense Cholesky up to 2,500 DOF, else CG to a
        1e-12 relative residual), or by dense Cholesky (1) or that CG (2)."""
        y = _d(y)
        p = np.zeros(len(y))
        if lib().orc_newton_system_solve(self.h, env, _dp(y), int(which), _dp(p)) != 0:
            raise RuntimeError("oracle linear solve failed")
        return p


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (results are bit-identical for
    any count; the library starts with 1).  Returns the count in use."""
    return lib().orc_set_threads(int(n))


# local functions -----------------------------------------------------------
def stencil_d2(x12, is_ee, derivs=False):
    x = _d(np.asarray(x12, dtype=np.float64).ravel())
    kind = np.zeros(1, dtype=np.int32)
    w = np.zeros(4)
    g = np.zeros(12) if derivs else None
    H = np.zeros(144) if derivs else None
    d2 = lib().orc_stencil_d2(_dp(x), int(is_ee), _ip(kind), _dp(w), _dp(g), _dp(H))
    return d2, int(kind[0]), w, g, (None if H is None else H.reshape(12, 12))


def pair_barrier(x12, is_ee, dhat, eps_x=1.0, project=True):
    x = _d(np.asarray(x12, dtype=np.float64).ravel())
    g = np.zeros(12)
    H = np.zeros(144)
    b = lib().orc_pair_barrier(_dp(x), int(is_ee), dhat, eps_x, int(project), _dp(g), _dp(H))
    return b, g, H.reshape(12, 12)


def barrier(d, dhat):
    return lib().orc_barrier_scalar(d, dhat)


def f0(y, eh):
    return lib().orc_f0(y, eh)


def f1(y, eh):
    return lib().orc_f1(y, eh)


def nh(F, mu, lam, project=False):
    F = _d(np.asarray(F, dtype=np.float64).ravel())
    g = np.zeros(9)
    H = np.zeros(81)
    v = lib().orc_nh(_dp(F), mu, lam, int(project), _dp(g), _dp(H))
    return v, g, H.reshape(9, 9)


def stvk(F, mu, lam, project=False):
    F = _d(np.asarray(F, dtype=np.float64).ravel())
    g = np.zeros(9)
    H = np.zeros(81)
    v = lib().orc_stvk(_dp(F), mu, lam, int(project), _dp(g), _dp(H))
    return v, g, H.reshape(9, 9)


def fcr(F, mu, lam, project=False):
    F = _d(np.asarray(F, dtype=np.float64).ravel())
    g = np.zeros(9)
    H = np.zeros(81)
    v = lib().orc_fcr(_dp(F), mu, lam, int(project), _dp(g), _dp(H))
    return v, g, H.reshape(9, 9)


def ortho(A):
    A = _d(np.asarray(A, dtype=np.float64).ravel())
    g = np.zeros(9)
    H = np.zeros(81)
    v = lib().orc_ortho(_dp(A), _dp(g), _dp(H))
    return v, g, H.reshape(9, 9)


def accd(x12, p12, is_ee, s=0.1, tc=1.0):
    x = _d(np.asarray(x12, dtype=np.float64).ravel())
    p = _d(np.asarray(p12, dtype=np.float64).ravel())
    it = np.zeros(1, dtype=np.int32)
    t = lib().orc_accd(_dp(x), _dp(p), int(is_ee), s, tc, _ip(it))
    return t, int(it[0])


def eigvals(A):
    A = _d(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    ev = np.zeros(n)
    lib().orc_eigvals(n, _dp(A.ravel()), _dp(ev))
    return np.sort(ev)


def brute_pairs(pos0, sv_body, b_class, b_env, edges, tris, infl, pos1=None, cap=1 << 22):
    """All valid PT / EE pairs with overlapping inflated (optionally swept)
    AABBs.  b_class: 0 soft, 1 affine dynamic, 2 fixed, 3 kinematic."""
    L = lib()
    pos0 = _d(pos0)
    pos1 = _d(pos1)
    svb = np.ascontiguousarray(sv_body, dtype=np.int32)
    bc = np.ascontiguousarray(b_class, dtype=np.int32)
    be = np.ascontiguousarray(b_env, dtype=np.int32)
    E = np.ascontiguousarray(edges, dtype=np.int32)
    T = np.ascontiguousarray(tris, dtype=np.int32)
    pt = np.zeros((cap, 4), dtype=np.int32)
    ee = np.zeros((cap, 4), dtype=np.int32)
    n = np.zeros(2, dtype=np.int64)
    L.orc_brute_pairs(len(pos0), _dp(pos0), _dp(pos1), _ip(svb), len(bc), _ip(bc), _ip(be), len(E), _ip(E),
                      len(T), _ip(T), infl, cap, _ip(pt), _ip(ee), n.ctypes.data_as(C.POINTER(C.c_long)))
    return pt[:n[0]].copy(), ee[:n[1]].copy()
