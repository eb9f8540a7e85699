"""Python binding of the zema C ABI (include/zema.h): argument marshalling only.

Every computation happens in libzema.so's CUDA kernels.  PyTorch supplies the
CUDA stream (and, optionally, device memory through its caching allocator).
There is no CPU fallback: without the built library or a GPU, calls raise.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref
from typing import Optional

import numpy as np

from . import scenes as _scenes

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libzema.so")

STATUS = {
    0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "INTERSECTING_INPUT", 5: "INVERTED_INPUT",
    6: "NEWTON_MAXITER", 7: "LINESEARCH", 8: "PCG_MAXITER", 9: "NONFINITE", 10: "FAULT_INJECTED", 11: "STATE",
}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Params(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double), ("eps_v", C.c_double),
        ("newton_tol_rel", C.c_double), ("gravity", C.c_double * 3), ("pcg_rel_tol", C.c_double),
        ("max_newton", C.c_int32), ("max_pcg", C.c_int32), ("max_al_rounds", C.c_int32),
        ("precision", C.c_int32), ("n_envs", C.c_int32), ("warm_start", C.c_int32), ("pcg_kind", C.c_int32),
        ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
        ("cell_size", C.c_double), ("pcg_cluster_size", C.c_int32), ("al_extrapolate", C.c_int32),
    ]


class StepStats(C.Structure):
    _fields_ = [
        ("steps", C.c_int64), ("newton_iters", C.c_int64), ("pcg_iters", C.c_int64), ("ls_halvings", C.c_int64),
        ("al_rounds", C.c_int64), ("warm_accepted", C.c_int64), ("max_candidates", C.c_int64),
        ("max_active", C.c_int64), ("dmin", C.c_double), ("kappa", C.c_double), ("energy", C.c_double),
        ("ms_phase", C.c_double * 6), ("pcg_refines", C.c_int64), ("warm_learned", C.c_int64),
        ("warm_fallback", C.c_int64),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms_phase"}
        d["ms_phase"] = dict(zip(["dcd", "energy", "hess", "linear", "ccd", "other"], list(self.ms_phase)))
        return d


class ZemaError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"zema status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


_lib = None

DP = C.POINTER(C.c_double)
IP = C.POINTER(C.c_int32)
LP = C.POINTER(C.c_int64)


def lib():
    """Load libzema.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"zema CUDA library not built ({LIB_PATH}); run paper_2311_05945_b300.build.build()")
    L = C.CDLL(LIB_PATH)
    L.zema_default_params.argtypes = [C.POINTER(Params)]
    L.zema_create_scene.argtypes = [C.POINTER(Params), C.POINTER(C.c_void_p)]
    L.zema_add_tet_body.argtypes = [C.c_void_p, C.c_int32, DP, C.c_int64, IP, C.c_int64, DP, DP, C.c_double,
                                    C.c_double, C.c_double, C.c_double, IP]
    L.zema_add_affine_body.argtypes = [C.c_void_p, C.c_int32, DP, C.c_int64, IP, C.c_int64, DP, DP, C.c_double,
                                       C.c_double, C.c_double, C.c_int32, IP]
    L.zema_finalize.argtypes = [C.c_void_p]
    L.zema_set_kinematic_target.argtypes = [C.c_void_p, C.c_int32, DP]
    L.zema_set_kinematic_targets.argtypes = [C.c_void_p, C.c_int64, IP, DP]
    L.zema_scene_state_size.argtypes = [C.c_void_p, LP]
    L.zema_get_scene_state.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, LP]
    L.zema_set_scene_state.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    L.zema_step.argtypes = [C.c_void_p, C.c_int32, C.POINTER(StepStats)]
    L.zema_get_state.argtypes = [C.c_void_p, C.c_int32, DP, C.c_int64, LP]
    L.zema_set_state.argtypes = [C.c_void_p, C.c_int32, DP, C.c_int64]
    L.zema_copy_soft_state_device.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    L.zema_scene_counts.argtypes = [C.c_void_p, LP]
    L.zema_get_kappa.argtypes = [C.c_void_p, C.c_int32, DP]
    L.zema_set_kappa.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double]
    L.zema_last_error.restype = C.c_char_p
    L.zema_last_error.argtypes = [C.c_void_p]
    L.zema_destroy_scene.argtypes = [C.c_void_p]
    L.zema_eval_energy_grad.argtypes = [C.c_void_p, C.c_int32, DP, DP]
    L.zema_candidates_raw.argtypes = [C.c_int64, DP, DP, IP, C.c_int64, IP, IP, C.c_int64, IP, C.c_int64, IP,
                                      C.c_double, C.c_double, C.c_int64, IP, IP, LP, C.c_void_p]
    L.zema_candidates_raw_noalloc.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                              C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_double,
                                              C.c_double, C.c_int64, C.c_void_p, C.c_void_p, LP, C.c_void_p]
    L.zema_local_barrier.argtypes = [C.c_int64, DP, IP, DP, C.c_double, DP, DP, DP, C.c_void_p]
    L.zema_local_distance.argtypes = [C.c_int64, DP, IP, DP, DP, C.c_void_p]
    L.zema_local_neo_hookean.argtypes = [C.c_int64, DP, C.c_double, C.c_double, DP, DP, DP, C.c_void_p]
    L.zema_local_elastic.argtypes = [C.c_int64, DP, C.c_double, C.c_double, C.c_int32, DP, DP, DP, C.c_void_p]
    L.zema_local_accd.argtypes = [C.c_int64, DP, DP, IP, DP, C.c_void_p]
    L.zema_launch_count.restype = C.c_longlong
    L.zema_launch_count.argtypes = []
    L.zema_profile_kernel.argtypes = [C.c_char_p]
    L.zema_profile_read.argtypes = [DP, C.POINTER(C.c_longlong), DP]
    FP = C.POINTER(C.c_float)
    L.zema_load_warmstart.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    L.zema_autotune.argtypes = [C.c_void_p]
    L.zema_checkpoint_size.argtypes = [C.c_void_p, LP]
    L.zema_save_checkpoint.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, LP]
    L.zema_load_checkpoint.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    L.zema_inject_fault.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
    L.zema_get_tuning.argtypes = [C.c_void_p, C.c_int32, IP, IP, FP, C.c_int32, IP]
    L.zema_record_warmstart.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
    L.zema_record_warmstart_affine.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
    L.zema_contact_forces.argtypes = [C.c_void_p, DP, C.c_int64]
    L.zema_set_material.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
    L.zema_add_prismatic_joint.argtypes = [C.c_void_p, C.c_int32, C.c_int32, DP, C.c_double, IP]
    L.zema_set_springs.argtypes = [C.c_void_p, C.c_int32, IP, C.c_int64, DP, C.c_double]
    L.zema_mlp_create.argtypes = [IP, C.c_int32, C.c_uint64, C.c_void_p, C.POINTER(C.c_void_p)]
    L.zema_mlp_destroy.argtypes = [C.c_void_p]
    L.zema_mlp_destroy.restype = None
    L.zema_mlp_n_params.argtypes = [C.c_void_p, LP]
    L.zema_mlp_get_params.argtypes = [C.c_void_p, FP, C.c_int64]
    L.zema_mlp_set_params.argtypes = [C.c_void_p, FP, C.c_int64]
    L.zema_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    L.zema_mlp_set_kernel.argtypes = [C.c_void_p, C.c_int32]
    L.zema_mlp_gradient.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, FP, C.c_int64, DP]
    L.zema_mlp_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_float,
                                      C.c_float, C.c_float, C.c_float, DP]
    _lib = L
    return L


def _d(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def _dp(a):
    return None if a is None else a.ctypes.data_as(DP)


def _ip(a):
    return None if a is None else a.ctypes.data_as(IP)


def _stream():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("zema needs a CUDA device")
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# torch-backed device allocator (device memory comes from PyTorch's caching allocator)
def _torch_alloc(nbytes, stream, ctx):
    import torch
    return int(torch.cuda.caching_allocator_alloc(int(nbytes)))


def _torch_free(ptr, stream, ctx):
    import torch
    torch.cuda.caching_allocator_delete(ptr)


_LIVE = weakref.WeakSet()


@atexit.register
def _close_all():
    # release device memory while PyTorch is still importable
    for sc in list(_LIVE):
        try:
            sc.close()
        except Exception:
            pass


_ALLOC = ALLOC_FN(_torch_alloc)
_FREE = FREE_FN(_torch_free)


def _check(r, handle=None):
    if r != 0:
        msg = ""
        if handle:
            m = lib().zema_last_error(handle)
            msg = m.decode() if m else ""
        raise ZemaError(r, msg)


class Scene:
    """A scene of the seeded generators loaded into the library."""

    def __init__(self, scene: _scenes.Scene, precision: Optional[int] = None, tol_scale: float = 1.0,
                 torch_alloc: bool = True, kappa: Optional[float] = None, pcg_kind: int = 0,
                 warm_start: int = 0, cell_size: float = 0.0, pcg_cluster_size: int = 0):
        L = lib()
        p = scene.params
        P = Params()
        L.zema_default_params(C.byref(P))
        P.dt = p.dt
        P.dhat = p.dhat
        P.kappa = p.kappa if kappa is None else kappa
        P.eps_v = p.eps_v
        P.newton_tol_rel = p.newton_tol_rel * tol_scale
        for k in range(3):
            P.gravity[k] = p.gravity[k]
        P.pcg_rel_tol = p.pcg_rel_tol
        P.max_newton = p.max_newton
        P.max_pcg = p.max_pcg
        P.max_al_rounds = p.max_al_rounds
        P.al_extrapolate = p.al_extrapolate
        P.precision = p.precision if precision is None else precision
        P.n_envs = scene.n_envs
        P.pcg_kind = pcg_kind
        P.warm_start = warm_start
        P.cell_size = cell_size
        P.pcg_cluster_size = pcg_cluster_size
        P.stream = _stream()
        if torch_alloc:
            P.alloc = _ALLOC
            P.free = _FREE
        self._P = P
        h = C.c_void_p()
        _check(L.zema_create_scene(C.byref(P), C.byref(h)))
        self.h = h
        self.scene = scene
        self.body_ids = []
        for kind, i in scene.body_order():
            bid = C.c_int32()
            if kind == "tet":
                b = scene.tets[i]
                X, T, x0, v0 = _d(b.X), _i(b.tets), _d(b.x0), _d(b.v0)
                r = L.zema_add_tet_body(h, b.env, _dp(X), len(X), _ip(T), len(T), _dp(x0), _dp(v0), b.E, b.nu,
                                        b.rho, b.mu, C.byref(bid))
            else:
                b = scene.affines[i]
                V, F, q0, qd = _d(b.V), _i(b.F), _d(b.q0), _d(b.qdot0)
                r = L.zema_add_affine_body(h, b.env, _dp(V), len(V), _ip(F), len(F), _dp(q0), _dp(qd), b.rho,
                                           b.stiffness, b.mu, b.mode, C.byref(bid))
            _check(r, h)
            self.body_ids.append(bid.value)
        self.n_tet = len(scene.tets)
        self.step_index = 0
        _LIVE.add(self)
        for i, b in enumerate(scene.tets):
            if b.model:
                _check(L.zema_set_material(h, self.body_ids[i], int(b.model)), h)
        for (i, verts, targets, k) in scene.springs:
            self.set_springs(i, verts, targets, k)
        for (a1, a2, axis, kappa) in scene.joints:
            ax = _d(axis)
            _check(L.zema_add_prismatic_joint(h, self.affine_body_id(a1), self.affine_body_id(a2), _dp(ax),
                                              float(kappa), None), h)
        _check(L.zema_finalize(h), h)

    def close(self):
        if getattr(self, "h", None):
            lib().zema_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self):
        """Tune the linear solve's CTAs per environment at the next solve."""
        _check(lib().zema_autotune(self.h), self.h)

    def tuning(self, precision=None):
        """(cluster schedule in use, {candidate: solve ms}) of the autotuner;
        a schedule is the CTAs per env, plus 100 for the two-CTAs-per-SM
        variant."""
        p = self._P.precision if precision is None else precision
        cs, n = C.c_int32(), C.c_int32()
        cap = 32
        cand = np.zeros(cap, dtype=np.int32)
        ms = np.zeros(cap, dtype=np.float32)
        _check(lib().zema_get_tuning(self.h, p, C.byref(cs), _ip(cand), ms.ctypes.data_as(C.POINTER(C.c_float)), cap,
                                     C.byref(n)), self.h)
        return cs.value, {int(cand[i]): float(ms[i]) for i in range(min(n.value, cap))}

    def load_warmstart(self, dims, theta):
        """Load a learned warm-start network: per soft vertex (dims[0] = 13,
        dims[-1] = 3) or per dynamic affine body (dims[0] = 40, dims[-1] = 12)."""
        blob = warmstart_blob(dims, theta)
        _check(lib().zema_load_warmstart(self.h, blob.ctypes.data_as(C.c_void_p), blob.nbytes), self.h)

    def record_warmstart(self, features=None, targets=None):
        """Record features (rows x 13) and scaled step displacements (rows x 3)
        of the soft vertices into CUDA float32 tensors during later steps."""
        if features is None:
            _check(lib().zema_record_warmstart(self.h, None, None, 0), self.h)
            return
        rows = min(features.shape[0], targets.shape[0])
        _check(lib().zema_record_warmstart(self.h, C.c_void_p(features.data_ptr()), C.c_void_p(targets.data_ptr()),
                                           rows), self.h)

    def set_springs(self, tet_index, verts, targets, k):
        """Spring constraints h^2 k |x - target|^2 on body-local vertices of a
        soft body (replacing its springs; allowed between steps)."""
        v = _i(verts)
        t = _d(targets)
        _check(lib().zema_set_springs(self.h, self.body_ids[tet_index], _ip(v), len(v), _dp(t), float(k)), self.h)

    def contact_forces(self) -> np.ndarray:
        """(n_bodies, 3) barrier contact force of every body at the current
        state, in newtons (gradient convention: the force on the body is the
        negative)."""
        n = len(self.body_ids)
        out = np.zeros(3 * n, dtype=np.float64)
        _check(lib().zema_contact_forces(self.h, _dp(out), out.size), self.h)
        return out.reshape(n, 3)

    def record_warmstart_affine(self, features=None, targets=None):
        """Record features (rows x 40) and scaled changes of q (rows x 12) of
        the dynamic affine bodies into CUDA float32 tensors during later steps."""
        if features is None:
            _check(lib().zema_record_warmstart_affine(self.h, None, None, 0), self.h)
            return
        rows = min(features.shape[0], targets.shape[0])
        _check(lib().zema_record_warmstart_affine(self.h, C.c_void_p(features.data_ptr()),
                                                  C.c_void_p(targets.data_ptr()), rows), self.h)

    def tet_body_id(self, i):
        return self.body_ids[i]

    def affine_body_id(self, i):
        return self.body_ids[self.n_tet + i]

    def set_kinematic_target(self, affine_index, q):
        """Target state q (12,) of a kinematic affine body for the next step."""
        qq = _d(q)
        _check(lib().zema_set_kinematic_target(self.h, self.affine_body_id(affine_index), _dp(qq)), self.h)

    def set_kinematic_targets(self, affine_indices, Q):
        """Targets Q (n, 12) of the kinematic affine bodies affine_indices
        (n,) for the next step, in one call."""
        ids = _i(np.array([self.affine_body_id(int(i)) for i in affine_indices], dtype=np.int32))
        QQ = _d(np.asarray(Q, dtype=np.float64).reshape(len(ids), 12))
        _check(lib().zema_set_kinematic_targets(self.h, len(ids), _ip(ids), _dp(QQ)), self.h)

    def apply_script(self):
        if self.scene.script is None:
            return
        arrays = getattr(self.scene.script, "arrays", None)
        if arrays is not None:
            idx, Q = arrays(self.step_index)
        else:
            targets = self.scene.script(self.step_index)
            idx = list(targets.keys())
            Q = np.array([targets[i] for i in idx], dtype=np.float64).reshape(len(idx), 12)
        if len(idx):
            self.set_kinematic_targets(idx, Q)

    def step(self, n: int = 1, script: bool = True) -> dict:
        """Advance n steps (the scene's kinematic script is applied before
        each); returns the summed statistics of the last call."""
        st = StepStats()
        total = None
        for _ in range(n):
            if script:
                self.apply_script()
            r = lib().zema_step(self.h, 1, C.byref(st))
            _check(r, self.h)
            self.step_index += 1
            d = st.as_dict()
            if total is None:
                total = d
            else:
                for k in ("steps", "newton_iters", "pcg_iters", "ls_halvings", "al_rounds", "warm_accepted",
                          "pcg_refines", "warm_learned", "warm_fallback"):
                    total[k] += d[k]
                for k in ("max_candidates", "max_active"):
                    total[k] = max(total[k], d[k])
                for k in ("dmin", "kappa", "energy"):
                    total[k] = d[k]
                for k in total["ms_phase"]:
                    total["ms_phase"][k] += d["ms_phase"][k]
        return total or {}

    def step_raw(self, n: int = 1) -> dict:
        """n steps in one library call (no script)."""
        st = StepStats()
        _check(lib().zema_step(self.h, n, C.byref(st)), self.h)
        self.step_index += n
        return st.as_dict()

    def save_checkpoint(self) -> tuple:
        """(checkpoint bytes, script step index): the whole scene's
        step-to-step state (zema_save_checkpoint)."""
        n = C.c_int64()
        _check(lib().zema_checkpoint_size(self.h, C.byref(n)), self.h)
        buf = np.zeros(n.value, dtype=np.uint8)
        w = C.c_int64()
        _check(lib().zema_save_checkpoint(self.h, buf.ctypes.data_as(C.c_void_p), n.value, C.byref(w)), self.h)
        return buf, self.step_index

    def load_checkpoint(self, ckpt):
        """Restore a (bytes, step index) pair of save_checkpoint, from this
        scene or one built from the same bodies (either precision)."""
        buf, step_index = ckpt
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().zema_load_checkpoint(self.h, buf.ctypes.data_as(C.c_void_p), buf.nbytes), self.h)
        self.step_index = step_index

    def inject_fault(self, kind: int, newton_iter: int = 0):
        """Arm one failure of the next step call (zema_inject_fault): 1 status
        word, 2 non-finite solve, 3 no line-search decrease; 0 disarms."""
        _check(lib().zema_inject_fault(self.h, int(kind), int(newton_iter)), self.h)

    def scene_state_size(self) -> int:
        n = C.c_int64()
        _check(lib().zema_scene_state_size(self.h, C.byref(n)), self.h)
        return n.value

    def get_scene_state(self) -> np.ndarray:
        """Every body's state, bodies back to back in order of addition."""
        out = np.zeros(self.scene_state_size())
        _check(lib().zema_get_scene_state(self.h, out.ctypes.data_as(C.c_void_p), len(out), None), self.h)
        return out

    def set_scene_state(self, arr):
        a = _d(arr)
        _check(lib().zema_set_scene_state(self.h, a.ctypes.data_as(C.c_void_p), len(a)), self.h)

    def get_scene_state_ptr(self, ptr, cap):
        """Into caller memory at ptr (host, e.g. pinned)."""
        _check(lib().zema_get_scene_state(self.h, C.c_void_p(ptr), cap, None), self.h)

    def set_scene_state_ptr(self, ptr, n):
        _check(lib().zema_set_scene_state(self.h, C.c_void_p(ptr), n), self.h)

    def get_state(self, body):
        cap = 1 << 24
        out = np.zeros(cap)
        w = C.c_int64()
        _check(lib().zema_get_state(self.h, body, _dp(out), cap, C.byref(w)), self.h)
        return out[:w.value].copy()

    def set_state(self, body, arr):
        a = _d(arr)
        _check(lib().zema_set_state(self.h, body, _dp(a), len(a)), self.h)

    def set_state_ptr(self, body, ptr, n):
        """zema_set_state from a raw host pointer (e.g. pinned memory)."""
        _check(lib().zema_set_state(self.h, body, C.cast(C.c_void_p(ptr), DP), n), self.h)

    def get_state_ptr(self, body, ptr, cap):
        """zema_get_state into a raw host pointer (e.g. pinned memory)."""
        w = C.c_int64()
        _check(lib().zema_get_state(self.h, body, C.cast(C.c_void_p(ptr), DP), cap, C.byref(w)), self.h)
        return w.value

    def tet_positions(self, i=0):
        st = self.get_state(self.tet_body_id(i))
        n = len(st) // 6
        return st[:3 * n].reshape(n, 3)

    def affine_q(self, i):
        return self.get_state(self.affine_body_id(i))[:12]

    def counts(self):
        out = np.zeros(8, dtype=np.int64)
        _check(lib().zema_scene_counts(self.h, out.ctypes.data_as(LP)), self.h)
        keys = ["n_verts", "n_tets", "n_affine", "n_sv", "n_edges", "n_tris", "n_nodes", "n_envs"]
        return dict(zip(keys, map(int, out)))

    def kappa(self, env=0):
        k = C.c_double()
        _check(lib().zema_get_kappa(self.h, env, C.byref(k)), self.h)
        return k.value

    def set_kappa(self, env, kappa, kappa_min):
        _check(lib().zema_set_kappa(self.h, env, kappa, kappa_min), self.h)

    def eval_energy_grad(self, apply_predictor=True, grad=True):
        """Total incremental potential per env and (optionally) the gradient
        in the caller's frame, bodies in order of addition."""
        if apply_predictor:
            self.apply_script()
        E = np.zeros(self.scene.n_envs)
        n = sum(3 * len(b.X) for b in self.scene.tets) + 12 * len(self.scene.affines)
        g = np.zeros(n) if grad else None
        _check(lib().zema_eval_energy_grad(self.h, 1 if apply_predictor else 0, _dp(E), _dp(g)), self.h)
        return E, g


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().zema_launch_count())


def profile_kernel(name: Optional[str]):
    """Time every launch of one library kernel with CUDA events (None stops)."""
    lib().zema_profile_kernel(None if name is None else name.encode())


def profile_read():
    """(ms total, launches, algorithmic bytes) since profile_kernel()."""
    ms = C.c_double()
    n = C.c_longlong()
    b = C.c_double()
    lib().zema_profile_read(C.byref(ms), C.byref(n), C.byref(b))
    return ms.value, n.value, b.value


# ---------------------------------------------------------------------------
# stand-alone kernels
# ---------------------------------------------------------------------------
def candidates_raw(pos0, sv_body, b_class, b_env, edges, tris, inflate, pos1=None, cell_size=0.0, cap=1 << 22):
    L = lib()
    pos0 = _d(pos0)
    pos1 = _d(pos1)
    svb, bc, be, E, T = _i(sv_body), _i(b_class), _i(b_env), _i(edges), _i(tris)
    pt = np.zeros((cap, 2), dtype=np.int32)
    ee = np.zeros((cap, 2), dtype=np.int32)
    n = np.zeros(2, dtype=np.int64)
    _check(L.zema_candidates_raw(len(pos0), _dp(pos0), _dp(pos1), _ip(svb), len(bc), _ip(bc), _ip(be), len(E), _ip(E),
                                 len(T), _ip(T), inflate, cell_size, cap, _ip(pt), _ip(ee), n.ctypes.data_as(LP),
                                 _stream()))
    if n[0] > cap or n[1] > cap:
        raise ZemaError(1, "candidate capacity exceeded")
    return pt[:n[0]].copy(), ee[:n[1]].copy()


def candidates_raw_noalloc(pos0, sv_body, b_class, b_env, edges, tris, inflate, cell_size, pt_out, ee_out,
                           pos1=None):
    """zema_candidates_raw_noalloc on CUDA tensors (float64 positions, int32
    index arrays; pt_out / ee_out int32 (cap, 2) tensors).  Returns the two
    pair counts; the pairs are in pt_out[:n_pt], ee_out[:n_ee]."""
    import torch

    def ptr(t):
        return None if t is None else C.c_void_p(t.data_ptr())

    for t in (pos0, sv_body, b_class, b_env, edges, tris, pt_out, ee_out):
        assert t.is_cuda and t.is_contiguous()
    n = np.zeros(2, dtype=np.int64)
    cap = min(pt_out.shape[0], ee_out.shape[0])
    _check(lib().zema_candidates_raw_noalloc(pos0.shape[0], ptr(pos0), ptr(pos1), ptr(sv_body), b_class.shape[0],
                                             ptr(b_class), ptr(b_env), edges.shape[0], ptr(edges), tris.shape[0],
                                             ptr(tris), inflate, cell_size, cap, ptr(pt_out), ptr(ee_out),
                                             n.ctypes.data_as(LP), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return int(n[0]), int(n[1])


def local_barrier(x12, is_ee, eps_x, dhat):
    x = _d(np.asarray(x12).reshape(-1, 12))
    n = len(x)
    ie = _i(np.broadcast_to(np.asarray(is_ee), (n,)))
    ep = _d(np.broadcast_to(np.asarray(eps_x, dtype=np.float64), (n,)))
    E, g, H = np.zeros(n), np.zeros((n, 12)), np.zeros((n, 12, 12))
    _check(lib().zema_local_barrier(n, _dp(x), _ip(ie), _dp(ep), dhat, _dp(E), _dp(g), _dp(H), _stream()))
    return E, g, H


def local_distance(x12, is_ee):
    x = _d(np.asarray(x12).reshape(-1, 12))
    n = len(x)
    ie = _i(np.broadcast_to(np.asarray(is_ee), (n,)))
    d2, w = np.zeros(n), np.zeros((n, 4))
    _check(lib().zema_local_distance(n, _dp(x), _ip(ie), _dp(d2), _dp(w), _stream()))
    return d2, w


def local_neo_hookean(F, mu, lam):
    F = _d(np.asarray(F).reshape(-1, 9))
    n = len(F)
    psi, g, H = np.zeros(n), np.zeros((n, 9)), np.zeros((n, 9, 9))
    _check(lib().zema_local_neo_hookean(n, _dp(F), mu, lam, _dp(psi), _dp(g), _dp(H), _stream()))
    return psi, g, H


def local_elastic(F, mu, lam, model):
    F = _d(np.asarray(F).reshape(-1, 9))
    n = len(F)
    psi, g, H = np.zeros(n), np.zeros((n, 9)), np.zeros((n, 9, 9))
    _check(lib().zema_local_elastic(n, _dp(F), mu, lam, int(model), _dp(psi), _dp(g), _dp(H), _stream()))
    return psi, g, H


def local_accd(x12, p12, is_ee):
    x = _d(np.asarray(x12).reshape(-1, 12))
    p = _d(np.asarray(p12).reshape(-1, 12))
    n = len(x)
    ie = _i(np.broadcast_to(np.asarray(is_ee), (n,)))
    t = np.zeros(n)
    _check(lib().zema_local_accd(n, _dp(x), _dp(p), _ip(ie), _dp(t), _stream()))
    return t


class Mlp:
    """A tensor-core MLP of the library (dims[0] -> ... -> dims[-1], ReLU
    between layers).  Inputs and targets are CUDA float32 tensors."""

    def __init__(self, dims, seed: int = 0):
        L = lib()
        self.dims = [int(d) for d in dims]
        d = np.array(self.dims, dtype=np.int32)
        h = C.c_void_p()
        _check(L.zema_mlp_create(_ip(d), len(self.dims) - 1, C.c_uint64(seed), _stream(), C.byref(h)))
        self.h = h
        n = C.c_int64()
        _check(L.zema_mlp_n_params(h, C.byref(n)))
        self.n_params = n.value

    def close(self):
        if getattr(self, "h", None):
            lib().zema_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_kernel(self, kind: int):
        """0: tcgen05 forward products (default), 1: warp-level mma.sync."""
        _check(lib().zema_mlp_set_kernel(self.h, kind))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().zema_mlp_get_params(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), self.n_params))
        return out

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib().zema_mlp_set_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float)), len(a)))

    @staticmethod
    def _dev(x):
        import torch
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
        return C.c_void_p(x.data_ptr())

    def forward(self, x):
        import torch
        y = torch.empty((x.shape[0], self.dims[-1]), dtype=torch.float32, device=x.device)
        _check(lib().zema_mlp_forward(self.h, self._dev(x), x.shape[0], self._dev(y)))
        return y

    def gradient(self, x, t):
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_double()
        _check(lib().zema_mlp_gradient(self.h, self._dev(x), self._dev(t), x.shape[0],
                                       g.ctypes.data_as(C.POINTER(C.c_float)), self.n_params, C.byref(loss)))
        return loss.value, g

    def train_step(self, x, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        loss = C.c_double()
        _check(lib().zema_mlp_train_step(self.h, self._dev(x), self._dev(t), x.shape[0], lr, beta1, beta2, eps,
                                         weight_decay, C.byref(loss)))
        return loss.value


WARMSTART_MAGIC = 0x5357455A


def warmstart_blob(dims, theta) -> np.ndarray:
    """The byte layout zema_load_warmstart reads, as a uint8 array."""
    dims = [int(d) for d in dims]
    head = np.array([WARMSTART_MAGIC, len(dims) - 1] + dims, dtype=np.uint32)
    return np.concatenate([head.view(np.uint8), np.ascontiguousarray(theta, dtype=np.float32).view(np.uint8)])


def read_warmstart_blob(blob: bytes):
    """(dims, theta) from a warm-start blob."""
    h = np.frombuffer(blob, dtype=np.uint32)
    assert h[0] == WARMSTART_MAGIC
    L = int(h[1])
    dims = [int(d) for d in h[2:3 + L]]
    theta = np.frombuffer(blob, dtype=np.float32, offset=4 * (3 + L)).copy()
    return dims, theta
