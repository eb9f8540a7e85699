"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/zema.h (no GPU needed)."""
import ctypes
import os
import re

from paper_2311_05945_b300 import build as zbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "zema.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zema_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("zema_create_scene", "zema_add_tet_body", "zema_add_affine_body", "zema_step", "zema_get_state"):
        assert must in names


def test_library_exports_all_declared_symbols():
    lib_path = zbuild.build()
    L = ctypes.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_product_path_does_not_import_oracle():
    # the package never imports, loads or links anything of the oracle
    pat = re.compile(r"^\s*(from\s+oracle|import\s+oracle)|ipc_oracle|libipc_oracle|orc_", re.M)
    pkg = os.path.join(ROOT, "paper_2311_05945_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not pat.search(txt), f


def test_product_path_fails_loudly_without_a_gpu():
    # no CPU fallback: where no CUDA device is visible, building a scene and
    # calling a local entry point raise instead of returning CPU results
    import numpy as np
    import pytest
    import torch

    from paper_2311_05945_b300 import scenes as S
    from paper_2311_05945_b300 import zema as Z
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is visible")
    with pytest.raises(RuntimeError):
        Z.Scene(S.scene_tiny_contact())
    with pytest.raises(RuntimeError):
        Z.local_distance(np.zeros((2, 12)), 0)


def test_default_params_match_the_header():
    # zema_default_params is host-only: its values are the ones include/zema.h
    # documents, read through the binding's structure layout
    from paper_2311_05945_b300.zema import Params
    L = ctypes.CDLL(zbuild.build())
    L.zema_default_params.argtypes = [ctypes.POINTER(Params)]
    p = Params()
    L.zema_default_params(ctypes.byref(p))
    assert (p.dt, p.dhat, p.eps_v, p.newton_tol_rel, p.pcg_rel_tol) == (0.01, 1e-3, 1e-3, 1e-3, 1e-4)
    assert p.kappa <= 0.0  # adaptive
    assert tuple(p.gravity) == (0.0, -9.81, 0.0)
    assert (p.max_newton, p.max_pcg, p.max_al_rounds) == (100, 10000, 10)
    assert (p.precision, p.n_envs, p.warm_start, p.pcg_kind) == (0, 1, 0, 0)
    assert (p.cell_size, p.pcg_cluster_size) == (0.0, 0)
    assert not p.stream and not p.alloc and not p.free



def test_create_scene_checks_its_parameters_on_the_host():
    # zema_create_scene validates the parameters before any device work:
    # the schedule pin accepts the documented codes only
    from paper_2311_05945_b300.zema import Params
    L = ctypes.CDLL(zbuild.build())
    L.zema_default_params.argtypes = [ctypes.POINTER(Params)]
    L.zema_create_scene.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]
    L.zema_destroy_scene.argtypes = [ctypes.c_void_p]

    def create(**kw):
        p = Params()
        L.zema_default_params(ctypes.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        h = ctypes.c_void_p()
        r = L.zema_create_scene(ctypes.byref(p), ctypes.byref(h))
        if r == 0:
            L.zema_destroy_scene(h)
        return r

    ok = [1, 2, 4, 8, 16, 101, 102, 104, 108, 116, 1001, 1002, 1004, 1101, 1102, 1104]
    for code in ok:
        assert create(pcg_cluster_size=code) == 0, code
    for code in (-1, 3, 6, 32, 100, 103, 132, 200, 1000, 1003, 1008, 1100, 1202, 2002):
        assert create(pcg_cluster_size=code) == 1, code
    assert create(pcg_kind=3) == 1 and create(pcg_kind=-1) == 1
    assert create(n_envs=0) == 1 and create(dt=0.0) == 1 and create(dhat=-1e-3) == 1
    assert create(eps_v=0.0) == 1 and create(cell_size=float("inf")) == 1
    assert create(n_envs=256, pcg_kind=2, cell_size=0.004) == 0

def _affine_adder():
    from paper_2311_05945_b300.zema import Params
    L = ctypes.CDLL(zbuild.build())
    DP, IP = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    L.zema_default_params.argtypes = [ctypes.POINTER(Params)]
    L.zema_create_scene.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]
    L.zema_add_affine_body.argtypes = [ctypes.c_void_p, ctypes.c_int32, DP, ctypes.c_int64, IP, ctypes.c_int64, DP,
                                       DP, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32, IP]
    L.zema_destroy_scene.argtypes = [ctypes.c_void_p]
    p = Params()
    L.zema_default_params(ctypes.byref(p))
    h = ctypes.c_void_p()
    # scene creation and body addition are host-only: no GPU needed
    assert L.zema_create_scene(ctypes.byref(p), ctypes.byref(h)) == 0

    def add(V, F):
        import numpy as np
        V = np.ascontiguousarray(V, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.int32)
        q = np.zeros(12)
        q[[3, 7, 11]] = 1.0
        bid = ctypes.c_int32()
        return L.zema_add_affine_body(h, 0, V.ctypes.data_as(DP), len(V), F.ctypes.data_as(IP), len(F),
                                      q.ctypes.data_as(DP), None, 1000.0, 1e8, 0.5, 0, ctypes.byref(bid))

    return add, lambda: L.zema_destroy_scene(h)


def test_affine_mesh_must_be_closed_and_outward():
    # Eq. 2's mass properties integrate over the enclosed volume: open,
    # inconsistently oriented, inward or degenerate surfaces are rejected
    # with ZEMA_ERR_INVALID_ARG at add time
    import numpy as np

    from paper_2311_05945_b300 import scenes as S
    add, close = _affine_adder()
    V, F = S.box_surface((0.1, 0.2, 0.3), 2)
    assert add(V, F) == 0
    assert add(V, F[:-1]) == 1                      # one face missing: open
    assert add(V, F[:, ::-1]) == 1                  # every face reversed: inward
    Fm = F.copy()
    Fm[0] = Fm[0, ::-1]
    assert add(V, Fm) == 1                          # one face flipped
    Fd = F.copy()
    Fd[0, 1] = Fd[0, 0]
    assert add(V, Fd) == 1                          # degenerate face
    Vs, Fs = S.uv_sphere_surface((0.1, 0.1, 0.1), 12, 12)
    assert add(Vs, Fs) == 0
    assert add(np.vstack([V, Vs + 1.0]), np.vstack([F, Fs + len(V)])) == 0  # two closed shells
    close()


def test_generated_affine_meshes_are_accepted():
    from paper_2311_05945_b300 import scenes as S
    add, close = _affine_adder()
    scenes = [S.scene_c1(), S.scene_c2(), S.scene_c3(n_envs=4), S.scene_c5(tets_per_body=300), S.scene_joint(),
              S.scene_slope(), S.scene_kinematic_track(), S.scene_free_fall(), S.scene_tiny_contact()]
    scenes += [S.scene_resolution(n) for n in S.RESOLUTION_SEGMENTS]
    # the pile variants the GPU tests, the benchmark and the training script build
    scenes += [S.scene_c5(n_steps=2, tets_per_body=100, n_soft=2, n_convex=1, n_nonconvex=1, n_seg=6, bin_subdiv=1),
               S.scene_c5(n_steps=2, tets_per_body=300, n_soft=2, n_convex=2, n_nonconvex=2, n_seg=8, bin_subdiv=1),
               S.scene_c5(n_steps=2, tets_per_body=300, n_seg=8, bin_subdiv=1),
               S.scene_c5(n_steps=2, tets_per_body=300, n_soft=4, n_convex=6, n_nonconvex=6, n_seg=16, bin_subdiv=2)]
    for sc in scenes:
        for a in sc.affines:
            assert add(a.V, a.F) == 0, sc.name
    close()


def test_tet_body_arguments_checked_at_add_time():
    # host-side checks of zema_add_tet_body: positive orientation (else
    # ZEMA_ERR_INVERTED_INPUT), index range, Poisson ratio in [0, 0.5), env
    import numpy as np

    from paper_2311_05945_b300.zema import Params
    L = ctypes.CDLL(zbuild.build())
    DP, IP = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    L.zema_default_params.argtypes = [ctypes.POINTER(Params)]
    L.zema_create_scene.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]
    L.zema_add_tet_body.argtypes = [ctypes.c_void_p, ctypes.c_int32, DP, ctypes.c_int64, IP, ctypes.c_int64, DP, DP,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, IP]
    L.zema_destroy_scene.argtypes = [ctypes.c_void_p]
    p = Params()
    L.zema_default_params(ctypes.byref(p))
    h = ctypes.c_void_p()
    assert L.zema_create_scene(ctypes.byref(p), ctypes.byref(h)) == 0
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    bid = ctypes.c_int32()

    def add(T, env=0, nu=0.4):
        T = np.ascontiguousarray(T, dtype=np.int32)
        return L.zema_add_tet_body(h, env, X.ctypes.data_as(DP), len(X), T.ctypes.data_as(IP), len(T), None, None,
                                   1e5, nu, 1000.0, 0.5, ctypes.byref(bid))

    assert add([[0, 1, 2, 3]]) == 0
    assert add([[0, 2, 1, 3]]) == 5          # negative orientation
    assert add([[0, 1, 2, 7]]) == 1          # index out of range
    assert add([[0, 1, 2, 3]], nu=0.5) == 1  # incompressible limit
    assert add([[0, 1, 2, 3]], env=1) == 1   # one env only
    L.zema_destroy_scene(h)


def _header_prototypes():
    src = open(os.path.join(ROOT, "include", "zema.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    protos = {}
    for m in re.finditer(r"([A-Za-z_][A-Za-z_0-9 \*]*?)\b(zema_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", src):
        ret, name, args = m.group(1).strip(), m.group(2), m.group(3).strip()
        params = [] if args in ("", "void") else [a.strip() for a in args.split(",")]
        protos[name] = (ret, params)
    return protos


def _kind_of_c(param):
    # pointer (or array) parameters, else the scalar type
    if "*" in param or "[" in param:
        return "ptr"
    t = re.sub(r"\bconst\b", "", param).split()
    return " ".join(t[:-1])


def test_binding_argtypes_match_the_header():
    # every entry point the binding declares takes the header's parameters:
    # the same count, a pointer where the header has one, the same scalar
    # type elsewhere, and the header's non-status return types
    import ctypes as C

    from paper_2311_05945_b300 import zema as Z
    scalar = {"int32_t": C.c_int32, "int64_t": C.c_int64, "uint64_t": C.c_uint64, "double": C.c_double,
              "float": C.c_float}
    protos = _header_prototypes()
    assert sorted(protos) == declared_symbols()
    L = Z.lib()
    checked = 0
    for name, (ret, params) in protos.items():
        f = getattr(L, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == len(params), name
        for a, p in zip(f.argtypes, params):
            k = _kind_of_c(p)
            if k == "ptr":
                assert a in (C.c_void_p, C.c_char_p) or hasattr(a, "_type_") and issubclass(a, C._Pointer), (name, p)
            else:
                assert a is scalar[k], (name, p, a)
        if ret == "const char*":
            assert f.restype is C.c_char_p, name
        elif ret == "long long":
            assert f.restype is C.c_longlong, name
        checked += 1
    assert checked == len(protos)


def test_mlp_create_checks_its_arguments_on_the_host():
    # widths 1..4096 and 1..16 layers are checked before any device work; on
    # a machine without a GPU a valid network fails with a status and no
    # handle instead of a CPU fallback
    import torch

    from paper_2311_05945_b300 import zema as Z
    L = Z.lib()

    def create(dims, n_layers=None):
        d = (ctypes.c_int32 * len(dims))(*dims)
        h = ctypes.c_void_p()
        r = L.zema_mlp_create(d, len(dims) - 1 if n_layers is None else n_layers, 7, None, ctypes.byref(h))
        return r, h.value

    assert create([13, 128, 3], n_layers=0) == (1, None)
    assert create([13] * 18, n_layers=17) == (1, None)
    assert create([13, 0, 3]) == (1, None)
    assert create([13, 4097, 3]) == (1, None)
    assert create([-1, 128, 3]) == (1, None)
    if not torch.cuda.is_available():
        r, h = create([13, 128, 128, 128, 3])
        assert (r, h) == (3, None)  # ZEMA_ERR_CUDA: no device


def test_local_entry_points_check_arguments_and_take_empty_input_on_the_host():
    # the per-stencil entry points check their arguments before any device
    # work, and an empty batch (n = 0) returns ZEMA_OK without one
    import numpy as np

    from paper_2311_05945_b300 import zema as Z
    L = Z.lib()
    DP, IP = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    d = np.zeros(16 * 144)
    i = np.zeros(16, dtype=np.int32)
    dp, ip = d.ctypes.data_as(DP), i.ctypes.data_as(IP)
    calls = {
        "barrier": lambda n, dhat=1e-3: L.zema_local_barrier(n, dp, ip, dp, dhat, dp, dp, dp, None),
        "distance": lambda n: L.zema_local_distance(n, dp, ip, dp, dp, None),
        "neo_hookean": lambda n: L.zema_local_neo_hookean(n, dp, 1.0, 1.0, dp, dp, dp, None),
        "elastic": lambda n, model=0: L.zema_local_elastic(n, dp, 1.0, 1.0, model, dp, dp, dp, None),
        "accd": lambda n: L.zema_local_accd(n, dp, dp, ip, dp, None),
    }
    for name, f in calls.items():
        assert f(0) == 0, name
        assert f(-1) == 1, name
    assert calls["barrier"](0, dhat=0.0) == 1
    assert calls["elastic"](0, model=3) == 1 and calls["elastic"](0, model=-1) == 1
    assert L.zema_local_distance(0, None, ip, dp, dp, None) == 1
    assert L.zema_local_accd(0, dp, None, ip, dp, None) == 1


def test_affine_body_arguments_checked_at_add_time():
    # host-side checks of zema_add_affine_body besides the mesh: env range,
    # density, stiffness, friction, mode (0 dynamic, 1 fixed, 2 kinematic),
    # the initial state; the message is kept for zema_last_error
    import numpy as np

    from paper_2311_05945_b300 import scenes as S
    from paper_2311_05945_b300 import zema as Z
    L = Z.lib()  # the binding's declared signatures
    DP, IP = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    p = Z.Params()
    L.zema_default_params(ctypes.byref(p))
    p.n_envs = 2
    h = ctypes.c_void_p()
    assert L.zema_create_scene(ctypes.byref(p), ctypes.byref(h)) == 0
    V, F = S.box_surface((0.1, 0.1, 0.1), 1)
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    q = np.zeros(12)
    q[[3, 7, 11]] = 1.0
    bid = ctypes.c_int32(-1)

    def add(env=0, rho=1000.0, stiffness=1e8, mu=0.5, mode=0, q0=q):
        return L.zema_add_affine_body(h, env, V.ctypes.data_as(DP), len(V), F.ctypes.data_as(IP), len(F),
                                      None if q0 is None else q0.ctypes.data_as(DP), None, rho, stiffness, mu,
                                      mode, ctypes.byref(bid))

    assert add(mode=0) == 0 and bid.value == 0
    assert add(env=1, mode=1) == 0 and add(env=1, mode=2) == 0 and bid.value == 2
    for bad in (dict(env=2), dict(env=-1), dict(rho=0.0), dict(stiffness=0.0), dict(mu=-0.1), dict(mode=3),
                dict(mode=-1), dict(q0=None), dict(rho=float("nan"))):
        assert add(**bad) == 1, bad
        assert L.zema_last_error(h) == b"invalid affine body arguments"
    L.zema_destroy_scene(h)


def test_material_spring_and_joint_calls_checked_before_the_first_step():
    # zema_set_material, zema_set_springs and zema_add_prismatic_joint check
    # their arguments on the host; before the first step they touch no device
    import numpy as np

    from paper_2311_05945_b300 import scenes as S
    from paper_2311_05945_b300 import zema as Z
    L = Z.lib()  # the binding's declared signatures
    DP, IP = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    p = Z.Params()
    L.zema_default_params(ctypes.byref(p))
    p.n_envs = 2
    h = ctypes.c_void_p()
    assert L.zema_create_scene(ctypes.byref(p), ctypes.byref(h)) == 0
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    T = np.array([[0, 1, 2, 3]], dtype=np.int32)
    bid = ctypes.c_int32()
    assert L.zema_add_tet_body(h, 0, X.ctypes.data_as(DP), 4, T.ctypes.data_as(IP), 1, None, None, 1e5, 0.4,
                               1000.0, 0.5, ctypes.byref(bid)) == 0                 # body 0: soft, env 0
    V, F = S.box_surface((0.1, 0.1, 0.1), 1)
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    q = np.zeros(12)
    q[[3, 7, 11]] = 1.0
    for env, mode in ((0, 0), (0, 1), (1, 0), (0, 1)):                          # bodies 1..4
        assert L.zema_add_affine_body(h, env, V.ctypes.data_as(DP), len(V), F.ctypes.data_as(IP), len(F),
                                      q.ctypes.data_as(DP), None, 1000.0, 1e8, 0.5, mode, ctypes.byref(bid)) == 0
    assert bid.value == 4
    # materials: soft bodies only, models 0..2
    assert [L.zema_set_material(h, 0, m) for m in (1, 2, 0)] == [0, 0, 0]
    assert L.zema_set_material(h, 0, 3) == 1 and L.zema_set_material(h, 1, 0) == 1
    assert L.zema_set_material(h, 9, 0) == 1
    # springs: vertex ids of the body, finite targets, finite k >= 0
    v = np.array([0, 3], dtype=np.int32)
    x = np.zeros((2, 3))

    def springs(body=0, verts=v, targets=x, k=10.0):
        return L.zema_set_springs(h, body, verts.ctypes.data_as(IP), len(verts), targets.ctypes.data_as(DP), k)

    assert springs() == 0
    assert L.zema_set_springs(h, 0, None, 0, None, 0.0) == 0
    assert springs(verts=np.array([0, 4], dtype=np.int32)) == 1
    assert springs(k=-1.0) == 1 and springs(k=float("inf")) == 1
    assert springs(targets=np.array([[0.0, 0.0, 0.0], [np.nan, 0.0, 0.0]])) == 1
    assert springs(body=1) == 1
    # prismatic joints: two distinct affine bodies of one env, one of them
    # dynamic, a nonzero finite axis
    jid = ctypes.c_int32(-1)
    ax = np.array([0.0, 2.0, 0.0])

    def joint(b1, b2, axis=ax, kappa=0.0):
        return L.zema_add_prismatic_joint(h, b1, b2, axis.ctypes.data_as(DP), kappa, ctypes.byref(jid))

    assert joint(1, 2) == 0 and jid.value == 0
    assert joint(1, 1) == 1 and joint(0, 1) == 1 and joint(1, 9) == 1
    assert joint(1, 2, kappa=float("inf")) == 1
    assert L.zema_last_error(h) == b"a prismatic joint needs two distinct affine bodies and an axis"
    assert joint(1, 3) == 1
    assert L.zema_last_error(h) == b"jointed bodies must share an env and at least one must be dynamic"
    assert joint(2, 4) == 1
    assert L.zema_last_error(h) == b"jointed bodies must share an env and at least one must be dynamic"
    assert joint(1, 2, axis=np.zeros(3)) == 1 and joint(1, 2, axis=np.array([np.nan, 1.0, 0.0])) == 1
    assert L.zema_last_error(h) == b"joint axis must be a nonzero finite vector"
    assert joint(4, 1) == 0 and jid.value == 1
    L.zema_destroy_scene(h)


def test_state_calls_before_the_first_step_are_host_only():
    # before the first step zema_get_state / zema_set_state read and write
    # the bodies' initial states on the host (tet body: x then v, nv x 3
    # each; affine body: q then qdot, 12 each, in the caller's frame); the
    # whole-scene state and checkpoint calls need a built scene and return
    # ZEMA_ERR_STATE
    import numpy as np

    from paper_2311_05945_b300 import scenes as S
    from paper_2311_05945_b300 import zema as Z
    L = Z.lib()
    DP, IP = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    p = Z.Params()
    L.zema_default_params(ctypes.byref(p))
    h = ctypes.c_void_p()
    assert L.zema_create_scene(ctypes.byref(p), ctypes.byref(h)) == 0
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    T = np.array([[0, 1, 2, 3]], dtype=np.int32)
    bid = ctypes.c_int32()
    assert L.zema_add_tet_body(h, 0, X.ctypes.data_as(DP), 4, T.ctypes.data_as(IP), 1, None, None, 1e5, 0.4,
                               1000.0, 0.5, ctypes.byref(bid)) == 0
    V, F = S.box_surface((0.1, 0.1, 0.1), 1)
    V = np.ascontiguousarray(V + 3.0, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    q = np.array([0.5, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0])
    assert L.zema_add_affine_body(h, 0, V.ctypes.data_as(DP), len(V), F.ctypes.data_as(IP), len(F),
                                  q.ctypes.data_as(DP), None, 1000.0, 1e8, 0.5, 0, ctypes.byref(bid)) == 0
    out = np.full(32, -1.0)
    n = ctypes.c_int64(-1)

    def get(body, cap):
        out[:] = -1.0
        return L.zema_get_state(h, body, out.ctypes.data_as(DP), cap, ctypes.byref(n))

    assert get(0, 24) == 0 and n.value == 24
    assert np.array_equal(out[:12], X.ravel()) and np.all(out[12:24] == 0.0) and np.all(out[24:] == -1.0)
    assert get(1, 24) == 0 and n.value == 24
    assert np.array_equal(out[:12], q) and np.all(out[12:24] == 0.0)
    assert get(0, 23) == 1 and get(1, 23) == 1 and get(2, 32) == 1 and get(-1, 32) == 1
    assert np.all(out == -1.0)
    st = np.arange(24, dtype=np.float64) * 0.01
    for body in (0, 1):
        assert L.zema_set_state(h, body, st.ctypes.data_as(DP), 24) == 0
        assert get(body, 24) == 0 and np.array_equal(out[:24], st)
        assert L.zema_set_state(h, body, st.ctypes.data_as(DP), 23) == 1
    assert L.zema_set_state(h, 0, None, 24) == 1
    STATE = 11
    m = ctypes.c_int64()
    assert L.zema_scene_state_size(h, ctypes.byref(m)) == STATE
    assert L.zema_get_scene_state(h, out.ctypes.data_as(ctypes.c_void_p), 32, ctypes.byref(m)) == STATE
    assert L.zema_set_scene_state(h, out.ctypes.data_as(ctypes.c_void_p), 32) == STATE
    assert L.zema_checkpoint_size(h, ctypes.byref(m)) == STATE
    assert L.zema_save_checkpoint(h, out.ctypes.data_as(ctypes.c_void_p), 256, ctypes.byref(m)) == STATE
    assert L.zema_copy_soft_state_device(h, None, None) == STATE
    L.zema_destroy_scene(h)
