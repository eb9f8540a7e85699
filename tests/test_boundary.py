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
    assert not p.stream and not p.alloc and not p.free
