"""A plain C99 program includes include/zema.h, links libzema.so and drives
the host-only part of the boundary (no GPU needed): default parameters,
parameter checks, scene creation, a body added and one rejected with its
status and message, and teardown.  This checks that the header is valid C
(no C++ or torch types) and that the entry points link from C.  The
binding's ctypes structures are checked against the C layout (size and
every field's offset)."""
import ctypes
import os
import subprocess

import pytest

from paper_2311_05945_b300 import build as zbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "zema.h"

int main(void) {
    zema_scene_params p;
    zema_scene* s = NULL;
    double X[12] = {0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1};
    int32_t good[4] = {0, 1, 2, 3}, flipped[4] = {0, 2, 1, 3};
    int32_t id = -1;
    zema_status r;

    zema_default_params(&p);
    printf("defaults %g %g %d %d\n", p.dt, p.dhat, p.max_newton, p.max_pcg);
    p.n_envs = 0;
    printf("n_envs0 %d\n", (int)zema_create_scene(&p, &s));
    zema_default_params(&p);
    p.pcg_cluster_size = 3;
    printf("schedule3 %d\n", (int)zema_create_scene(&p, &s));
    zema_default_params(&p);
    p.n_envs = 2;
    r = zema_create_scene(&p, &s);
    printf("create %d %d\n", (int)r, s != NULL);
    if (r != ZEMA_OK) return 1;
    r = zema_add_tet_body(s, 1, X, 4, good, 1, NULL, NULL, 1e5, 0.4, 1000.0, 0.5, &id);
    printf("add %d %d\n", (int)r, (int)id);
    r = zema_add_tet_body(s, 0, X, 4, flipped, 1, NULL, NULL, 1e5, 0.4, 1000.0, 0.5, &id);
    printf("inverted %d %d\n", (int)r, zema_last_error(s) != NULL && strlen(zema_last_error(s)) > 0);
    r = zema_add_tet_body(s, 2, X, 4, good, 1, NULL, NULL, 1e5, 0.4, 1000.0, 0.5, &id);
    printf("env2 %d\n", (int)r);
    zema_destroy_scene(s);
    zema_destroy_scene(NULL);
    printf("done\n");
    return 0;
}
"""


def test_c99_client_links_and_drives_the_host_calls(tmp_path):
    lib = zbuild.build()
    src = tmp_path / "client.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", libdir, "-lzema", f"-Wl,-rpath,{libdir}"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("no C compiler")
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split("\n")
    assert out[:8] == ["defaults 0.01 0.001 100 10000", "n_envs0 1", "schedule3 1", "create 0 1", "add 0 0",
                       "inverted 5 1", "env2 1", "done"], out


def _c_layout(tmp_path, struct, fields):
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "zema.h"', "int main(void) {",
             f'    printf("sizeof %zu\\n", sizeof({struct}));']
    for f in fields:
        lines.append(f'    printf("{f} %zu\\n", offsetof({struct}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / f"{struct}.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / struct
    try:
        subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("no C compiler")
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split()
    return {k: int(v) for k, v in zip(out[0::2], out[1::2])}


def test_binding_structures_match_the_c_layout(tmp_path):
    # the ctypes structures of the binding have the C structures' size and
    # every field at the C offset, field by field
    from paper_2311_05945_b300.zema import Params, StepStats
    for struct, cls in (("zema_scene_params", Params), ("zema_step_stats", StepStats)):
        names = [f for f, _ in cls._fields_]
        c = _c_layout(tmp_path, struct, names)
        assert c["sizeof"] == ctypes.sizeof(cls), struct
        for f in names:
            assert c[f] == getattr(cls, f).offset, (struct, f)
