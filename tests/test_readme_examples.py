"""The README's examples stay valid: the C example compiles against the
header and links to the library; the Python example parses and uses only
names the package defines."""
import ast
import os
import re
import subprocess

import pytest

from paper_2311_05945_b300 import build as zbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _block(lang):
    text = open(os.path.join(ROOT, "README.md")).read()
    m = re.search(r"```" + lang + r"\n(.*?)```", text, re.S)
    assert m, f"no {lang} example"
    return m.group(1)


def test_readme_c_example_compiles_and_links(tmp_path):
    # the C example of the README stays valid against the header and links
    lib = zbuild.build()
    src = tmp_path / "example.c"
    src.write_text(_block("c"))
    libdir = os.path.dirname(lib)
    try:
        subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(tmp_path / "example"), "-L", libdir,
                        "-lzema", f"-Wl,-rpath,{libdir}"], check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("no C compiler")


def test_readme_python_example_uses_existing_names():
    from paper_2311_05945_b300 import scenes, zema
    tree = ast.parse(_block("python"))
    mods = {"zema": zema, "scenes": scenes}
    handles = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Assign) and isinstance(node.value, ast.Call):
            f = node.value.func
            if isinstance(f, ast.Attribute) and isinstance(f.value, ast.Name) and f.value.id == "zema" \
                    and f.attr == "Scene":
                handles.update(t.id for t in node.targets if isinstance(t, ast.Name))
    assert handles, "the example builds no Scene"
    seen = 0
    for node in ast.walk(tree):
        if isinstance(node, ast.Attribute) and isinstance(node.value, ast.Name):
            if node.value.id in mods:
                assert hasattr(mods[node.value.id], node.attr), node.attr
                seen += 1
            elif node.value.id in handles:
                assert hasattr(zema.Scene, node.attr), node.attr
                seen += 1
    assert seen >= 6
