"""CPU-side checks of the boundary: the library builds, loads and exports every entry point
declared in include/odyssey.h, and the ctypes layouts match the header's structs."""
import os
import re
import subprocess

import pytest

from paper_1601_02063_gb300 import binding as B
from paper_1601_02063_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "odyssey.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(odx_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return cuda_build.build()


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (odx_\w+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    # the binding wraps exactly the declared set
    assert sorted(B.SYMBOLS) == declared


def test_binding_loads_all_symbols(libpath):
    L = B.lib()
    for name in B.SYMBOLS:
        assert hasattr(L, name)
    assert "sm_103a" in B.odx_version()


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "odyssey.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(odx_scene),'
                   ' sizeof(odx_ray_record), sizeof(odx_launch), sizeof(odx_stats),'
                   ' offsetof(odx_scene, rtol_fp32), offsetof(odx_ray_record, g));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    import ctypes as C
    assert vals == [C.sizeof(B.odx_scene), C.sizeof(B.odx_ray_record), C.sizeof(B.odx_launch),
                    C.sizeof(B.odx_stats), B.odx_scene.rtol_fp32.offset,
                    B.odx_ray_record.g.offset]


def test_host_side_torus_norm_matches_oracle(orc):
    """Host-only helper (no device work): the library's Gauss-Legendre normalisation and the
    oracle's Simpson rule agree."""
    for a in (0.94, 0.998):
        assert abs(B.odx_torus_norm(a) - orc.torus_norm(a)) < 1e-10 * orc.torus_norm(a)


def test_error_strings():
    assert B.error_string(B.OK) == "ok"
    assert B.error_string(B.ERR_INVALID_ARG) == "invalid argument"
