"""The C ABI: header declarations, exported symbols and struct layouts (CPU only; no
compute call is made)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "raptor.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:raptor_status|void|int|const char\*)\s+(raptor_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


def test_library_exports_every_declared_symbol(built):
    names = _declared()
    assert len(names) >= 15
    L = C.CDLL(built.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(built.EXPORTS) | {"raptor_version"}


def test_struct_layout_matches_header(built):
    """Compile a C program against raptor.h with gcc and compare sizes/offsets with the
    ctypes mirrors used by the binding."""
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "raptor.h"
int main(void){
 printf("%zu %zu %zu %zu %zu\n", sizeof(raptor_camera_desc), offsetof(raptor_camera_desc, max_steps),
        offsetof(raptor_camera_desc, r_fp64), offsetof(raptor_camera_desc, t_delay), offsetof(raptor_camera_desc, flags));
 printf("%zu %zu %zu %zu %zu\n", sizeof(raptor_plasma_desc), offsetof(raptor_plasma_desc, fields),
        offsetof(raptor_plasma_desc, n1), offsetof(raptor_plasma_desc, x1_min), offsetof(raptor_plasma_desc, gamma_ad));
 return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    cam = [int(v) for v in out[0].split()]
    pl = [int(v) for v in out[1].split()]
    CD, PD = built.CameraDesc, built.PlasmaDesc
    assert cam == [C.sizeof(CD), CD.max_steps.offset, CD.r_fp64.offset, CD.t_delay.offset, CD.flags.offset]
    assert pl == [C.sizeof(PD), PD.fields.offset, PD.n1.offset, PD.x1_min.offset, PD.gamma_ad.offset]


def test_header_declarations_cite_the_paper():
    txt = open(HEADER).read()
    for key in ["Eqs. 24-28", "Eqs. 7-15", "Eqs. 20-23", "Eqs. 35-36", "Eqs. 41-44", "Eqs. 45-46", "App. A.2", "sec. 5"]:
        assert key in txt, key


def test_product_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1801_10452_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                t = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in t.replace("the oracle", ""), f


def test_binding_fails_loudly_without_library(monkeypatch, built):
    import paper_1801_10452_b300 as R

    monkeypatch.setattr(R, "_lib", None)
    monkeypatch.setattr(R, "LIB_PATH", "/nonexistent/libraptor.so")
    with pytest.raises(RuntimeError):
        R.lib()
