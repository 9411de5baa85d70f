"""The C-ABI library builds, loads, exports every symbol include/md.h declares,
and rejects bad parameters on the host (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def md():
    from paper_2109_10876_gb300 import build
    build.build()
    from paper_2109_10876_gb300 import md as m
    return m


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(md_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(md):
    names = declared_functions()
    assert "md_create" in names and "md_step" in names and len(names) >= 10
    lib = C.CDLL(md.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_checked_build_exports_the_same_symbols(md):
    """The checked build (-DMD_CHECKED) exports every declared symbol, and
    md_build_flags (no device call) tells the two builds apart."""
    from paper_2109_10876_gb300 import build
    assert os.path.exists(build.LIB_CHECKED)
    checked = C.CDLL(build.LIB_CHECKED)
    for n in declared_functions():
        assert hasattr(checked, n), f"{n} declared in include/ but not exported by the checked build"
    assert checked.md_build_flags() == md.MD_BUILD_CHECKED
    assert C.CDLL(md.LIB_PATH).md_build_flags() == 0


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of `struct` from the C compiler reading include/md.h."""
    inc = os.path.join(ROOT, "include")
    src = tmp_path / "layout.c"
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "md.h"', "int main(void) {",
             f'    printf("%zu\\n", sizeof({struct}));']
    lines += [f'    printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["    return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    return int(out[0]), [int(t) for t in out[1:]]


@pytest.mark.parametrize("name", ["md_params", "md_stats"])
def test_structs_match_the_header_layout(md, name, tmp_path):
    """The ctypes mirrors have the C layout of include/md.h: size and every
    field offset, as the C compiler computes them."""
    st = getattr(md, name)
    fields = [f for f, _ in st._fields_]
    size, offs = _c_layout(name, fields, tmp_path)
    assert C.sizeof(st) == size
    assert [getattr(st, f).offset for f in fields] == offs


def test_box_too_small_and_bad_args_are_rejected_on_host(md):
    with pytest.raises(md.MDError) as e:
        md.md_create(10, [5.0, 5.0, 5.0], skin=0.3)   # 5 < 2 * (2.5 + 0.3)
    assert e.value.status == md.MD_ERR_BOX_TOO_SMALL
    for kw in (dict(dt=0.0), dict(mass=-1.0), dict(skin=-0.1), dict(potential=7), dict(precision=3),
               dict(eps=0.0), dict(sigma=-1.0), dict(list_capacity=-2), dict(langevin_gamma=-1.0)):
        with pytest.raises(md.MDError) as e:
            md.md_create(10, [20.0, 20.0, 20.0], **kw)
        assert e.value.status == md.MD_ERR_ARG, kw
    with pytest.raises(md.MDError) as e:
        md.md_create([5, 5], [[20.0] * 3, [20.0] * 3], bonds=[[2, 7]])   # bond across replicas
    assert e.value.status == md.MD_ERR_ARG
