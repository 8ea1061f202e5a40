"""Host-side checks: the C-ABI library builds, loads and exports every entry
point declared in include/lqr.h; host-side argument validation and the
segment partition need no GPU."""
import ctypes
import os
import re

import pytest

from paper_1809_06360_gb300 import build as pbuild
from paper_1809_06360_gb300 import lqr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return lqr.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(lqr_[a-z0-9_]+)\s*\(", src, re.M))
    return names


def test_header_declares_the_binding_exports():
    assert _declared() == set(lqr.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(10):
        assert lqr.lqr_status_string(code)


def test_partition_host_logic(lib):
    assert lqr.lqr_partition(12, 4, 128, 8) == [16 * j for j in range(9)]
    b = lqr.lqr_partition(3, 1, 10, 3)
    assert b == [0, 3, 6, 10]
    # segments shorter than ceil(n/m) cannot reach an arbitrary end state
    with pytest.raises(lqr.LqrError) as e:
        lqr.lqr_partition(12, 4, 128, 64)
    assert e.value.status == 3
    with pytest.raises(lqr.LqrError):
        lqr.lqr_partition(12, 4, 128, 0)
    with pytest.raises(lqr.LqrError):
        lqr.lqr_partition(12, 4, 8, 9)


STRUCTS = ["lqr_problem", "lqr_solution", "lqr_opts", "lqr_report_t", "lqr_nl_model", "lqr_sqp_opts",
           "lqr_sqp_report"]


def test_binding_structs_match_header_layout(tmp_path):
    """Every struct the binding passes across the C ABI has, in ctypes, the size
    and field offsets that a C compiler gives the declaration in include/lqr.h
    (gcc on a small program that prints sizeof and offsetof): a field added on
    one side only would shift every later field."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lqr.h"', "int main(void) {"]
    for st in STRUCTS:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (st, st))
        for name, _ in getattr(lqr, st)._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (st, name, st, name))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        st, field, value = line.split()
        got[(st, field)] = int(value)
    for st in STRUCTS:
        cls = getattr(lqr, st)
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for name, _ in cls._fields_:
            assert got[(st, name)] == getattr(cls, name).offset, (st, name)
