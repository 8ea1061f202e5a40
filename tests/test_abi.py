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
