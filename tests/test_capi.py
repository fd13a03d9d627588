"""CPU-side checks of the C ABI library: it builds, loads, and exports every
symbol that include/ggf.h declares (no compute calls without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_01737_gb300 import build
    path = build.build()
    from paper_2412_01737_gb300 import ggf
    return path, ggf.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "ggf.h")).read()
    return sorted(set(re.findall(r"\b(ggf_[a-z_]+)\s*\(", txt)))


def test_header_symbols_exported(lib):
    path, handle = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ggf_\w+)", out))
    decl = declared_symbols()
    assert decl, "no declarations parsed"
    missing = [s for s in decl if s not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for s in decl:
        assert hasattr(handle, s)


def test_binding_covers_header(lib):
    from paper_2412_01737_gb300 import ggf
    assert sorted(ggf.EXPORTS) == declared_symbols()

