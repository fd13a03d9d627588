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
    return sorted(set(re.findall(r"\b(ggf_[a-z0-9_]+)\s*\(", txt)))


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



def header_defines():
    txt = open(os.path.join(ROOT, "include", "ggf.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define (GGF_[A-Z0-9_]+) (-?\d+)", txt)}
    enum = {k: int(v) for k, v in re.findall(r"\b(GGF_[A-Z]+)\s*=\s*(\d+)", txt)}
    return defs, enum


def test_binding_constants_match_header():
    from paper_2412_01737_gb300 import ggf
    defs, enum = header_defines()
    pairs = {"GGF_Z2": ggf.Z2, "GGF_U1": ggf.U1, "GGF_SU2": ggf.SU2, "GGF_FP64": ggf.FP64, "GGF_FP32": ggf.FP32,
             "GGF_MEM_DEVICE": ggf.MEM_DEVICE, "GGF_MEM_HOST": ggf.MEM_HOST, "GGF_N_OBS": ggf.N_OBS,
             "GGF_OBS_PLAQUETTE": ggf.OBS_PLAQUETTE, "GGF_KT_RATIO": ggf.KT_RATIO,
             "GGF_KT_UPDATE": ggf.KT_UPDATE, "GGF_KT_REFRESH": ggf.KT_REFRESH, "GGF_KT_FLUSH": ggf.KT_FLUSH,
             "GGF_KT_GATHER": ggf.KT_GATHER, "GGF_KT_APPLY": ggf.KT_APPLY, "GGF_NET_PARAMS": ggf.NET_PARAMS,
             "GGF_PAIRS_NORM": ggf.PAIRS_NORM, "GGF_PAIRS_ELECTRIC": ggf.PAIRS_ELECTRIC,
             "GGF_PAIRS_SITE": ggf.PAIRS_SITE, "GGF_PAIRS_LINK": ggf.PAIRS_LINK,
             "GGF_PAIRS_FIELD": ggf.PAIRS_FIELD, "GGF_PAIRS_FOUR": ggf.PAIRS_FOUR}
    for name, val in pairs.items():
        assert defs[name] == val, name
    assert len(enum) == len(ggf.STATUS)
    for name, val in enum.items():
        assert ggf.STATUS[val] == name
