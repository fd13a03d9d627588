"""The tensor-core flush's producer index arithmetic (csrc/ggf_flush_layout.cuh),
built for the host by tests/hostemu/emu_flush_layout.cu -- on CPU.

Each producer thread copies 16-byte pieces of the operand planes of a stage
(copy slot idx = thread + t * 256) and writes their tf32 hi/lo splits into
the no-swizzle K-major core-matrix layout that the MMA descriptors read.  The
checks: the slots of a 128- or 256-row plane cover every (row, 4-column group)
exactly once; the 16-byte shared stores of each 8-thread phase of a warp hit
32 distinct banks; a warp's global reads of the chunk-major panel fall on four
128-byte lines.
"""
import ctypes
import os
import shutil
import subprocess
from collections import Counter

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
PGROUP = 256          # producer threads


@pytest.fixture(scope="module")
def lay(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("emu") / "libflushlayout.so")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-gencode",
                    "arch=compute_103a,code=sm_103a", "-o", out,
                    os.path.join(HERE, "hostemu", "emu_flush_layout.cu")], check=True, capture_output=True)
    return ctypes.CDLL(out)


def _layout(lay, n, NP=4096):
    row = np.zeros(n, dtype=np.int32)
    kq = np.zeros(n, dtype=np.int32)
    off = np.zeros(n, dtype=np.uint32)
    pan = np.zeros(n, dtype=np.uint64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    lay.emu_flush_layout(ctypes.c_int(n), ctypes.c_int(NP), p(row), p(kq), p(off), p(pan))
    return row, kq, off, pan


@pytest.mark.parametrize("NR", [128, 256])
def test_slots_cover_the_plane_once(lay, NR):
    row, kq, off, _ = _layout(lay, 2 * NR)
    assert set(zip(row.tolist(), kq.tolist())) == {(r, k) for r in range(NR) for k in (0, 4)}
    assert len(set(off.tolist())) == 2 * NR
    assert off.max() + 16 <= NR * 8 * 4          # inside the plane (NR rows x 8 tf32)


@pytest.mark.parametrize("NR", [128, 256])
def test_split_stores_are_conflict_free(lay, NR):
    _, _, off, _ = _layout(lay, 2 * NR)
    for w0 in range(0, 2 * NR, 32):
        for ph in range(4):
            banks = Counter()
            for a in off[w0 + 8 * ph: w0 + 8 * ph + 8]:
                for i in range(4):
                    banks[(int(a) // 4 + i) % 32] += 1
            assert max(banks.values()) == 1, (w0, ph)


@pytest.mark.parametrize("NR", [128, 256])
def test_panel_reads_are_coalesced(lay, NR):
    _, _, _, pan = _layout(lay, 2 * NR)
    for w0 in range(0, 2 * NR, 32):
        byte = pan[w0:w0 + 32].astype(np.int64) * 4
        assert len({int(b) // 128 for b in byte}) == 4
        assert len(set(byte.tolist())) == 32


# ---- pre-split operand blocks (flush in chain waves) -------------------------

def _cm(row, k):
    """Core-matrix byte offset of (row, k) in a KC = 8 wide plane: 8-row x
    16-byte core matrices, 128 bytes apart along k, 256 bytes between 8-row
    groups (the layout the MMA descriptors of the flush read)."""
    return (row // 8) * 256 + (k // 4) * 128 + (row % 8) * 16 + (k % 4) * 4


@pytest.mark.parametrize("cplx,N,KRM,pairs,n", [(0, 300, 12, 2, 3), (1, 300, 12, 3, 2), (0, 512, 16, 1, 1),
                                                (1, 128, 8, 1, 2)])
def test_presplit_blocks_tile_the_scratch(lay, cplx, N, KRM, pairs, n):
    """Every 16-byte hi/lo piece the split pass writes has its own place, all
    inside the scratch, and together they fill it: the two bulk copies of a
    stage then read only bytes the split pass wrote."""
    NP = (N + 255) // 256 * 256
    KP = (KRM + 7) // 8 * 8
    cap = n * pairs * 2 * (2 if cplx else 1) * NP * (KP // 4)
    rec = np.zeros((cap, 10), dtype=np.uint64)
    m = lay.emu_ps_layout(ctypes.c_int(cplx), ctypes.c_int(N), ctypes.c_int(KRM), ctypes.c_int(pairs),
                          ctypes.c_int(n), rec.ctypes.data_as(ctypes.c_void_p), ctypes.c_longlong(cap))
    assert m == cap
    lay.emu_ps_bytes.restype = ctypes.c_ulonglong
    total = lay.emu_ps_bytes(ctypes.c_int(cplx), ctypes.c_int(N), ctypes.c_int(KRM), ctypes.c_int(pairs),
                             ctypes.c_int(n))
    none = np.uint64(2**64 - 1)
    offs = np.concatenate([rec[:, 6], rec[:, 7], rec[:, 8][rec[:, 8] != none], rec[:, 9][rec[:, 9] != none]])
    assert np.all(offs % 16 == 0)
    assert len(np.unique(offs)) == len(offs)
    assert offs.max() + 16 <= total and len(offs) * 16 == total


@pytest.mark.parametrize("cplx", [0, 1])
def test_presplit_blocks_hold_the_stage_layout(lay, cplx):
    """Inside each block the pieces sit where the per-tile producers of the
    other flush kernel put them in a stage: V (A operand) hi/lo planes of 128
    rows, then the U (B operand) hi and lo parts -- 256 rows for real pairs,
    the composite [-U_i ; U_r ; U_i] for complex pairs."""
    N, KRM, pairs, n = 300, 12, 2, 2
    NP = 512
    KP = 16
    cap = n * pairs * 2 * (2 if cplx else 1) * NP * (KP // 4)
    rec = np.zeros((cap, 10), dtype=np.uint64)
    lay.emu_ps_layout(ctypes.c_int(cplx), ctypes.c_int(N), ctypes.c_int(KRM), ctypes.c_int(pairs), ctypes.c_int(n),
                      rec.ctypes.data_as(ctypes.c_void_p), ctypes.c_longlong(cap))
    lay.emu_ps_off.restype = ctypes.c_ulonglong
    plane = 128 * 8 * 4
    for c, p, uv, pl, row, k, hi, lo, hi2, lo2 in rec.astype(object):
        ur = 128 if (uv == 0 or cplx) else 256
        blk = lay.emu_ps_off(ctypes.c_int(cplx), ctypes.c_int(N), ctypes.c_int(KRM), ctypes.c_int(pairs),
                             ctypes.c_int(n), ctypes.c_int(uv), ctypes.c_int(c), ctypes.c_int(p),
                             ctypes.c_int(row // ur), ctypes.c_int(k // 8))
        r, kk = row % ur, k % 8
        if uv == 0:
            assert hi - blk == 2 * pl * plane + _cm(r, kk) and lo == hi + plane
        elif not cplx:
            assert hi - blk == _cm(r, kk) and lo == hi + 2 * plane
        else:
            assert hi - blk == _cm((128 if pl == 0 else 256) + r, kk) and lo == hi + 3 * plane
            if pl == 1:
                assert hi2 - blk == _cm(r, kk) and lo2 == hi2 + 3 * plane
