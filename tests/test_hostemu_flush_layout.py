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
