"""The allocation-free weight entry point (for callers that cannot allocate
device memory when they need log N(G)) agrees with ggf_logweight.

Collected last on purpose: it runs after every other test in a full run and
also passes alone in a fresh process.  Two calls in a row check that the
shared fixed scratch carries nothing from one call into the next."""
import ctypes

import numpy as np
import pytest

import ggf_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,grp,nv,K", [(4, gi.Z2, 1, 1), (3, gi.U1, 2, 3), (8, gi.Z2, 1, 2),
                                        (8, gi.U1, 2, 4)])
def test_noalloc_matches_logweight(L, grp, nv, K):
    """Two calls in a row agree with ggf_logweight at 1e-10; the last case is
    the largest accepted M (N = 1024) with K = 4, whose complex items are
    factored one at a time in the fixed scratch."""
    import torch
    from paper_2412_01737_gb300 import GGF
    from paper_2412_01737_gb300.ggf import load
    p = gi.make_problem(L, grp, nv, K, bond_scale=0.2)
    ctx = GGF(0)
    ctx.init_problem(p)
    lib = load()
    for call, seed in enumerate((1, 2)):
        links = gi.random_links(p, (5 if L < 8 or K < 4 else 2) + call, seed=seed)
        want = ctx.logweight(links)                      # existing entry point, host buffers
        dl = torch.from_numpy(links).cuda()
        out = torch.full((len(links),), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.cuda.current_stream().cuda_stream
        rc = lib.ggf_logweight_noalloc(ctx.h, len(links), ctypes.c_void_p(dl.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st))
        assert rc == 0, lib.ggf_last_error(ctx.h)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-10 * max(1.0, np.abs(want).max())
    ctx.close()


def test_noalloc_rejects_too_large():
    import torch
    from paper_2412_01737_gb300 import GGF, GGFError
    p = gi.make_problem(12, gi.Z2, 1, 1)                 # N = 1152 > 1024
    ctx = GGF(0)
    ctx.init_problem(p)
    dl = torch.from_numpy(gi.random_links(p, 1)).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(GGFError, match="fixed-scratch maximum"):
        ctx.logweight_noalloc(dl, out)
    ctx.close()


def test_noalloc_allocates_nothing():
    """After a first call (which looks up the scratch address), further calls
    leave the device's free memory unchanged."""
    import torch
    from paper_2412_01737_gb300 import GGF
    p = gi.make_problem(6, gi.U1, 2, 2, bond_scale=0.2)
    ctx = GGF(0)
    ctx.init_problem(p)
    dl = torch.from_numpy(gi.random_links(p, 3, seed=4)).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.logweight_noalloc(dl, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        ctx.logweight_noalloc(dl, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ctx.close()
