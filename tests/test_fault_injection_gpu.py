"""Fault injection on a GPU: a NaN written into one chain's cached inverse.

Selected only explicitly (``-m gpu_fault``): the run ``-m gpu`` does not
include it, and without CUDA it is skipped.  The bordered-Pfaffian ratio of a
proposal whose W_SS block is not finite is 0, so the chain rejects the links
that read the poisoned element, the call returns normally, the other chains
are unaffected, and a refresh rebuilds the inverse from the links.
"""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import weight

pytestmark = pytest.mark.gpu_fault


def _cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_nan_in_inverse_stalls_one_link_until_refresh():
    if not _cuda():
        pytest.skip("needs a CUDA GPU")
    from tests.gpu_util import ctx_for
    p = gi.make_problem(3, gi.Z2, 1, 1, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.cold_links(p, 4), precision=0, refresh_every=10 ** 9, seed=3)
    # link 0's support: source end of site 0 (+x end) and target end on site 1
    B, h2 = 8 * p.n_v, 2 * p.n_v
    i = 0 * B + 1 * h2          # first Majorana of site 0's +x end
    ctx.debug_poison_inverse(0, 0, i, i + 1)
    obs = ctx.sample(3)
    fin = ctx.chains_links()
    assert fin[0, 0] == 1                                  # link 0 of chain 0 never accepted
    assert np.isfinite(obs[:, 1:, :]).all()                # the other chains are unaffected
    W = ctx.chains_inverse(0, 0, p.N)
    assert not np.isfinite(W).all()
    # a refresh rebuilds W from the links
    ctx2 = ctx_for(p)
    ctx2.chains_init(np.ascontiguousarray(fin), precision=0, refresh_every=1, seed=4)
    ctx2.debug_poison_inverse(0, 0, i, i + 1)
    obs2 = ctx2.sample(2)
    assert np.isfinite(ctx2.chains_inverse(0, 0, p.N)).all()
    lk = ctx2.chains_links()
    assert abs(obs2[-1, 0, 1] - weight.Weights(p).log_norm(lk[0])) <= 1e-8
    ctx.close()
    ctx2.close()
