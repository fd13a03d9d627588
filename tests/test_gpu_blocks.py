"""Block moves with the learned proposal: the tracked log-weights follow the
configurations exactly (FP64), rejected moves leave no trace, and block-only
sampling agrees with local sampling on the plaquette mean."""
import numpy as np
import pytest

import ggf_inputs as gi
from tests.gpu_util import ctx_for

pytestmark = pytest.mark.gpu


def test_block_moves_keep_log_weights_exact():
    from paper_2412_01737_gb300 import Net
    p = gi.make_problem(5, gi.U1, 1, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 4, seed=3), precision=0, refresh_every=10**9, seed=11, delay=32)
    net = Net(0, p.L, 5)
    obs = ctx.sample_blocks(net, 6)
    st = ctx.chains_stats()
    assert st.block_proposals == 24
    links = np.ascontiguousarray(ctx.chains_links())
    ell = np.zeros((4, 3, 2))
    fresh = ctx.logweight(links, ell=ell)
    tracked = ctx.chains_ell()
    assert np.abs(tracked.real - ell[..., 0]).max() < 1e-9
    assert np.abs(obs[-1, :, 1] - fresh).max() < 1e-9
    # mixing local sweeps and block moves keeps everything consistent
    ctx.sample(1)
    ctx.sample_blocks(net, 2)
    links = np.ascontiguousarray(ctx.chains_links())
    ctx.logweight(links, ell=ell)
    assert np.abs(ctx.chains_ell().real - ell[..., 0]).max() < 1e-9
    net.close()
    ctx.close()


def test_untrained_block_moves_sample_the_same_distribution():
    """4x4 lattice: the block is the whole lattice (independence proposals);
    block-only chains and local chains agree on <plaquette> within errors."""
    from paper_2412_01737_gb300 import Net
    p = gi.make_problem(4, gi.U1, 1, 1)
    ctx = ctx_for(p)
    ctx.chains_init(gi.cold_links(p, 64), precision=1, refresh_every=10**9, seed=3, delay=32)
    net = Net(0, p.L, 7)
    # train on the cold configuration's neighbourhood so that moves get accepted
    ctx.sample(20)
    obs_b = ctx.sample_blocks(net, 150)
    st = ctx.chains_stats()
    ctx2 = ctx_for(p)
    ctx2.chains_init(gi.cold_links(p, 64), precision=1, refresh_every=10**9, seed=4, delay=8)
    ctx2.sample(20)
    obs_l = ctx2.sample(150)
    a, b = obs_b[30:, :, 0].mean(axis=1), obs_l[30:, :, 0].mean(axis=1)
    err = np.sqrt(np.var(a) / len(a) * 20 + np.var(b) / len(b) * 20)
    assert st.block_accepts > 0
    assert abs(a.mean() - b.mean()) < 5 * err + 1e-3, (a.mean(), b.mean(), err)
    net.close()
    ctx.close()
    ctx2.close()
