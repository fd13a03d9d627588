"""What the trained network adds: trained on configurations of the plain
local sampler, its block proposals are accepted far more often than those of
the untrained network (which the exact MH step otherwise rejects), and every
accepted block move resamples 32 links at once."""
import numpy as np
import pytest

import ggf_inputs as gi
from tests.gpu_util import ctx_for

pytestmark = pytest.mark.gpu


def test_trained_proposal_gains_acceptance():
    import torch
    from paper_2412_01737_gb300 import Net
    p = gi.make_problem(8, gi.U1, 1, 1)
    ctx = ctx_for(p)
    ctx.chains_init(gi.cold_links(p, 64), precision=1, refresh_every=10**9, seed=21, delay=32)
    ctx.sample(30)
    data = []
    for _ in range(20):
        ctx.sample(2)
        data.append(ctx.chains_links())
    data = np.concatenate(data)
    fresh = Net(0, p.L, 1)
    st0 = ctx.chains_stats()
    ctx.sample_blocks(fresh, 10)
    st1 = ctx.chains_stats()
    acc_untrained = (st1.block_accepts - st0.block_accepts) / (st1.block_proposals - st0.block_proposals)
    net = Net(0, p.L, 1)
    losses = net.train(torch.from_numpy(data).cuda(), 64, 400, 2e-3)
    ctx.sample_blocks(net, 10)
    st2 = ctx.chains_stats()
    acc_trained = (st2.block_accepts - st1.block_accepts) / (st2.block_proposals - st1.block_proposals)
    print(f"block acceptance untrained {acc_untrained:.4f} trained {acc_trained:.4f}; "
          f"loss {losses[:10].mean():.2f} -> {losses[-10:].mean():.2f}")
    assert losses[-10:].mean() < losses[:10].mean()
    assert acc_trained > max(2 * acc_untrained, 0.01)
    fresh.close()
    net.close()
    ctx.close()
