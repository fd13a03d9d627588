"""Graph-captured sweeps replay exactly what eager launches do, and the
grouped launch of uneven problems (one parent graph per sweep) gives each
problem the same chains as sampling it alone."""
import numpy as np
import pytest

import ggf_inputs as gi
from tests.gpu_util import ctx_for

pytestmark = pytest.mark.gpu


def run(p, graph, precision, delay, refresh, n_chains=3, sweeps=4, seed=17):
    ctx = ctx_for(p)
    ctx.chains_init(gi.cold_links(p, n_chains), precision=precision, refresh_every=refresh, seed=seed,
                    delay=delay, graph=graph)
    obs = ctx.sample(sweeps)
    links = ctx.chains_links()
    st = ctx.chains_stats()
    ctx.close()
    return obs, links, st


@pytest.mark.parametrize("precision,delay", [(0, 1), (0, 4), (1, 8)])
def test_graph_matches_eager(precision, delay):
    p = gi.make_problem(3, gi.U1, 2, 2, bond_scale=0.3)
    a = run(p, 1, precision, delay, refresh=6)
    b = run(p, 0, precision, delay, refresh=6)
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[0], b[0])
    assert a[2].refreshes == b[2].refreshes > 0
    assert a[2].launches == b[2].launches


def test_group_matches_individual():
    from paper_2412_01737_gb300.ggf import sample_group
    probs = [(gi.make_problem(3, gi.Z2, 1, 1), 0, 4, 5),
             (gi.make_problem(4, gi.U1, 2, 2, bond_scale=0.2), 1, 8, 10),
             (gi.make_problem(2, gi.U1, 1, 3, bond_scale=0.3), 0, 1, 7)]
    solo = [run(p, 1, prec, d, r, n_chains=2 + k, sweeps=3, seed=5 + k) for k, (p, prec, d, r) in enumerate(probs)]
    ctxs = []
    for k, (p, prec, d, r) in enumerate(probs):
        c = ctx_for(p)
        c.chains_init(gi.cold_links(p, 2 + k), precision=prec, refresh_every=r, seed=5 + k, delay=d, graph=1)
        ctxs.append(c)
    obs = sample_group(ctxs, 3)
    for k, c in enumerate(ctxs):
        assert np.array_equal(c.chains_links(), solo[k][1])
        assert np.array_equal(obs[k], solo[k][0])
        c.close()
