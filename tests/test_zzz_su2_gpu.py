"""GPU parity of the SU(2) path: log N(G) against the oracle's covariance
route, plaquettes, gauge invariance, FP64 Metropolis decisions (immediate
and batched updates) against the oracle's exact chain under the shared
Philox stream, FP32 chains replayed through the oracle, and the observables
computed from the chains' inverses.
"""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import fermionic, mcmc, observables, weight
from tests.gpu_util import ctx_for

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,K", [(1, 1), (2, 2), (3, 3), (4, 2)])
def test_logweight_matches_oracle(L, K):
    p = gi.make_problem(L, gi.SU2, 2, K, bond_scale=0.3)
    links = np.ascontiguousarray(gi.random_links(p, 3, seed=21))
    ctx = ctx_for(p)
    got = ctx.logweight(links)
    W = weight.Weights(p)
    want = np.array([W.log_norm(G) for G in links])
    assert np.abs(got - want).max() <= 1e-10
    pl = ctx.observable(links)
    assert np.abs(pl - observables.plaquette_mean(gi.SU2, L, links)).max() <= 1e-13
    h = gi.random_links(gi.make_problem(L, gi.SU2, 2, 1), 1, seed=3)[0][:p.V]
    hg = np.ascontiguousarray(gi.gauge_transform(p, links, h))
    assert np.abs(ctx.logweight(hg) - got).max() <= 1e-10
    ctx.close()


@pytest.mark.parametrize("delay", [1, 4])
@pytest.mark.parametrize("L,K,nch,nsw", [(2, 1, 3, 6), (2, 2, 2, 4), (3, 1, 2, 3)])
def test_fp64_decisions_match_oracle(L, K, nch, nsw, delay):
    p = gi.make_problem(L, gi.SU2, 2, K, bond_scale=0.3)
    start = gi.random_links(p, nch, seed=9)
    ctx = ctx_for(p)
    ctx.chains_init(np.ascontiguousarray(start), precision=0, refresh_every=8, seed=77, width=1.0, delay=delay)
    obs = ctx.sample(nsw)
    fin = ctx.chains_links()
    st = ctx.chains_stats()
    ctx.close()
    W = weight.Weights(p)
    for c in range(nch):
        lk, ob, _ = mcmc.run_chain(p, W, start[c], 77, c, 0, nsw, width=1.0)
        assert np.array_equal(ob[:, 2], obs[:, c, 2])
        assert np.abs(lk - fin[c]).max() <= 1e-12
        assert np.abs(ob[:, 0] - obs[:, c, 0]).max() <= 1e-12
        assert np.abs(ob[:, 1] - obs[:, c, 1]).max() <= 1e-10
    assert st.proposals == nch * nsw * p.n_links
    assert 0 < st.accepts < st.proposals
    assert st.max_drift < 1e-9


@pytest.mark.parametrize("delay", [1, 8])
def test_fp32_chains_replayed_through_oracle(delay):
    p = gi.make_problem(3, gi.SU2, 2, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(np.ascontiguousarray(gi.cold_links(p, 3)), precision=1, refresh_every=16, seed=5, width=1.0,
                    delay=delay)
    obs = ctx.sample(4)
    fin = ctx.chains_links()
    st = ctx.chains_stats()
    ctx.close()
    W = weight.Weights(p)
    want = np.array([W.log_norm(G) for G in fin])
    assert np.abs(obs[-1, :, 1] - want).max() <= 1e-4
    assert np.abs(np.linalg.norm(fin, axis=-1) - 1.0).max() <= 1e-12
    assert st.max_drift < 1e-3


def test_fermion_bilinears():
    p = gi.make_problem(2, gi.SU2, 2, 2, bond_scale=0.3)
    links = np.ascontiguousarray(gi.random_links(p, 2, seed=4))
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=0)
    site, link = ctx.chains_fermion()
    fe = fermionic.Fermionic(p)
    for c in range(2):
        rs, rl = fe.bilinears(links[c])
        assert np.abs(site[c] - rs).max() <= 1e-10
        assert np.abs(link[c] - rl).max() <= 1e-10
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_casimir_matches_oracle(precision, tol):
    from oracle import electric
    p = gi.make_problem(3, gi.SU2, 2, 2, bond_scale=0.3)
    links = np.ascontiguousarray(gi.random_links(p, 2, seed=12))
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=precision)
    got = ctx.chains_electric()
    el = electric.Electric(p)
    for c in range(2):
        ref = el.f_electric(links[c])
        assert np.abs(got[c] - ref).max() <= tol * max(1.0, np.abs(ref).max())
    ctx.close()


def test_checkpoint_resume_bit_exact(tmp_path):
    p = gi.make_problem(2, gi.SU2, 2, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(np.ascontiguousarray(gi.cold_links(p, 3)), refresh_every=4, seed=3, width=1.0, delay=4)
    ctx.sample(2)
    ck = tmp_path / "su2.ckpt"
    ctx.checkpoint(ck)
    a = ctx.sample(3)
    la = ctx.chains_links()
    ctx.close()
    ctx2 = ctx_for(p)
    ctx2.resume(ck)
    b = ctx2.sample(3)
    lb = ctx2.chains_links()
    ctx2.close()
    assert np.array_equal(la, lb)
    assert np.array_equal(a[:, :, 2], b[:, :, 2])


def test_su2_gradient_on_gpu_matches_oracle_on_the_same_samples():
    """The reweighted gradient along an SU(2)-symmetric site rotation
    (magnetic, Casimir and density terms) from the GPU against the same
    estimator evaluated by the oracle on the same sampled configurations."""
    from paper_2412_01737_gb300 import optimize
    from tests.test_optimize import _OracleCtx
    p = gi.make_problem(2, gi.SU2, 2, 2, bond_scale=0.3)
    sctx = ctx_for(p)
    sctx.chains_init(gi.random_links(p, 32, seed=5), precision=0, seed=4)
    sctx.sample(2)
    links = np.ascontiguousarray(sctx.chains_links())
    sctx.close()
    gens = gi._su2_generators(gi._site_slots_su2(p.n_v))
    A = np.random.default_rng(3).normal(size=(p.m_s, p.m_s))
    X = optimize.commutant_generator(A - A.T, gens)
    dirs = [lambda t: optimize.rotate_sites(p, X, t)]
    kw = dict(c_plaquette=-1.0, c_electric=0.5 * np.ones(p.n_links), c_site=0.4 * np.ones(p.V))
    gctx = ctx_for(p)
    e_gpu, g_gpu = optimize.energy_gradient(gctx, p, links, dirs, **kw)
    gctx.close()
    e_ref, g_ref = optimize.energy_gradient(_OracleCtx(), p, links, dirs, **kw)
    assert abs(g_ref[0]) > 1e-4
    assert abs(e_gpu - e_ref) <= 1e-10 * max(1.0, abs(e_ref))
    assert abs(g_gpu[0] - g_ref[0]) <= 1e-6 * max(1.0, abs(g_ref[0]))
