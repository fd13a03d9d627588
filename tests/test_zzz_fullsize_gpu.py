"""Parity at the benchmark's full problem size and launch shapes: 16x16 U(1),
n_v = 2 (M 4096 x 4096), K = 4, FP32 chains with batches of 16 links (one
rank-128 tensor-core flush per batch), on 32 chains (the per-chain launch
shapes of the 256-chain benchmark, a tenth of its memory).

The oracle's exact Metropolis is too slow at N = 4096 (minutes per pair
term), so the checks are: the per-sweep plaquettes against the oracle's
plaquettes of the final links, and the tracked FP32 log-weights against the
FP64 log N(G) of the same configurations at an absolute 1e-4.  The FP64 value
comes from ggf_logweight (the site-by-site Pfaffian), which
tests/test_gpu_refresh.py pins to the oracle at this lattice size
(16 x 16, n_v = 2, against values the oracle wrote into tests/golden/) and
per pair at 8 x 8 with K = 4.
"""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle.observables import plaquette_mean
from tests.gpu_util import ctx_for

pytestmark = pytest.mark.gpu


def test_u1_16x16_k4_batched_fp32():
    p = gi.make_problem(16, gi.U1, 2, 4, seed=20241202)
    ctx = ctx_for(p)
    n = 32
    ctx.chains_init(gi.cold_links(p, n), precision=1, refresh_every=1 << 30, seed=20241202, delay=16)
    obs = ctx.sample(2)
    fin = ctx.chains_links()
    st = ctx.chains_stats()
    assert np.isfinite(obs).all()
    assert np.abs(obs[-1, :, 0] - plaquette_mean(gi.U1, 16, fin)).max() <= 1e-12
    assert 0 < st.accepts < st.proposals
    fresh = ctx.logweight(np.ascontiguousarray(fin))
    tracked = obs[-1, :, 1]
    assert np.abs(tracked - fresh).max() <= 1e-4
    ctx.close()


def test_u1_16x16_fermion_properties_fp32():
    """At the benchmark's lattice and n_v, properties that hold in every
    configuration whatever the size: the Majorana bilinears of a Hermitian
    state are imaginary (i <c_a c_b> real), the densities lie in [0, 1], and
    the staggered charge sum_s q_s <n_s> vanishes (charge-conserving site
    tensors, neutral bond pairs)."""
    p = gi.make_problem(16, gi.U1, 2, 2, seed=20241202, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 4, seed=5), precision=1, refresh_every=1 << 30, seed=3, delay=16)
    ctx.sample(1)
    site, link = ctx.chains_fermion()
    n = (1 + 1j * site) / 2
    assert np.abs(site.real).max() <= 1e-4
    assert np.abs(link.real).max() <= 1e-4
    assert n.real.min() >= -1e-4 and n.real.max() <= 1 + 1e-4
    assert np.abs(n @ p.q_phys).max() <= 1e-3
    ctx.close()


@pytest.mark.parametrize("K", [1, 2])
def test_z2_16x16_batched_fp32(K):
    """16x16 Z2, n_v = 1 (M 2048 x 2048), the largest Z2 cell of the uneven
    batch: FP32 chains with batches of 16 links, from the cold start.

    Without a refresh, every accepted flip adds the FP32 error of the cached
    inverse to the tracked log-weight; a Z2 flip is a large change (a sign, not
    a small angle), so over three sweeps (~1.4e3 accepts per chain) the
    tracked value drifts by ~1.5e-6 per accept.  The test bounds that at
    3e-6 per accept.  With a refresh every 32 accepts each chain is refreshed
    at the end of every sweep (the fresh FP64 log-weight resets the tracked
    one, the Newton step refines the inverse), so the drift, both at the
    refreshes and at the last sweep, is that of one sweep's accepts only:
    the refresh does not let the error accumulate."""
    p = gi.make_problem(16, gi.Z2, 1, K, seed=20241202 + K)
    n = 8
    for refresh in (1 << 30, 32):
        ctx = ctx_for(p)
        ctx.chains_init(gi.cold_links(p, n), precision=1, refresh_every=refresh, seed=77 + K, delay=16)
        obs = ctx.sample(3)
        fin = ctx.chains_links()
        st = ctx.chains_stats()
        assert np.isfinite(obs).all()
        assert np.abs(obs[-1, :, 0] - plaquette_mean(gi.Z2, 16, fin)).max() <= 1e-12
        assert 0 < st.accepts < st.proposals
        fresh = ctx.logweight(np.ascontiguousarray(fin))
        err = np.abs(obs[-1, :, 1] - fresh).max()
        per_chain = st.accepts / n
        if refresh > st.accepts:
            assert st.refreshes == 0
            assert err <= 3e-6 * per_chain, (err, per_chain)
        else:
            assert st.refreshes == 3 * n
            assert err <= 1.5 * 3e-6 * per_chain / 3, (err, per_chain)
            assert st.max_drift <= 1.5 * 3e-6 * per_chain / 3, (st.max_drift, per_chain)
        ctx.close()
