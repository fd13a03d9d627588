"""Pins of the Z2 electric (link-flip) observable of Sec. 5.3 in the oracle.

The covariance route (a Pfaffian of the composed covariance on one link end)
is checked against explicit Fock-space vectors, which are the definition.
"""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import electric, fock


def _fock_f(fp, G):
    """f_E(G) for every link from explicit vectors."""
    lam = fp.p.lam
    v = (lam[:, None] * fp.psi(G)).sum(axis=0)
    nv = np.vdot(v, v)
    out = []
    for l in range(fp.p.n_links):
        w = (lam[:, None] * fp.psi(electric.flipped(G, l))).sum(axis=0)
        out.append(np.vdot(v, w) / nv)
    return np.array(out)


@pytest.mark.parametrize("K,seed", [(1, 4), (2, 5)])
def test_covariance_route_matches_fock_2x2(K, seed):
    p = gi.make_problem(2, gi.Z2, 1, K, bond_scale=0.3)
    G = gi.random_links(p, 1, seed=seed)[0]
    ref = _fock_f(fock.FockPEPS(p), G)
    cov = electric.Electric(p).f_electric(G)
    assert np.abs(ref).max() > 0.1
    assert np.abs(cov - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("K", [1, 2])
def test_covariance_route_matches_fock_two_modes_per_end(K):
    """n_v = 2 (four Majoranas per link end, (-1)^{n_v} = +1) on the 1x1
    torus, every configuration."""
    p = gi.make_problem(1, gi.Z2, 2, K, bond_scale=0.4)
    fp, el = fock.FockPEPS(p), electric.Electric(p)
    for G in gi.all_z2_configs(p):
        ref = _fock_f(fp, G)
        assert np.abs(el.f_electric(G) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("K", [1, 2, 3])
def test_exhaustive_expectation_matches_fock_1x1(K):
    """<X_l> = sum_G <psi(G)|psi(G^(l))> / sum_G <psi(G)|psi(G)> on the 1x1
    torus (two self-links, four configurations), against explicit vectors."""
    p = gi.make_problem(1, gi.Z2, 1, K, bond_scale=0.4)
    fp = fock.FockPEPS(p)
    cfgs = gi.all_z2_configs(p)
    vec = {tuple(G): (p.lam[:, None] * fp.psi(G)).sum(axis=0) for G in cfgs}
    num = np.zeros(p.n_links, dtype=complex)
    den = 0.0
    for G in cfgs:
        v = vec[tuple(G)]
        den += np.vdot(v, v).real
        for l in range(p.n_links):
            num[l] += np.vdot(v, vec[tuple(electric.flipped(G, l).astype(np.int8))])
    ref = num / den
    got = electric.Electric(p).expectation_exhaustive(cfgs)
    assert np.abs(got - ref).max() <= 1e-12
    assert np.abs(ref.imag).max() <= 1e-14


def test_gauge_invariance_and_bounds_2x2():
    """f_E is gauge invariant (the flip commutes with Z2 gauge transformations);
    the exhaustive expectation of the Hermitian flip is real and at most 1."""
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    el = electric.Electric(p)
    G = gi.random_links(p, 2, seed=9)
    h = np.array([1, -1, -1, 1], dtype=np.int8)
    hG = gi.gauge_transform(p, G, h)
    for a, b in zip(G, hG):
        fa, fb = el.f_electric(a), el.f_electric(b)
        assert np.abs(fa - fb).max() <= 1e-12 * np.abs(fa).max()
    x = el.expectation_exhaustive(gi.all_z2_configs(p))
    assert np.abs(x.imag).max() <= 1e-12
    assert np.abs(x.real).max() <= 1.0
    assert np.abs(x.real).max() > 0.05


def test_u1_rejected():
    p = gi.make_problem(2, gi.U1, 1, 1)
    with pytest.raises(ValueError):
        electric.Electric(p)
