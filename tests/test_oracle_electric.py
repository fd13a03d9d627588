"""Pins of the electric observables of Sec. 5.3 in the oracle (Z2 link flip,
U(1) Casimir).

The covariance route (Wick's theorem on the composed covariance of one link
end) is checked against explicit Fock-space vectors, which are the
definition (for U(1) the single-link integral itself, by exact quadrature).
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


@pytest.mark.parametrize("L,n_v,K", [(2, 1, 1), (2, 1, 2), (1, 2, 1), (1, 2, 2)])
def test_u1_covariance_route_matches_quadrature(L, n_v, K):
    """U(1): <Q_l^2> from Gamma_O against the single-link integral of
    <G|J^2|g; G> with the overlap, by exact quadrature on explicit vectors."""
    p = gi.make_problem(L, gi.U1, n_v, K, bond_scale=0.3)
    fp, el = fock.FockPEPS(p), electric.Electric(p)
    # on 2x2 an x link and a y link from each sublattice (each needs 8 contractions)
    ls = [0, 3, 5, 6] if L == 2 else list(range(p.n_links))
    for G in gi.random_links(p, 1 if L == 2 else 3, seed=5):
        ref = np.array([electric.f_electric_u1_fock(fp, G, l) for l in ls])
        assert np.abs(ref).max() > 0.1
        assert np.abs(el.f_electric(G)[ls] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_u1_gauge_invariance_and_positive_casimir():
    p = gi.make_problem(2, gi.U1, 1, 2, bond_scale=0.3)
    el = electric.Electric(p)
    G = gi.random_links(p, 2, seed=9)
    alpha = np.array([0.3, -1.1, 2.0, 0.7])
    for a, b in zip(G, gi.gauge_transform(p, G, alpha)):
        fa, fb = el.f_electric(a), el.f_electric(b)
        assert np.abs(fa - fb).max() <= 1e-12 * np.abs(fa).max()
    # <J_l^2> over p(G) on the 1x1 torus: N(G) and N(G) f_E(G) are
    # trigonometric polynomials of degree <= 2 n_v in each angle, so an 8 x 8
    # product grid integrates both exactly
    q = gi.make_problem(1, gi.U1, 1, 2, bond_scale=0.4)
    th = 2 * np.pi * np.arange(8) / 8
    grid = np.array([[a, b] for a in th for b in th])
    x = electric.Electric(q).expectation_exhaustive(grid)
    assert np.abs(x.imag).max() <= 1e-12
    assert x.real.min() >= 0.0 and x.real.max() > 0.01


@pytest.mark.parametrize("K", [1, 2])
def test_su2_casimir_matches_quadrature(K):
    """SU(2): (3/4) <n_0 + n_1 - 2 n_0 n_1> of the source doublet from Gamma_O
    against -sum_a d^2/d eps_a^2 of the overlap under right translations of
    the ket's link, by exact quadrature on explicit vectors (1x1 torus)."""
    p = gi.make_problem(1, gi.SU2, 2, K, bond_scale=0.3)
    fp, el = fock.FockPEPS(p), electric.Electric(p)
    for G in gi.random_links(p, 2, seed=7):
        ref = np.array([electric.f_electric_su2_fock(fp, G, l) for l in range(p.n_links)])
        assert np.abs(ref).max() > 0.1
        assert np.abs(el.f_electric(G) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_su2_casimir_gauge_invariance():
    p = gi.make_problem(2, gi.SU2, 2, 2, bond_scale=0.3)
    el = electric.Electric(p)
    G = gi.random_links(p, 2, seed=9)
    h = gi.random_links(p, 1, seed=10)[0][:p.V]
    for a, b in zip(G, gi.gauge_transform(p, G, h)):
        fa, fb = el.f_electric(a), el.f_electric(b)
        assert np.abs(fa - fb).max() <= 1e-11 * np.abs(fa).max()


@pytest.mark.parametrize("L,n_v,K", [(2, 1, 1), (2, 1, 2), (1, 2, 2)])
def test_u1_field_matches_quadrature(L, n_v, K):
    """<J_l> from Gamma_O against -i d/dtheta' of the overlap (explicit vectors)."""
    p = gi.make_problem(L, gi.U1, n_v, K, bond_scale=0.3)
    fp, el = fock.FockPEPS(p), electric.Electric(p)
    ls = [0, 3, 5, 6] if L == 2 else list(range(p.n_links))
    for G in gi.random_links(p, 1 if L == 2 else 3, seed=5):
        ref = np.array([electric.f_field_u1_fock(fp, G, l) for l in ls])
        assert np.abs(ref).max() > 0.1
        assert np.abs(el.field(G)[ls] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("L,n_v,K", [(2, 1, 2), (3, 1, 2), (3, 2, 2), (1, 2, 1)])
def test_u1_gauss_law_per_configuration(L, n_v, K):
    """Site tensors conserve the total charge and bond pairs are neutral, so in
    every configuration sum_out <J> - sum_in <J> + q_s <n_s> = 0 at each site
    (the field from oracle.electric, the density from oracle.fermionic)."""
    from oracle import fermionic
    p = gi.make_problem(L, gi.U1, n_v, K, bond_scale=0.3)
    el, fe = electric.Electric(p), fermionic.Fermionic(p)
    for G in gi.random_links(p, 3, seed=9):
        J = el.field(G)
        site, _ = fe.bilinears(G)
        n = (1 + 1j * site) / 2
        assert np.abs(J).max() > 0.05
        for s in range(p.V):
            x, y = s % L, s // L
            out_l = [2 * s, 2 * s + 1]
            in_l = [2 * (y * L + (x - 1) % L), 2 * (((y - 1) % L) * L + x) + 1]
            div = sum(J[l] for l in out_l) - sum(J[l] for l in in_l)
            assert abs(div + p.q_phys[s] * n[s]) <= 1e-12
