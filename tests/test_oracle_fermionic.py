"""Pins of the fermionic observables of Sec. 5.2 in the oracle.

The covariance route (Gamma_eff = A + B W B^T per pair, Wick's theorem) is
checked against explicit Fock vectors, which are the definition, and against
symmetries that hold whatever the route: Z2 gauge covariance of the link
bilinears, reality of Hermitian bilinears in each configuration, and zero
staggered charge for U(1).
"""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import fermionic, fock


@pytest.mark.parametrize("L,grp,n_v,K", [
    (2, gi.Z2, 1, 1), (2, gi.Z2, 1, 2), (2, gi.U1, 1, 2), (1, gi.Z2, 2, 2), (1, gi.U1, 2, 2),
])
def test_covariance_route_matches_fock(L, grp, n_v, K):
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    fp, fe = fock.FockPEPS(p), fermionic.Fermionic(p)
    for G in gi.random_links(p, 1 if L == 2 else 3, seed=5):
        s0, l0 = fermionic.bilinears_fock(fp, G)
        s1, l1 = fe.bilinears(G)
        assert np.abs(l0).max() > 0.1
        assert np.abs(s1 - s0).max() <= 1e-12
        assert np.abs(l1 - l0).max() <= 1e-12


def test_higher_monomials_match_fock():
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    fp, fe = fock.FockPEPS(p), fermionic.Fermionic(p)
    G = gi.random_links(p, 1, seed=12)[0]
    for idx in [(0, 1, 2, 3), (1, 4, 6, 7), (0, 2, 3, 5, 6, 7), (5, 0, 3, 6)]:
        ref = fermionic.monomial_fock(fp, G, idx)
        assert abs(fe.monomial(G, idx) - ref) <= 1e-12


def test_z2_gauge_covariance_and_hermiticity():
    """psi_s -> h_s psi_s under a Z2 gauge transformation, so the link block
    picks up h_s h_t and the densities are invariant; i c_a c_b (a != b) is
    Hermitian, so i times each bilinear is real in every configuration."""
    p = gi.make_problem(3, gi.Z2, 1, 2, bond_scale=0.3)
    fe = fermionic.Fermionic(p)
    G = gi.random_links(p, 2, seed=3)
    h = np.array([1, -1, 1, 1, -1, -1, 1, 1, -1], dtype=np.int8)
    hG = gi.gauge_transform(p, G, h)
    for a, b in zip(G, hG):
        sa, la = fe.bilinears(a)
        sb, lb = fe.bilinears(b)
        assert np.abs(sa - sb).max() <= 1e-12
        for l in range(p.n_links):
            s, t = fermionic._link_sites(p, l)
            assert np.abs(lb[l] - h[s] * h[t] * la[l]).max() <= 1e-12
        assert np.abs((1j * sa).imag).max() <= 1e-12
        assert np.abs((1j * la).imag).max() <= 1e-12
        n = (1 + 1j * sa).real / 2
        assert n.min() >= -1e-12 and n.max() <= 1 + 1e-12


def test_u1_staggered_charge_is_zero():
    """The site tensors commute with the U(1) charge and the bonds are
    neutral, so every psi(G) carries zero staggered charge:
    sum_s q_s <n_s> = 0 in each configuration."""
    p = gi.make_problem(3, gi.U1, 1, 2, bond_scale=0.3)
    fe = fermionic.Fermionic(p)
    for G in gi.random_links(p, 3, seed=21):
        s, _ = fe.bilinears(G)
        n = (1 + 1j * s).real / 2
        assert n.sum() > 1e-3
        assert abs(np.sum(p.q_phys * n)) <= 1e-12


@pytest.mark.parametrize("L,grp,n_v,K", [
    (2, gi.Z2, 1, 2),
    (2, gi.U1, 1, 2),
    (1, gi.U1, 2, 2),     # self-links: F_s F_t on one site (1 - n_s for q_s > 0)
    (1, gi.Z2, 2, 1),
])
def test_link_terms_match_fock(L, grp, n_v, K):
    """T_l(G) = u_l <F_s F_t> from the link block against explicit psi and
    psi^dag matrices on the Fock vectors."""
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    fp, fe = fock.FockPEPS(p), fermionic.Fermionic(p)
    for G in gi.random_links(p, 2, seed=13):
        ref = fermionic.link_terms_fock(fp, G)
        got = fe.link_terms(G)
        assert np.abs(ref).max() > 1e-3
        assert np.abs(got - ref).max() <= 1e-12


@pytest.mark.parametrize("L,grp", [(2, gi.U1), (3, gi.U1), (2, gi.Z2), (3, gi.Z2)])
def test_link_terms_gauge_invariant(L, grp):
    """T_l(G^h) = T_l(G) for random gauge transformations h, while the
    bilinear with the conjugate link factor, u_l^* F_s F_t, is not invariant
    for U(1) (its phase moves by 2 (alpha_s - alpha_t))."""
    p = gi.make_problem(L, grp, 1, 2, bond_scale=0.3)
    fe = fermionic.Fermionic(p)
    rng = np.random.default_rng(7)
    for G in gi.random_links(p, 2, seed=17):
        h = rng.uniform(0, 2 * np.pi, p.V) if grp == gi.U1 else rng.choice([-1, 1], p.V)
        Gh = gi.gauge_transform(p, G[None], h)[0]
        T, Th = fe.link_terms(G), fe.link_terms(Gh)
        assert np.abs(T).max() > 1e-3
        assert np.abs(Th - T).max() <= 1e-12
        if grp == gi.U1:
            u, uh = np.exp(1j * G), np.exp(1j * Gh)
            wrong, wrongh = T / u ** 2, Th / uh ** 2      # u^* F_s F_t
            assert np.abs(wrongh - wrong).max() > 1e-3


def test_u1_charge_violating_bilinears_vanish():
    """On the 3x3 torus the wrap-around links join equal charges; there
    psi_s psi_t and psi_s^dag psi_t^dag (the combinations that change the
    total charge by 2) vanish in every configuration, while the link term
    (psi_s psi_t^dag for q = +1) does not."""
    p = gi.make_problem(3, gi.U1, 1, 2, bond_scale=0.3)
    fe = fermionic.Fermionic(p)
    same = [l for l in range(p.n_links)
            if p.q_phys[fermionic._link_sites(p, l)[0]] == p.q_phys[fermionic._link_sites(p, l)[1]]]
    assert same
    for G in gi.random_links(p, 2, seed=19):
        _, blk = fe.bilinears(G)
        T = fe.link_terms(G)
        for l in same:
            for e in (1, -1):
                a = np.array([1.0, 1j * e])
                assert abs(0.25 * a @ blk[l] @ a) <= 1e-13
        assert np.abs(T[same]).max() > 1e-3
