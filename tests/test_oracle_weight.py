"""Pin the covariance route (oracle.weight) to the brute-force Fock
contraction (oracle.fock) and to the invariants the paper states."""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import fock, weight

CASES = [
    # (L, group, n_v, K, site_mode, bond_mode, bond_scale)
    (2, gi.Z2, 1, 1, "random", "random", 0.3),
    (2, gi.Z2, 1, 2, "random", "random", 0.3),
    (2, gi.U1, 1, 2, "sublattice", "random", 0.3),
    (1, gi.U1, 2, 3, "random", "random", 0.3),
    (1, gi.Z2, 2, 2, "random", "uniform", 0.3),
]


@pytest.mark.parametrize("case", CASES)
def test_covariance_route_equals_fock(case):
    L, grp, nv, K, sm, bm, bs = case
    p = gi.make_problem(L, grp, nv, K, site_mode=sm, bond_mode=bm, bond_scale=bs)
    F, W = fock.FockPEPS(p), weight.Weights(p)
    for links in gi.random_links(p, 3, seed=11):
        Nf = F.n_matrix(links)
        Nw = np.exp(W.log_n_matrix(links))
        assert np.abs(Nf - Nw).max() <= 1e-11 * np.abs(Nf).max()
        assert abs(W.log_norm(links) - np.log(F.norm(links))) < 1e-11


def test_exhaustive_z2_normalisation_and_positivity():
    """Sum over all 256 configs of the 2x2 Z2 lattice: N(G) >= 0 with Im N_nn = 0,
    and the total weight agrees with the Fock route on a sample."""
    p = gi.make_problem(2, gi.Z2, 1, 2)
    W = weight.Weights(p)
    cfgs = gi.all_z2_configs(p)
    logs = np.array([W.log_norm(c) for c in cfgs])
    assert np.all(np.isfinite(logs))
    F = fock.FockPEPS(p)
    for c in cfgs[::37]:
        assert abs(np.exp(W.log_norm(c)) - F.norm(c)) < 1e-11 * F.norm(c)
    for c in cfgs[::51]:
        lnm = W.log_n_matrix(c)
        nm = np.exp(lnm)
        assert np.allclose(nm, nm.conj().T, rtol=1e-12, atol=0)
        assert np.all(np.abs(np.imag(np.diag(nm))) < 1e-12 * np.abs(np.diag(nm)))
    p_g = np.exp(logs - logs.max())
    p_g /= p_g.sum()
    assert abs(p_g.sum() - 1) < 1e-14 and np.all(p_g > 0)


@pytest.mark.parametrize("grp", [gi.Z2, gi.U1])
def test_gauge_invariance(grp):
    """p(G) is invariant under site gauge transformations (Sec. 2.2, Sec. 3.1)."""
    p = gi.make_problem(3, grp, 1, 2)
    W = weight.Weights(p)
    rng = np.random.default_rng(4)
    links = gi.random_links(p, 2, seed=3)
    for _ in range(2):
        h = rng.choice([1, -1], size=p.V) if grp == gi.Z2 else rng.uniform(0, 2 * np.pi, p.V)
        lt = gi.gauge_transform(p, links, h)
        assert not np.allclose(lt, links)
        for a, b in zip(links, lt):
            assert abs(W.log_norm(a) - W.log_norm(b)) < 1e-10


def test_lambda_special_cases():
    p = gi.make_problem(2, gi.U1, 1, 2, bond_scale=0.3)
    W = weight.Weights(p)
    links = gi.random_links(p, 1, seed=2)[0]
    lnm = W.log_n_matrix(links)
    # global phase of lambda leaves N unchanged
    lam = p.lam
    for th in (0.3, 2.0):
        assert abs(weight.combine(lnm, lam * np.exp(1j * th)) - weight.combine(lnm, lam)) < 1e-13
    # lambda = (1, 0) reduces to the single Gaussian
    assert abs(weight.combine(lnm, np.array([1, 0], dtype=complex)) - lnm[0, 0].real) < 1e-13
    # B_2 = B_1 gives N = |lambda_1 + lambda_2|^2 N_11
    q = gi.make_problem(2, gi.U1, 1, 2, distinct_bonds=False)
    Wq = weight.Weights(q)
    lq = Wq.log_n_matrix(links)
    want = np.log(abs(q.lam.sum()) ** 2) + lq[0, 0].real
    assert abs(Wq.log_norm(links) - want) < 1e-11


def test_pure_site_covariance_and_twist_orthogonal():
    p = gi.make_problem(2, gi.U1, 2, 1)
    GA = weight.gamma_A(p)
    assert np.allclose(GA @ GA.T, np.eye(GA.shape[0]), atol=1e-13)
    O = weight.twist_matrix(p, gi.random_links(p, 1)[0])
    assert np.allclose(O @ O.T, np.eye(O.shape[0]), atol=1e-14)
    assert abs(np.linalg.det(O) - 1) < 1e-12


def test_transition_covariance_is_pure():
    """Covariance of |b_n><b_m|/<b_m|b_n> squares to -1 (a rank-one Gaussian operator)."""
    p = gi.make_problem(1, gi.U1, 2, 3, bond_scale=0.4)
    bd = weight.BondData(p)
    r = p.r
    for n in range(3):
        for m in range(3):
            G = bd.G[n, m, 0]
            assert np.allclose(G @ G, -np.eye(r), atol=1e-12)
            assert np.allclose(G, -G.T, atol=1e-13)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("grp,n_v", [(gi.Z2, 1), (gi.U1, 2), (gi.SU2, 2)])
def test_reduced_virtual_matrix_identity(grp, n_v, L):
    """The sampler works on the virtual-mode matrix D + O Gamma_X O^T only.
    For pure site covariances the full-space Pf(Gamma_A(G) + 0 (+) Gamma_X) of
    the covariance route equals its Pfaffian times prod_s sign(Gamma_s[0, 1])
    (the sites' physical blocks), for every pair and configuration, although
    the physical-virtual coupling is non-zero; for a mixed site covariance
    the ratio is not of modulus one."""
    from oracle.pfaffian import log_pfaffian
    p = gi.make_problem(L, grp, n_v, 2, bond_scale=0.3)
    W = weight.Weights(p)
    virt = np.array([i for i in range(p.m_s * p.V) if i % p.m_s >= 2])
    sign = np.prod([np.sign(p.gamma_site[s][0, 1]) for s in range(p.V)])

    def ratio(GA, links, nm):
        O = weight.twist_matrix(p, links)
        la, ph = log_pfaffian(O.T @ GA @ O + W.GX[nm])
        Ov = O[np.ix_(virt, virt)]
        lb, pb = log_pfaffian(GA[np.ix_(virt, virt)] + Ov @ W.GX[nm][np.ix_(virt, virt)] @ Ov.T)
        return np.exp((la + np.log(complex(ph))) - (lb + np.log(complex(pb))))

    for links in gi.random_links(p, 3, seed=3):
        for nm in [(0, 0), (0, 1), (1, 0)]:
            assert abs(ratio(W.GA, links, nm) - sign) <= 1e-12
    if grp != gi.SU2:        # the SU(2) physical singlet does not couple
        assert np.abs(p.gamma_site[0][:2, 2:]).max() > 0.05
    assert abs(abs(ratio(0.8 * W.GA, links, (0, 1))) - 1.0) > 0.1
