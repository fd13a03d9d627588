"""Pins of the lambda optimisation in the oracle (oracle/variational.py).

On the 2x2 Z2 lattice everything is exhaustive: the Hermitian forms built
from summed local matrices must reproduce the direct expectations computed
with any other lambda; the generalised eigenvector must minimise the energy;
and independent samples of p_lambda0 must estimate the same energy.
"""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import electric, fermionic, variational as va, weight
from oracle.observables import plaquette_values


@pytest.fixture(scope="module")
def setup():
    p = gi.make_problem(2, gi.Z2, 1, 3, bond_scale=0.3)
    cfgs = gi.all_z2_configs(p)
    return p, cfgs, va.exhaustive(p, cfgs)


def test_forms_reproduce_direct_expectations(setup):
    p, cfgs, S = setup
    rng = np.random.default_rng(1)
    pl = plaquette_values(gi.Z2, 2, cfgs).mean(axis=1)
    for _ in range(2):
        z = rng.normal(size=p.K) + 1j * rng.normal(size=p.K)
        lam = z / np.linalg.norm(z)
        q = va.with_lambda(p, lam)
        W = weight.Weights(q)
        logs = np.array([W.log_norm(G) for G in cfgs])
        w = np.exp(logs - logs.max())
        w /= w.sum()
        assert abs(va.expectation(S["plaquette"], S["norm"], lam) - np.sum(w * pl)) <= 1e-13
        ref_el = electric.Electric(q).expectation_exhaustive(cfgs)
        assert np.abs(va.expectation(S["electric"], S["norm"], lam) - ref_el).max() <= 1e-13
        fe = fermionic.Fermionic(q)
        ref_d = sum(wi * fe.bilinears(G)[0] for wi, G in zip(w, cfgs))
        assert np.abs(va.expectation(S["density"], S["norm"], lam) - ref_d).max() <= 1e-13
        four = lambda G: np.array([fe.monomial(G, [2 * (l // 2), 2 * (l // 2) + 1,
                                                   2 * fermionic._link_sites(q, l)[1],
                                                   2 * fermionic._link_sites(q, l)[1] + 1])
                                   for l in range(q.n_links)])
        ref_f = sum(wi * four(G) for wi, G in zip(w, cfgs))
        assert np.abs(va.expectation(S["four"], S["norm"], lam) - ref_f).max() <= 1e-13
        ref_t = sum(wi * fe.link_terms(G) for wi, G in zip(w, cfgs))
        assert np.abs(ref_t).max() > 1e-3
        assert np.abs(va.expectation(S["hopping"], S["norm"], lam) - ref_t).max() <= 1e-13
        hop = S["hopping"] + np.conj(np.swapaxes(S["hopping"], 1, 2))      # T + T^dag
        assert np.abs(va.expectation(hop, S["norm"], lam) - 2 * ref_t.real).max() <= 1e-13


def test_linear_method_minimises_the_energy(setup):
    p, cfgs, S = setup
    assert np.abs(S["norm"] - S["norm"].conj().T).max() <= 1e-14
    assert np.linalg.eigvalsh(S["norm"]).min() > 0
    H = -1.0 * S["plaquette"] + 0.5 * S["electric"].sum(axis=0)
    assert np.abs(H - H.conj().T).max() <= 1e-12          # Hermitian once summed over G
    E0, lam0 = va.linear_method(H, S["norm"])
    assert abs(va.expectation(H, S["norm"], lam0) - E0) <= 1e-12
    rng = np.random.default_rng(2)
    for _ in range(200):
        z = rng.normal(size=p.K) + 1j * rng.normal(size=p.K)
        assert va.expectation(H, S["norm"], z).real >= E0 - 1e-12
    # the sampling weights of the problem are not the optimum
    assert va.expectation(H, S["norm"], p.lam).real > E0 + 1e-3
    # a lattice-gauge energy with every term: magnetic, electric, staggered
    # mass (n_s = (1 + i c_2s c_2s+1) / 2; the bilinear itself is
    # anti-Hermitian) and hopping (T + T^dag)
    hop = S["hopping"].sum(axis=0)
    H2 = (-1.0 * S["plaquette"] + 0.5 * S["electric"].sum(axis=0)
          + 0.4 * np.einsum("s,snm->nm", p.q_phys.astype(float), 0.5 * (S["norm"] + 1j * S["density"]))
          + 0.3 * (hop + hop.conj().T))
    assert np.abs(H2 - H2.conj().T).max() <= 1e-12
    E2, lam2 = va.linear_method(H2, S["norm"])
    for _ in range(200):
        z = rng.normal(size=p.K) + 1j * rng.normal(size=p.K)
        assert va.expectation(H2, S["norm"], z).real >= E2 - 1e-12


def test_sampled_matrices_estimate_the_energy(setup):
    """Independent samples of p_lambda0 (drawn from the exhaustive
    distribution) estimate Hbar and Nbar, hence E(lambda), within errors."""
    p, cfgs, S = setup
    W = weight.Weights(p)
    logs = np.array([W.log_norm(G) for G in cfgs])
    w = np.exp(logs - logs.max())
    w /= w.sum()
    rng = np.random.default_rng(3)
    idx = rng.choice(len(cfgs), size=4000, p=w)
    lm = va.LocalMatrices(p)
    cache = {}
    Hs, Ns = [], []
    for i in idx:
        if i not in cache:
            loc = lm(cfgs[i])
            cache[i] = (-1.0 * loc["plaquette"] + 0.5 * loc["electric"].sum(axis=0), loc["norm"])
        Hs.append(cache[i][0])
        Ns.append(cache[i][1])
    Hs, Ns = np.array(Hs), np.array(Ns)
    H = -1.0 * S["plaquette"] + 0.5 * S["electric"].sum(axis=0)
    _, lam0 = va.linear_method(H, S["norm"])
    e_loc = np.einsum("n,inm,m->i", np.conj(lam0), Hs, lam0)
    n_loc = np.einsum("n,inm,m->i", np.conj(lam0), Ns, lam0)
    est = e_loc.mean() / n_loc.mean()
    # delta-method error of a ratio of means
    r = (e_loc - est * n_loc) / n_loc.mean()
    err = np.sqrt(np.mean(np.abs(r) ** 2) / len(idx))
    assert abs(est - va.expectation(H, S["norm"], lam0)) <= 5 * err


@pytest.mark.parametrize("grp,n_v,K", [(gi.Z2, 1, 2), (gi.U1, 1, 2), (gi.U1, 2, 1), (gi.SU2, 2, 2)])
def test_site_score_matches_finite_differences(grp, n_v, K):
    """d log N(G) along a rotation of one sublattice's site states by a
    generator of their commutant equals sum_s tr(S_s^T dD_s)."""
    import dataclasses
    import scipy.linalg
    p = gi.make_problem(2, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 1, seed=5)[0]
    S = va.score_sites(p, links)
    rng = np.random.default_rng(1)
    A = rng.normal(size=(p.m_s, p.m_s))
    A = A - A.T
    if grp == gi.U1:
        A = gi._project_commutant(A, gi.site_charges(p.n_v, +1))
    elif grp == gi.SU2:
        A = gi._project_commutant_su2(A, gi._su2_generators(gi._site_slots_su2(p.n_v)))

    def log_n(eps):
        O = scipy.linalg.expm(eps * A)
        gs = p.gamma_site.copy()
        for s in range(p.V):
            if p.q_phys[s] == 1:
                gs[s] = O @ gs[s] @ O.T
        return weight.Weights(dataclasses.replace(p, gamma_site=gs)).log_norm(links)

    h = 1e-5
    fd = (log_n(h) - log_n(-h)) / (2 * h)
    an = sum(np.sum(S[s] * (A @ p.gamma_site[s] - p.gamma_site[s] @ A)[2:, 2:])
             for s in range(p.V) if p.q_phys[s] == 1)
    assert abs(an) > 1e-3
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


def test_wilson_energy_gradient_is_a_covariance_with_the_score():
    """d<W>/d theta = E_p[(W(G) - <W>) sum_s tr(S_s^T dD_s/d theta)] for a
    rotation theta of one sublattice's site states (exhaustive 2x2 Z2)."""
    import dataclasses
    import scipy.linalg
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    cfgs = gi.all_z2_configs(p)
    pl = plaquette_values(gi.Z2, 2, cfgs).mean(axis=1)
    rng = np.random.default_rng(6)
    A = rng.normal(size=(p.m_s, p.m_s))
    A = A - A.T

    def mean_w(eps):
        O = scipy.linalg.expm(eps * A)
        gs = p.gamma_site.copy()
        for s in range(p.V):
            if p.q_phys[s] == 1:
                gs[s] = O @ gs[s] @ O.T
        W = weight.Weights(dataclasses.replace(p, gamma_site=gs))
        logs = np.array([W.log_norm(G) for G in cfgs])
        w = np.exp(logs - logs.max())
        return np.sum(w * pl) / w.sum()

    h = 1e-5
    fd = (mean_w(h) - mean_w(-h)) / (2 * h)
    W = weight.Weights(p)
    logs = np.array([W.log_norm(G) for G in cfgs])
    w = np.exp(logs - logs.max())
    w /= w.sum()
    dD = {s: (A @ p.gamma_site[s] - p.gamma_site[s] @ A)[2:, 2:] for s in range(p.V) if p.q_phys[s] == 1}
    dlog = np.array([sum(np.sum(S[s] * dD[s]) for s in dD) for S in (va.score_sites(p, G) for G in cfgs)])
    mw = np.sum(w * pl)
    an = np.sum(w * (pl - mw) * dlog)
    assert abs(an) > 1e-3
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


@pytest.mark.parametrize("grp,n_v", [(gi.Z2, 1), (gi.U1, 1), (gi.U1, 2), (gi.SU2, 2)])
def test_link_score_matches_finite_differences_k1(grp, n_v):
    """K = 1: d log N(G) along a rotation of every link's bond state by a
    generator of the bond commutant equals Re sum_l tr(U[l]^T dGamma_B[l])."""
    import dataclasses
    import scipy.linalg
    p = gi.make_problem(2, grp, n_v, 1, bond_scale=0.3)
    links = gi.random_links(p, 1, seed=5)[0]
    U = va.score_links(p, links)[0]
    rng = np.random.default_rng(2)
    A = rng.normal(size=(p.r, p.r))
    A = A - A.T
    if grp == gi.U1:
        A = gi._project_commutant(A, np.concatenate([p.q_src, -p.q_src]))
    elif grp == gi.SU2:
        A = gi._project_commutant_su2(A, gi._su2_generators(gi._bond_slots_su2(p.n_v)))

    def log_n(eps):
        O = scipy.linalg.expm(eps * A)
        gb = np.einsum("ij,nljk,mk->nlim", O, p.gamma_bond, O)
        return weight.Weights(dataclasses.replace(p, gamma_bond=gb)).log_norm(links)

    h = 1e-5
    fd = (log_n(h) - log_n(-h)) / (2 * h)
    an = sum(np.sum(U[l] * (A @ p.gamma_bond[0, l] - p.gamma_bond[0, l] @ A)).real for l in range(p.n_links))
    assert abs(an) > 1e-3
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


def test_energies_respect_the_variational_bounds(setup):
    """H = -h sum_l X_l - J sum_p W_p acts on the 2^8 link states of the 2x2
    Z2 torus (X_l flips link l, W_p is diagonal).  Every energy the per-pair
    matrices give -- for random lambda and for the optimum -- is a genuine
    quantum expectation, hence within H's spectrum."""
    p, cfgs, S = setup
    h, J = 0.7, 1.3
    idx = {tuple(G): k for k, G in enumerate(cfgs)}
    Hm = np.zeros((len(cfgs), len(cfgs)))
    pl = plaquette_values(gi.Z2, 2, cfgs)
    for k, G in enumerate(cfgs):
        Hm[k, k] = -J * pl[k].sum()
        for l in range(p.n_links):
            g2 = G.copy()
            g2[l] = -g2[l]
            Hm[idx[tuple(g2)], k] += -h
    ev = np.linalg.eigvalsh(Hm)
    Hbar = -J * p.V * S["plaquette"] - h * S["electric"].sum(axis=0)
    E0, lam0 = va.linear_method(Hbar, S["norm"])
    assert ev[0] - 1e-9 <= E0 <= ev[-1] + 1e-9
    rng = np.random.default_rng(5)
    for _ in range(50):
        z = rng.normal(size=p.K) + 1j * rng.normal(size=p.K)
        e = va.expectation(Hbar, S["norm"], z).real
        assert ev[0] - 1e-9 <= e <= ev[-1] + 1e-9
        assert e >= E0 - 1e-9


def test_site_gradient_step_lowers_a_wilson_energy():
    """E = -<mean plaquette> on the 2x2 Z2 torus (exhaustive).  The gradient
    with respect to a rotation exp(A) of the even-sublattice site states,
    A = sum_k theta_k E_k over the antisymmetric basis, is the covariance of
    the plaquette with sum_s tr(S_s^T dD_s/d theta_k); a small step against
    it lowers E, by the amount the gradient predicts to first order."""
    import dataclasses
    import scipy.linalg
    p = gi.make_problem(2, gi.Z2, 1, 1, bond_scale=0.3)
    cfgs = gi.all_z2_configs(p)
    pl = plaquette_values(gi.Z2, 2, cfgs).mean(axis=1)

    def energy(q):
        W = weight.Weights(q)
        logs = np.array([W.log_norm(G) for G in cfgs])
        w = np.exp(logs - logs.max())
        return -np.sum(w * pl) / w.sum(), w / w.sum()

    E, w = energy(p)
    scores = [va.score_sites(p, G) for G in cfgs]
    m = p.m_s
    basis = []
    for a in range(m):
        for b in range(a + 1, m):
            Ek = np.zeros((m, m))
            Ek[a, b], Ek[b, a] = 1.0, -1.0
            basis.append(Ek)
    even = [s for s in range(p.V) if p.q_phys[s] == 1]
    grad = np.zeros(len(basis))
    for k, Ek in enumerate(basis):
        dlog = np.array([sum(np.sum(S[s] * (Ek @ p.gamma_site[s] - p.gamma_site[s] @ Ek)[2:, 2:]) for s in even)
                         for S in scores])
        grad[k] = -np.sum(w * (pl - np.sum(w * pl)) * dlog)      # dE/dtheta_k
    assert np.linalg.norm(grad) > 1e-3
    eta = 0.05 / np.linalg.norm(grad)
    O = scipy.linalg.expm(-eta * sum(g * Ek for g, Ek in zip(grad, basis)))
    gs = p.gamma_site.copy()
    for s in even:
        gs[s] = O @ gs[s] @ O.T
    E2, _ = energy(dataclasses.replace(p, gamma_site=gs))
    predicted = -eta * np.dot(grad, grad)
    assert E2 < E
    assert abs((E2 - E) - predicted) <= 0.2 * abs(predicted)


def test_u1_field_forms_reproduce_direct_expectations():
    """U(1) on the 1x1 torus, on an 8 x 8 angle grid that integrates the
    terms exactly: the per-pair field forms, contracted with another lambda,
    give the grid expectation of <J_l> computed directly with that lambda."""
    from oracle import electric
    p = gi.make_problem(1, gi.U1, 1, 2, bond_scale=0.4)
    th = 2 * np.pi * np.arange(8) / 8
    grid = np.array([[a, b] for a in th for b in th])
    S = va.exhaustive(p, grid)
    rng = np.random.default_rng(4)
    for _ in range(2):
        z = rng.normal(size=p.K) + 1j * rng.normal(size=p.K)
        lam = z / np.linalg.norm(z)
        q = va.with_lambda(p, lam)
        W = weight.Weights(q)
        logs = np.array([W.log_norm(G) for G in grid])
        w = np.exp(logs - logs.max())
        w /= w.sum()
        el = electric.Electric(q)
        direct = sum(wi * el.field(G) for wi, G in zip(w, grid))
        got = va.expectation(S["field"], S["norm"], lam)
        assert np.abs(direct).max() > 1e-3
        assert np.abs(got - direct).max() <= 1e-12
