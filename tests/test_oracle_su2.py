"""Pins of the SU(2) extension of the oracle (non-Abelian links, Sec. 2 and
App. A: the twist psi^dag -> psi^dag D(g) on every doublet of a source end).

* the Majorana rotation of the twist against explicit Fock operators;
* the weight by the covariance route against explicit Fock vectors (1x1);
* on the U(1) subgroup exp(i theta sigma_z) the SU(2) code reproduces the
  pinned U(1) code (weights, plaquettes, proposals);
* gauge invariance of the weight and of the plaquette under
  g_l -> h_t^dag g_l h_s, and SU(2) invariance of the generated inputs;
* the Metropolis chain with the SU(2) proposal against independent Haar
  importance sampling of the same expectation.
"""
import dataclasses

import numpy as np
import pytest
import scipy.linalg

import ggf_inputs as gi
from oracle import fock, mcmc, observables, weight
from oracle.observables import tau_int


def _haar(n, seed):
    q = np.random.default_rng(seed).normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def test_doublet_rotation_matches_fock():
    """U c_a U^dag = sum_b R_ab c_b for U = exp(sum (log u)_{ba} psi^dag_b psi_a)."""
    ann, cre = fock.fermion_ops(2)
    cs = fock.majoranas(2)
    for q in _haar(3, 1):
        u = weight.su2_matrix(q)
        lg = scipy.linalg.logm(u)
        H = sum(lg[b, a] * (cre[b] @ ann[a]) for a in range(2) for b in range(2)).toarray()
        U = scipy.linalg.expm(H)
        # the defining action on creators
        for j in range(2):
            lhs = U @ cre[j].toarray() @ U.conj().T
            rhs = sum(u[k, j] * cre[k].toarray() for k in range(2))
            assert np.abs(lhs - rhs).max() <= 1e-12
        R = weight.doublet_rotation(u)
        for a in range(4):
            lhs = U @ cs[a].toarray() @ U.conj().T
            rhs = sum(R[a, b] * cs[b].toarray() for b in range(4))
            assert np.abs(lhs - rhs).max() <= 1e-12


@pytest.mark.parametrize("K", [1, 2])
def test_covariance_route_matches_fock_1x1(K):
    p = gi.make_problem(1, gi.SU2, 2, K, bond_scale=0.3)
    fp, W = fock.FockPEPS(p), weight.Weights(p)
    for G in gi.random_links(p, 3, seed=3):
        nf = fp.n_matrix(G)
        nc = np.exp(W.log_n_matrix(G))
        assert np.abs(nc - nf).max() <= 1e-12 * np.abs(nf).max()
        assert abs(W.log_norm(G) - np.log(fp.norm(G))) <= 1e-12


def test_u1_subgroup_reproduces_u1():
    p = gi.make_problem(2, gi.SU2, 2, 2, bond_scale=0.3)
    pu = dataclasses.replace(p, group=gi.U1)          # q_src = (+1, -1): D = diag(e^{i t}, e^{-i t})
    th = gi.random_links(pu, 2, seed=5)
    q = np.zeros(th.shape + (4,))
    q[..., 0], q[..., 3] = np.cos(th), np.sin(th)
    Ws, Wu = weight.Weights(p), weight.Weights(pu)
    for a, b in zip(q, th):
        assert np.abs(weight.twist_matrix(p, a) - weight.twist_matrix(pu, b)).max() <= 1e-15
        assert abs(Ws.log_norm(a) - Wu.log_norm(b)) <= 1e-12
    assert np.abs(observables.plaquette_values(gi.SU2, 2, q) - observables.plaquette_values(gi.U1, 2, th)).max() \
        <= 1e-14
    # the proposal along n = z is the U(1) move (before wrapping)
    for t, u in [(0.3, 0.9), (2.0, 0.1)]:
        g = np.array([np.cos(t), 0.0, 0.0, np.sin(t)])
        new = mcmc.propose(gi.SU2, g, u, 0.5, 1.0, 0.0)
        d = 0.5 * (u - 0.5)
        assert np.abs(new - [np.cos(t + d), 0.0, 0.0, np.sin(t + d)]).max() <= 1e-15


def test_gauge_invariance_and_symmetric_inputs():
    p = gi.make_problem(3, gi.SU2, 2, 2, bond_scale=0.3)
    W = weight.Weights(p)
    G = gi.random_links(p, 2, seed=8)
    h = _haar(p.V, 9)
    hG = gi.gauge_transform(p, G, h)
    for a, b in zip(G, hG):
        assert abs(W.log_norm(a) - W.log_norm(b)) <= 1e-11
        assert np.abs(observables.plaquette_values(gi.SU2, 3, a) -
                      observables.plaquette_values(gi.SU2, 3, b)).max() <= 1e-13
    # site: D on source ends (+x, +y), conj(D) on target ends, singlet physical mode;
    # bond: D on the source end, conj(D) on the target end
    for q in _haar(3, 4):
        u = weight.su2_matrix(q)
        R, Rc = weight.doublet_rotation(u), weight.doublet_rotation(u.conj())
        Rs = np.eye(p.m_s)
        for e in range(4):
            a = 2 + 4 * e
            Rs[a:a + 4, a:a + 4] = R if e % 2 else Rc
        Rb = scipy.linalg.block_diag(R, Rc)
        for s in range(p.V):
            assert np.abs(Rs @ p.gamma_site[s] @ Rs.T - p.gamma_site[s]).max() <= 1e-12
        for n in range(p.K):
            assert np.abs(Rb @ p.gamma_bond[n, 0] @ Rb.T - p.gamma_bond[n, 0]).max() <= 1e-12
    # the virtual ends are coupled (a non-trivial symmetric site state)
    assert np.abs(p.gamma_site[0][6:10, 2:6]).max() > 0.05


def test_plaquette_special_cases():
    p = gi.make_problem(3, gi.SU2, 2, 1)
    cold = gi.cold_links(p, 1)
    assert np.abs(observables.plaquette_values(gi.SU2, 3, cold) - 1.0).max() <= 1e-15
    flip = cold.copy()
    flip[0, 2 * 4, 0] = -1.0                # the centre element -1 on the x link from site 4
    v = observables.plaquette_values(gi.SU2, 3, flip)[0]
    assert v[4] == -1.0 and v[1] == -1.0 and np.sum(v == -1.0) == 2


def test_proposal_is_reversible_and_unitary():
    g = _haar(1, 2)[0]
    for u, uz, uf in [(0.8, 0.3, 0.6), (0.05, 0.99, 0.1)]:
        new = mcmc.propose(gi.SU2, g, u, 1.3, uz, uf)
        assert abs(new @ new - 1.0) <= 1e-15
        back = mcmc.propose(gi.SU2, new, 1.0 - u, 1.3, uz, uf)
        assert np.abs(back - g).max() <= 1e-14


def test_metropolis_matches_haar_importance_sampling():
    """<plaquette> on the 1x1 torus: Metropolis with the SU(2) proposal
    against sum_i N(G_i) W(G_i) / sum_i N(G_i) over independent Haar samples."""
    p = gi.make_problem(1, gi.SU2, 2, 1, bond_scale=0.3, site_scale=1.5)
    W = weight.Weights(p)
    G = gi.random_links(p, 20000, seed=11)
    logs = np.array([W.log_norm(g) for g in G])
    w = np.exp(logs - logs.max())
    w /= w.sum()
    pl = observables.plaquette_values(gi.SU2, 1, G)[:, 0]
    imp = np.sum(w * pl)
    se_imp = np.sqrt(np.sum(w ** 2 * (pl - imp) ** 2))
    runs = []
    for ch in range(16):
        _, obs, _ = mcmc.run_chain(p, W, gi.cold_links(p, 1)[0], 5, ch, 0, 500, width=2.0)
        runs.append(obs[50:, 0])
    runs = np.array(runs)
    tau, _ = tau_int(runs)
    se_mc = runs.std() * np.sqrt(2 * tau / runs.size)
    assert abs(runs.mean() - imp) <= 4 * np.hypot(se_imp, se_mc)
    # the test has power: the weighting moves the mean far from the Haar value
    assert abs(pl.mean() - imp) > 8 * np.hypot(se_imp, se_mc)
