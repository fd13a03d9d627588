"""The algebra of the GPU observable kernels (electric, fermionic), in numpy.

Electric (Sec. 5.3; Z2 link flip, U(1) Casimir):

The kernel works on the reduced virtual-mode matrix with the twist on the
bond side, M = D + O Gamma_X O^T, W = M^{-1}, and for link l with source-end
Majoranas S computes
    Gamma_O[S, S] = i 1 - (1 + i D)[S, site] W[site, link] (1 + i O Gamma_X O^T)[link, S]
and from it R_nm = (-1)^{n_v} Pf(Gamma_O[S, S]) (Z2) or <Q_l^2> (U(1)),
from the B x r block of W between the source site and the link only, with the
(m, n) order of a pair n < m taken from conj(W_nm) and conj(Gamma_X^nm).
These checks restate that recipe and compare it with the oracle's f_E (which
has the twist on the site side and the full covariance route), and check the
two facts it rests on: the block restriction and M_mn = conj(M_nm).

Fermionic (Sec. 5.2): the physical covariance A + B W B^T of each pair from
the B x B block of W between two sites, A and B untwisted.
"""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import electric, pfaffian, weight


def _gpu_picture(p, links):
    """Reduced D, per-pair twisted bond blocks and inverses, and link indices."""
    virt = np.array([i for i in range(p.m_s * p.V) if i % p.m_s >= 2])
    pos = -np.ones(p.m_s * p.V, dtype=int)
    pos[virt] = np.arange(virt.size)
    N, B, h2 = virt.size, 8 * p.n_v, 2 * p.n_v
    D = np.zeros((N, N))
    for s in range(p.V):
        D[s * B:(s + 1) * B, s * B:(s + 1) * B] = p.gamma_site[s][2:, 2:]
    idx = [pos[np.array(ix)] for ix in weight.link_majoranas(p)]
    O = weight.twist_matrix(p, links)[np.ix_(virt, virt)]   # acts on source ends only
    bd = weight.BondData(p)
    tw = {nm: O @ bd.embedded(*nm)[np.ix_(virt, virt)] @ O.T
          for nm in [(n, m) for n in range(p.K) for m in range(p.K)]}
    return D, tw, idx, B, h2


def _kernel_ratio(p, D, W, Gtw, S, site, lk):
    h2 = S.size
    left = np.eye(D.shape[0])[S][:, site] + 1j * D[np.ix_(S, site)]
    right = np.eye(D.shape[0])[np.ix_(lk, S)] + 1j * Gtw[np.ix_(lk, S)]
    G = 1j * np.eye(h2) - left @ W[np.ix_(site, lk)] @ right
    if p.group == gi.Z2:
        return (-1) ** p.n_v * pfaffian.pfaffian(G)
    if p.group == gi.SU2:
        return 0.75 * ((2 + G[0, 1] + G[2, 3]) / 2 - 2 * (1 + G[0, 1] + G[2, 3] + pfaffian.pfaffian(G)) / 4)
    q = p.q_src
    val = sum(q[j] ** 2 * (1 + G[2 * j, 2 * j + 1]) / 2 for j in range(p.n_v))
    if p.n_v == 2:
        val += 2 * q[0] * q[1] * (1 + G[0, 1] + G[2, 3] + pfaffian.pfaffian(G)) / 4
    return val


@pytest.mark.parametrize("L,grp,n_v,K", [(3, gi.Z2, 1, 2), (2, gi.Z2, 1, 3), (2, gi.Z2, 2, 2),
                                         (3, gi.U1, 1, 2), (2, gi.U1, 2, 3), (2, gi.SU2, 2, 2)])
def test_block_recipe_matches_oracle(L, grp, n_v, K):
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    el, Wt = electric.Electric(p), weight.Weights(p)
    for links in gi.random_links(p, 2, seed=17):
        D, tw, idx, B, h2 = _gpu_picture(p, links)
        lnm = Wt.log_n_matrix(links)
        Nnm = np.exp(lnm - lnm.real.max())
        f = np.zeros(p.n_links, dtype=complex)
        for n in range(p.K):
            for m in range(n, p.K):
                Wnm = np.linalg.inv(D + tw[n, m])
                if m > n:
                    # the (m, n) order from the stored (n, m) inverse
                    assert np.abs(np.linalg.inv(D + tw[m, n]) - Wnm.conj()).max() <= 1e-10 * np.abs(Wnm).max()
                for l in range(p.n_links):
                    s = l // 2
                    site = np.arange(s * B, (s + 1) * B)
                    S, lk = idx[l][:h2], idx[l]
                    Rf = _kernel_ratio(p, D, Wnm, tw[n, m], S, site, lk)
                    f[l] += np.conj(p.lam[n]) * p.lam[m] * Nnm[n, m] * Rf
                    if m > n:
                        Rr = _kernel_ratio(p, D, Wnm.conj(), tw[n, m].conj(), S, site, lk)
                        f[l] += np.conj(p.lam[m]) * p.lam[n] * Nnm[m, n] * Rr
        f /= np.einsum("n,m,nm->", np.conj(p.lam), p.lam, Nnm)
        ref = el.f_electric(links)
        assert np.abs(f - ref).max() <= 1e-11 * np.abs(ref).max()


def test_block_restriction_is_exact():
    """(1 + i D) W (1 + i Gamma_tw) on S x S equals the full product: D is
    block diagonal by site and Gamma_tw by link."""
    p = gi.make_problem(3, gi.Z2, 1, 1, bond_scale=0.3)
    links = gi.random_links(p, 1, seed=2)[0]
    D, tw, idx, B, h2 = _gpu_picture(p, links)
    W = np.linalg.inv(D + tw[0, 0])
    one = np.eye(D.shape[0])
    full = (one + 1j * D) @ W @ (one + 1j * tw[0, 0])
    for l in range(p.n_links):
        s = l // 2
        site = np.arange(s * B, (s + 1) * B)
        S, lk = idx[l][:h2], idx[l]
        blk = (one[S][:, site] + 1j * D[np.ix_(S, site)]) @ W[np.ix_(site, lk)] @ \
              (one[np.ix_(lk, S)] + 1j * tw[0, 0][np.ix_(lk, S)])
        assert np.abs(blk - full[np.ix_(S, S)]).max() <= 1e-12 * np.abs(full).max()


@pytest.mark.parametrize("L,grp,n_v,K", [(3, gi.Z2, 1, 2), (2, gi.U1, 1, 3), (2, gi.U1, 2, 2)])
def test_fermion_block_recipe_matches_oracle(L, grp, n_v, K):
    """The fermionic kernel's recipe: Gamma_eff^nm[a, b] = A_s (s = t) +
    B_s W_nm[site s, site t] B_t^T with untwisted A, B and the bond-side twist;
    the (m, n) order of a pair uses the conjugate of the same product."""
    from oracle import fermionic
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    fe, Wt = fermionic.Fermionic(p), weight.Weights(p)
    B = 8 * n_v
    virt = np.array([i for i in range(p.m_s * p.V) if i % p.m_s >= 2])
    for links in gi.random_links(p, 2, seed=23):
        O = weight.twist_matrix(p, links)[np.ix_(virt, virt)]
        D = np.zeros((B * p.V, B * p.V))
        for s in range(p.V):
            D[s * B:(s + 1) * B, s * B:(s + 1) * B] = p.gamma_site[s][2:, 2:]
        lnm = Wt.log_n_matrix(links)
        Nnm = np.exp(lnm - lnm.real.max())
        acc = np.zeros((p.n_links, 2, 2), dtype=complex)
        acc_site = np.zeros(p.V, dtype=complex)
        den = 0.0
        for n in range(p.K):
            for m in range(n, p.K):
                GX = Wt.GX[n, m][np.ix_(virt, virt)]
                Wnm = np.linalg.inv(D + O @ GX @ O.T)
                wnm = np.conj(p.lam[n]) * p.lam[m] * Nnm[n, m]

                def X(s, t, Wm):
                    Bs, Bt = p.gamma_site[s][:2, 2:], p.gamma_site[t][:2, 2:]
                    return Bs @ Wm[s * B:(s + 1) * B, t * B:(t + 1) * B] @ Bt.T
                terms = [(wnm, Wnm, False)] + ([(np.conj(wnm), Wnm, True)] if m > n else [])
                for wt, Wm, cj in terms:
                    den += wt.real
                    for s in range(p.V):
                        x = X(s, s, Wm)
                        acc_site[s] += wt * (x.conj() if cj else x)[0, 1]
                    for l in range(p.n_links):
                        s, t = fermionic._link_sites(p, l)
                        x = X(s, t, Wm)
                        acc[l] += wt * (x.conj() if cj else x)
        site = -1j * (acc_site / den + np.array([p.gamma_site[s][0, 1] for s in range(p.V)]))
        link = -1j * acc / den
        for l in range(p.n_links):
            s, t = fermionic._link_sites(p, l)
            if s == t:
                link[l] += -1j * p.gamma_site[s][:2, :2]
                link[l][0, 0] = link[l][1, 1] = 1.0
        rs, rl = fe.bilinears(links)
        assert np.abs(site - rs).max() <= 1e-11
        assert np.abs(link - rl).max() <= 1e-11
