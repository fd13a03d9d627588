"""Variational optimisation of the superposition weights lambda_n (Sec. 4,
Sec. 5; the Ansatz's parameters are meant to be optimised against an energy
built from the observables of Sec. 5).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For fixed Gaussians every per-configuration quantity of Secs. 5.1-5.3 is a
Hermitian form in lambda:
    N(G)   = lambda^dag N(G) lambda,          N(G)_nm  = N_nm(G),
    O(G)   = lambda^dag Ohat(G) lambda,       Ohat(G)_nm = N_nm(G) o_nm(G),
with o_nm the per-pair normalised expectation: W(G) for a Wilson loop (the
same for every pair), R_nm(G) for the electric term (oracle.electric), and
-i Gamma_eff^nm[a, b] for a Majorana bilinear (oracle.fermionic).  Hence
    <O>_lambda = lambda^dag Obar lambda / lambda^dag Nbar lambda,
    Obar = sum_G Ohat(G),  Nbar = sum_G N(G)
(integrals over the group for U(1)), and the lambda minimising an energy
E = sum_k c_k <O_k> is the lowest generalised eigenvector of
    (sum_k c_k Obar_k) lambda = E Nbar lambda.
Samples G_i of p_lambda0 estimate both matrices up to the common factor
1 / sum_G N_lambda0(G): Obar ~ mean_i Ohat(G_i) / N_lambda0(G_i).  Per
configuration the local matrices are returned in that normalised form
(Ohat(G) / N_lambda0(G), N(G) / N_lambda0(G)), which needs no absolute scale.

Also the score d log N(G) / d D_s of the site blocks (score_sites), which
gives exact gradients of Wilson-loop energies with respect to the site
parameters: dE = E_p[(W(G) - E) sum_s tr(S_s^T dD_s)], and its counterpart
for the link blocks of every pair (score_links; for K = 1 the bond gradient).

Pinned (tests/test_oracle_variational.py): the site and (K = 1) link scores
against central finite differences of log N(G) along commutant generators of
the site and bond states (Z2, U(1), SU(2)); on the 2x2 Z2 lattice, for random lambda, the Hermitian forms
built from exhaustive sums reproduce the direct exhaustive expectations of
the plaquette, the link flip, the densities and the link terms computed with that lambda; the generalised eigenvector minimises the energy
over random lambda; the forms are Hermitian and Nbar positive definite.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg

from . import electric, fermionic, weight
from .pfaffian import pfaffian
from .observables import plaquette_values


class LocalMatrices:
    """Per-configuration K x K matrices for the observables of Sec. 5."""

    def __init__(self, p):
        self.p = p
        self.W = weight.Weights(p)
        self.el = electric.Electric(p)
        self.fe = fermionic.Fermionic(p)

    def __call__(self, links):
        """dict of K x K (or (n, K, K)) arrays divided by N_lambda0(G):
        'norm' N(G); 'plaquette' mean plaquette; 'electric' per link;
        'field' per link (U(1): the electric field <J_l>); 'four' per link
        (<c_2s c_2s+1 c_2t c_2t+1>, the density-density part);
        'density' per site (the bilinear c_2s c_2s+1); 'hopping' per link
        (Z2 and U(1): the gauge-invariant link term T_l; T_l^dag has the
        conjugate transpose over n, m)."""
        p = self.p
        lnm = self.W.log_n_matrix(links)
        logN = weight.combine(lnm, p.lam)
        Nn = np.exp(lnm - logN)                                  # N(G) / N_lambda0(G)
        out = {"norm": Nn}
        out["plaquette"] = Nn * plaquette_values(p.group, p.L, links).mean()
        R = self.el.ratios(links)                                # [n, m, l]
        out["electric"] = np.moveaxis(Nn[:, :, None] * R, 2, 0)  # [l, n, m]
        if p.group == weight.U1:
            out["field"] = np.moveaxis(Nn[:, :, None] * self.el.field_ratios(links), 2, 0)
        Ge = self.fe.gamma_eff(links)
        dens = np.zeros((p.V, p.K, p.K), dtype=complex)
        for (n, m), G in Ge.items():
            for s in range(p.V):
                dens[s, n, m] = Nn[n, m] * (-1j) * G[2 * s, 2 * s + 1]
        out["density"] = dens
        four = np.zeros((p.n_links, p.K, p.K), dtype=complex)
        for l in range(p.n_links):
            s, t = fermionic._link_sites(p, l)
            ix = [2 * s, 2 * s + 1, 2 * t, 2 * t + 1]
            for (n, m), G in Ge.items():
                four[l, n, m] = Nn[n, m] * (-1.0 if s == t else pfaffian(-1j * G[np.ix_(ix, ix)]))
        out["four"] = four
        if p.group == weight.SU2:      # link terms are defined for Z2 and U(1)
            return out
        blk = np.zeros((p.n_links, 2, 2, p.K, p.K), dtype=complex)
        for l in range(p.n_links):
            s, t = fermionic._link_sites(p, l)
            for a in range(2):
                for b in range(2):
                    i, j = 2 * s + a, 2 * t + b
                    for (n, m), G in Ge.items():
                        blk[l, a, b, n, m] = Nn[n, m] * (1.0 if i == j else -1j * G[i, j])
        out["hopping"] = fermionic.link_terms_from_block(p, links, blk)
        return out


def exhaustive(p, configs, weights=None):
    """Sums over an explicit list of configurations (optionally weighted, e.g.
    quadrature weights) of the local matrices, all divided by the same
    constant sum_G N_lambda0(G).  Returns the dict of summed matrices."""
    lm = LocalMatrices(p)
    W = lm.W
    logs = np.array([W.log_norm(G) for G in configs])
    wts = np.exp(logs - logs.max())
    if weights is not None:
        wts = wts * weights
    wts = wts / wts.sum()                                        # p_lambda0 on the list
    acc = None
    for w, G in zip(wts, configs):
        loc = lm(G)
        if acc is None:
            acc = {k: w * v for k, v in loc.items()}
        else:
            for k, v in loc.items():
                acc[k] = acc[k] + w * v
    return acc


def expectation(Obar, Nbar, lam):
    """lambda^dag Obar lambda / lambda^dag Nbar lambda (Obar may carry leading axes)."""
    lam = np.asarray(lam)
    num = np.einsum("n,...nm,m->...", np.conj(lam), Obar, lam)
    den = np.einsum("n,nm,m->", np.conj(lam), Nbar, lam)
    return num / den


def linear_method(Hbar, Nbar):
    """Lowest generalised eigenpair of (Hbar + Hbar^dag)/2 lambda = E Nbar lambda
    (Nbar Hermitian positive definite); lambda normalised to unit 2-norm with
    lambda_0 real positive."""
    H = 0.5 * (Hbar + Hbar.conj().T)
    Nm = 0.5 * (Nbar + Nbar.conj().T)
    w, v = scipy.linalg.eigh(H, Nm)
    lam = v[:, 0]
    lam = lam / np.linalg.norm(lam)
    if abs(lam[0]) > 0:
        lam = lam * (abs(lam[0]) / lam[0])
    return float(w[0]), lam


def score_sites(p, links) -> np.ndarray:
    """d log N(G) / d D_s[i][j] for every site s (V, B, B), B = 8 n_v, D_s the
    site's virtual covariance block, entries treated as independent.  For
    pure site states N_nm(G) is Pf(D + O Gamma_X O^T) times a constant, and
    d log Pf(M) = (1/2) tr(M^{-1} dM), so
        S_s = Re sum_nm lambda_n^* lambda_m (N_nm(G) / N(G)) (1/2) W_nm[s, s]^T
    with W_nm[s, s] the site's diagonal block of (D + O Gamma_X^nm O^T)^{-1}.
    A variation of the site parameters changes log N(G) by sum_ij S_ij dD_ij."""
    W = weight.Weights(p)
    lnm = W.log_n_matrix(links)
    logN = weight.combine(lnm, p.lam)
    B = 8 * p.n_v
    virt = np.array([i for i in range(p.m_s * p.V) if i % p.m_s >= 2])
    Ov = weight.twist_matrix(p, links)[np.ix_(virt, virt)]
    D = np.zeros((B * p.V, B * p.V))
    for s in range(p.V):
        D[s * B:(s + 1) * B, s * B:(s + 1) * B] = p.gamma_site[s][2:, 2:]
    S = np.zeros((p.V, B, B))
    for n in range(p.K):
        for m in range(p.K):
            Wnm = np.linalg.inv(D + Ov @ W.GX[n, m][np.ix_(virt, virt)] @ Ov.T)
            wt = np.conj(p.lam[n]) * p.lam[m] * np.exp(lnm[n, m] - logN)
            for s in range(p.V):
                S[s] += (wt * 0.5 * Wnm[s * B:(s + 1) * B, s * B:(s + 1) * B].T).real
    return S


def score_links(p, links) -> np.ndarray:
    """Per pair p (diagonal pairs, then n < m) and link l, the r x r complex
    block U_p[l] = (w_p N_p / N(G)) (1/2) (O_l^T W_p[l, l] O_l)^T, with w_p the
    pair weight (|lambda_n|^2, or 2 lambda_n^* lambda_m), N_p = N_nm(G),
    W_p[l, l] the block of (D + O Gamma_X^p O^T)^{-1} on the link's r
    Majoranas and O_l the link's twist.  Since d log Pf(M) = (1/2) tr(W dM),
        d log N(G) = Re sum_p sum_l tr(U_p[l]^T dGamma_X^p[l])
                     + Re sum_p (w_p N_p / N(G)) d log c_p,
    c_p the pair's G-independent constant (for K = 1 the second term
    vanishes and Gamma_X = Gamma_B, so this is the bond gradient)."""
    W = weight.Weights(p)
    lnm = W.log_n_matrix(links)
    logN = weight.combine(lnm, p.lam)
    B = 8 * p.n_v
    virt = np.array([i for i in range(p.m_s * p.V) if i % p.m_s >= 2])
    pos = -np.ones(p.m_s * p.V, dtype=int)
    pos[virt] = np.arange(virt.size)
    idx = [pos[np.array(ix)] for ix in weight.link_majoranas(p)]
    Ov = weight.twist_matrix(p, links)[np.ix_(virt, virt)]
    D = np.zeros((B * p.V, B * p.V))
    for s in range(p.V):
        D[s * B:(s + 1) * B, s * B:(s + 1) * B] = p.gamma_site[s][2:, 2:]
    pairs = [(n, n) for n in range(p.K)] + [(n, m) for n in range(p.K) for m in range(n + 1, p.K)]
    out = np.zeros((len(pairs), p.n_links, p.r, p.r), dtype=complex)
    for k, (n, m) in enumerate(pairs):
        Wnm = np.linalg.inv(D + Ov @ W.GX[n, m][np.ix_(virt, virt)] @ Ov.T)
        wp = abs(p.lam[n]) ** 2 if n == m else 2 * np.conj(p.lam[n]) * p.lam[m]
        f = wp * np.exp(lnm[n, m] - logN)
        for l in range(p.n_links):
            ii = idx[l]
            Ol = Ov[np.ix_(ii, ii)]
            out[k, l] = f * 0.5 * (Ol.T @ Wnm[np.ix_(ii, ii)] @ Ol).T
    return out


def with_lambda(p, lam):
    """The same problem with other superposition weights."""
    return dataclasses.replace(p, lam=np.asarray(lam, dtype=np.complex128))
