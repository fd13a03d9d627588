"""Fermionic observables of the gauged superposition (Sec. 5.2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A fermionic observable is a Majorana monomial c^x on the physical modes times
a string of link operators W(F), diagonal in G.  Per configuration
    F(G) = W(F, G) sum_nm lambda_n^* lambda_m <psi_n(G)| c^x |psi_m(G)> / N(G).
This module evaluates the Majorana part, Sec. 5.2's per-configuration
expectation; the link factor W(F, G) belongs to the operator.

Two routes:

1. Fock (the definition, tiny lattices): explicit vectors psi_n(G) from
   oracle.fock and explicit Majorana matrices on the physical modes (site s
   carries c_{2s}, c_{2s+1}).
2. Covariance (Wick's theorem): contracting the virtual modes of the site
   state with the bond operator X_nm leaves a Gaussian operator on the
   physical modes with covariance
       Gamma_eff^nm = A + B W B^T,   W = (D_G + Gamma_X^nm)^{-1},
   where [[A, B], [-B^T, D_G]] is Gamma_{A(G)} split into physical and virtual
   Majoranas (the twist acts on D_G and B only).  Then
       <psi_n(G)| c_{a1} ... c_{a2k} |psi_m(G)> = N_nm(G) Pf(-i Gamma_eff^nm[x, x])
   for distinct indices x = (a1, ..., a2k) in that order; for a bilinear,
   N_nm(G) (-i Gamma_eff^nm[a, b]).  This is the Pfaffian formula of Sec. 5.2
   with the virtual modes integrated out first.

Outputs per configuration: the site bilinear c_{2s} c_{2s+1} (density
n_s = (1 + i <c_{2s} c_{2s+1}>) / 2) and, per link l = (s -> t), the 2 x 2
block <c_{2s+alpha} c_{2t+beta}> from which hoppings psi_s^dag psi_t,
pairings psi_s psi_t and their conjugates follow.

Pinned (tests/test_oracle_fermionic.py): the covariance route against the
Fock route (Z2 and U(1), K = 1, 2, 2x2 and 1x1 lattices, n_v = 1, 2),
four- and six-Majorana monomials against Fock, Z2 gauge covariance of the
link block (C_l(hG) = h_s h_t C_l(G)) and gauge invariance of the densities,
i <c_a c_b> real and 0 <= <n_s> <= 1 in every configuration, zero staggered
charge sum_s q_s <n_s> for U(1) in every configuration.
"""
from __future__ import annotations

import numpy as np

from . import fock, weight
from .pfaffian import pfaffian


def _link_sites(p, l):
    s, d = l // 2, l % 2
    x, y = s % p.L, s // p.L
    t = (y * p.L + (x + 1) % p.L) if d == 0 else (((y + 1) % p.L) * p.L + x)
    return s, t


def _expect(p, v, idx) -> complex:
    cs = fock.majoranas(p.V)
    w = v.copy()
    for a in reversed(list(idx)):
        w = cs[a] @ w
    return complex(np.vdot(v, w) / np.vdot(v, v))


def monomial_fock(fp: fock.FockPEPS, links, idx) -> complex:
    """sum_nm lambda_n^* lambda_m <psi_n|c_{idx[0]} c_{idx[1]} ...|psi_m> / N(G)
    from explicit vectors; idx are physical Majorana indices (2s + alpha)."""
    p = fp.p
    return _expect(p, (p.lam[:, None] * fp.psi(links)).sum(axis=0), idx)


def bilinears_fock(fp: fock.FockPEPS, links):
    """(site[V], link[n_links, 2, 2]) by explicit vectors."""
    p = fp.p
    v = (p.lam[:, None] * fp.psi(links)).sum(axis=0)
    site = np.array([_expect(p, v, (2 * s, 2 * s + 1)) for s in range(p.V)])
    link = np.zeros((p.n_links, 2, 2), dtype=complex)
    for l in range(p.n_links):
        s, t = _link_sites(p, l)
        for al in range(2):
            for be in range(2):
                link[l, al, be] = _expect(p, v, (2 * s + al, 2 * t + be))
    return site, link


class Fermionic:
    """Covariance route to the Majorana expectations of Sec. 5.2."""

    def __init__(self, p):
        self.p = p
        self.W = weight.Weights(p)
        m_s = p.m_s
        self.virt = np.array([i for i in range(m_s * p.V) if i % m_s >= 2])
        self.phys = np.array([i for i in range(m_s * p.V) if i % m_s < 2])

    def gamma_eff(self, links) -> dict:
        """Gamma_eff^nm on the 2V physical Majoranas, every ordered pair."""
        p = self.p
        O = weight.twist_matrix(p, links)
        GA = O.T @ self.W.GA @ O
        ph, vi = self.phys, self.virt
        A, B, D = GA[np.ix_(ph, ph)], GA[np.ix_(ph, vi)], GA[np.ix_(vi, vi)]
        out = {}
        for n in range(p.K):
            for m in range(p.K):
                Wnm = np.linalg.inv(D + self.W.GX[n, m][np.ix_(vi, vi)])
                out[n, m] = A + B @ Wnm @ B.T
        return out

    def _weights(self, links):
        lnm = self.W.log_n_matrix(links)
        Nnm = np.exp(lnm - lnm.real.max())
        w = np.conj(self.p.lam)[:, None] * self.p.lam[None, :] * Nnm
        return w / w.sum()

    def monomial(self, links, idx) -> complex:
        """The Fock route's quantity by Pfaffians (distinct indices, even count)."""
        idx = list(idx)
        if len(idx) % 2 or len(set(idx)) != len(idx):
            raise ValueError("distinct indices, even count")
        w, Ge = self._weights(links), self.gamma_eff(links)
        tot = 0.0 + 0.0j
        for (n, m), G in Ge.items():
            tot += w[n, m] * pfaffian(-1j * G[np.ix_(idx, idx)])
        return complex(tot)

    def bilinears(self, links):
        """(site[V], link[n_links, 2, 2]) as in bilinears_fock."""
        p = self.p
        w, Ge = self._weights(links), self.gamma_eff(links)
        C = sum(w[n, m] * (-1j) * G for (n, m), G in Ge.items())
        site = np.array([C[2 * s, 2 * s + 1] for s in range(p.V)])
        link = np.zeros((p.n_links, 2, 2), dtype=complex)
        for l in range(p.n_links):
            s, t = _link_sites(p, l)
            for al in range(2):
                for be in range(2):
                    a, b = 2 * s + al, 2 * t + be
                    link[l, al, be] = 1.0 if a == b else C[a, b]
        return site, link
