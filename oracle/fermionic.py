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

Gauge-invariant link terms.  A fermion bilinear across link l = (s -> t)
becomes gauge invariant with the link operator u_l(G) (Z2: g_l; U(1):
e^{i theta_l}, diagonal in G) when the bilinear carries the charge that the
link operator removes: with the Gauss generator sum_out J - sum_in J + q_s n_s
(J = -i d/dtheta, so [J_l, e^{i theta_l}] = e^{i theta_l}), the operator
    T_l = u_l F_s F_t,  F_s = psi_s (q_s > 0) or psi_s^dag (q_s < 0),
                        F_t = psi_t^dag (q_t > 0) or psi_t (q_t < 0)
commutes with every generator (for staggered charges it is the pair term
psi_s psi_t or psi_s^dag psi_t^dag; T_l + T_l^dag is the link's hopping term).
Per configuration T_l(G) = u_l(G) <F_s F_t>_G, with psi = (c_0 + i c_1) / 2,
a linear combination of the link block.  For Z2 every bilinear times g_l is
invariant; the same F are used.

Pinned (tests/test_oracle_fermionic.py): the covariance route against the
Fock route (Z2 and U(1), K = 1, 2, 2x2 and 1x1 lattices, n_v = 1, 2),
four- and six-Majorana monomials against Fock, Z2 gauge covariance of the
link block (C_l(hG) = h_s h_t C_l(G)) and gauge invariance of the densities,
i <c_a c_b> real and 0 <= <n_s> <= 1 in every configuration, zero staggered
charge sum_s q_s <n_s> for U(1) in every configuration.  Link terms: the
covariance route against explicit psi / psi^dag matrices on Fock vectors
(Z2, U(1); 1x1, 2x2; n_v = 1, 2), per-configuration gauge invariance while
the bilinear with the opposite phase (u_l^* F_s F_t) is not invariant, and
zero charge-violating bilinears on links between equal charges (3x3 torus).
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


def link_signs(q_s: int, q_t: int):
    """(e_s, e_t) with F = (c_0 + i e c_1) / 2: e = +1 is psi, -1 is psi^dag."""
    return (1 if q_s > 0 else -1), (-1 if q_t > 0 else 1)


def link_phase(p, links, l) -> complex:
    """u_l(G): the Z2 element, or e^{i theta_l} for U(1)."""
    if p.group == weight.Z2:
        return complex(int(links[l]))
    return complex(np.exp(1j * float(links[l])))


def link_terms_fock(fp: fock.FockPEPS, links) -> np.ndarray:
    """T_l(G) (n_links,) from explicit vectors and explicit annihilation
    operators psi_s = (c_{2s} + i c_{2s+1}) / 2."""
    p = fp.p
    v = (p.lam[:, None] * fp.psi(links)).sum(axis=0)
    cs = fock.majoranas(p.V)
    out = np.zeros(p.n_links, dtype=complex)
    for l in range(p.n_links):
        s, t = _link_sites(p, l)
        psi_s = 0.5 * (cs[2 * s] + 1j * cs[2 * s + 1])
        psi_t = 0.5 * (cs[2 * t] + 1j * cs[2 * t + 1])
        Fs = psi_s if p.q_phys[s] > 0 else psi_s.conj().T
        Ft = psi_t.conj().T if p.q_phys[t] > 0 else psi_t
        out[l] = link_phase(p, links, l) * np.vdot(v, Fs @ (Ft @ v)) / np.vdot(v, v)
    return out


def link_terms_from_block(p, links, block) -> np.ndarray:
    """T_l(G) from link blocks block[l, alpha, beta] = <c_{2s+alpha} c_{2t+beta}>
    (or per-pair parts with trailing axes): u_l (1/4) sum a_alpha b_beta block,
    a = (1, i e_s), b = (1, i e_t)."""
    out = np.zeros((p.n_links,) + block.shape[3:], dtype=complex)
    for l in range(p.n_links):
        s, t = _link_sites(p, l)
        es, et = link_signs(p.q_phys[s], p.q_phys[t])
        a, b = np.array([1.0, 1j * es]), np.array([1.0, 1j * et])
        out[l] = link_phase(p, links, l) * 0.25 * np.einsum("a,b,ab...->...", a, b, block[l])
    return out


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

    def link_terms(self, links) -> np.ndarray:
        """Gauge-invariant link terms T_l(G) (n_links,) by the covariance route."""
        _, link = self.bilinears(links)
        return link_terms_from_block(self.p, links, link)
