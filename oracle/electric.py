"""Electric-field observable of a Z2 gauge field (Sec. 5.3).

For Z2 the electric operator of link l acts in the group-element basis as the
flip X_l |G> = |G^(l)>, G^(l) being G with g_l -> -g_l (the electric energy of
the link is a linear function of X_l; its normalisation and sign belong to the
Hamiltonian, not to the state).  Sec. 5.3 writes <X_l> = sum_G p(G) f_E(G) with

    f_E(G) = sum_nm lambda_n^* lambda_m <psi_n(G)|psi_m(G^(l))> / N(G),

a bra/ket-asymmetric overlap, since <G|X_l|G~> vanishes unless G~ = G^(l).

Two routes:

1. Fock (the definition, tiny lattices): explicit vectors psi_n(G) from
   oracle.fock.
2. Covariance: psi_m(G^(l)) = <B_m| U(G) P_l |A>, where P_l is the parity of
   the modes of the source end of link l (the end that carries the twist),
   P_l = prod_j (-i c_2j c_2j+1) over that end's n_v modes.  Hence
       R_nm = <psi_n(G)|psi_m(G^(l))> / <psi_n(G)|psi_m(G)>
   is the expectation of P_l (on the right) in the Gaussian operator
   sigma_G X_nm, sigma_G the reduced state of the twisted sites on the virtual
   modes (covariance D_G, the virtual block of Gamma_{A(G)}) and X_nm the bond
   operator of covariance Gamma_X (as in oracle.weight).  By Wick's theorem,
   with <c_a c_b> = delta_ab - i Gamma_ab,
       R_nm = (-1)^{n_v} Pf(Gamma_O[S, S])
   over the 2 n_v Majoranas S of that end, and composing the two Gaussian
   operators (Gamma_X^2 = -1) gives
       Gamma_O = i 1 - (1 + i D_G) W (1 + i Gamma_X),  W = (D_G + Gamma_X)^{-1}.
   Then f_E(G) = sum_nm lambda_n^* lambda_m N_nm(G) R_nm / N(G) with N_nm(G)
   from oracle.weight.

Pinned (tests/test_oracle_electric.py): the covariance route against the Fock
route on 2x2 Z2 lattices (K = 1, 2; every link; random configurations) and
on the 1x1 torus with n_v = 2 (every configuration);
gauge invariance of f_E; the exhaustive <X_l> on the 2x2 lattice is real and
at most 1 in modulus.
"""
from __future__ import annotations

import numpy as np

from . import fock, weight
from .pfaffian import pfaffian

Z2 = 0


def flipped(links: np.ndarray, l: int) -> np.ndarray:
    g = np.array(links, dtype=float).copy()
    g[l] = -g[l]
    return g


def f_electric_fock(fp: fock.FockPEPS, links: np.ndarray, l: int) -> complex:
    """f_E(G) for link l from explicit vectors (the definition)."""
    lam = fp.p.lam
    v = (lam[:, None] * fp.psi(links)).sum(axis=0)
    w = (lam[:, None] * fp.psi(flipped(links, l))).sum(axis=0)
    return complex(np.vdot(v, w) / np.vdot(v, v))


class Electric:
    """Covariance route to f_E(G) for every link of a Z2 problem."""

    def __init__(self, p):
        if p.group != Z2:
            raise ValueError("the link-flip observable is defined for Z2")
        self.p = p
        self.W = weight.Weights(p)
        m_s = p.m_s
        self.virt = np.array([i for i in range(m_s * p.V) if i % m_s >= 2])
        pos = -np.ones(m_s * p.V, dtype=int)
        pos[self.virt] = np.arange(self.virt.size)
        h = 2 * p.n_v
        self.S = [pos[np.array(ix[:h])] for ix in weight.link_majoranas(p)]
        self.GX = {nm: g[np.ix_(self.virt, self.virt)] for nm, g in self.W.GX.items()}

    def ratios(self, links: np.ndarray) -> np.ndarray:
        """R[n, m, l] = <psi_n(G)|psi_m(G^(l))> / <psi_n(G)|psi_m(G)>."""
        p = self.p
        O = weight.twist_matrix(p, links)
        D = (O.T @ self.W.GA @ O)[np.ix_(self.virt, self.virt)]
        one = np.eye(D.shape[0])
        out = np.zeros((p.K, p.K, p.n_links), dtype=complex)
        for n in range(p.K):
            for m in range(p.K):
                GX = self.GX[n, m]
                Wi = np.linalg.inv(D + GX)
                GO = 1j * one - (one + 1j * D) @ Wi @ (one + 1j * GX)
                for l in range(p.n_links):
                    s = self.S[l]
                    out[n, m, l] = (-1) ** p.n_v * pfaffian(GO[np.ix_(s, s)])
        return out

    def f_electric(self, links: np.ndarray) -> np.ndarray:
        """f_E(G) for every link (complex; its expectation over p(G) is real)."""
        p = self.p
        lnm = self.W.log_n_matrix(links)
        ref = lnm.real.max()
        Nnm = np.exp(lnm - ref)
        w = np.conj(p.lam)[:, None] * p.lam[None, :] * Nnm
        R = self.ratios(links)
        return np.einsum("nm,nml->l", w, R) / w.sum()

    def expectation_exhaustive(self, configs: np.ndarray) -> np.ndarray:
        """<X_l> = sum_G p(G) f_E(G) over an explicit list of configurations."""
        num = np.zeros(self.p.n_links, dtype=complex)
        logs, fs = [], []
        for G in configs:
            logs.append(self.W.log_norm(G))
            fs.append(self.f_electric(G))
        logs = np.array(logs)
        wts = np.exp(logs - logs.max())
        for wt, f in zip(wts, fs):
            num += wt * f
        return num / wts.sum()
