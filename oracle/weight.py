"""Covariance-matrix route to N_nm(G), N(G) and p(G) (Sec. 3.2, Sec. 5).

Steps, in the paper's order and notation:

1. Gamma_A = (+)_s Gamma_{A,s} over the full (physical + virtual) Majorana
   space, site-major with each site in the layout
   [phys(2) | end -x | end +x | end -y | end +y].
2. O(G): identity except on the source-end Majoranas of every link, where
   Z2 gives g_l * 1 and U(1) gives, per mode of charge q, the rotation
   [[cos q theta, sin q theta], [-sin q theta, cos q theta]] (this is
   U(G) c_a U(G)^dag = O_ab c_b for U(G) = prod exp(i theta q n)).  SU(2)
   acts on each doublet (modes 2k, 2k + 1) of the end by the Gaussian unitary
   with U psi^dag_j U^dag = sum_k psi^dag_k u_kj, u the link's 2 x 2 matrix,
   whose Majorana rotation has rows
   c_2j -> sum_k Re u_kj c_2k + Im u_kj c_2k+1 and
   c_2j+1 -> sum_k -Im u_kj c_2k + Re u_kj c_2k+1 (the U(1) rotation for a
   diagonal u).
   Gamma_{A(G)} = O^T Gamma_A O  (Sec. 5).
3. Numerator tr(rho_{A(G)} (1 x rho_{B_n})(1 x rho_{B_m})): the product of
   the two bond density matrices is Gaussian (Bravyi-Gosset),
   rho_{B_n} rho_{B_m} = tr(rho_{B_n} rho_{B_m}) X_nm with
   X_nm = |B_n><B_m| / <B_m|B_n>; for a pure Gaussian rho and a Gaussian
   operator X of covariance Gamma_X on n_tot modes,
   tr(rho X) = 2^{-n_tot} Pf(Gamma_rho) Pf(Gamma_rho + Gamma_X)  (Sec. 3.2
   gives the Hermitian case tr(rho1 rho2) = Pf((Gamma1 + Gamma2)/2) up to
   this sign/normalisation reading).  The identity on the physical modes is
   2^{n_ph} times the state of covariance 0.
4. Denominator <B_n|B_m> with the reference B_0 and <B_n|B_0> real positive
   (Sec. 5).  Per-link factors are taken from explicit link-space vectors
   (oracle.fock), so the phase convention is applied literally.
5. N_nm(G) = numerator / <B_n|B_m>,  N(G) = sum_nm lambda_n^* lambda_m
   N_nm(G), p(G) = N(G) / sum_G N(G)  (Sec. 5, Sec. 5.1).

The transition covariance of X_nm on one link is computed from its
definition (i/2) tr(X [c_a, c_b]) on the 2^(2 n_v)-dimensional link space.

Pinned (tests/test_oracle_weight.py): against the brute-force Fock
contraction (oracle.fock) for Z2 and U(1), K = 1, 2, 3; invariants
(N >= 0, Im N = 0, N_mn = conj N_nm, gauge invariance, lambda phase
invariance, B_2 = B_1 => N = |lambda_1 + lambda_2|^2 N_11); exhaustive
normalisation on the 2x2 Z2 lattice; for pure site covariances the
full-space Pfaffian equals the virtual-only Pf(D_G + Gamma_X) times the fixed
sign prod_s sign(Gamma_s[0, 1]) (Z2, U(1), SU(2), L = 1..4; not for a mixed
one).
SU(2) (tests/test_oracle_su2.py): the doublet rotation against explicit
Fock operators, N_nm against the Fock contraction on the 1x1 torus, the U(1)
code on the subgroup exp(i theta sigma_z), gauge invariance under
g_l -> h_t^dag g_l h_s.
The absolute U(1) and SU(2) normalisations sum_G N(G) (integrals over the
group) are parity unpinned; only ratios and observables are compared.
"""
from __future__ import annotations

import numpy as np

from . import fock
from .pfaffian import log_pfaffian

Z2, U1, SU2 = 0, 1, 2


def su2_matrix(q) -> np.ndarray:
    """a0 1 + i (a1 sigma_x + a2 sigma_y + a3 sigma_z) for a unit quaternion."""
    a0, a1, a2, a3 = (float(x) for x in q)
    return np.array([[complex(a0, a3), complex(a2, a1)], [complex(-a2, a1), complex(a0, -a3)]])


def doublet_rotation(u) -> np.ndarray:
    """Majorana rotation (4 x 4) of the Gaussian unitary psi^dag -> psi^dag u
    on one doublet."""
    R = np.zeros((4, 4))
    for j in range(2):
        for k in range(2):
            R[2 * j, 2 * k], R[2 * j, 2 * k + 1] = u[k, j].real, u[k, j].imag
            R[2 * j + 1, 2 * k], R[2 * j + 1, 2 * k + 1] = -u[k, j].imag, u[k, j].real
    return R


def twist_matrix(p, links) -> np.ndarray:
    """O(G) on the full site-major Majorana space."""
    m_s, n_v, L = p.m_s, p.n_v, p.L
    n = m_s * p.V
    O = np.eye(n)
    for l in range(p.n_links):
        s, d = l // 2, l % 2
        base = s * m_s + 2 + (2 * d + 1) * 2 * n_v
        if p.group == SU2:
            R = doublet_rotation(su2_matrix(links[l]))
            for k in range(n_v // 2):
                i0 = base + 4 * k
                O[i0:i0 + 4, i0:i0 + 4] = R
            continue
        for j in range(n_v):
            i0 = base + 2 * j
            if p.group == Z2:
                O[i0, i0] = O[i0 + 1, i0 + 1] = float(links[l])
            else:
                ph = int(p.q_src[j]) * float(links[l])
                c, s_ = np.cos(ph), np.sin(ph)
                O[i0, i0], O[i0, i0 + 1], O[i0 + 1, i0], O[i0 + 1, i0 + 1] = c, s_, -s_, c
    return O


def gamma_A(p) -> np.ndarray:
    n = p.m_s * p.V
    G = np.zeros((n, n))
    for s in range(p.V):
        G[s * p.m_s:(s + 1) * p.m_s, s * p.m_s:(s + 1) * p.m_s] = p.gamma_site[s]
    return G


class BondData:
    """Per-link bond quantities from explicit link-space vectors."""

    def __init__(self, p):
        self.p = p
        self.vec = fock.bond_states(p.gamma_bond)      # (K, 2V, 2^(2 n_v))
        K, nl = p.K, p.n_links
        r = p.r
        self.G = np.zeros((K, K, nl, r, r), dtype=complex)   # covariance of |b_n><b_m|/<b_m|b_n>
        self.ov = np.zeros((K, K, nl), dtype=complex)         # <b_m|b_n>
        for n in range(K):
            for m in range(K):
                for l in range(nl):
                    bn, bm = self.vec[n, l], self.vec[m, l]
                    self.ov[n, m, l] = np.vdot(bm, bn)
                    self.G[n, m, l] = fock.covariance_of(bn, bra=bm)

    def log_overlap(self, n, m) -> complex:
        """log <B_m|B_n> (product over links, B_0 phase convention)."""
        return complex(np.sum(np.log(self.ov[n, m])))

    def embedded(self, n, m) -> np.ndarray:
        """Gamma_X of X_nm on the full Majorana space (zero on physical)."""
        p = self.p
        n_full = p.m_s * p.V
        out = np.zeros((n_full, n_full), dtype=complex)
        idx = link_majoranas(p)
        for l in range(p.n_links):
            ii = idx[l]
            out[np.ix_(ii, ii)] += self.G[n, m, l]
        return out


def link_majoranas(p):
    """Full-space Majorana indices of each link, order [source end | target end]."""
    out = []
    L, n_v, m_s = p.L, p.n_v, p.m_s
    for l in range(p.n_links):
        s, d = l // 2, l % 2
        x, y = s % L, s // L
        t = (y * L + (x + 1) % L) if d == 0 else (((y + 1) % L) * L + x)
        a0 = s * m_s + 2 + (2 * d + 1) * 2 * n_v
        b0 = t * m_s + 2 + (2 * d) * 2 * n_v
        out.append(list(range(a0, a0 + 2 * n_v)) + list(range(b0, b0 + 2 * n_v)))
    return out


class Weights:
    """log N_nm(G) and log N(G) by the covariance route."""

    def __init__(self, p):
        self.p = p
        self.GA = gamma_A(p)
        self.bond = BondData(p)
        la, ph = log_pfaffian(self.GA)
        self.log_pf_A = complex(la + np.log(complex(ph)))
        self.n_virt = 4 * p.n_v * p.V               # virtual complex modes
        self.GX = {}
        for n in range(p.K):
            for m in range(p.K):
                self.GX[n, m] = self.bond.embedded(n, m)

    def log_n_nm(self, links, n, m) -> complex:
        """log N_nm(G) (complex; exp gives N_nm)."""
        O = twist_matrix(self.p, links)
        GAG = O.T @ self.GA @ O
        la, ph = log_pfaffian(GAG + self.GX[n, m])
        log_tr = -self.n_virt * np.log(2.0) + self.log_pf_A + la + np.log(complex(ph))
        # numerator = tr(rho_n rho_m) tr(rho_A X_nm), tr(rho_n rho_m) = |<B_n|B_m>|^2
        lo = self.bond.log_overlap(n, m)           # log <B_m|B_n>
        log_num = 2 * lo.real + log_tr
        log_den = np.conj(lo)                       # log <B_n|B_m>
        return complex(log_num - log_den)

    def log_n_matrix(self, links) -> np.ndarray:
        K = self.p.K
        out = np.zeros((K, K), dtype=complex)
        for n in range(K):
            for m in range(n, K):
                out[n, m] = self.log_n_nm(links, n, m)
                out[m, n] = np.conj(out[n, m])
        return out

    def log_norm(self, links) -> float:
        """log N(G), N(G) = sum_nm lambda_n^* lambda_m N_nm(G); -inf if N <= 0."""
        lnm = self.log_n_matrix(links)
        return combine(lnm, self.p.lam)


def combine(lnm: np.ndarray, lam: np.ndarray) -> float:
    K = lam.size
    a = lnm.real.max()
    s = 0.0 + 0.0j
    for n in range(K):
        for m in range(K):
            s += np.conj(lam[n]) * lam[m] * np.exp(lnm[n, m] - a)
    if s.real <= 0.0:
        return -np.inf
    return float(a + np.log(s.real))

