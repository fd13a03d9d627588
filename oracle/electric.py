"""Electric-field observables of Sec. 5.3: the Z2 link flip and the U(1) and
SU(2) Casimirs J_l^2.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 5.3 writes <J_l^2> = sum_G p(G) f_E(G) with the single-link integral
    f_E(G) = int dg <G|J_l^2|g; G> sum_nm lambda_n^* lambda_m <psi_n(G)|psi_m(g; G)> / N(G),
|g; G> being G with link l set to g.

Z2: the electric term of a link is a linear function of the flip X_l
|G> = |G^(l)> (G^(l): g_l -> -g_l), so the integral has the diagonal term
(value 1) and the flip term
    f_X(G) = sum_nm lambda_n^* lambda_m <psi_n(G)|psi_m(G^(l))> / N(G),
which is what this module returns for Z2 (the Hamiltonian's coefficients are
left out).

U(1): in the angle basis J = -i d/dtheta, so the integral is -d^2/dtheta'^2 of
the ket's overlap at theta' = theta_l.  The ket depends on theta' only
through the twist exp(i theta' Q_l) of the source-end modes,
Q_l = sum_j q_j n_j, so the overlap is a trigonometric polynomial with
frequencies |Q| <= n_v and
    f_E(G) = sum_nm lambda_n^* lambda_m <psi_n(G)| Q_l^2 |psi_m(G)>_ket / N(G),
Q_l^2 inserted on the ket's source-end modes before the contraction.

SU(2): J^2 = sum_a J_a J_a with J_a the generators of right translations
g -> g exp(i eps sigma_a / 2) of the ket's link (the left and right Casimirs
agree); the twist of g exp(i eps sigma_a / 2) is U(g) exp(i eps Q^a), so
f_E inserts sum_a (Q^a)^2, Q^a = psi^dag (sigma_a / 2) psi on the source
doublet, which is (3/4)(n_0 + n_1 - 2 n_0 n_1).

Two routes:

1. Fock (the definition, tiny lattices): explicit vectors.  Z2: psi(G^(l)).
   U(1): the single-link integral itself, by quadrature over theta' on a
   grid of 8 angles, exact for frequencies |Q| <= 3.  SU(2): the Laplacian
   along each generator, by quadrature over eps on 8 points of [0, 4 pi).
2. Covariance: the insertion acts on the source-end Majoranas S of link l
   (the end that carries the twist).  Composing the sites' virtual state
   (covariance D_G, the virtual block of Gamma_{A(G)}) with the bond operator
   X_nm (covariance Gamma_X, Gamma_X^2 = -1) gives a Gaussian operator whose
   normalised covariance is
       Gamma_O = i 1 - (1 + i D_G) W (1 + i Gamma_X),  W = (D_G + Gamma_X)^{-1},
   and Wick's theorem with <c_a c_b> = -i Gamma_O[a, b] (a != b) gives
     Z2:   R_nm = (-1)^{n_v} Pf(Gamma_O[S, S])   (the parity of the end),
     SU(2): R_nm = (3/4) (<n_0> + <n_1> - 2 <n_0 n_1>),
     U(1): R_nm = <Q_l^2> = sum_j q_j^2 <n_j> + 2 sum_{j<k} q_j q_k <n_j n_k>,
           <n_j> = (1 + G_{2j,2j+1}) / 2,
           <n_j n_k> = (1 + G_{2j,2j+1} + G_{2k,2k+1} + Pf G[2j,2j+1,2k,2k+1]) / 4,
   G = Gamma_O[S, S].  Then f = sum_nm lambda_n^* lambda_m N_nm(G) R_nm / N(G)
   with N_nm(G) from oracle.weight.

Pinned (tests/test_oracle_electric.py): Z2: the covariance route against the
Fock route on 2x2 lattices (K = 1, 2; every link; random configurations) and
on the 1x1 torus with n_v = 2 (every configuration); gauge invariance; the
exhaustive <X_l> on the 1x1 torus against explicit vectors, and on the 2x2
lattice real and at most 1 in modulus.  U(1): the covariance route against
the quadrature of the definition (2x2, K = 1, 2; 1x1, n_v = 2); gauge
invariance; <J_l^2> over p(G) on the 1x1 torus (exact product quadrature) is
real and non-negative.  SU(2): the covariance route against the quadrature
of the definition (1x1, K = 1, 2); gauge invariance.  U(1) field <J_l> (the
insertion of Q_l, -i d/dtheta'): against the quadrature of the definition,
and Gauss's law in every configuration, sum_out <J> - sum_in <J> + q_s <n_s>
= 0 with the density from oracle.fermionic.
"""
from __future__ import annotations

import numpy as np

from . import fock, weight
from .pfaffian import pfaffian

Z2, U1, SU2 = 0, 1, 2
N_QUAD = 8
_PAULI = [np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]]),
          np.array([[1, 0], [0, -1]], dtype=complex)]


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


def f_electric_u1_fock(fp: fock.FockPEPS, links: np.ndarray, l: int) -> complex:
    """U(1) f_E(G) for link l: the single-link integral of <G|J^2|g; G>
    against the overlap, by quadrature over the ket's angle (the overlap is a
    trigonometric polynomial of degree <= n_v <= 2, so 8 points are exact)."""
    p = fp.p
    lam = p.lam
    v = (lam[:, None] * fp.psi(links)).sum(axis=0)
    th = 2.0 * np.pi * np.arange(N_QUAD) / N_QUAD
    phi = np.zeros(N_QUAD, dtype=complex)
    for k, t in enumerate(th):
        g = np.array(links, dtype=float).copy()
        g[l] = t
        phi[k] = np.vdot(v, (lam[:, None] * fp.psi(g)).sum(axis=0))
    Q = np.fft.fftfreq(N_QUAD, 1.0 / N_QUAD)           # integer frequencies
    c = np.fft.fft(phi) / N_QUAD                        # phi(t) = sum_Q c_Q e^{i Q t}
    return complex(np.sum(Q ** 2 * c * np.exp(1j * Q * links[l])) / np.vdot(v, v))


def f_field_u1_fock(fp: fock.FockPEPS, links: np.ndarray, l: int) -> complex:
    """U(1) electric field <J_l> for link l: -i d/dtheta' of the ket's overlap
    at theta' = theta_l (the single-link integral with <G|J|g; G>), by the
    same exact quadrature as f_electric_u1_fock."""
    p = fp.p
    lam = p.lam
    v = (lam[:, None] * fp.psi(links)).sum(axis=0)
    th = 2.0 * np.pi * np.arange(N_QUAD) / N_QUAD
    phi = np.zeros(N_QUAD, dtype=complex)
    for k, t in enumerate(th):
        g = np.array(links, dtype=float).copy()
        g[l] = t
        phi[k] = np.vdot(v, (lam[:, None] * fp.psi(g)).sum(axis=0))
    Q = np.fft.fftfreq(N_QUAD, 1.0 / N_QUAD)
    c = np.fft.fft(phi) / N_QUAD
    return complex(np.sum(Q * c * np.exp(1j * Q * links[l])) / np.vdot(v, v))


def f_electric_su2_fock(fp: fock.FockPEPS, links: np.ndarray, l: int) -> complex:
    """SU(2) f_E(G) for link l: the Casimir J^2 = sum_a J_a J_a, J_a the
    generators of right translations g -> g exp(i eps sigma_a / 2) of the
    ket's link, i.e. -sum_a d^2/d eps_a^2 of the overlap at eps = 0.  Along
    each generator the overlap is a trigonometric polynomial in eps / 2 of
    degree <= 2 (period 4 pi), so 8 points on [0, 4 pi) give it exactly."""
    import scipy.linalg
    from .weight import su2_matrix
    p = fp.p
    lam = p.lam
    v = (lam[:, None] * fp.psi(links)).sum(axis=0)
    u = su2_matrix(links[l])
    k = np.fft.fftfreq(N_QUAD, 1.0 / N_QUAD)           # phi(e) = sum_k c_k e^{i k e / 2}
    tot = 0.0 + 0.0j
    for sig in _PAULI:
        phi = np.zeros(N_QUAD, dtype=complex)
        for j in range(N_QUAD):
            w = u @ scipy.linalg.expm(0.5j * (4.0 * np.pi * j / N_QUAD) * sig)
            g = np.array(links, dtype=float).copy()
            g[l] = [w[0, 0].real, w[0, 1].imag, w[0, 1].real, w[0, 0].imag]
            phi[j] = np.vdot(v, (lam[:, None] * fp.psi(g)).sum(axis=0))
        c = np.fft.fft(phi) / N_QUAD
        tot += np.sum((k / 2.0) ** 2 * c)
    return complex(tot / np.vdot(v, v))


class Electric:
    """Covariance route to f_E(G) for every link (Z2 flip, U(1) or SU(2) J^2)."""

    def __init__(self, p):
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
        """R[n, m, l]: the insertion's normalised expectation for pair (n, m);
        Z2: <psi_n(G)|psi_m(G^(l))> / <psi_n(G)|psi_m(G)>."""
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
                    out[n, m, l] = self._insertion(GO[np.ix_(s, s)])
        return out

    def _insertion(self, G) -> complex:
        """Normalised expectation of the insertion on one source end."""
        p = self.p
        if p.group == Z2:
            return (-1) ** p.n_v * pfaffian(G)
        if p.group == SU2:
            # sum_a (Q^a)^2 on one doublet = (3/4)(n_0 + n_1 - 2 n_0 n_1)
            occ = [(1.0 + G[2 * j, 2 * j + 1]) / 2.0 for j in range(2)]
            pair = (1.0 + G[0, 1] + G[2, 3] + pfaffian(G)) / 4.0
            return 0.75 * (occ[0] + occ[1] - 2.0 * pair)
        q = p.q_src
        occ = [(1.0 + G[2 * j, 2 * j + 1]) / 2.0 for j in range(p.n_v)]
        val = sum(q[j] ** 2 * occ[j] for j in range(p.n_v))
        for j in range(p.n_v):
            for k in range(j + 1, p.n_v):
                ix = [2 * j, 2 * j + 1, 2 * k, 2 * k + 1]
                pair = (1.0 + G[2 * j, 2 * j + 1] + G[2 * k, 2 * k + 1] + pfaffian(G[np.ix_(ix, ix)])) / 4.0
                val = val + 2 * q[j] * q[k] * pair
        return val

    def field_ratios(self, links: np.ndarray) -> np.ndarray:
        """F[n, m, l]: the normalised expectation of the twist charge
        Q_l = sum_j q_j n_j inserted on the ket for pair (n, m),
        <Q_l> = sum_j q_j (1 + G_{2j,2j+1}) / 2 with G = Gamma_O[S, S]."""
        p = self.p
        if p.group != U1:
            raise ValueError("the electric field insertion is defined for U(1)")
        O = weight.twist_matrix(p, links)
        D = (O.T @ self.W.GA @ O)[np.ix_(self.virt, self.virt)]
        one = np.eye(D.shape[0])
        out = np.zeros((p.K, p.K, p.n_links), dtype=complex)
        for n in range(p.K):
            for m in range(p.K):
                GX = self.GX[n, m]
                GO = 1j * one - (one + 1j * D) @ np.linalg.inv(D + GX) @ (one + 1j * GX)
                for l in range(p.n_links):
                    G = GO[np.ix_(self.S[l], self.S[l])]
                    out[n, m, l] = sum(p.q_src[j] * (1.0 + G[2 * j, 2 * j + 1]) / 2.0 for j in range(p.n_v))
        return out

    def field(self, links: np.ndarray) -> np.ndarray:
        """U(1) electric field <J_l> per link (complex per configuration): the
        pairs' field_ratios combined with lambda_n^* lambda_m N_nm(G) / N(G)."""
        p = self.p
        lnm = self.W.log_n_matrix(links)
        Nnm = np.exp(lnm - lnm.real.max())
        w = np.conj(p.lam)[:, None] * p.lam[None, :] * Nnm
        return np.einsum("nm,nml->l", w, self.field_ratios(links)) / w.sum()

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
        """sum_G p(G) f_E(G) over an explicit list of configurations (Z2: all
        of them; U(1): a product grid that integrates exactly)."""
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
