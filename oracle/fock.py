"""Brute-force Fock-space construction of the gauged superposition of
Gaussian PEPS (Sec. 3, Sec. 3.1, Sec. 4) on tiny lattices.

Everything here is the definition written out on explicit state vectors:

* Jordan-Wigner occupation basis; mode k of an n-mode register is bit
  (n-1-k) of the basis index, so a tensor product of blocks of consecutive
  modes is a Kronecker product of their vectors.
* Majoranas c_{2i} = psi_i + psi_i^dag, c_{2i+1} = -i (psi_i - psi_i^dag)
  (Sec. 3.2) act as signed bit flips.
* A pure Gaussian state with covariance Gamma (Gamma_ab = (i/2)<[c_a,c_b]>,
  Sec. 3.2) is the ground state of H = -(i/4) sum_ab Gamma_ab c_a c_b.
* The gauge twist U(G) (Sec. 3.1) multiplies every basis state by
  exp(i theta_l sum_j q_j n_j) over the source-end modes of every link
  (Z2: (-1)^(sum_j n_j) for g_l = -1).  SU(2) acts on each doublet of a
  source end (modes 2k, 2k + 1) by exp(sum_{alpha beta} (log u)_{beta alpha}
  psi^dag_beta psi_alpha), so that psi^dag_alpha -> sum_beta psi^dag_beta
  u_{beta alpha} (Sec. 2, the Wigner matrix acting on the fermion modes).
* psi_n(G) = <B_n| U(G) |A> (Sec. 4): |A> is the product of site states, <B_n|
  the product of link states, the contraction runs over the virtual modes;
  N_nm(G) = <psi_n(G)|psi_m(G)> and N(G) = || sum_n lambda_n psi_n(G) ||^2.
* Bond phases follow the convention <B_n|B_0> real positive (Sec. 5), with
  B_0 := B_1 and the per-link factors each made real positive.

Pinned (tests/test_oracle_fock.py): vacuum covariance, Gamma -> state ->
Gamma round trip, the SU(2) twist's action on creators
(tests/test_oracle_su2.py), the worked two-mode contraction of App. C, overlaps against
|<a|b>|^2 computed from explicit vectors, fermionic reordering against
explicit operator products.
"""
from __future__ import annotations

import functools
import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg

Z2, U1, SU2 = 0, 1, 2


@functools.lru_cache(maxsize=32)
def majoranas(n: int):
    """Sparse matrices of the 2n Majoranas on n modes."""
    dim = 1 << n
    idx = np.arange(dim)
    ops = []
    for i in range(n):
        bit = n - 1 - i
        occ = (idx >> bit) & 1
        # Jordan-Wigner string over modes 0..i-1 (higher bits)
        before = idx >> (bit + 1)
        par = np.zeros(dim, dtype=np.int64)
        t = before.copy()
        while t.any():
            par ^= t & 1
            t >>= 1
        js = 1 - 2 * par
        tgt = idx ^ (1 << bit)
        c0 = sp.csr_matrix((js.astype(complex), (tgt, idx)), shape=(dim, dim))
        # c_{2i+1} |n> = i * js * (1 - 2 n_i) |n ^ e_i>
        c1 = sp.csr_matrix((1j * js * (1 - 2 * occ), (tgt, idx)), shape=(dim, dim))
        ops += [c0, c1]
    return ops


def state_from_covariance(gamma: np.ndarray) -> np.ndarray:
    """Pure Gaussian state with covariance gamma (ground state of
    -(i/4) sum Gamma_ab c_a c_b)."""
    n = gamma.shape[0] // 2
    cs = majoranas(n)
    dim = 1 << n
    H = sp.csr_matrix((dim, dim), dtype=complex)
    for a in range(2 * n):
        for b in range(a + 1, 2 * n):
            if gamma[a, b] != 0.0:
                # Gamma_ab c_a c_b + Gamma_ba c_b c_a = 2 Gamma_ab c_a c_b  (a != b)
                H = H + (-0.5j * gamma[a, b]) * (cs[a] @ cs[b])
    w, v = np.linalg.eigh(H.toarray())
    if w.size > 1 and w[1] - w[0] < 1e-8:
        raise ValueError("covariance is not pure: degenerate ground state")
    return v[:, 0]


def covariance_of(state: np.ndarray, bra: np.ndarray | None = None) -> np.ndarray:
    """(i/2) <bra|[c_a,c_b]|state> / <bra|state>; bra = state gives the
    covariance, another bra the transition covariance."""
    n = int(round(np.log2(state.size)))
    cs = majoranas(n)
    if bra is None:
        bra = state
    norm = np.vdot(bra, state)
    cv = [c @ state for c in cs]
    G = np.zeros((2 * n, 2 * n), dtype=complex)
    for a in range(2 * n):
        ca_bra = cs[a].conj().T @ bra  # <bra| c_a = (c_a^dag |bra>)^dag, c_a Hermitian
        for b in range(2 * n):
            if a != b:
                G[a, b] = 1j * np.vdot(ca_bra, cv[b]) / norm  # (i/2)<[c_a,c_b]> = i<c_a c_b>
    return G


def reorder(state: np.ndarray, perm) -> np.ndarray:
    """Rewrite a state given in mode order (0..n-1) in the new order where new
    mode k is old mode perm[k]; fermionic signs from reordering the creation
    operators of every basis state."""
    perm = np.asarray(perm)
    n = perm.size
    newpos = np.empty(n, dtype=np.int64)
    newpos[perm] = np.arange(n)
    idx = np.arange(1 << n)
    occ = [((idx >> (n - 1 - k)) & 1).astype(np.int8) for k in range(n)]
    parity = np.zeros(1 << n, dtype=np.int8)
    new_idx = np.zeros(1 << n, dtype=np.int64)
    for i in range(n):
        new_idx |= occ[i].astype(np.int64) << (n - 1 - newpos[i])
        for j in range(i + 1, n):
            if newpos[i] > newpos[j]:
                parity ^= occ[i] & occ[j]
    out = np.zeros_like(state)
    out[new_idx] = state * (1 - 2 * parity.astype(np.int64))
    return out


def fermion_ops(n: int):
    """(annihilators, creators) of n modes from the Majoranas:
    psi = (c_{2i} + i c_{2i+1}) / 2, psi^dag = (c_{2i} - i c_{2i+1}) / 2."""
    cs = majoranas(n)
    ann = [(cs[2 * i] + 1j * cs[2 * i + 1]) * 0.5 for i in range(n)]
    cre = [(cs[2 * i] - 1j * cs[2 * i + 1]) * 0.5 for i in range(n)]
    return ann, cre


def contract(state: np.ndarray, phys, virt, bra_virt: np.ndarray) -> np.ndarray:
    """<B| state over the modes `virt` (an even bra given in the order of
    `virt`); returns the amplitudes over the modes `phys` in their order.
    The state is first rewritten in the order phys + virt."""
    Phi = reorder(state, list(phys) + list(virt))
    Phi = Phi.reshape(1 << len(phys), -1)
    return Phi @ np.conj(bra_virt)


class Lattice:
    """Mode bookkeeping for the Fock construction."""

    def __init__(self, L: int, n_v: int):
        self.L, self.n_v = L, n_v
        self.V = L * L
        self.mps = 1 + 4 * n_v               # modes per site
        self.n_modes = self.V * self.mps

    def site_mode(self, s, e=None, j=0):
        """Global mode index: physical mode (e None) or virtual mode j of end e."""
        base = s * self.mps
        return base if e is None else base + 1 + e * self.n_v + j

    def neighbour(self, s, d):
        x, y = s % self.L, s // self.L
        return (y * self.L + (x + 1) % self.L) if d == 0 else (((y + 1) % self.L) * self.L + x)

    def link_modes(self, l):
        """(source-end modes, target-end modes) of link l."""
        s, d = l // 2, l % 2
        t = self.neighbour(s, d)
        a = [self.site_mode(s, 2 * d + 1, j) for j in range(self.n_v)]
        b = [self.site_mode(t, 2 * d, j) for j in range(self.n_v)]
        return a, b


def bond_states(gamma_bond: np.ndarray) -> np.ndarray:
    """Per-link Fock vectors of all K bond states, phases fixed by
    <b_n|b_0> > 0 (b_0 = b_1), and b_0 by its largest amplitude > 0."""
    K, nl = gamma_bond.shape[:2]
    out = []
    for n in range(K):
        row = []
        for l in range(nl):
            v = state_from_covariance(gamma_bond[n, l])
            if n == 0:
                k = np.argmax(np.abs(v))
                v = v * (np.abs(v[k]) / v[k])
            else:
                ov = np.vdot(v, out[0][l])      # <b_n|b_0>
                v = v * (ov / abs(ov))          # makes <b_n|b_0> real positive
            row.append(v)
        out.append(row)
    return np.array(out)


class FockPEPS:
    """Explicit-vector PEPS: psi_n(G) for every bond state n."""

    def __init__(self, problem):
        p = problem
        self.p = p
        self.lat = Lattice(p.L, p.n_v)
        lat = self.lat
        if lat.n_modes > 22:
            raise ValueError("Fock construction limited to <= 22 modes")
        # |A> = kron of site states (site-major order, site modes consecutive)
        A = np.ones(1, dtype=complex)
        for s in range(p.V):
            A = np.kron(A, state_from_covariance(p.gamma_site[s]))
        self.A = A
        n = lat.n_modes
        self.phys = [lat.site_mode(s) for s in range(p.V)]
        self.virt = [m for m in range(n) if m not in set(self.phys)]
        # occupation of every mode for every basis index
        idx = np.arange(1 << n)
        self.occ = np.array([((idx >> (n - 1 - k)) & 1) for k in range(n)], dtype=np.int8)
        # <B_n| on the virtual modes in site-major virtual order
        bs = bond_states(p.gamma_bond)
        link_order = []
        for l in range(p.n_links):
            a, b = lat.link_modes(l)
            link_order += a + b
        perm = list(link_order)
        # state in link-major order -> site-major virtual order
        new_order = self.virt                  # new mode k = global mode virt[k]
        old_index = {m: k for k, m in enumerate(perm)}
        perm_old = [old_index[m] for m in new_order]
        self.B = []
        for nb in range(p.K):
            v = np.ones(1, dtype=complex)
            for l in range(p.n_links):
                v = np.kron(v, bs[nb, l])
            self.B.append(reorder(v, perm_old))
        self.B = np.array(self.B)

    def twist_phase(self, links: np.ndarray) -> np.ndarray:
        """Diagonal of U(G) in the occupation basis."""
        p, lat = self.p, self.lat
        ang = np.zeros(self.A.size)
        for l in range(p.n_links):
            a, _ = lat.link_modes(l)
            for j, m in enumerate(a):
                if p.group == Z2:
                    if links[l] == -1:
                        ang += np.pi * self.occ[m]
                else:
                    ang += float(links[l]) * int(p.q_src[j]) * self.occ[m]
        if p.group == Z2:
            return 1.0 - 2.0 * (np.round(ang / np.pi).astype(np.int64) % 2)
        return np.exp(1j * ang)

    def twisted_state(self, links: np.ndarray) -> np.ndarray:
        """U(G) |A>."""
        if self.p.group != SU2:
            return self.twist_phase(links) * self.A
        from .weight import su2_matrix
        ann, cre = fermion_ops(self.lat.n_modes)
        Phi = self.A.astype(complex)
        for l in range(self.p.n_links):
            a, _ = self.lat.link_modes(l)
            lg = scipy.linalg.logm(su2_matrix(links[l]))
            for k in range(self.p.n_v // 2):
                m = (a[2 * k], a[2 * k + 1])
                H = sum(lg[b, al] * (cre[m[b]] @ ann[m[al]]) for b in range(2) for al in range(2))
                Phi = scipy.sparse.linalg.expm_multiply(sp.csr_matrix(H), Phi)
        return Phi

    def psi(self, links: np.ndarray) -> np.ndarray:
        """(K, 2^V) physical amplitudes psi_n(G) = <B_n| U(G) |A>."""
        Phi = self.twisted_state(links)
        return np.array([contract(Phi, self.phys, self.virt, b) for b in self.B])

    def n_matrix(self, links: np.ndarray) -> np.ndarray:
        """N_nm(G) = <psi_n|psi_m>."""
        ps = self.psi(links)
        return ps.conj() @ ps.T

    def norm(self, links: np.ndarray) -> float:
        """N(G) = sum_nm lambda_n^* lambda_m N_nm(G)."""
        ps = self.psi(links)
        v = (self.p.lam[:, None] * ps).sum(axis=0)
        return float(np.vdot(v, v).real)
