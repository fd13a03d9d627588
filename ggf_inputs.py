"""Seeded synthetic inputs for the gauged Gaussian fermionic PEPS sampler.

This module is shared by the tests, ``bench.py`` and ``__graft_entry__``.  It
only *generates* problem instances -- the variational parameters of the
Ansatz of Sec. 4 (site covariance Gamma_A, bond covariances Gamma_{B_n},
superposition weights lambda_n, cf. Sec. 5) and link configurations.  It holds
none of the method's arithmetic (no twist, no weight, no ratio, no update):
both the FP64 oracle and the CUDA library consume what it returns.

Conventions (shared input contract, restated in include/ggf.h):

* L x L periodic square lattice, site s = y*L + x, V = L*L sites.
* Link l = 2*s + d, d = 0 (x) / 1 (y), joins the +d end of site s (the
  "source" end, which carries the gauge twist, Sec. 3.1) to the -d end of
  site s + e_d.
* Per site, 1 physical complex fermion and n_v virtual complex modes on each
  of the 4 link ends.  Majoranas c_{2i} = psi_i + psi_i^dag,
  c_{2i+1} = -i (psi_i - psi_i^dag) (Sec. 3.2); site Majorana layout
  [phys(2) | end -x (2 n_v) | end +x | end -y | end +y], m_s = 2 + 8 n_v.
* Covariance Gamma_ab = (i/2) <[c_a, c_b]> (Sec. 3.2); the vacuum of one mode
  is [[0,-1],[1,0]] (the matrix J below).
* Bond covariance per link, layout [source end (2 n_v) | target end (2 n_v)],
  r = 4 n_v Majoranas.
* Group Z2 (link value g = +-1), U(1) (link angle theta in [0, 2 pi)) or
  SU(2) (unit quaternion (a0, a1, a2, a3), the group element
  a0 1 + i (a1 sigma_x + a2 sigma_y + a3 sigma_z); links stored as
  (n_cfg, 2V, 4) float64).
  Under U(1) a mode of charge q picks up the phase exp(i q phi); in Majorana
  space that is the rotation [[cos q phi, sin q phi], [-sin q phi, cos q phi]].
  Charges: physical (-1)^(x+y) (staggered, Sec. 2.4); virtual mode j on a
  source end +1 (j even) / -1 (j odd), on a target end the opposite sign, so
  that every bond pair is neutral.  Under Z2 every mode is odd (the group acts
  as fermion parity) and any Gaussian state is symmetric.
* SU(2) (n_v even): the n_v modes of a link end form n_v / 2 doublets
  (modes 2k, 2k + 1).  A group element u acts on a doublet as
  psi^dag_alpha -> sum_beta psi^dag_beta u_{beta alpha}; source ends carry u,
  target ends its complex conjugate, and the physical mode is a singlet, so
  every bond pair sum_alpha psi^dag_{a alpha} psi^dag_{b alpha} is invariant
  and the site covariance lies in the commutant of that action.  A gauge
  transformation h (one element per site) maps the link (s -> t) to
  h_t^dag g h_s (on the U(1) subgroup exp(i theta sigma_z) this is
  theta + alpha_s - alpha_t, as for U(1)).
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.linalg

Z2, U1, SU2 = 0, 1, 2


@dataclasses.dataclass
class Problem:
    L: int
    group: int            # Z2 or U1
    n_v: int
    K: int
    gamma_site: np.ndarray  # (V, m_s, m_s) float64
    gamma_bond: np.ndarray  # (K, 2V, r, r) float64
    lam: np.ndarray         # (K,) complex128, unit 2-norm
    q_src: np.ndarray       # (n_v,) int32 charges of the source-end modes
    q_phys: np.ndarray      # (V,) int32

    @property
    def V(self):
        return self.L * self.L

    @property
    def n_links(self):
        return 2 * self.V

    @property
    def m_s(self):
        return 2 + 8 * self.n_v

    @property
    def r(self):
        return 4 * self.n_v

    @property
    def N(self):
        """Number of virtual Majoranas on the lattice."""
        return 8 * self.n_v * self.V


def vacuum(n_modes: int) -> np.ndarray:
    return np.kron(np.eye(n_modes), np.array([[0.0, -1.0], [1.0, 0.0]]))


def _rot(phi):
    c, s = np.cos(phi), np.sin(phi)
    return np.array([[c, s], [-s, c]])


def site_charges(n_v: int, q_phys: int) -> np.ndarray:
    """Charges of the 1 + 4 n_v site modes in site layout order."""
    src = np.array([1 if j % 2 == 0 else -1 for j in range(n_v)])
    q = [q_phys]
    for e in range(4):
        q.extend(list(src if e % 2 == 1 else -src))
    return np.array(q, dtype=np.int64)


def _rotation(charges, phi):
    return scipy.linalg.block_diag(*[_rot(q * phi) for q in charges])


def _project_commutant(A, charges, n_phi=16):
    """Group average of a generator over U(1): keeps the symmetric part."""
    out = np.zeros_like(A)
    for k in range(n_phi):
        R = _rotation(charges, 2 * np.pi * k / n_phi)
        out += R.T @ A @ R
    return out / n_phi


def su2(q) -> np.ndarray:
    """2 x 2 unitary of a unit quaternion (a0, a1, a2, a3)."""
    a0, a1, a2, a3 = q
    return np.array([[a0 + 1j * a3, 1j * a1 + a2], [1j * a1 - a2, a0 - 1j * a3]])


def _quat_of(u) -> np.ndarray:
    return np.array([u[0, 0].real, u[0, 1].imag, u[0, 1].real, u[0, 0].imag])


def _majorana_rep(u) -> np.ndarray:
    """Real 2n x 2n rotation R with U c_a U^dag = sum_b R_ab c_b for the
    Gaussian unitary U with U psi^dag_j U^dag = sum_k psi^dag_k u_kj."""
    n = u.shape[0]
    R = np.zeros((2 * n, 2 * n))
    for j in range(n):
        for k in range(n):
            R[2 * j, 2 * k], R[2 * j, 2 * k + 1] = u[k, j].real, u[k, j].imag
            R[2 * j + 1, 2 * k], R[2 * j + 1, 2 * k + 1] = -u[k, j].imag, u[k, j].real
    return R


_PAULI = [np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]]),
          np.array([[1, 0], [0, -1]], dtype=complex)]


def _su2_generators(slots):
    """so(m) generators of the SU(2) action on a mode register; slots lists,
    per doublet, (first Majorana, conjugate?) (other Majoranas untouched)."""
    m = max(a for a, _ in slots) + 4
    gens = []
    for sig in _PAULI:
        Xi = np.zeros((m, m))
        for a, conj in slots:
            # the Majorana representation is real-linear in u, so the
            # generator of u = exp(i t sigma / 2) is the map applied to i sigma / 2
            x = 0.5j * sig
            Xi[a:a + 4, a:a + 4] = _majorana_rep(x.conj() if conj else x)
        gens.append(Xi)
    return gens


def _project_commutant_su2(A, gens):
    """Orthogonal projection of an antisymmetric A onto the antisymmetric
    matrices that commute with every generator (the SU(2) commutant)."""
    n = A.shape[0]
    iu = np.triu_indices(n, 1)
    basis = []
    for a, b in zip(*iu):
        E = np.zeros((n, n))
        E[a, b], E[b, a] = 1.0, -1.0
        basis.append(E)
    M = np.array([np.concatenate([(Xi @ E - E @ Xi).ravel() for Xi in gens]) for E in basis]).T
    _, sv, vt = np.linalg.svd(M)
    null = vt[np.sum(sv > 1e-8 * sv.max()):]
    coef = A[iu]
    coef = null.T @ (null @ coef)
    out = np.zeros((n, n))
    out[iu] = coef
    return out - out.T


def _site_slots_su2(n_v):
    """Doublet slots of one site (layout [phys(2) | -x | +x | -y | +y])."""
    slots = []
    for e in range(4):
        for k in range(n_v // 2):
            slots.append((2 + e * 2 * n_v + 4 * k, e % 2 == 0))   # target ends (-x, -y) conjugate
    return slots


def _bond_slots_su2(n_v):
    return [(4 * k, False) for k in range(n_v // 2)] + [(2 * n_v + 4 * k, True) for k in range(n_v // 2)]


def _rand_antisym(rng, n, scale):
    X = rng.normal(size=(n, n)) * scale
    return np.triu(X, 1) - np.triu(X, 1).T


def max_entangled_bond(n_v: int) -> np.ndarray:
    """Covariance of prod_j (1 + psi^dag_{a,j} psi^dag_{b,j})/sqrt(2) |0>
    built as a pi/4 rotation of the vacuum that mixes end a with end b."""
    r = 4 * n_v
    O = np.eye(r)
    c, s = np.cos(np.pi / 4), np.sin(np.pi / 4)
    for j in range(n_v):
        a0, a1 = 2 * j, 2 * j + 1
        b0, b1 = 2 * n_v + 2 * j, 2 * n_v + 2 * j + 1
        # +pi/4 in the (a0, b0) plane, -pi/4 in the (a1, b1) plane
        O[a0, a0], O[a0, b0], O[b0, a0], O[b0, b0] = c, s, -s, c
        O[a1, a1], O[a1, b1], O[b1, a1], O[b1, b1] = c, -s, s, c
    return O @ vacuum(2 * n_v) @ O.T


def make_problem(L: int, group: int, n_v: int, K: int, seed: int = 20241202,
                 site_scale: float = 0.5, bond_scale: float = 0.05,
                 site_mode: str = "sublattice", bond_mode: str = "uniform",
                 distinct_bonds: bool = True) -> Problem:
    """Seeded instance.  site_mode: 'sublattice' (one Gamma per sublattice)
    or 'random' (independent per site).  bond_mode: 'uniform' (same bond on
    every link) or 'random' (independent per link).  With distinct_bonds
    False, every B_n equals B_1."""
    if group == SU2 and n_v % 2:
        raise ValueError("SU(2) needs n_v even (doublets)")
    rng = np.random.default_rng(seed)
    V = L * L
    m_s, r = 2 + 8 * n_v, 4 * n_v
    q_src = np.array([1 if j % 2 == 0 else -1 for j in range(n_v)], dtype=np.int32)
    q_phys = np.array([(-1) ** ((s % L) + (s // L)) for s in range(V)], dtype=np.int32)

    def one_site(qp):
        A = _rand_antisym(rng, m_s, site_scale)
        if group == U1:
            A = _project_commutant(A, site_charges(n_v, qp))
        elif group == SU2:
            A = _project_commutant_su2(A, _su2_generators(_site_slots_su2(n_v)))
        O = scipy.linalg.expm(A)
        return O @ vacuum(m_s // 2) @ O.T

    gamma_site = np.zeros((V, m_s, m_s))
    if site_mode == "sublattice":
        types = {+1: one_site(+1), -1: one_site(-1)}
        for s in range(V):
            gamma_site[s] = types[int(q_phys[s])]
    else:
        for s in range(V):
            gamma_site[s] = one_site(int(q_phys[s]))

    bond_q = np.concatenate([q_src, -q_src])

    def one_bond(n):
        g1 = max_entangled_bond(n_v)
        if n == 0 or not distinct_bonds:
            return g1
        A = _rand_antisym(rng, r, bond_scale)
        if group == U1:
            A = _project_commutant(A, bond_q)
        elif group == SU2:
            A = _project_commutant_su2(A, _su2_generators(_bond_slots_su2(n_v)))
        O = scipy.linalg.expm(A)
        return O @ g1 @ O.T

    gamma_bond = np.zeros((K, 2 * V, r, r))
    for n in range(K):
        if bond_mode == "uniform":
            gamma_bond[n, :] = one_bond(n)
        else:
            for l in range(2 * V):
                gamma_bond[n, l] = one_bond(n)
    z = rng.normal(size=K) + 1j * rng.normal(size=K)
    lam = z / np.linalg.norm(z)
    return Problem(L, group, n_v, K, gamma_site, gamma_bond, lam.astype(np.complex128),
                   q_src, q_phys)


def cold_links(p: Problem, n_cfg: int = 1) -> np.ndarray:
    if p.group == Z2:
        return np.ones((n_cfg, p.n_links), dtype=np.int8)
    if p.group == SU2:
        out = np.zeros((n_cfg, p.n_links, 4))
        out[..., 0] = 1.0
        return out
    return np.zeros((n_cfg, p.n_links), dtype=np.float64)


def random_links(p: Problem, n_cfg: int, seed: int = 7) -> np.ndarray:
    """Haar-random link values (SU(2): normalised Gaussian quaternions)."""
    rng = np.random.default_rng(seed)
    if p.group == Z2:
        return rng.choice(np.array([1, -1], dtype=np.int8), size=(n_cfg, p.n_links))
    if p.group == SU2:
        q = rng.normal(size=(n_cfg, p.n_links, 4))
        return q / np.linalg.norm(q, axis=-1, keepdims=True)
    return rng.uniform(0.0, 2 * np.pi, size=(n_cfg, p.n_links))


def all_z2_configs(p: Problem) -> np.ndarray:
    """Every Z2 link configuration (2^(2V) rows); small lattices only."""
    nl = p.n_links
    idx = np.arange(2 ** nl)[:, None]
    bits = (idx >> np.arange(nl)[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)


def gauge_transform(p: Problem, links: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Apply a site gauge transformation h (V,) to links (n, 2V): the link
    from s to t = s + e_d becomes (Z2) h_s g h_t, (U(1)) theta + alpha_s -
    alpha_t, (SU(2), h (V, 4) quaternions) h_t^dag g h_s."""
    L = p.L
    out = links.copy()
    for s in range(p.V):
        x, y = s % L, s // L
        for d in range(2):
            t = ((y * L + (x + 1) % L) if d == 0 else (((y + 1) % L) * L + x))
            l = 2 * s + d
            if p.group == Z2:
                out[:, l] = links[:, l] * h[s] * h[t]
            elif p.group == SU2:
                for c in range(links.shape[0]):
                    out[c, l] = _quat_of(su2(h[t]).conj().T @ su2(links[c, l]) @ su2(h[s]))
            else:
                out[:, l] = np.mod(links[:, l] + h[s] - h[t], 2 * np.pi)
    return out
