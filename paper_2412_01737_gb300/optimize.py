"""Variational optimisation: the superposition weights lambda and the site
and bond parameters for a given energy.

For fixed Gaussians every per-configuration quantity of Secs. 5.1-5.3 is a
Hermitian form in lambda, so with the per-pair parts that
``GGF.chains_pairs`` returns (N_nm(G) o_nm(G) / N(G), expectations over the
chains' p(G)),

    <E>_lambda = lambda^dag Hbar lambda / lambda^dag Nbar lambda,

and the lambda that minimises it is the lowest generalised eigenvector of
Hbar lambda = E Nbar lambda.  ``accumulate`` samples with the context's
current lambda and estimates Hbar and Nbar for an energy

    E = c_plaquette <mean plaquette> + sum_l c_electric[l] <f_E,l>
        + sum_s c_site[s] <n_s> + sum_{l,a,b} c_link[l,a,b] <i c_{2s+a} c_{2t+b}>
        + sum_l c_hop[l] <T_l + T_l^dag> + sum_l c_field[l] <J_l>   (U(1))
        + sum_l c_nn[l] <n_s n_t>   (l = (s -> t), density-density)

with the Hermitian operators n_s = (1 + i c_2s c_2s+1) / 2 and i c c (the
Majorana bilinears themselves are anti-Hermitian), so that for real
coefficients every local matrix is Hermitian.  Any coefficient may be
omitted; T_l is the gauge-invariant link term of ``GGF.chains_link_terms``,
whose per-pair parts enter as T + T^H over the pair indices.  The couplings,
and thus the Hamiltonian, are the caller's.  ``linear_method`` solves for the
new lambda, which ``GGF.init_gaussians`` takes before sampling again;
``forms`` does what ``accumulate`` does for an explicit list of
configurations.

``energy_gradient`` gives the derivative of any such energy along directions
in the space of site and bond parameters (``rotate_sites``, ``rotate_bonds``:
orthogonal rotations, which keep the Gaussians pure; ``u1_generator``
projects a generator onto the U(1)-symmetric ones, ``commutant_generator``
onto those of any group given its generators), from configurations
sampled at the current parameters: for a problem p' near p,
    E(p') = sum_i r_i h'(G_i) / sum_i r_i,   r_i = N'(G_i) / N(G_i),
exactly for samples of p (Sec. 5.1: p(G) = N(G) / sum_G N(G)), with h' the
local energy of the configuration under p'; central differences of this
reweighted energy on the same samples estimate the gradient (every term,
including the electric and fermionic ones and the dependence of the pair
weights, at O(delta^2) plus the sampling error).

``descend`` alternates the exact lambda update with gradient steps along
given parameter directions, from the configurations a sampler returns.

``wilson_score`` gives the gradient of a Wilson-loop energy with respect to
the site blocks, as the covariance of the plaquette with the score
d log N(G) / d D_s (``GGF.chains_score``); ``wilson_link_score`` does the same
for the link blocks (for K = 1 the bond covariances).  For the other terms
use ``energy_gradient``.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg

from .ggf import FP64, PAIRS_ELECTRIC, PAIRS_FIELD, PAIRS_FOUR, PAIRS_LINK, PAIRS_NORM, PAIRS_SITE


def local_energy(pairs: dict, plaquette: np.ndarray, c_plaquette=0.0, c_electric=None, c_site=None,
                 c_link=None, c_hop=None, c_field=None, c_nn=None) -> np.ndarray:
    """(n_chains, K, K) local matrices of the energy from one sweep's per-pair
    parts (dict with keys 'norm', 'electric', 'site', 'link' as returned by
    GGF.chains_pairs, 'hop' the per-pair link terms of GGF.chains_link_terms,
    'field' the PAIRS_FIELD parts, 'four' the PAIRS_FOUR parts; c_nn needs
    'site' and 'four')
    and the chains' mean plaquettes."""
    H = c_plaquette * plaquette[:, None, None] * pairs["norm"]
    if c_electric is not None:
        H = H + np.einsum("l,clnm->cnm", np.asarray(c_electric, dtype=complex), pairs["electric"])
    if c_site is not None:
        cs = np.asarray(c_site, dtype=complex)
        H = H + 0.5 * (cs.sum() * pairs["norm"] + 1j * np.einsum("s,csnm->cnm", cs, pairs["site"]))
    if c_link is not None:
        H = H + 1j * np.einsum("lab,clabnm->cnm", np.asarray(c_link, dtype=complex), pairs["link"])
    if c_hop is not None:
        T = np.einsum("l,clnm->cnm", np.asarray(c_hop, dtype=float), pairs["hop"])
        H = H + T + np.conj(np.swapaxes(T, 1, 2))
    if c_field is not None:
        H = H + np.einsum("l,clnm->cnm", np.asarray(c_field, dtype=complex), pairs["field"])
    if c_nn is not None:
        # n_s n_t = (1 + i A_s + i A_t - A_s A_t) / 4, A_s = c_2s c_2s+1
        cn = np.asarray(c_nn, dtype=complex)
        V = pairs["site"].shape[1]
        src = np.arange(cn.size) // 2
        dst = np.array([_link_target(l, int(round(np.sqrt(V)))) for l in range(cn.size)])
        site = pairs["site"]
        H = H + 0.25 * (cn.sum() * pairs["norm"] + 1j * np.einsum("l,clnm->cnm", cn, site[:, src])
                        + 1j * np.einsum("l,clnm->cnm", cn, site[:, dst])
                        - np.einsum("l,clnm->cnm", cn, pairs["four"]))
    return H


def _link_target(l, L):
    """Site t of link l = (s -> t): s + e_x for even l, s + e_y for odd l."""
    s, d = l // 2, l % 2
    x, y = s % L, s // L
    return y * L + (x + 1) % L if d == 0 else ((y + 1) % L) * L + x


def accumulate(ctx, n_sweeps: int, c_plaquette=0.0, c_electric=None, c_site=None, c_link=None, c_hop=None,
               charges=None, c_field=None, c_nn=None):
    """Run n_sweeps sweeps of ctx's chains and return (Hbar, Nbar), the means
    over chains and sweeps of the energy's and the norm's per-pair parts
    (c_hop needs the sites' physical charges)."""
    if c_hop is not None and charges is None:
        raise ValueError("c_hop needs the sites' physical charges")
    Hbar, Nbar, n = 0.0, 0.0, 0
    for _ in range(n_sweeps):
        obs = ctx.sample(1)
        pairs = {"norm": ctx.chains_pairs(PAIRS_NORM)}
        if c_electric is not None:
            pairs["electric"] = ctx.chains_pairs(PAIRS_ELECTRIC)
        if c_site is not None or c_nn is not None:
            pairs["site"] = ctx.chains_pairs(PAIRS_SITE)
        if c_link is not None:
            pairs["link"] = ctx.chains_pairs(PAIRS_LINK)
        if c_hop is not None:
            pairs["hop"] = ctx.chains_link_terms(charges, pairs=True)[1]
        if c_field is not None:
            pairs["field"] = ctx.chains_pairs(PAIRS_FIELD)
        if c_nn is not None:
            pairs["four"] = ctx.chains_pairs(PAIRS_FOUR)
        H = local_energy(pairs, obs[0, :, 0], c_plaquette, c_electric, c_site, c_link, c_hop, c_field, c_nn)
        Hbar = Hbar + H.sum(axis=0)
        Nbar = Nbar + pairs["norm"].sum(axis=0)
        n += H.shape[0]
    return Hbar / n, Nbar / n


def forms(ctx, links, weights=None, c_plaquette=0.0, c_electric=None, c_site=None, c_link=None, c_hop=None,
          charges=None, c_field=None, c_nn=None):
    """(Hbar, Nbar) as in ``accumulate``, from an explicit list of
    configurations (samples of ctx's problem, or every configuration with
    weights p(G)): they become FP64 chains of ctx, whose per-pair parts are
    averaged."""
    if c_hop is not None and charges is None:
        raise ValueError("c_hop needs the sites' physical charges")
    links = np.ascontiguousarray(links)
    ctx.chains_init(links, precision=FP64, refresh_every=1 << 30, delay=1)
    pairs = {"norm": ctx.chains_pairs(PAIRS_NORM)}
    if c_electric is not None:
        pairs["electric"] = ctx.chains_pairs(PAIRS_ELECTRIC)
    if c_site is not None or c_nn is not None:
        pairs["site"] = ctx.chains_pairs(PAIRS_SITE)
    if c_link is not None:
        pairs["link"] = ctx.chains_pairs(PAIRS_LINK)
    if c_hop is not None:
        pairs["hop"] = ctx.chains_link_terms(charges, pairs=True)[1]
    if c_field is not None:
        pairs["field"] = ctx.chains_pairs(PAIRS_FIELD)
    if c_nn is not None:
        pairs["four"] = ctx.chains_pairs(PAIRS_FOUR)
    pl = np.asarray(ctx.observable(links), dtype=float)
    H = local_energy(pairs, pl, c_plaquette, c_electric, c_site, c_link, c_hop, c_field, c_nn)
    w = np.full(len(links), 1.0 / len(links)) if weights is None else np.asarray(weights, float) / np.sum(weights)
    return np.einsum("c,cnm->nm", w, H), np.einsum("c,cnm->nm", w, pairs["norm"])


def descend(ctx, p, sampler, directions, n_iter, lr, delta=1e-3, **couplings):
    """Variational optimisation of lambda and of the site and bond parameters.
    Per iteration: configurations from sampler(p) -> (links, weights or None);
    lambda <- the lowest generalised eigenvector of their forms (exact for
    the sampled Gaussians); fresh configurations for the new problem; one
    gradient step t_k = -lr dE/dt_k along each direction (callables
    (p, t) -> problem, e.g. ``lambda q, t: rotate_sites(q, A, t)``), applied
    in order.  ctx is re-initialised throughout (not a sampling context).
    Returns the final problem and the energies after each lambda update."""
    energies = []
    for _ in range(n_iter):
        links, w = sampler(p)
        ctx.init_problem(p)
        H, N = forms(ctx, links, w, **couplings)
        E, lam = linear_method(H, N)
        energies.append(E)
        p = dataclasses.replace(p, lam=np.asarray(lam, dtype=np.complex128))
        if not directions:
            continue
        links, w = sampler(p)
        dirs = [(lambda t, d=d, q=p: d(q, t)) for d in directions]
        _, g = energy_gradient(ctx, p, links, dirs, delta=delta, weights=w, **couplings)
        for d, gk in zip(directions, g):
            p = d(p, -lr * gk)
    return p, energies


def wilson_score(ctx, n_sweeps: int):
    """Run n_sweeps sweeps and return (<W>, C): the mean plaquette and, per
    site, the covariance C_s = E_p[(W(G) - <W>) S_s(G)] of the chains' mean
    plaquette with the site scores S_s = d log N(G) / d D_s
    (GGF.chains_score).  A change dD_s of the site blocks (through the
    site parameters, keeping the states pure) changes <W> by
    sum_s sum_ij C_s[i, j] dD_s[i, j]: the exact gradient of a Wilson-loop
    energy with respect to the site parameters."""
    sw, ss, sws, n = 0.0, 0.0, 0.0, 0
    for _ in range(n_sweeps):
        obs = ctx.sample(1)
        S = ctx.chains_score()
        w = obs[0, :, 0]
        sw = sw + w.sum()
        ss = ss + S.sum(axis=0)
        sws = sws + np.einsum("c,csij->sij", w, S)
        n += w.shape[0]
    mw = sw / n
    return mw, sws / n - mw * ss / n


def wilson_link_score(ctx, n_sweeps: int):
    """As wilson_score for the link blocks: (<W>, C) with
    C = E_p[(W(G) - <W>) U(G)] (P, 2V, r, r complex), U the per-pair link
    scores of GGF.chains_link_score.  For K = 1 a change dGamma_B[l] of the
    bond blocks changes <W> by Re sum_l tr(C[0, l]^T dGamma_B[l])."""
    sw, su, swu, n = 0.0, 0.0, 0.0, 0
    for _ in range(n_sweeps):
        obs = ctx.sample(1)
        U = ctx.chains_link_score()
        w = obs[0, :, 0]
        sw = sw + w.sum()
        su = su + U.sum(axis=0)
        swu = swu + np.einsum("c,cplij->plij", w, U)
        n += w.shape[0]
    mw = sw / n
    return mw, swu / n - mw * su / n


def linear_method(Hbar: np.ndarray, Nbar: np.ndarray):
    """(E, lambda): the lowest generalised eigenpair of the Hermitian parts of
    Hbar and Nbar; lambda has unit 2-norm and lambda_0 real non-negative."""
    H = 0.5 * (Hbar + Hbar.conj().T)
    Nm = 0.5 * (Nbar + Nbar.conj().T)
    w, v = scipy.linalg.eigh(H, Nm)
    lam = v[:, 0] / np.linalg.norm(v[:, 0])
    if abs(lam[0]) > 0:
        lam = lam * (abs(lam[0]) / lam[0])
    return float(w[0]), lam


def energy(Hbar: np.ndarray, Nbar: np.ndarray, lam) -> float:
    """lambda^dag Hbar lambda / lambda^dag Nbar lambda (real part)."""
    lam = np.asarray(lam, dtype=complex)
    return float((np.conj(lam) @ Hbar @ lam / (np.conj(lam) @ Nbar @ lam)).real)


def local_energies(ctx, links, c_plaquette=0.0, c_electric=None, c_site=None, c_link=None, c_hop=None,
                   charges=None, batch=None, c_field=None, c_nn=None):
    """(log N(G), h(G)) for every configuration in links under ctx's current
    problem: h(G) the per-configuration value of the energy of
    ``local_energy`` (complex; its mean over p is real).  The configurations
    become FP64 chains of ctx (replacing any it holds), `batch` of them at a
    time (all by default; each holds its P inverses in FP64)."""
    links = np.ascontiguousarray(links)
    if batch is not None and len(links) > batch:
        parts = [local_energies(ctx, links[i:i + batch], c_plaquette, c_electric, c_site, c_link, c_hop, charges,
                                c_field=c_field, c_nn=c_nn) for i in range(0, len(links), batch)]
        return np.concatenate([a for a, _ in parts]), np.concatenate([b for _, b in parts])
    logN = np.asarray(ctx.logweight(links), dtype=float)
    h = c_plaquette * np.asarray(ctx.observable(links), dtype=complex)
    if all(c is None for c in (c_electric, c_site, c_link, c_hop, c_field, c_nn)):
        return logN, h
    ctx.chains_init(links, precision=FP64, refresh_every=1 << 30, delay=1)
    if c_electric is not None:
        h = h + ctx.chains_electric() @ np.asarray(c_electric, dtype=complex)
    if c_site is not None or c_link is not None or c_nn is not None:
        site, link = ctx.chains_fermion()
        if c_site is not None:
            h = h + (0.5 * (1.0 + 1j * site)) @ np.asarray(c_site, dtype=complex)
        if c_link is not None:
            h = h + 1j * np.einsum("lab,clab->c", np.asarray(c_link, dtype=complex), link)
    if c_hop is not None:
        if charges is None:
            raise ValueError("c_hop needs the sites' physical charges")
        T = ctx.chains_link_terms(charges)
        h = h + 2.0 * T.real @ np.asarray(c_hop, dtype=float)
    if c_field is not None:
        h = h + ctx.chains_electric_field() @ np.asarray(c_field, dtype=complex)
    if c_nn is not None:
        cn = np.asarray(c_nn, dtype=complex)
        L = int(round(np.sqrt(site.shape[1])))
        src = np.arange(cn.size) // 2
        dst = np.array([_link_target(l, L) for l in range(cn.size)])
        four = ctx.chains_fermion4()
        nn = 0.25 * (1.0 + 1j * site[:, src] + 1j * site[:, dst] - four)
        h = h + nn @ cn
    return logN, h


def reweighted_energy(logN0, logN1, h1, weights=None) -> float:
    """sum_i w_i r_i h1_i / sum_i w_i r_i (real part), r_i = exp(logN1_i - logN0_i):
    the energy under the problem of (logN1, h1) from configurations sampled
    under that of logN0 (w_i = 1 for samples; pass p0(G) for an explicit list)."""
    d = np.asarray(logN1, dtype=float) - np.asarray(logN0, dtype=float)
    r = np.exp(d - d.max())
    if weights is not None:
        r = r * np.asarray(weights, dtype=float)
    return float((np.sum(r * np.asarray(h1)) / np.sum(r)).real)


def u1_generator(A, charges):
    """The part of an antisymmetric generator A (Majorana basis, mode j on
    Majoranas 2j, 2j+1) that commutes with the U(1) action, which turns the
    Majorana pair of a mode of charge q by the angle q phi: the average of
    R(phi)^T A R(phi) over phi.  Its entries are trigonometric polynomials of
    degree at most 2 max|q|, so 4 max|q| + 2 equally spaced angles give the
    average exactly.  Rotations it generates keep a symmetric state
    symmetric (site charges: the physical mode, then the virtual modes)."""
    q = np.asarray(charges, dtype=float)
    n_phi = 4 * int(np.max(np.abs(q))) + 2
    out = np.zeros_like(np.asarray(A, dtype=float))
    for k in range(n_phi):
        phi = 2.0 * np.pi * k / n_phi
        R = np.zeros_like(out)
        for j, qj in enumerate(q):
            c, sn = np.cos(qj * phi), np.sin(qj * phi)
            R[2 * j:2 * j + 2, 2 * j:2 * j + 2] = [[c, sn], [-sn, c]]
        out += R.T @ A @ R
    return out / n_phi


def commutant_generator(A, generators, tol=1e-10):
    """Orthogonal (Frobenius) projection of an antisymmetric A onto the
    antisymmetric matrices that commute with every given generator of a
    group action (so(m) matrices, e.g. the SU(2) action on a site's
    doublets).  C(X) = sum_a [T_a, [T_a, X]] maps antisymmetric matrices to
    antisymmetric ones, is symmetric and negative semi-definite, and vanishes
    exactly on that commutant, so the projection is onto C's null space."""
    A = np.asarray(A, dtype=float)
    n = A.shape[0]
    iu = np.triu_indices(n, 1)
    basis = np.zeros((len(iu[0]), n, n))
    for k, (a, b) in enumerate(zip(*iu)):
        basis[k, a, b], basis[k, b, a] = 2 ** -0.5, -(2 ** -0.5)
    Ts = [np.asarray(T, dtype=float) for T in generators]

    def C(X):
        out = np.zeros_like(X)
        for T in Ts:
            Y = T @ X - X @ T
            out += T @ Y - Y @ T
        return out

    Cm = np.array([[np.sum(Bi * C(Bj)) for Bj in basis] for Bi in basis])
    w, v = np.linalg.eigh(0.5 * (Cm + Cm.T))
    null = v[:, np.abs(w) <= tol * max(1.0, np.abs(w).max())]
    coef = np.einsum("kab,ab->k", basis, A)
    return np.einsum("k,kab->ab", null @ (null.T @ coef), basis)


def rotate_sites(p, generator, t, sites=None):
    """The problem with the site covariances rotated, Gamma_s -> O Gamma_s O^T,
    O = expm(t A) for the antisymmetric m_s x m_s generator A (in the commutant
    of the group action, so the symmetry is kept), on the given sites (all by
    default).  A pure state stays pure."""
    O = scipy.linalg.expm(t * np.asarray(generator, dtype=float))
    gs = np.array(p.gamma_site, copy=True)
    for s in (range(gs.shape[0]) if sites is None else sites):
        gs[s] = O @ gs[s] @ O.T
    return dataclasses.replace(p, gamma_site=gs)


def rotate_bonds(p, n, generator, t):
    """The problem with bond state n rotated on every link, Gamma_{B_n} ->
    O Gamma_{B_n} O^T, O = expm(t A) for an antisymmetric r x r generator A."""
    O = scipy.linalg.expm(t * np.asarray(generator, dtype=float))
    gb = np.array(p.gamma_bond, copy=True)
    for l in range(gb.shape[1]):
        gb[n, l] = O @ gb[n, l] @ O.T
    return dataclasses.replace(p, gamma_bond=gb)


def energy_gradient(ctx, p, links, directions, delta=1e-3, weights=None, batch=None, **couplings):
    """dE/dt at t = 0 along each direction (a callable t -> problem, e.g.
    ``lambda t: rotate_sites(p, A, t)``), by central differences of the
    reweighted energy on the configurations `links` sampled under p (or an
    explicit list with weights p(G)).  couplings and batch as for
    ``local_energies``.
    It re-initialises ctx for every offset, so use a context other than the
    sampling one; ctx is left holding p (with FP64 chains at `links` if a
    coupling needed them).  Returns (E(p), gradient)."""
    ctx.init_problem(p)
    logN0, h0 = local_energies(ctx, links, batch=batch, **couplings)
    e0 = reweighted_energy(logN0, logN0, h0, weights)
    grad = []
    for d in directions:
        e = []
        for t in (delta, -delta):
            ctx.init_problem(d(t))
            logN, h = local_energies(ctx, links, batch=batch, **couplings)
            e.append(reweighted_energy(logN0, logN, h, weights))
        grad.append((e[0] - e[1]) / (2.0 * delta))
    ctx.init_problem(p)
    return e0, np.array(grad)
