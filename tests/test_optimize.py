"""Host logic of the variational optimiser (paper_2412_01737_gb300/optimize.py),
on CPU: the generalised eigensolver against the oracle's, the local energy
contraction against explicit sums, the accumulation loop with a stand-in
context that serves the oracle's local matrices, the reweighted gradients
against exhaustive finite differences (Z2, and U(1) on an exact angle grid)
and the site score, the descent loop, and the symmetric generators."""
import numpy as np

import ggf_inputs as gi
from oracle import variational
from paper_2412_01737_gb300 import optimize
from paper_2412_01737_gb300.ggf import PAIRS_ELECTRIC, PAIRS_FIELD, PAIRS_FOUR, PAIRS_NORM, PAIRS_SITE


def test_linear_method_matches_oracle():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    B = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    H, N = A + A.conj().T, B @ B.conj().T + np.eye(4)
    e1, l1 = optimize.linear_method(H, N)
    e2, l2 = variational.linear_method(H, N)
    assert abs(e1 - e2) <= 1e-12 and np.abs(l1 - l2).max() <= 1e-10
    assert abs(optimize.energy(H, N, l1) - e1) <= 1e-12


class _ScoreStub:
    """Serves oracle scores and plaquettes of fixed configurations."""

    def __init__(self, p, configs):
        from oracle.observables import plaquette_values
        self.S = np.array([variational.score_sites(p, G) for G in configs])
        self.w = plaquette_values(p.group, p.L, configs).mean(axis=1)

    def sample(self, n):
        return np.stack([self.w, np.zeros_like(self.w), np.zeros_like(self.w)], axis=-1)[None]

    def chains_score(self):
        return self.S


def test_wilson_score_is_the_sample_covariance():
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    stub = _ScoreStub(p, gi.random_links(p, 5, seed=3))
    mw, C = optimize.wilson_score(stub, 3)
    assert abs(mw - stub.w.mean()) <= 1e-14
    want = np.mean([(w - stub.w.mean()) * S for w, S in zip(stub.w, stub.S)], axis=0)
    assert np.abs(C - want).max() <= 1e-13


class _Stub:
    """Serves per-pair parts of fixed configurations, one per chain."""

    def __init__(self, p, configs):
        self.p, self.cfgs = p, configs
        self.lm = variational.LocalMatrices(p)
        self.loc = [self.lm(G) for G in configs]

    def sample(self, n):
        from oracle.observables import plaquette_values
        pl = plaquette_values(self.p.group, self.p.L, self.cfgs).mean(axis=1)
        return np.stack([pl, np.zeros_like(pl), np.zeros_like(pl)], axis=-1)[None]

    def chains_pairs(self, what):
        key = {PAIRS_NORM: "norm", PAIRS_ELECTRIC: "electric", PAIRS_SITE: "density"}[what]
        return np.array([d[key] for d in self.loc])

    def chains_link_terms(self, charges, pairs=False):
        assert pairs and np.array_equal(charges, self.p.q_phys)
        return None, np.array([d["hopping"] for d in self.loc])


def test_accumulate_contracts_the_energy():
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    cfgs = gi.random_links(p, 3, seed=2)
    stub = _Stub(p, cfgs)
    ce = np.linspace(0.1, 0.8, p.n_links)
    cs = np.linspace(-0.3, 0.3, p.V)
    ch = np.linspace(-0.2, 0.4, p.n_links)
    H, N = optimize.accumulate(stub, 2, c_plaquette=-1.5, c_electric=ce, c_site=cs, c_hop=ch, charges=p.q_phys)
    hop = [np.einsum("l,lnm->nm", ch, d["hopping"]) for d in stub.loc]
    want_H = np.mean([-1.5 * stub.sample(1)[0, c, 0] * d["norm"] + np.einsum("l,lnm->nm", ce, d["electric"])
                      + np.einsum("s,snm->nm", cs, 0.5 * (d["norm"] + 1j * d["density"]))
                      + hop[c] + hop[c].conj().T
                      for c, d in enumerate(stub.loc)], axis=0)
    want_N = np.mean([d["norm"] for d in stub.loc], axis=0)
    assert np.abs(H - want_H).max() <= 1e-13
    assert np.abs(N - want_N).max() <= 1e-13


def test_hopping_energy_is_twice_the_real_part():
    """local_energy's hopping term: lambda^dag (sum_l c_l (T_l + T_l^H)) lambda
    equals sum_l c_l 2 Re T_l(G) per configuration, with the per-pair link
    terms built from the oracle's per-pair blocks."""
    from oracle import fermionic, variational
    p = gi.make_problem(3, gi.U1, 1, 2, bond_scale=0.3)
    fe, lm = fermionic.Fermionic(p), variational.LocalMatrices(p)
    ch = np.linspace(-0.5, 0.7, p.n_links)
    for G in gi.random_links(p, 2, seed=8):
        Nn = lm(G)["norm"]
        Ge = fe.gamma_eff(G)
        blk = np.zeros((p.n_links, 2, 2, p.K, p.K), dtype=complex)
        for l in range(p.n_links):
            s, t = fermionic._link_sites(p, l)
            for a in range(2):
                for b in range(2):
                    i, j = 2 * s + a, 2 * t + b
                    for (n, m), Gm in Ge.items():
                        blk[l, a, b, n, m] = Nn[n, m] * (1.0 if i == j else -1j * Gm[i, j])
        hop = fermionic.link_terms_from_block(p, G, blk)
        H = optimize.local_energy({"norm": Nn[None], "hop": hop[None]}, np.zeros(1), c_hop=ch)[0]
        assert np.abs(H - H.conj().T).max() <= 1e-13
        got = np.conj(p.lam) @ H @ p.lam
        want = np.sum(ch * 2 * fe.link_terms(G).real)
        assert abs(got - want) <= 1e-12


class _OracleCtx:
    """The binding calls that energy_gradient makes, answered by the oracle."""

    def init_problem(self, q):
        from oracle import electric, fermionic, weight
        self.p, self.W = q, weight.Weights(q)
        self.el, self.fe = electric.Electric(q), fermionic.Fermionic(q)
        self.links = None

    def logweight(self, links):
        return np.array([self.W.log_norm(G) for G in links])

    def observable(self, links):
        from oracle.observables import plaquette_mean
        return plaquette_mean(self.p.group, self.p.L, links)

    def chains_init(self, links, **kw):
        self.links = links

    def chains_electric(self):
        return np.array([self.el.f_electric(G) for G in self.links])

    def chains_fermion(self):
        out = [self.fe.bilinears(G) for G in self.links]
        return np.array([o[0] for o in out]), np.array([o[1] for o in out])

    def chains_link_terms(self, charges, pairs=False):
        assert np.array_equal(charges, self.p.q_phys)
        T = np.array([self.fe.link_terms(G) for G in self.links])
        if not pairs:
            return T
        from oracle import variational
        lm = variational.LocalMatrices(self.p)
        return T, np.array([lm(G)["hopping"] for G in self.links])

    def chains_pairs(self, what):
        from oracle import variational
        lm = variational.LocalMatrices(self.p)
        key = {PAIRS_NORM: "norm", PAIRS_ELECTRIC: "electric", PAIRS_SITE: "density", PAIRS_FIELD: "field",
               PAIRS_FOUR: "four"}[what]
        return np.array([lm(G)[key] for G in self.links])

    def chains_electric_field(self):
        return np.array([self.el.field(G) for G in self.links])

    def chains_fermion4(self):
        from oracle import fermionic
        p = self.p
        out = []
        for G in self.links:
            row = []
            for l in range(p.n_links):
                s, t = fermionic._link_sites(p, l)
                row.append(-1.0 if s == t else self.fe.monomial(G, [2 * s, 2 * s + 1, 2 * t, 2 * t + 1]))
            out.append(row)
        return np.array(out, dtype=complex)


def _OracleCtx_at(q):
    ctx = _OracleCtx()
    ctx.init_problem(q)
    return ctx


def _exact_energy(q, cfgs, ce, cs, ch, cn=None):
    from oracle import fermionic, variational as va
    S = va.exhaustive(q, cfgs)
    hop = np.einsum("l,lnm->nm", ch, S["hopping"])
    H = (-1.0 * S["plaquette"] + np.einsum("l,lnm->nm", ce, S["electric"])
         + np.einsum("s,snm->nm", cs, 0.5 * (S["norm"] + 1j * S["density"])) + hop + hop.conj().T)
    if cn is not None:
        for l in range(q.n_links):
            s, t = fermionic._link_sites(q, l)
            H = H + cn[l] * 0.25 * (S["norm"] + 1j * S["density"][s] + 1j * S["density"][t] - S["four"][l])
    return float(va.expectation(H, S["norm"], q.lam).real)


def test_reweighted_gradient_matches_exact_finite_differences():
    """On the 2x2 Z2 lattice with every configuration weighted by p(G), the
    reweighted energies at p(+-delta) equal the exhaustive expectations of
    the Hermitian forms at those parameters (another route), for a site and
    a bond direction and an energy with every term."""
    from oracle import weight
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    cfgs = gi.all_z2_configs(p)
    W = weight.Weights(p)
    logs = np.array([W.log_norm(G) for G in cfgs])
    w0 = np.exp(logs - logs.max())
    w0 /= w0.sum()
    rng = np.random.default_rng(3)
    A = rng.normal(size=(p.m_s, p.m_s))
    A = A - A.T
    Bg = rng.normal(size=(p.r, p.r))
    Bg = Bg - Bg.T
    ce = np.linspace(0.2, 0.6, p.n_links)
    cs = 0.4 * p.q_phys.astype(float)
    ch = 0.3 * np.ones(p.n_links)
    cn = np.linspace(-0.5, 0.5, p.n_links)
    dirs = [lambda t: optimize.rotate_sites(p, A, t), lambda t: optimize.rotate_bonds(p, 1, Bg, t)]
    delta = 1e-3
    kw = dict(c_plaquette=-1.0, c_electric=ce, c_site=cs, c_hop=ch, charges=p.q_phys, c_nn=cn)
    e0, g = optimize.energy_gradient(_OracleCtx(), p, cfgs, dirs, delta=delta, weights=w0, batch=100, **kw)
    assert abs(e0 - _exact_energy(p, cfgs, ce, cs, ch, cn)) <= 1e-12
    H, N = optimize.forms(_OracleCtx_at(p), cfgs, w0, **kw)
    assert abs(optimize.energy(H, N, p.lam) - e0) <= 1e-12
    for k, d in enumerate(dirs):
        fd = (_exact_energy(d(delta), cfgs, ce, cs, ch, cn) - _exact_energy(d(-delta), cfgs, ce, cs, ch, cn)) / (2 * delta)
        assert abs(fd) > 1e-3
        assert abs(g[k] - fd) <= 1e-9 * max(1.0, abs(fd))


def test_reweighted_gradient_of_a_wilson_energy_matches_the_score():
    """For a plaquette energy the reweighted central difference along a site
    rotation agrees with the analytic gradient sum_s tr(C_s^T dD_s/dt),
    C_s = E_p[(W - <W>) S_s] with the site scores S_s (O(delta^2))."""
    from oracle import variational as va, weight
    from oracle.observables import plaquette_mean
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    cfgs = gi.all_z2_configs(p)
    W = weight.Weights(p)
    logs = np.array([W.log_norm(G) for G in cfgs])
    w0 = np.exp(logs - logs.max())
    w0 /= w0.sum()
    A = np.random.default_rng(4).normal(size=(p.m_s, p.m_s))
    A = A - A.T
    _, g = optimize.energy_gradient(_OracleCtx(), p, cfgs, [lambda t: optimize.rotate_sites(p, A, t)],
                                    delta=1e-4, weights=w0, c_plaquette=1.0)
    pl = plaquette_mean(p.group, p.L, cfgs)
    mw = np.sum(w0 * pl)
    C = sum(wi * (x - mw) * va.score_sites(p, G) for wi, x, G in zip(w0, pl, cfgs))
    dD = [(A @ p.gamma_site[s] - p.gamma_site[s] @ A)[2:, 2:] for s in range(p.V)]
    want = sum(np.sum(C[s] * dD[s]) for s in range(p.V))
    assert abs(want) > 1e-4
    assert abs(g[0] - want) <= 1e-6


def test_u1_generator_keeps_the_symmetry():
    """Rotating one sublattice's site covariance with a projected generator
    keeps it invariant under the U(1) action and keeps log N(G) gauge
    invariant; the unprojected generator breaks both."""
    from oracle import weight
    p = gi.make_problem(2, gi.U1, 1, 2, bond_scale=0.3)
    plus = [s for s in range(p.V) if p.q_phys[s] > 0]
    q = gi.site_charges(p.n_v, 1)
    rng = np.random.default_rng(6)
    A = rng.normal(size=(p.m_s, p.m_s))
    A = A - A.T
    Ap = optimize.u1_generator(A, q)
    assert np.abs(Ap + Ap.T).max() <= 1e-14
    assert np.abs(optimize.u1_generator(Ap, q) - Ap).max() <= 1e-13       # a projection
    G = gi.random_links(p, 1, seed=3)
    h = rng.uniform(0, 2 * np.pi, p.V)
    Gh = gi.gauge_transform(p, G, h)
    for gen, symmetric in ((Ap, True), (A, False)):
        r = optimize.rotate_sites(p, gen, 0.3, sites=plus)
        R = gi._rotation(q, 0.7)
        inv = np.abs(R @ r.gamma_site[plus[0]] @ R.T - r.gamma_site[plus[0]]).max()
        W = weight.Weights(r)
        gauge = abs(W.log_norm(G[0]) - W.log_norm(Gh[0]))
        if symmetric:
            assert inv <= 1e-12 and gauge <= 1e-10
        else:
            assert inv > 1e-3 and gauge > 1e-6



def test_descend_lowers_the_energy():
    """Two iterations of lambda updates and gradient steps along a site and a
    bond rotation on the 2x2 Z2 lattice (every configuration, weighted by
    p(G)): each lambda update is the exact optimum for its Gaussians, and
    the steps lower the exact energy further."""
    from oracle import weight
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    cfgs = gi.all_z2_configs(p)

    def sampler(q):
        W = weight.Weights(q)
        logs = np.array([W.log_norm(G) for G in cfgs])
        w = np.exp(logs - logs.max())
        return cfgs, w / w.sum()

    rng = np.random.default_rng(9)
    A = rng.normal(size=(p.m_s, p.m_s))
    A = 0.2 * (A - A.T)
    Bg = rng.normal(size=(p.r, p.r))
    Bg = 0.2 * (Bg - Bg.T)
    ce = 0.5 * np.ones(p.n_links)
    cs = 0.4 * p.q_phys.astype(float)
    ch = 0.3 * np.ones(p.n_links)
    kw = dict(c_plaquette=-1.0, c_electric=ce, c_site=cs, c_hop=ch, charges=p.q_phys)
    dirs = [lambda q, t: optimize.rotate_sites(q, A, t), lambda q, t: optimize.rotate_bonds(q, 1, Bg, t)]
    e_start = _exact_energy(p, cfgs, ce, cs, ch)
    q, hist = optimize.descend(_OracleCtx(), p, sampler, dirs, n_iter=2, lr=0.05, **kw)
    # the first lambda update is the exact optimum for the starting Gaussians
    from oracle import variational as va
    S = va.exhaustive(p, cfgs)
    hop = np.einsum("l,lnm->nm", ch, S["hopping"])
    H = (-1.0 * S["plaquette"] + np.einsum("l,lnm->nm", ce, S["electric"])
         + np.einsum("s,snm->nm", cs, 0.5 * (S["norm"] + 1j * S["density"])) + hop + hop.conj().T)
    E0, _ = va.linear_method(H, S["norm"])
    assert abs(hist[0] - E0) <= 1e-9
    assert hist[0] < e_start - 1.0
    e_final = _exact_energy(q, cfgs, ce, cs, ch)
    assert hist[1] < hist[0] - 1e-4
    assert e_final < hist[1] + 1e-9


def test_commutant_generator_for_su2_keeps_gauge_invariance():
    """Projected onto the commutant of the SU(2) action on a site's doublets,
    a generator commutes with that action (and the projection is
    idempotent); rotating the site covariances with it keeps log N(G)
    invariant under SU(2) gauge transformations, which the unprojected
    generator breaks.  For a U(1) action it agrees with u1_generator."""
    from oracle import weight
    p = gi.make_problem(1, gi.SU2, 2, 1, bond_scale=0.3)
    gens = gi._su2_generators(gi._site_slots_su2(p.n_v))
    rng = np.random.default_rng(12)
    A = rng.normal(size=(p.m_s, p.m_s))
    A = A - A.T
    X = optimize.commutant_generator(A, gens)
    assert np.abs(X + X.T).max() <= 1e-13
    assert max(np.abs(T @ X - X @ T).max() for T in gens) <= 1e-10
    assert np.abs(optimize.commutant_generator(X, gens) - X).max() <= 1e-10
    assert np.abs(X).max() > 1e-2
    G = gi.random_links(p, 1, seed=4)
    h = np.array([gi._quat_of(gi.su2(q)) for q in rng.normal(size=(p.V, 4))])
    h = h / np.linalg.norm(h, axis=1, keepdims=True)
    Gh = gi.gauge_transform(p, G, h)
    for gen, symmetric in ((X, True), (A, False)):
        W = weight.Weights(optimize.rotate_sites(p, gen, 0.3))
        d = abs(W.log_norm(G[0]) - W.log_norm(Gh[0]))
        assert (d <= 1e-10) if symmetric else (d > 1e-6)
    # U(1): the same projection as the exact group average
    q = gi.site_charges(1, 1)
    T = np.zeros((len(q) * 2, len(q) * 2))
    for j, qj in enumerate(q):
        T[2 * j, 2 * j + 1], T[2 * j + 1, 2 * j] = qj, -qj
    B = rng.normal(size=T.shape)
    B = B - B.T
    assert np.abs(optimize.commutant_generator(B, [T]) - optimize.u1_generator(B, q)).max() <= 1e-10


def test_reweighted_gradient_u1_on_an_exact_grid():
    """U(1) on the 1x1 torus, every configuration of an 8 x 8 angle grid
    weighted by N(G) (a grid that integrates the energy's terms exactly): the
    reweighted central difference along a U(1)-symmetric site rotation
    equals the finite difference of the grid expectations of the Hermitian
    forms (magnetic, Casimir, density, link and field terms); the forms of an
    explicit weighted list give the same energy."""
    from oracle import variational as va, weight
    p = gi.make_problem(1, gi.U1, 1, 2, bond_scale=0.4)
    th = 2 * np.pi * np.arange(8) / 8
    grid = np.array([[a, b] for a in th for b in th])
    W = weight.Weights(p)
    logs = np.array([W.log_norm(G) for G in grid])
    w0 = np.exp(logs - logs.max())
    w0 /= w0.sum()
    A = np.random.default_rng(8).normal(size=(p.m_s, p.m_s))
    Ap = optimize.u1_generator(A - A.T, gi.site_charges(p.n_v, int(p.q_phys[0])))
    ce, cs, ch, cf = np.array([0.5, 0.7]), np.array([0.4]), np.array([0.3, -0.2]), np.array([0.25, -0.6])

    def exact(q):
        S = va.exhaustive(q, grid)
        hop = np.einsum("l,lnm->nm", ch, S["hopping"])
        H = (-1.0 * S["plaquette"] + np.einsum("l,lnm->nm", ce, S["electric"])
             + np.einsum("s,snm->nm", cs, 0.5 * (S["norm"] + 1j * S["density"])) + hop + hop.conj().T
             + np.einsum("l,lnm->nm", cf, S["field"]))
        return float(va.expectation(H, S["norm"], q.lam).real)

    d = lambda t: optimize.rotate_sites(p, Ap, t)
    kw = dict(c_plaquette=-1.0, c_electric=ce, c_site=cs, c_hop=ch, charges=p.q_phys, c_field=cf)
    e0, g = optimize.energy_gradient(_OracleCtx(), p, grid, [d], delta=1e-3, weights=w0, **kw)
    H, N = optimize.forms(_OracleCtx_at(p), grid, w0, **kw)
    assert abs(optimize.energy(H, N, p.lam) - exact(p)) <= 1e-12
    fd = (exact(d(1e-3)) - exact(d(-1e-3))) / 2e-3
    assert abs(e0 - exact(p)) <= 1e-12
    assert abs(fd) > 1e-3
    assert abs(g[0] - fd) <= 1e-9 * max(1.0, abs(fd))
