"""GPU parity of the per-configuration observables computed from the chains'
cached inverses: the electric observables of Sec. 5.3 (Z2 link flip, U(1)
Casimir and field, Gauss's law), the fermionic ones of Sec. 5.2 (bilinears,
four-point function, gauge-invariant link terms), their per-pair parts, the
scores, Wilson and Polyakov loops, in-memory chain states, and the
variational helpers built on them (lambda optimisation, reweighted
gradients, descent).  The oracle evaluates the observables by the full
covariance route (itself pinned to explicit Fock vectors).  FP64 chains agree
to 1e-10 relative, FP32 chains to 1e-4.
"""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import electric, fermionic
from tests.gpu_util import ctx_for

pytestmark = pytest.mark.gpu


def _check(p, ctx, links, tol):
    got = ctx.chains_electric()
    el = electric.Electric(p)
    assert got.shape == (links.shape[0], p.n_links)
    for c in range(links.shape[0]):
        ref = el.f_electric(links[c])
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(got[c] - ref).max() <= tol * scale, (c, np.abs(got[c] - ref).max())


@pytest.mark.parametrize("L,n_v,K,nch", [
    (2, 1, 1, 3),
    (2, 1, 3, 2),
    (3, 1, 2, 3),
    (2, 2, 2, 2),
    (9, 1, 2, 2),      # 162 links: two thread blocks per chain, ragged tail
])
def test_fp64_initial_configurations(L, n_v, K, nch):
    p = gi.make_problem(L, gi.Z2, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, nch, seed=31)
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=0, seed=5)
    _check(p, ctx, links, 1e-10)
    ctx.close()


@pytest.mark.parametrize("delay", [1, 8])
def test_fp64_after_sampling(delay):
    """After sweeps (immediate and batched updates) the inverses the
    observable reads are those of the chains' current links."""
    p = gi.make_problem(4, gi.Z2, 1, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 3, seed=4), precision=0, seed=11, delay=delay, refresh_every=1000)
    ctx.sample(3)
    links = ctx.chains_links()
    _check(p, ctx, links, 1e-10)
    ctx.close()


@pytest.mark.parametrize("n_v", [1, 2])
def test_fp32_chains(n_v):
    p = gi.make_problem(4 if n_v == 1 else 2, gi.Z2, n_v, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=8), precision=1, seed=3, delay=8 if n_v == 1 else 1)
    ctx.sample(2)
    links = ctx.chains_links()
    _check(p, ctx, links, 1e-4)
    ctx.close()


def test_device_output_matches_host():
    torch = pytest.importorskip("torch")
    p = gi.make_problem(3, gi.Z2, 1, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=6), precision=0, seed=1)
    host = ctx.chains_electric()
    dev = torch.zeros((2, p.n_links, 2), dtype=torch.float64, device="cuda")
    ctx.chains_electric(out=dev)
    ctx.sync()
    d = dev.cpu().numpy()
    assert np.array_equal(d[..., 0] + 1j * d[..., 1], host)
    ctx.close()


@pytest.mark.parametrize("L,n_v,K,nch", [(2, 1, 2, 2), (3, 1, 3, 2), (2, 2, 2, 2)])
def test_u1_casimir_fp64(L, n_v, K, nch):
    p = gi.make_problem(L, gi.U1, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, nch, seed=33)
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=0, seed=5)
    _check(p, ctx, links, 1e-10)
    ctx.close()


def test_u1_casimir_fp32_after_sampling():
    p = gi.make_problem(4, gi.U1, 1, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=14), precision=1, seed=3, delay=8)
    ctx.sample(2)
    _check(p, ctx, ctx.chains_links(), 1e-4)
    ctx.close()


def _check_fermion(p, ctx, links, tol):
    site, link = ctx.chains_fermion()
    fe = fermionic.Fermionic(p)
    assert site.shape == (links.shape[0], p.V) and link.shape == (links.shape[0], p.n_links, 2, 2)
    for c in range(links.shape[0]):
        rs, rl = fe.bilinears(links[c])
        assert np.abs(site[c] - rs).max() <= tol, (c, np.abs(site[c] - rs).max())
        assert np.abs(link[c] - rl).max() <= tol, (c, np.abs(link[c] - rl).max())


@pytest.mark.parametrize("L,grp,n_v,K,nch", [
    (2, gi.Z2, 1, 2, 2),
    (3, gi.U1, 1, 3, 2),
    (2, gi.U1, 2, 2, 2),
    (1, gi.Z2, 1, 2, 2),     # self-links: both Majoranas of a link on one site
    (9, gi.Z2, 1, 1, 2),     # 243 items: two thread blocks per chain, ragged tail
])
def test_fermion_fp64_initial_configurations(L, grp, n_v, K, nch):
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, nch, seed=41)
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=0, seed=5)
    _check_fermion(p, ctx, links, 1e-10)
    ctx.close()


@pytest.mark.parametrize("precision,delay,tol", [(0, 4, 1e-10), (1, 8, 1e-4)])
def test_fermion_after_sampling(precision, delay, tol):
    p = gi.make_problem(4, gi.U1, 1, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=4), precision=precision, seed=13, delay=delay)
    ctx.sample(2)
    _check_fermion(p, ctx, ctx.chains_links(), tol)
    ctx.close()


def test_fermion_site_only_and_device_buffers():
    torch = pytest.importorskip("torch")
    p = gi.make_problem(3, gi.Z2, 1, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=6), precision=0, seed=1)
    hs, hl = ctx.chains_fermion()
    ds = torch.zeros((2, p.V, 2), dtype=torch.float64, device="cuda")
    ctx.chains_fermion(site=ds)
    ctx.sync()
    d = ds.cpu().numpy()
    assert np.array_equal(d[..., 0] + 1j * d[..., 1], hs)
    ctx.close()


@pytest.mark.parametrize("L,grp,n_v,K,prec,tol", [
    (3, gi.Z2, 1, 3, 0, 1e-10),
    (2, gi.U1, 2, 2, 0, 1e-10),
    (4, gi.U1, 1, 2, 1, 1e-4),
])
def test_pair_parts_match_oracle(L, grp, n_v, K, prec, tol):
    """ggf_chains_pairs against the oracle's local matrices, and contracting
    them with lambda gives the combined observables."""
    from oracle import variational
    from paper_2412_01737_gb300.ggf import PAIRS_NORM, PAIRS_ELECTRIC, PAIRS_SITE, PAIRS_LINK
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=51)
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=prec, seed=2)
    norm = ctx.chains_pairs(PAIRS_NORM)
    elp = ctx.chains_pairs(PAIRS_ELECTRIC)
    sitep = ctx.chains_pairs(PAIRS_SITE)
    linkp = ctx.chains_pairs(PAIRS_LINK)
    el = ctx.chains_electric()
    site, link = ctx.chains_fermion()
    lm = variational.LocalMatrices(p)
    fe = fermionic.Fermionic(p)
    lam = p.lam
    for c in range(2):
        ref = lm(links[c])
        sc = max(1.0, np.abs(ref["norm"]).max())
        assert np.abs(norm[c] - ref["norm"]).max() <= tol * sc
        assert np.abs(elp[c] - ref["electric"]).max() <= tol * max(1.0, np.abs(ref["electric"]).max())
        assert np.abs(sitep[c] - ref["density"]).max() <= tol * max(1.0, np.abs(ref["density"]).max())
        Ge = fe.gamma_eff(links[c])
        for l in range(p.n_links):
            s_, t_ = fermionic._link_sites(p, l)
            for a in range(2):
                for b in range(2):
                    want = np.zeros((K, K), dtype=complex)
                    for (n, m), G in Ge.items():
                        i, j = 2 * s_ + a, 2 * t_ + b
                        want[n, m] = ref["norm"][n, m] * (1.0 if i == j else -1j * G[i, j])
                    assert np.abs(linkp[c, l, a, b] - want).max() <= tol * max(1.0, np.abs(want).max())
        contract = lambda X: np.einsum("n,...nm,m->...", np.conj(lam), X, lam)
        assert abs(contract(norm[c]) - 1.0) <= tol
        assert np.abs(contract(elp[c]) - el[c]).max() <= tol * max(1.0, np.abs(el[c]).max())
        assert np.abs(contract(sitep[c]) - site[c]).max() <= tol
        assert np.abs(contract(linkp[c]) - link[c]).max() <= tol
    ctx.close()


def test_lambda_optimisation_end_to_end():
    """Sample with the problem's lambda, estimate the per-pair matrices of
    E = -<plaquette> + 0.5 sum_l <X_l> on the GPU, solve for lambda, and
    check with the exhaustive oracle that the new lambda is near the optimum."""
    from oracle import variational
    from paper_2412_01737_gb300 import optimize
    p = gi.make_problem(2, gi.Z2, 1, 3, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 512, seed=61), precision=0, seed=8)
    ctx.sample(3)
    Hbar, Nbar = optimize.accumulate(ctx, 20, c_plaquette=-1.0, c_electric=0.5 * np.ones(p.n_links))
    ctx.close()
    _, lam = optimize.linear_method(Hbar, Nbar)
    S = variational.exhaustive(p, gi.all_z2_configs(p))
    H = -1.0 * S["plaquette"] + 0.5 * S["electric"].sum(axis=0)
    E0, _ = variational.linear_method(H, S["norm"])
    e_new = variational.expectation(H, S["norm"], lam).real
    e_old = variational.expectation(H, S["norm"], p.lam).real
    assert e_old - E0 > 3.0
    assert e_new < E0 + 0.5


def test_gauge_theory_energy_optimisation():
    """As above with every term of a lattice-gauge energy: magnetic,
    electric, staggered mass and the hopping through the gauge-invariant
    link terms (exhaustive optimum -2.6996, sampling lambda +1.380; i.i.d.
    samples of the same size land within 4e-4 of the optimum)."""
    from oracle import variational
    from paper_2412_01737_gb300 import optimize
    p = gi.make_problem(2, gi.Z2, 1, 3, bond_scale=0.3)
    mass = 0.4 * p.q_phys.astype(float)
    hopc = 0.3 * np.ones(p.n_links)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 512, seed=62), precision=0, seed=9)
    ctx.sample(3)
    Hbar, Nbar = optimize.accumulate(ctx, 20, c_plaquette=-1.0, c_electric=0.5 * np.ones(p.n_links), c_site=mass,
                                     c_hop=hopc, charges=p.q_phys)
    ctx.close()
    _, lam = optimize.linear_method(Hbar, Nbar)
    S = variational.exhaustive(p, gi.all_z2_configs(p))
    hop = np.einsum("l,lnm->nm", hopc, S["hopping"])
    H = (-1.0 * S["plaquette"] + 0.5 * S["electric"].sum(axis=0)
         + np.einsum("s,snm->nm", mass, 0.5 * (S["norm"] + 1j * S["density"])) + hop + hop.conj().T)
    E0, _ = variational.linear_method(H, S["norm"])
    e_new = variational.expectation(H, S["norm"], lam).real
    e_old = variational.expectation(H, S["norm"], p.lam).real
    assert e_old - E0 > 3.0
    assert e_new < E0 + 0.5


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_site_score_matches_oracle(precision, tol):
    from oracle import variational
    p = gi.make_problem(3, gi.U1, 2, 2, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=71)
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=precision, seed=3)
    S = ctx.chains_score()
    ctx.close()
    for c in range(2):
        ref = variational.score_sites(p, links[c])
        assert np.abs(S[c] - ref).max() <= tol * max(1.0, np.abs(ref).max())


def test_wilson_gradient_estimate_matches_exact():
    """The sampled covariance of the plaquette with the site score against
    the exact gradient of <W> along a rotation of one sublattice's sites
    (exhaustive 2x2 Z2 through the oracle)."""
    from oracle import variational, weight
    from oracle.observables import plaquette_values
    from paper_2412_01737_gb300 import optimize
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    rng = np.random.default_rng(6)
    A = rng.normal(size=(p.m_s, p.m_s))
    A = A - A.T
    dD = {s: (A @ p.gamma_site[s] - p.gamma_site[s] @ A)[2:, 2:] for s in range(p.V) if p.q_phys[s] == 1}
    cfgs = gi.all_z2_configs(p)
    W = weight.Weights(p)
    logs = np.array([W.log_norm(G) for G in cfgs])
    w = np.exp(logs - logs.max())
    w /= w.sum()
    pl = plaquette_values(gi.Z2, 2, cfgs).mean(axis=1)
    dlog = np.array([sum(np.sum(S[s] * dD[s]) for s in dD) for S in (variational.score_sites(p, G) for G in cfgs)])
    exact = np.sum(w * (pl - np.sum(w * pl)) * dlog)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 1024, seed=81), precision=0, seed=9)
    ctx.sample(3)
    ests = []
    for _ in range(8):
        _, C = optimize.wilson_score(ctx, 4)
        ests.append(sum(np.sum(C[s] * dD[s]) for s in dD))
    ctx.close()
    ests = np.array(ests)
    se = ests.std(ddof=1) / np.sqrt(len(ests))
    assert abs(ests.mean() - exact) <= max(5 * se, 0.2 * abs(exact))


@pytest.mark.parametrize("L,grp,n_v,K,prec,tol", [
    (3, gi.Z2, 1, 3, 0, 1e-10),
    (2, gi.U1, 2, 2, 0, 1e-10),
    (4, gi.U1, 1, 2, 1, 1e-4),
])
def test_four_point_matches_oracle(L, grp, n_v, K, prec, tol):
    """<c_2s c_2s+1 c_2t c_2t+1> per link against the oracle's monomial, and
    the density-density correlation it gives lies in [0, 1] (n_s n_t is a
    projector)."""
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=91)
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=prec, seed=4)
    f4 = ctx.chains_fermion4()
    site, _ = ctx.chains_fermion()
    ctx.close()
    fe = fermionic.Fermionic(p)
    for c in range(2):
        for l in range(p.n_links):
            s_, t_ = fermionic._link_sites(p, l)
            want = fe.monomial(links[c], (2 * s_, 2 * s_ + 1, 2 * t_, 2 * t_ + 1))
            assert abs(f4[c, l] - want) <= tol
            nn = (1 + 1j * site[c, s_] + 1j * site[c, t_] - f4[c, l]) / 4
            assert abs(nn.imag) <= 1e-6 and -1e-6 <= nn.real <= 1 + 1e-6


@pytest.mark.parametrize("L,grp,n_v,K,prec,tol", [
    (2, gi.U1, 2, 2, 0, 1e-10),
    (3, gi.Z2, 1, 3, 0, 1e-10),
    (4, gi.U1, 1, 2, 1, 1e-4),
])
def test_link_score_matches_oracle(L, grp, n_v, K, prec, tol):
    from oracle import variational
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=95)
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=prec, seed=6)
    U = ctx.chains_link_score()
    ctx.close()
    for c in range(2):
        ref = variational.score_links(p, links[c])
        assert np.abs(U[c] - ref).max() <= tol * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("grp,n_v", [(gi.Z2, 1), (gi.U1, 1), (gi.SU2, 2)])
def test_wilson_and_polyakov_loops_match_oracle(grp, n_v):
    from oracle.observables import polyakov_values, wilson_loop_values
    p = gi.make_problem(4, grp, n_v, 1)
    links = np.ascontiguousarray(gi.random_links(p, 3, seed=97))
    ctx = ctx_for(p)
    for R, T in ((1, 1), (2, 1), (2, 3), (4, 4)):
        got = ctx.wilson_loop(links, R, T)
        assert np.abs(got - wilson_loop_values(grp, 4, links, R, T).mean(axis=1)).max() <= 1e-13
    got = ctx.polyakov_loop(links)
    assert np.abs(got - polyakov_values(grp, 4, links).mean(axis=1)).max() <= 1e-13
    assert np.abs(ctx.wilson_loop(links, 1, 1) - ctx.observable(links)).max() <= 1e-14
    ctx.close()


def test_state_save_load_continues_bit_exact():
    from paper_2412_01737_gb300 import GGFError
    p = gi.make_problem(3, gi.U1, 1, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.cold_links(p, 3), precision=1, seed=5, delay=4)
    ctx.sample(2)
    state = ctx.save_state()
    a = ctx.sample(3)
    la = ctx.chains_links()
    ctx.load_state(state)
    b = ctx.sample(3)
    lb = ctx.chains_links()
    assert np.array_equal(a, b) and np.array_equal(la, lb)
    bad = state.copy()
    bad[:8] = 0
    with pytest.raises(GGFError):
        ctx.load_state(bad)
    ctx.close()


def test_waves_match_separate_contexts():
    """Two waves paged through one context reproduce two resident contexts."""
    from paper_2412_01737_gb300.waves import Waves
    p = gi.make_problem(3, gi.Z2, 1, 2, bond_scale=0.3)
    starts = [gi.random_links(p, 4, seed=s) for s in (1, 2)]
    ctx = ctx_for(p)
    wv = Waves(ctx, starts, seed=100, precision=0, delay=4)
    obs = wv.sample(3)
    obs2 = wv.sample(2)
    links = wv.links()
    ctx.close()
    for w in range(2):
        c = ctx_for(p)
        c.chains_init(starts[w], precision=0, delay=4, seed=100 + 7919 * w)
        ref = c.sample(3)
        ref2 = c.sample(2)
        assert np.array_equal(obs[w], ref) and np.array_equal(obs2[w], ref2)
        assert np.array_equal(links[w], c.chains_links())
        c.close()


def _divergence(L, J):
    """(n, V) sum over the links leaving a site minus the links entering it."""
    V = L * L
    s = np.arange(V)
    x, y = s % L, s // L
    left = 2 * (y * L + (x - 1) % L)
    down = 2 * (((y - 1) % L) * L + x) + 1
    return J[:, 2 * s] + J[:, 2 * s + 1] - J[:, left] - J[:, down]


@pytest.mark.parametrize("L,n_v,K,prec,tol", [(3, 1, 2, 0, 1e-10), (2, 2, 3, 0, 1e-10), (4, 1, 2, 1, 1e-4)])
def test_u1_field_matches_oracle(L, n_v, K, prec, tol):
    p = gi.make_problem(L, gi.U1, n_v, K, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=17), precision=prec, seed=7, delay=8 if prec else 1)
    ctx.sample(2)
    links = ctx.chains_links()
    J = ctx.chains_electric_field()
    el = electric.Electric(p)
    for c in range(2):
        ref = el.field(links[c])
        assert np.abs(J[c] - ref).max() <= tol * max(1.0, np.abs(ref).max())
    ctx.close()


@pytest.mark.parametrize("L,n_v,K,prec,tol", [(8, 1, 2, 0, 1e-10), (16, 2, 2, 1, 1e-4)])
def test_u1_gauss_law_from_gpu_outputs(L, n_v, K, prec, tol):
    """Gauss's law holds in every configuration at any size: the divergence of
    the field plus the physical charge density vanishes, both read from the
    chains' inverses after sampling (the 16x16 case at the benchmark's n_v)."""
    p = gi.make_problem(L, gi.U1, n_v, K, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 4, seed=23), precision=prec, seed=9, delay=16 if prec else 4)
    ctx.sample(1)
    J = ctx.chains_electric_field()
    site, _ = ctx.chains_fermion()
    n = (1 + 1j * site) / 2
    resid = _divergence(L, J) + p.q_phys[None, :] * n
    assert np.abs(J).max() > 0.01
    assert np.abs(resid).max() <= tol, np.abs(resid).max()
    ctx.close()


def test_u1_field_rejects_other_groups():
    p = gi.make_problem(2, gi.Z2, 1, 1)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 1, seed=1), precision=0, seed=1)
    with pytest.raises(RuntimeError):
        ctx.chains_electric_field()
    ctx.close()


@pytest.mark.parametrize("L,grp,n_v,K,prec,tol", [
    (2, gi.Z2, 1, 2, 0, 1e-10),
    (3, gi.U1, 1, 2, 0, 1e-10),    # odd torus: wrap-around links join equal charges
    (2, gi.U1, 2, 3, 0, 1e-10),
    (4, gi.U1, 1, 2, 1, 1e-4),
])
def test_link_terms_match_oracle(L, grp, n_v, K, prec, tol):
    """Gauge-invariant link terms and their per-pair parts against the
    oracle; the parts contract with lambda to the combined terms."""
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=61), precision=prec, seed=4, delay=8 if prec else 1)
    if prec:
        ctx.sample(2)
    links = ctx.chains_links()
    T, Tp = ctx.chains_link_terms(p.q_phys, pairs=True)
    fe = fermionic.Fermionic(p)
    for c in range(2):
        ref = fe.link_terms(links[c])
        assert np.abs(T[c] - ref).max() <= tol, np.abs(T[c] - ref).max()
        con = np.einsum("n,lnm,m->l", np.conj(p.lam), Tp[c], p.lam)
        assert np.abs(con - T[c]).max() <= tol
    ctx.close()


@pytest.mark.parametrize("grp", [gi.Z2, gi.U1])
def test_link_terms_gauge_invariant_on_gpu(grp):
    """Chains started at G and at a gauge transform of G give the same link
    terms (each from its own inverse), at a size the oracle does not run."""
    p = gi.make_problem(8, grp, 1, 2, bond_scale=0.3)
    G = gi.random_links(p, 1, seed=63)
    rng = np.random.default_rng(5)
    h = rng.uniform(0, 2 * np.pi, p.V) if grp == gi.U1 else rng.choice([-1, 1], p.V)
    Gh = gi.gauge_transform(p, G, h)
    ctx = ctx_for(p)
    ctx.chains_init(np.ascontiguousarray(np.concatenate([G, Gh])), precision=0, seed=1)
    T = ctx.chains_link_terms(p.q_phys)
    assert np.abs(T[0]).max() > 1e-3
    assert np.abs(T[1] - T[0]).max() <= 1e-10
    ctx.close()


def test_link_terms_device_buffers_and_errors():
    torch = pytest.importorskip("torch")
    from paper_2412_01737_gb300 import GGFError
    p = gi.make_problem(3, gi.U1, 1, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=6), precision=0, seed=1)
    T = ctx.chains_link_terms(p.q_phys)
    dev = torch.zeros((2, p.n_links, 2), dtype=torch.float64, device="cuda")
    ctx.chains_link_terms(p.q_phys, out=dev)
    d = dev.cpu().numpy()
    assert np.array_equal(d[..., 0] + 1j * d[..., 1], T)
    with pytest.raises(GGFError):
        ctx.chains_link_terms(np.zeros(p.V, dtype=np.int32))
    ctx.close()
    s = gi.make_problem(1, gi.SU2, 2, 1)
    cs = ctx_for(s)
    cs.chains_init(gi.random_links(s, 1, seed=2), precision=0, seed=1)
    with pytest.raises(GGFError):
        cs.chains_link_terms(np.ones(s.V, dtype=np.int32))
    cs.close()


def test_reweighted_energy_gradient_on_gpu():
    """energy_gradient through the GPU context (log-weights, Wilson loops,
    electric, fermionic and link terms of every configuration), with the 256
    configurations of the 2x2 Z2 lattice weighted by p(G): equals the
    central difference of the oracle's exhaustive energies along a site and
    a bond rotation."""
    from oracle import variational as va, weight
    from paper_2412_01737_gb300 import optimize
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    cfgs = np.ascontiguousarray(gi.all_z2_configs(p))
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

    def exact(q):
        S = va.exhaustive(q, cfgs)
        hop = np.einsum("l,lnm->nm", ch, S["hopping"])
        H = (-1.0 * S["plaquette"] + np.einsum("l,lnm->nm", ce, S["electric"])
             + np.einsum("s,snm->nm", cs, 0.5 * (S["norm"] + 1j * S["density"])) + hop + hop.conj().T)
        return float(va.expectation(H, S["norm"], q.lam).real)

    dirs = [lambda t: optimize.rotate_sites(p, A, t), lambda t: optimize.rotate_bonds(p, 1, Bg, t)]
    delta = 1e-3
    ctx = ctx_for(p)
    e0, g = optimize.energy_gradient(ctx, p, cfgs, dirs, delta=delta, weights=w0, c_plaquette=-1.0,
                                     c_electric=ce, c_site=cs, c_hop=ch, charges=p.q_phys)
    ctx.close()
    assert abs(e0 - exact(p)) <= 1e-9
    for k, d in enumerate(dirs):
        fd = (exact(d(delta)) - exact(d(-delta))) / (2 * delta)
        assert abs(g[k] - fd) <= 1e-6 * max(1.0, abs(fd)), (k, g[k], fd)


def test_descend_with_gpu_samples():
    """Two iterations of optimize.descend with configurations sampled by GPU
    chains (512 chains, 10 recorded sweeps) and the forms and gradients
    computed through the library: the energy of the final parameters (exact,
    exhaustive oracle) is far below the starting one (start +0.78, exact
    lambda optimum -2.21 for the starting Gaussians)."""
    from oracle import variational as va
    from paper_2412_01737_gb300 import optimize
    p = gi.make_problem(2, gi.Z2, 1, 2, bond_scale=0.3)
    cfgs = gi.all_z2_configs(p)
    rng = np.random.default_rng(9)
    A = rng.normal(size=(p.m_s, p.m_s))
    A = 0.2 * (A - A.T)
    Bg = rng.normal(size=(p.r, p.r))
    Bg = 0.2 * (Bg - Bg.T)
    ce = 0.5 * np.ones(p.n_links)
    cs = 0.4 * p.q_phys.astype(float)
    ch = 0.3 * np.ones(p.n_links)
    kw = dict(c_plaquette=-1.0, c_electric=ce, c_site=cs, c_hop=ch, charges=p.q_phys)
    sctx = ctx_for(p)

    def sampler(q):
        sctx.init_problem(q)
        sctx.chains_init(gi.random_links(q, 512, seed=71), precision=0, seed=12)
        sctx.sample(5)
        out = []
        for _ in range(10):
            sctx.sample(1)
            out.append(sctx.chains_links().copy())
        return np.ascontiguousarray(np.concatenate(out)), None

    def exact(q):
        S = va.exhaustive(q, cfgs)
        hop = np.einsum("l,lnm->nm", ch, S["hopping"])
        H = (-1.0 * S["plaquette"] + np.einsum("l,lnm->nm", ce, S["electric"])
             + np.einsum("s,snm->nm", cs, 0.5 * (S["norm"] + 1j * S["density"])) + hop + hop.conj().T)
        return float(va.expectation(H, S["norm"], q.lam).real)

    gctx = ctx_for(p)
    dirs = [lambda q, t: optimize.rotate_sites(q, A, t), lambda q, t: optimize.rotate_bonds(q, 1, Bg, t)]
    q, hist = optimize.descend(gctx, p, sampler, dirs, n_iter=2, lr=0.05, **kw)
    gctx.close()
    sctx.close()
    assert abs(hist[0] - (-2.2105)) <= 0.3
    assert exact(q) < exact(p) - 2.5


@pytest.mark.parametrize("grp", [gi.Z2, gi.U1])
def test_link_terms_and_field_on_the_1x1_torus(grp):
    """Self-links (both ends on one site): the link term is u_l <psi psi^dag>
    = u_l (1 - <n>) for a positive charge (the oracle agrees to 1e-15), and
    the U(1) field of the two self-links matches the oracle."""
    p = gi.make_problem(1, grp, 2, 2, bond_scale=0.3)
    links = gi.random_links(p, 3, seed=81)
    ctx = ctx_for(p)
    ctx.chains_init(links, precision=0, seed=2)
    T = ctx.chains_link_terms(p.q_phys)
    site, _ = ctx.chains_fermion()
    fe = fermionic.Fermionic(p)
    for c in range(3):
        assert np.abs(T[c] - fe.link_terms(links[c])).max() <= 1e-10
        u = links[c].astype(float) if grp == gi.Z2 else np.exp(1j * links[c])
        n = (1 + 1j * site[c, 0]) / 2
        assert np.abs(T[c] - u * (1 - n)).max() <= 1e-10
    if grp == gi.U1:
        J = ctx.chains_electric_field()
        el = electric.Electric(p)
        for c in range(3):
            assert np.abs(J[c] - el.field(links[c])).max() <= 1e-10
    ctx.close()


def test_loop_and_pair_argument_errors():
    """Rejected arguments come back as errors with the context still usable:
    loops larger than the lattice, an unknown per-pair quantity; an empty
    batch of configurations is a no-op."""
    from paper_2412_01737_gb300 import GGFError
    p = gi.make_problem(3, gi.U1, 1, 2, bond_scale=0.3)
    links = np.ascontiguousarray(gi.random_links(p, 2, seed=7))
    ctx = ctx_for(p)
    with pytest.raises(GGFError):
        ctx.wilson_loop(links, 4, 1)
    with pytest.raises(GGFError):
        ctx.wilson_loop(links, 1, 0)
    assert ctx.wilson_loop(np.ascontiguousarray(links[:0]), 1, 1).shape == (0,)
    ctx.chains_init(links, precision=0, seed=1)
    with pytest.raises(GGFError):
        ctx.chains_pairs(7, out=np.zeros((2, p.K, p.K, 2)))
    from oracle.observables import wilson_loop_values
    assert np.abs(ctx.wilson_loop(links, 3, 3) - wilson_loop_values(gi.U1, 3, links, 3, 3).mean(axis=1)).max() <= 1e-13
    ctx.close()


def test_u1_gradient_on_gpu_matches_oracle_on_the_same_samples():
    """The reweighted gradient along a U(1)-symmetric site rotation from the
    GPU (log-weights, Wilson loops, electric, fermionic and link terms of
    every sample under the offset parameters) against the same estimator
    evaluated by the oracle on the same sampled configurations (3x3 torus,
    K = 2): equal up to rounding."""
    from paper_2412_01737_gb300 import optimize
    from tests.test_optimize import _OracleCtx
    p = gi.make_problem(3, gi.U1, 1, 2, bond_scale=0.3)
    sctx = ctx_for(p)
    sctx.chains_init(gi.random_links(p, 64, seed=5), precision=0, seed=4)
    sctx.sample(3)
    links = np.ascontiguousarray(sctx.chains_links())
    sctx.close()
    rng = np.random.default_rng(2)
    A = rng.normal(size=(p.m_s, p.m_s))
    A = A - A.T
    plus = [s for s in range(p.V) if p.q_phys[s] > 0]
    Ap = optimize.u1_generator(A, gi.site_charges(p.n_v, 1))
    dirs = [lambda t: optimize.rotate_sites(p, Ap, t, sites=plus)]
    kw = dict(c_plaquette=-1.0, c_electric=0.5 * np.ones(p.n_links), c_site=0.4 * p.q_phys.astype(float),
              c_hop=0.3 * np.ones(p.n_links), charges=p.q_phys)
    gctx = ctx_for(p)
    e_gpu, g_gpu = optimize.energy_gradient(gctx, p, links, dirs, **kw)
    gctx.close()
    e_ref, g_ref = optimize.energy_gradient(_OracleCtx(), p, links, dirs, **kw)
    assert abs(e_gpu - e_ref) <= 1e-10 * max(1.0, abs(e_ref))
    assert abs(g_gpu[0] - g_ref[0]) <= 1e-6 * max(1.0, abs(g_ref[0]))


@pytest.mark.parametrize("L,n_v,K,prec,tol", [(3, 1, 2, 0, 1e-10), (2, 2, 3, 0, 1e-10), (4, 1, 2, 1, 1e-4)])
def test_field_pair_parts_match_oracle(L, n_v, K, prec, tol):
    """PAIRS_FIELD against the oracle's per-pair field forms; contracted with
    lambda they give ggf_chains_electric_field.  Rejected for Z2 chains."""
    from oracle import variational
    from paper_2412_01737_gb300 import GGFError
    from paper_2412_01737_gb300.ggf import PAIRS_FIELD
    p = gi.make_problem(L, gi.U1, n_v, K, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=19), precision=prec, seed=3, delay=8 if prec else 1)
    if prec:
        ctx.sample(2)
    links = ctx.chains_links()
    fp = ctx.chains_pairs(PAIRS_FIELD)
    J = ctx.chains_electric_field()
    ctx.close()
    lm = variational.LocalMatrices(p)
    for c in range(2):
        ref = lm(links[c])["field"]
        assert np.abs(fp[c] - ref).max() <= tol * max(1.0, np.abs(ref).max())
        con = np.einsum("n,lnm,m->l", np.conj(p.lam), fp[c], p.lam)
        assert np.abs(con - J[c]).max() <= tol * max(1.0, np.abs(J[c]).max())
    z = gi.make_problem(2, gi.Z2, 1, 2)
    zc = ctx_for(z)
    zc.chains_init(gi.random_links(z, 1, seed=1), precision=0, seed=1)
    with pytest.raises(GGFError):
        zc.chains_pairs(PAIRS_FIELD, out=np.zeros((1, z.n_links, 2, 2, 2)))
    zc.close()


@pytest.mark.parametrize("L,grp,n_v,K,prec,tol", [
    (3, gi.Z2, 1, 3, 0, 1e-10),
    (2, gi.U1, 2, 2, 0, 1e-10),
    (1, gi.U1, 1, 2, 0, 1e-10),     # self-links: -N_nm / N(G)
    (4, gi.U1, 1, 2, 1, 1e-4),
])
def test_four_point_pair_parts_match_oracle(L, grp, n_v, K, prec, tol):
    """PAIRS_FOUR against the oracle's per-pair four-point forms; contracted
    with lambda they give ggf_chains_fermion4."""
    from oracle import variational
    from paper_2412_01737_gb300.ggf import PAIRS_FOUR
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 2, seed=29), precision=prec, seed=3, delay=8 if prec else 1)
    if prec:
        ctx.sample(2)
    links = ctx.chains_links()
    fp = ctx.chains_pairs(PAIRS_FOUR)
    f4 = ctx.chains_fermion4()
    ctx.close()
    lm = variational.LocalMatrices(p)
    for c in range(2):
        ref = lm(links[c])["four"]
        assert np.abs(fp[c] - ref).max() <= tol * max(1.0, np.abs(ref).max())
        con = np.einsum("n,lnm,m->l", np.conj(p.lam), fp[c], p.lam)
        assert np.abs(con - f4[c]).max() <= tol
