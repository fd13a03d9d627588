"""GPU parity of the periodic refresh (Sec. 5: N_nm(G) = c_nm Pf(M_nm(G))).

The refresh gives a chain fresh log-weights from the site-by-site FP64
Pfaffian and, for FP32 chains, refines the cached inverse by a Newton step on
the tensor cores.  Checked against the oracle: the refreshed per-pair
log-weights against the oracle's full-space Pfaffian route (1e-10 relative
magnitude, 1e-9 phase), the refreshed FP32 inverse element by element against
numpy's inverse of the reduced matrix D + O Gamma_X O^T built from the
oracle's covariances, and the FP64 log-weights at the largest lattice with a
complex pair against values the oracle wrote into tests/golden/."""
import json
import os

import numpy as np
import pytest

import ggf_inputs as gi
from oracle import weight
from tests.gpu_util import ctx_for, oracle_log_nm, phase_dist

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def reduced_matrix(p, G, n, m):
    """D + O(G) Gamma_X^{nm} O(G)^T on the virtual Majoranas, from the oracle."""
    W = weight.Weights(p)
    virt = np.array([i for i in range(p.m_s * p.V) if i % p.m_s >= 2])
    Ov = weight.twist_matrix(p, G)[np.ix_(virt, virt)]
    B = 8 * p.n_v
    D = np.zeros((B * p.V, B * p.V))
    for s in range(p.V):
        D[s * B:(s + 1) * B, s * B:(s + 1) * B] = p.gamma_site[s][2:, 2:]
    M = D + Ov @ W.GX[n, m][np.ix_(virt, virt)] @ Ov.T
    return M.real if n == m else M


@pytest.mark.parametrize("L,grp,nv,K", [(4, gi.U1, 2, 2), (3, gi.Z2, 1, 2)])
def test_newton_step_on_fresh_inverse(L, grp, nv, K):
    """Right after chains_init the FP32 inverse is the rounded FP64 one: its
    residual is at the FP32 floor, it agrees with numpy's inverse of the
    oracle's reduced matrix, and a Newton step keeps both."""
    from paper_2412_01737_gb300 import FP32
    p = gi.make_problem(L, grp, nv, K, bond_scale=0.3)
    ctx = ctx_for(p)
    links = gi.random_links(p, 2, seed=L + K)
    ctx.chains_init(links, precision=FP32, refresh_every=10**9, seed=9, delay=4)
    lc, pr = ctx.get_constants()
    N = 8 * nv * L * L
    for k, (n, m) in enumerate(pr):
        want = np.linalg.inv(reduced_matrix(p, links[1], n, m))
        got = ctx.chains_inverse(1, k, N)
        got = got.real if n == m else got
        r0 = ctx.chains_refine(1, k, apply=False)
        r1 = ctx.chains_refine(1, k, apply=True)
        r2 = ctx.chains_refine(1, k, apply=False)
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
        assert r0 < 1e-5 and r1 == r0 and r2 < 1e-5
        got = ctx.chains_inverse(1, k, N)
        got = got.real if n == m else got
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    ctx.close()


@pytest.mark.parametrize("L,grp,nv,K,delay", [(4, gi.U1, 2, 2, 4), (3, gi.Z2, 1, 2, 1), (4, gi.U1, 1, 3, 8)])
def test_fp32_refresh_every_sweep(L, grp, nv, K, delay):
    """refresh_every = 1: every chain that accepted is refreshed after each
    sweep, so its log-weights are the fresh FP64 values and its inverse the
    Newton-refined one."""
    from paper_2412_01737_gb300 import FP32
    p = gi.make_problem(L, grp, nv, K, bond_scale=0.3)
    ctx = ctx_for(p)
    nch = 3
    ctx.chains_init(gi.random_links(p, nch, seed=L + K), precision=FP32, refresh_every=1, seed=9, delay=delay)
    ctx.sample(3)
    st = ctx.chains_stats()
    assert st.refreshes > 0
    assert st.dense_refreshes == 0
    assert 0.0 < st.max_resid < 1e-4
    links = ctx.chains_links()
    ell = ctx.chains_ell()
    lc, pr = ctx.get_constants()
    Wo = weight.Weights(p)
    onm = oracle_log_nm(Wo, links)
    N = 8 * nv * L * L
    for k, (n, m) in enumerate(pr):
        g = lc[k] + ell[:, k]
        o = onm[:, n, m]
        assert np.abs(g.real - o.real).max() <= 1e-10 * max(1.0, np.abs(o.real).max())
        if n != m:
            assert phase_dist(g.imag, o.imag).max() <= 1e-9
        for c in range(nch):
            want = np.linalg.inv(reduced_matrix(p, links[c], n, m))
            got = ctx.chains_inverse(c, k, N)
            if n == m:
                got = got.real
            assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    ctx.close()


def test_logweight_8x8_u1_k4_pairs():
    """N = 1024, K = 4 (four real and six complex pairs), per-pair magnitude
    and phase against the oracle."""
    p = gi.make_problem(8, gi.U1, 2, 4, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=31)
    ctx = ctx_for(p)
    ell = np.zeros((2, 10, 2))
    got = ctx.logweight(links, ell=ell)
    W = weight.Weights(p)
    want = np.array([W.log_norm(c) for c in links])
    assert np.abs(got - want).max() <= 1e-10 * max(1.0, np.abs(want).max())
    lc, pr = ctx.get_constants()
    onm = oracle_log_nm(W, links)
    for k, (n, m) in enumerate(pr):
        g = lc[k] + ell[:, k, 0] + 1j * ell[:, k, 1]
        o = onm[:, n, m]
        assert np.abs(g.real - o.real).max() <= 1e-10 * max(1.0, np.abs(o.real).max())
        if n != m:
            assert phase_dist(g.imag, o.imag).max() <= 1e-9
    ctx.close()


def test_logweight_16x16_u1_k2_golden():
    """16 x 16 U(1), n_v = 2 (N = 4096), K = 2: log N(G) and the three pair
    terms of one seeded configuration against the oracle's values, written by
    tests/golden/make_fullsize_u1.py (a 4608 x 4608 complex Pfaffian per pair
    on the full physical + virtual space)."""
    with open(os.path.join(HERE, "golden", "u1_16x16_nv2_k2.json")) as f:
        gold = json.load(f)
    p = gi.make_problem(16, gi.U1, 2, 2, seed=gold["seed"], bond_scale=gold["bond_scale"])
    links = gi.random_links(p, 1, seed=gold["links_seed"])
    ctx = ctx_for(p)
    ell = np.zeros((1, 3, 2))
    got = ctx.logweight(links, ell=ell)
    assert abs(got[0] - gold["log_norm"]) <= 1e-10 * max(1.0, abs(gold["log_norm"]))
    lc, pr = ctx.get_constants()
    for k, (n, m) in enumerate(pr):
        o = complex(*gold["log_n_nm"][f"{n}{m}"])
        g = lc[k] + ell[0, k, 0] + 1j * ell[0, k, 1]
        assert abs(g.real - o.real) <= 1e-10 * max(1.0, abs(o.real))
        if n != m:
            assert phase_dist(np.array([g.imag]), np.array([o.imag])).max() <= 1e-9
    ctx.close()


def test_newton_step_repairs_a_perturbed_inverse():
    """A Newton step (three-product split for a residual of 1e-3, one product
    below 1e-4) brings an inverse with a perturbed entry back to the FP32
    floor: the perturbation is planted in W on the device through the
    diagnostic hook, and the refined W matches numpy's inverse again."""
    from paper_2412_01737_gb300 import FP32
    p = gi.make_problem(4, gi.U1, 2, 2, bond_scale=0.3)
    ctx = ctx_for(p)
    links = gi.random_links(p, 1, seed=12)
    ctx.chains_init(links, precision=FP32, refresh_every=10**9, seed=9, delay=4)
    N = 8 * 2 * 16
    lc, pr = ctx.get_constants()
    for k, (n, m) in enumerate(pr):
        want = np.linalg.inv(reduced_matrix(p, links[0], n, m))
        ctx.debug_scale_inverse(0, k, 1.0 + 1e-3)
        r0 = ctx.chains_refine(0, k, apply=True)
        assert 5e-4 < r0 < 5e-2
        r1 = ctx.chains_refine(0, k, apply=True)
        assert r1 < 1e-5 < r0
        r2 = ctx.chains_refine(0, k, apply=False)
        assert r2 < 1e-5
        got = ctx.chains_inverse(0, k, N)
        got = got.real if n == m else got
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    ctx.close()


def test_newton_step_at_full_size():
    """At the benchmark's matrix order (16x16 U(1), n_v = 2, K = 2: N = 4096,
    real and complex pairs) a planted 1e-3 scaling of each pair's FP32
    inverse is repaired by the tensor-core Newton steps (a three-product step
    for the 1e-3 residual, then the residual at the level of the freshly
    factored inverse)."""
    from paper_2412_01737_gb300 import FP32
    p = gi.make_problem(16, gi.U1, 2, 2, seed=20241202)
    ctx = ctx_for(p)
    ctx.chains_init(gi.random_links(p, 1, seed=3), precision=FP32, refresh_every=10**9, seed=9, delay=16)
    for k in range(3):
        fresh = ctx.chains_refine(0, k, apply=False)
        assert fresh < 1e-5
        ctx.debug_scale_inverse(0, k, 1.0 + 1e-3)
        r0 = ctx.chains_refine(0, k, apply=True)
        assert 5e-4 < r0 < 5e-2
        ctx.chains_refine(0, k, apply=True)
        r2 = ctx.chains_refine(0, k, apply=False)
        assert r2 <= max(2 * fresh, 1e-5), (k, fresh, r2)
    ctx.close()
