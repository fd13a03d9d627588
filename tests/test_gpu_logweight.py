"""GPU parity of ggf_logweight against the FP64 oracle (covariance route).

Tolerance: |Delta log N| <= 1e-10 (FP64 path).  Per-pair terms: the GPU's
c_nm Pf(M_nm(G)) on the reduced virtual matrix against the oracle's full
(physical + virtual) Pfaffian route, magnitude and phase."""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import weight
from tests.gpu_util import ctx_for, oracle_log_nm, phase_dist

pytestmark = pytest.mark.gpu
TOL = 1e-10


def check(p, links, pairs=True):
    ctx = ctx_for(p)
    W = weight.Weights(p)
    P = p.K * (p.K + 1) // 2
    ell = np.zeros((len(links), P, 2))
    got = ctx.logweight(links, ell=ell)
    want = np.array([W.log_norm(c) for c in links])
    assert np.all(np.isfinite(got))
    assert np.abs(got - want).max() <= TOL * max(1.0, np.abs(want).max())
    if pairs:
        lc, pr = ctx.get_constants()
        onm = oracle_log_nm(W, links)
        for k, (n, m) in enumerate(pr):
            g = lc[k] + ell[:, k, 0] + 1j * ell[:, k, 1]
            o = onm[:, n, m]
            assert np.abs(g.real - o.real).max() <= TOL * max(1.0, np.abs(o.real).max())
            if n != m:
                assert phase_dist(g.imag, o.imag).max() <= 1e-9
    ctx.close()


def test_z2_exhaustive_2x2_k1():
    p = gi.make_problem(2, gi.Z2, 1, 1)
    check(p, gi.all_z2_configs(p))


def test_z2_2x2_k2_random_sites():
    p = gi.make_problem(2, gi.Z2, 1, 2, site_mode="random", bond_mode="random", bond_scale=0.3)
    check(p, np.ascontiguousarray(gi.all_z2_configs(p)[::9]))


@pytest.mark.parametrize("L,nv,K", [(2, 1, 2), (1, 2, 3), (2, 2, 2), (3, 2, 4)])
def test_u1_random(L, nv, K):
    p = gi.make_problem(L, gi.U1, nv, K, bond_scale=0.3, site_mode="random", bond_mode="random")
    check(p, gi.random_links(p, 5, seed=L * 10 + K))


@pytest.mark.parametrize("L,grp,nv,K", [(5, gi.Z2, 1, 1), (6, gi.U1, 1, 2), (5, gi.U1, 2, 2)])
def test_several_tiles_ragged(L, grp, nv, K):
    # N = 8 n_v L^2 = 200, 288, 400: several 32-wide tiles with a ragged tail
    p = gi.make_problem(L, grp, nv, K, bond_scale=0.2)
    check(p, gi.random_links(p, 3, seed=5), pairs=(K > 1))


def test_cfg2_full_size_sampled():
    """8x8 Z2, K=1 (M is 512 x 512): sampled configurations."""
    p = gi.make_problem(8, gi.Z2, 1, 1)
    check(p, gi.random_links(p, 3, seed=8), pairs=False)


def test_gauge_invariance_on_gpu():
    p = gi.make_problem(4, gi.U1, 2, 2, bond_scale=0.2)
    ctx = ctx_for(p)
    links = gi.random_links(p, 2, seed=4)
    h = np.random.default_rng(0).uniform(0, 2 * np.pi, p.V)
    a = ctx.logweight(links)
    b = ctx.logweight(np.ascontiguousarray(gi.gauge_transform(p, links, h)))
    assert np.abs(a - b).max() < 1e-10
    ctx.close()


def test_device_tensors_and_plaquette():
    import torch
    p = gi.make_problem(3, gi.U1, 1, 2)
    ctx = ctx_for(p)
    links = gi.random_links(p, 6, seed=2)
    host = ctx.logweight(links)
    dl = torch.from_numpy(links).cuda()
    dev = ctx.logweight(dl)
    torch.cuda.synchronize()
    assert np.abs(dev.cpu().numpy() - host).max() == 0.0
    from oracle.observables import plaquette_mean
    pl = ctx.observable(links)
    assert np.abs(pl - plaquette_mean(p.group, p.L, links)).max() < 1e-13
    ctx.close()


def test_bad_arguments_raise():
    from paper_2412_01737_gb300 import GGF, GGFError
    c = GGF(0)
    with pytest.raises(GGFError):
        c.init_lattice(0)
    c.init_lattice(2)
    with pytest.raises(GGFError):
        c.init_group(gi.U1, 3, [1, -1, 1])
    c.close()
