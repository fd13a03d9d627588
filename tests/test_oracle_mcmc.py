"""Pin the oracle sampler to the exhaustive distribution of the 2x2 Z2
lattice and check the U(1) proposal/wrap rule."""
import numpy as np

import ggf_inputs as gi
from oracle import mcmc, weight
from oracle.observables import plaquette_mean, tau_int


def test_z2_chain_matches_exhaustive_distribution():
    p = gi.make_problem(2, gi.Z2, 1, 1)
    W = weight.Weights(p)
    cfgs = gi.all_z2_configs(p)
    logs = np.array([W.log_norm(c) for c in cfgs])
    pg = np.exp(logs - logs.max())
    pg /= pg.sum()
    wl = plaquette_mean(p.group, p.L, cfgs)
    exact_w = float(pg @ wl)
    _, obs, _ = mcmc.run_chain(p, W, gi.cold_links(p)[0], 20241202, 0, 0, 6000)
    series = obs[200:, 0]
    tau, _ = tau_int(series[None, :])
    err = series.std() * np.sqrt(2 * max(tau, 0.5) / series.size)
    assert abs(series.mean() - exact_w) < 4 * err + 1e-12
    # distribution of the plaquette mean over its values {-1, 0, 1, -0.5, 0.5}
    vals = np.unique(wl)
    exp_p = np.array([pg[wl == v].sum() for v in vals])
    obs_p = np.array([(series == v).mean() for v in vals])
    n_eff = series.size / (2 * max(tau, 0.5))
    mask = exp_p > 0.02
    chi2 = n_eff * np.sum((obs_p[mask] - exp_p[mask]) ** 2 / exp_p[mask])
    assert chi2 < 30.0
    assert np.all(obs_p[exp_p == 0] == 0)


def test_u1_proposal_wraps_into_range():
    for th, u in [(6.2, 0.99), (0.01, 0.0), (3.0, 0.5), (2 * np.pi - 1e-17, 0.5)]:
        t = mcmc.propose(gi.U1, th, u, 0.5)
        assert 0.0 <= t < 2 * np.pi
    assert mcmc.propose(gi.Z2, -1, 0.3, 0.5) == 1


def test_u1_chain_runs_and_logs_consistent():
    p = gi.make_problem(2, gi.U1, 1, 2)
    W = weight.Weights(p)
    links, obs, dec = mcmc.run_chain(p, W, gi.cold_links(p)[0], 5, 3, 10, 3, record_decisions=True)
    assert len(dec) == 3 * p.n_links
    assert abs(obs[-1, 1] - W.log_norm(links)) < 1e-12
    for (_, _, acc, u, R) in dec:
        assert acc == (u < R)
