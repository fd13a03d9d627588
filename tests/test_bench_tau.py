"""The benchmark's autocorrelation estimate (Madras-Sokal window, c = 5)
against the closed form of an AR(1) process: x_{t+1} = rho x_t + e_t has
normalised autocorrelation rho^t, so tau_int = 1/2 + sum_{t>=1} rho^t =
(1 + rho) / (2 (1 - rho)).  CPU only."""
import numpy as np
import pytest

import bench


def _ar1(rho, chains, T, seed):
    rng = np.random.default_rng(seed)
    x = np.empty((chains, T))
    x[:, 0] = rng.standard_normal(chains)
    e = rng.standard_normal((chains, T)) * np.sqrt(1 - rho * rho)
    for t in range(1, T):
        x[:, t] = rho * x[:, t - 1] + e[:, t]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8, 0.9])
def test_tau_int_matches_ar1_closed_form(rho):
    want = (1 + rho) / (2 * (1 - rho))
    tau, window, closed = bench.tau_int(_ar1(rho, 64, 4000, seed=int(rho * 10)))
    assert closed and window >= 5 * tau - 1
    # the window truncation (c = 5) biases tau low by at most ~rho^(5 tau)
    assert abs(tau - want) <= 0.05 * want + 0.02, (tau, want)


def test_short_series_reports_an_open_window():
    tau, window, closed = bench.tau_int(_ar1(0.95, 8, 20, seed=3))
    assert not closed and window == 19


def test_tau_report_takes_the_larger_series_and_removes_common_drift():
    chains, T = 32, 3000
    plaq = _ar1(0.5, chains, T, seed=1)
    logn = _ar1(0.9, chains, T, seed=2)
    drift = np.linspace(0, 50, T)[None, :]          # common to all chains
    ser = np.stack([plaq + drift, logn - drift], axis=2)
    tau, closed, det = bench.tau_report(ser)
    assert closed
    assert det["plaquette"]["tau"] < det["logN"]["tau"] == tau
    assert abs(tau - 9.5) <= 0.05 * 9.5 + 0.02
