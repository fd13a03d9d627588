"""Helpers shared by the GPU tests."""
import numpy as np


def ctx_for(p):
    from paper_2412_01737_gb300 import GGF
    c = GGF(0)
    c.init_problem(p)
    return c


def oracle_log_nm(W, links):
    """(n_cfg, K, K) complex log N_nm from the oracle."""
    return np.array([W.log_n_matrix(c) for c in links])


def phase_dist(a, b):
    return np.abs(np.angle(np.exp(1j * (a - b))))
