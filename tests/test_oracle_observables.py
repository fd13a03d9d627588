import numpy as np

import ggf_inputs as gi
from oracle.observables import plaquette_values, tau_int, plaquette_links


def test_plaquette_z2_single_flip():
    L = 3
    links = np.ones((1, 2 * L * L), dtype=np.int8)
    links[0, 2 * 4 + 0] = -1           # x-link from site 4
    v = plaquette_values(gi.Z2, L, links)[0]
    # that link borders the plaquette at site 4 (as +l1) and at site 1 (as -l3)
    assert v[4] == -1 and v[1] == -1 and np.sum(v == -1) == 2


def test_plaquette_u1_orientation():
    L = 2
    th = np.zeros((1, 8))
    pl = plaquette_links(L)
    s = 0
    th[0, pl[s, 0]] += 0.1
    th[0, pl[s, 1]] += 0.2
    th[0, pl[s, 2]] += 0.4
    v = plaquette_values(gi.U1, L, th)[0]
    # on a 2x2 torus each link belongs to two plaquettes; plaquette 0 sees 0.1 + 0.2 - 0.4
    assert abs(v[0] - np.cos(0.1 + 0.2 - 0.4 - th[0, pl[0, 3]])) < 1e-15


def test_tau_int_ar1():
    rng = np.random.default_rng(0)
    a = 0.8
    x = np.zeros((64, 4000))
    x[:, 0] = rng.normal(size=64)
    for t in range(1, x.shape[1]):
        x[:, t] = a * x[:, t - 1] + np.sqrt(1 - a * a) * rng.normal(size=64)
    tau, _ = tau_int(x)
    assert abs(tau - (1 + a) / (2 * (1 - a))) < 0.25
