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



def test_loops_reduce_to_plaquettes_and_products():
    from oracle.observables import plaquette_values, wilson_loop_values
    for grp in (gi.Z2, gi.U1, gi.SU2):
        p = gi.make_problem(3, grp, 2 if grp == gi.SU2 else 1, 1)
        G = gi.random_links(p, 2, seed=4)
        assert np.abs(wilson_loop_values(grp, 3, G, 1, 1) - plaquette_values(grp, 3, G)).max() <= 1e-14
    # Z2: a rectangle is the product of the plaquettes it encloses
    p = gi.make_problem(4, gi.Z2, 1, 1)
    G = gi.random_links(p, 3, seed=5)
    P1 = plaquette_values(gi.Z2, 4, G)
    W23 = wilson_loop_values(gi.Z2, 4, G, 2, 3)
    for s in range(16):
        x, y = s % 4, s // 4
        inside = [((y + b) % 4) * 4 + (x + a) % 4 for a in range(2) for b in range(3)]
        assert np.array_equal(W23[:, s], np.prod(P1[:, inside], axis=1))


def test_loops_gauge_invariant():
    from oracle.observables import polyakov_values, wilson_loop_values
    for grp, nv in ((gi.Z2, 1), (gi.U1, 1), (gi.SU2, 2)):
        p = gi.make_problem(3, grp, nv, 1)
        G = gi.random_links(p, 2, seed=6)
        if grp == gi.Z2:
            h = np.array([1, -1, -1, 1, 1, -1, 1, -1, 1], dtype=np.int8)
        elif grp == gi.U1:
            h = np.random.default_rng(1).uniform(0, 2 * np.pi, p.V)
        else:
            h = gi.random_links(p, 1, seed=7)[0][:p.V]
        hG = gi.gauge_transform(p, G, h)
        for R, T in ((1, 2), (2, 2), (3, 1)):
            assert np.abs(wilson_loop_values(grp, 3, G, R, T) - wilson_loop_values(grp, 3, hG, R, T)).max() <= 1e-12
        assert np.abs(polyakov_values(grp, 3, G) - polyakov_values(grp, 3, hG)).max() <= 1e-12


def test_winding_loops_z2():
    from oracle.observables import polyakov_values, wilson_loop_values
    p = gi.make_problem(4, gi.Z2, 1, 1)
    G = gi.random_links(p, 2, seed=8)
    Pk = polyakov_values(gi.Z2, 4, G)
    W = wilson_loop_values(gi.Z2, 4, G, 2, 4)            # T = L: two winding loops, x and x + 2
    for s in range(4):
        assert np.array_equal(W[:, s], Pk[:, s % 4] * Pk[:, (s + 2) % 4])
    cold = gi.cold_links(p, 1)
    cold[0, 2 * (1 * 4 + 2) + 1] = -1                    # the y link from site (2, 1)
    Pc = polyakov_values(gi.Z2, 4, cold)[0]
    assert Pc[2] == -1 and np.sum(Pc == -1) == 1
