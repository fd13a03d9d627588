"""Sequential-sweep Metropolis sampling of p(G) = N(G) / N (Sec. 5.1).

The weight is sign-free, so plain Metropolis over link configurations
applies.  One sweep proposes every link l = 0 .. 2V-1 in order:

* Z2: g_l -> -g_l.
* U(1): theta_l -> theta_l + w (u_prop - 1/2), wrapped into [0, 2 pi) by one
  conditional add/subtract of 2 pi (w is the full proposal width).
* SU(2): g_l -> r g_l with r = cos d + i sin d (n . sigma), d = w (u_prop - 1/2),
  n the unit vector (sqrt(1 - z^2) cos phi, sqrt(1 - z^2) sin phi, z) with
  z = 2 u_z - 1, phi = 2 pi u_phi (Philox words 2 and 3), the product
  renormalised to a unit quaternion.  r and r^dag are equally likely, so the
  proposal is symmetric with respect to the Haar measure; on the U(1)
  subgroup exp(i theta sigma_z) with n = z it is the U(1) move.
* Accept iff u_acc < N(G') / N(G); a proposal with N(G') <= 0 is rejected.

Random numbers come from oracle.philox with counter (sweep, link, 0, 0) and
key (seed, chain).  Every proposal recomputes log N(G') from scratch with
oracle.weight (no low-rank updates), so this is the exact reference for the
sampler's accept/reject decisions.

Per sweep it records: plaquette mean, log N(G) at the end of the sweep and
the sweep's acceptance rate.

Pinned (tests/test_oracle_mcmc.py): on the 2x2 Z2 lattice the visit
histogram of a long chain agrees with the exhaustive p(G) (chi^2) and the
plaquette mean with sum_G p(G) W(G) within 4 sigma.  SU(2)
(tests/test_oracle_su2.py): the proposal is reversible, unitary and the U(1)
move on the subgroup; on the 1x1 torus the chain's plaquette mean agrees with
Haar importance sampling within 4 sigma.
"""
from __future__ import annotations

import numpy as np

from .philox import draws4
from .observables import plaquette_mean
from .weight import Weights

Z2, U1, SU2 = 0, 1, 2
TWO_PI = 2.0 * np.pi


def quat_mul(a, b):
    """Quaternion product in the (a0, a1, a2, a3) <-> a0 + i a.sigma convention."""
    a0, av = a[0], np.asarray(a[1:])
    b0, bv = b[0], np.asarray(b[1:])
    # (a0 + i a.s)(b0 + i b.s) = a0 b0 - a.b + i (a0 b + b0 a - a x b)
    v = a0 * bv + b0 * av - np.cross(av, bv)
    return np.array([a0 * b0 - av @ bv, *v])


def propose(group: int, value, u_prop: float, width: float, u_z: float = 0.0, u_phi: float = 0.0):
    if group == Z2:
        return -value
    if group == SU2:
        d = width * (u_prop - 0.5)
        z = 2.0 * u_z - 1.0
        rho = np.sqrt(max(0.0, 1.0 - z * z))
        ph = TWO_PI * u_phi
        r = np.array([np.cos(d), np.sin(d) * rho * np.cos(ph), np.sin(d) * rho * np.sin(ph), np.sin(d) * z])
        q = quat_mul(r, np.asarray(value, dtype=np.float64))
        return q / np.sqrt(q @ q)
    th = float(value) + width * (u_prop - 0.5)
    if th >= TWO_PI:
        th -= TWO_PI
    elif th < 0.0:
        th += TWO_PI
    return th


def run_chain(p, weights: Weights, links0, seed: int, chain: int, sweep0: int, n_sweeps: int,
              width: float = 0.5, record_decisions: bool = False):
    links = np.array(links0, copy=True)
    logN = weights.log_norm(links)
    if not np.isfinite(logN):
        raise ValueError("initial configuration has N(G) <= 0")
    obs = np.zeros((n_sweeps, 3))
    decisions = []
    for k in range(n_sweeps):
        sw = sweep0 + k
        acc = 0
        for l in range(p.n_links):
            u_acc, u_prop, u_z, u_phi = draws4(seed, chain, sw, l)
            new = links.copy()
            new[l] = propose(p.group, links[l], u_prop, width, u_z, u_phi)
            logN_new = weights.log_norm(new)
            R = np.exp(logN_new - logN) if np.isfinite(logN_new) else 0.0
            accept = bool(u_acc < R)
            if record_decisions:
                decisions.append((sw, l, accept, float(u_acc), float(R)))
            if accept:
                links, logN = new, logN_new
                acc += 1
        obs[k] = (plaquette_mean(p.group, p.L, links)[0], logN, acc / p.n_links)
    return links, obs, decisions
