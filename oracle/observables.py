"""Observables on link configurations and Monte Carlo error analysis.

* Plaquette Wilson loop (Sec. 2.3): the diagonal value of the plaquette
  operator is the trace of the oriented product of the four link group
  elements; for Z2 that is g1 g2 g3 g4, for U(1) cos(theta1 + theta2 -
  theta3 - theta4) (real part of the U(1) character).  The plaquette at site
  s uses link (s, x), link (s + e_x, y), link (s + e_y, x) reversed and
  link (s, y) reversed.  SU(2): the link label g enters the twist as
  psi^dag -> psi^dag D(g) (the right-regular action of App. A), under which
  the weight is invariant for g_l -> h_t^dag g_l h_s, so the covariant link
  matrix is g^dag and the plaquette is (1/2) tr(g1^dag g2^dag g3 g4) (real
  for SU(2); cos(theta1 + theta2 - theta3 - theta4) on the U(1) subgroup
  exp(i theta sigma_z)).  <W> = sum_G p(G) W(G) (Sec. 5.1).
* General Wilson loops (Sec. 5.1): R x T rectangles and loops winding once
  around the torus along y, with the same orientation rule (a forward step
  contributes the covariant link matrix, a backward step its inverse, in
  path order).
* Integrated autocorrelation time with the automatic window of Madras &
  Sokal (J. Stat. Phys. 50, 1988): tau(W) = 1/2 + sum_{t=1..W} rho(t),
  smallest W with W >= c tau(W), c = 5.

Pinned (tests/test_oracle_observables.py): plaquette against a loop-by-loop
product on hand-built configurations, tau_int against the closed form
(1 + a) / (2 (1 - a)) of an AR(1) series.  SU(2) (tests/test_oracle_su2.py):
cold configuration, a centre element on one link, the U(1) subgroup, gauge
invariance.  Loops (tests/test_oracle_observables.py): 1 x 1 rectangles equal
the plaquettes; a Z2 R x T loop is the product of the plaquettes it encloses;
gauge invariance (Z2, U(1), SU(2)); an L x T rectangle equals the product of
two winding loops for Z2; a centre element on one y link flips exactly the
winding loop through it.
"""
from __future__ import annotations

import numpy as np

Z2, U1, SU2 = 0, 1, 2


def plaquette_links(L: int):
    """(V, 4) link ids: +l1, +l2, -l3, -l4 around each plaquette."""
    out = []
    for s in range(L * L):
        x, y = s % L, s // L
        sx = y * L + (x + 1) % L
        sy = ((y + 1) % L) * L + x
        out.append((2 * s + 0, 2 * sx + 1, 2 * sy + 0, 2 * s + 1))
    return np.array(out, dtype=np.int64)


def plaquette_values(group: int, L: int, links: np.ndarray) -> np.ndarray:
    """(n_cfg, V) plaquette values."""
    pl = plaquette_links(L)
    if group == SU2:
        from .weight import su2_matrix
        links = np.asarray(links, dtype=np.float64)
        if links.ndim == 2:
            links = links[None]
        out = np.zeros((links.shape[0], L * L))
        for c in range(links.shape[0]):
            for s in range(L * L):
                g = [su2_matrix(links[c, k]) for k in pl[s]]
                out[c, s] = 0.5 * np.trace(g[0].conj().T @ g[1].conj().T @ g[2] @ g[3]).real
        return out
    links = np.atleast_2d(links)
    if group == Z2:
        g = links.astype(np.int64)
        return (g[:, pl[:, 0]] * g[:, pl[:, 1]] * g[:, pl[:, 2]] * g[:, pl[:, 3]]).astype(np.float64)
    th = links.astype(np.float64)
    return np.cos(th[:, pl[:, 0]] + th[:, pl[:, 1]] - th[:, pl[:, 2]] - th[:, pl[:, 3]])


def _steps_rect(L: int, s: int, R: int, T: int):
    """(link, forward) steps of the R x T rectangle with lower-left corner s:
    R steps +x, T steps +y, R steps -x, T steps -y."""
    x, y = s % L, s // L
    out = []
    for k in range(R):
        out.append((2 * (y * L + (x + k) % L), True))
    for k in range(T):
        out.append((2 * (((y + k) % L) * L + (x + R) % L) + 1, True))
    for k in range(R):
        out.append((2 * (((y + T) % L) * L + (x + R - 1 - k) % L), False))
    for k in range(T):
        out.append((2 * (((y + T - 1 - k) % L) * L + x) + 1, False))
    return out


def _loop_value(group: int, links_c: np.ndarray, steps) -> float:
    """Trace of the oriented product along a closed path: a forward step
    contributes the covariant link matrix (Z2 g, U(1) e^{i theta} with the
    real part taken at the end, SU(2) u^dag), a backward step its inverse."""
    if group == Z2:
        return float(np.prod([int(links_c[l]) for l, _ in steps]))
    if group == U1:
        return float(np.cos(sum(float(links_c[l]) * (1 if fw else -1) for l, fw in steps)))
    from .weight import su2_matrix
    M = np.eye(2, dtype=complex)
    for l, fw in steps:
        u = su2_matrix(links_c[l])
        M = M @ (u.conj().T if fw else u)
    return float(0.5 * np.trace(M).real)


def wilson_loop_values(group: int, L: int, links: np.ndarray, R: int, T: int) -> np.ndarray:
    """(n_cfg, V) R x T rectangular Wilson loops (R along x, T along y) at
    every lower-left corner (Sec. 5.1); R = T = 1 is the plaquette."""
    links = np.asarray(links)
    if (group == SU2 and links.ndim == 2) or (group != SU2 and links.ndim == 1):
        links = links[None]
    return np.array([[_loop_value(group, lc, _steps_rect(L, s, R, T)) for s in range(L * L)] for lc in links])


def polyakov_values(group: int, L: int, links: np.ndarray) -> np.ndarray:
    """(n_cfg, L) loops winding once around the torus along y at every x
    (a closed path through the periodic boundary, Sec. 5.1)."""
    links = np.asarray(links)
    if (group == SU2 and links.ndim == 2) or (group != SU2 and links.ndim == 1):
        links = links[None]
    out = []
    for lc in links:
        out.append([_loop_value(group, lc, [(2 * (y * L + x) + 1, True) for y in range(L)]) for x in range(L)])
    return np.array(out)


def plaquette_mean(group: int, L: int, links: np.ndarray) -> np.ndarray:
    return plaquette_values(group, L, links).mean(axis=1)


def tau_int(series: np.ndarray, c: float = 5.0):
    """Integrated autocorrelation time of (n_chains, T) series (chains pooled
    after removing the grand mean).  Returns (tau, window)."""
    x = np.atleast_2d(np.asarray(series, dtype=np.float64))
    x = x - x.mean()
    T = x.shape[1]
    var = np.mean(x * x)
    if var == 0.0 or T < 2:
        return 0.5, 0
    tau = 0.5
    for t in range(1, T):
        rho = np.mean(x[:, :-t] * x[:, t:]) / var
        tau += rho
        if t >= c * tau:
            return float(tau), t
    return float(tau), T - 1
