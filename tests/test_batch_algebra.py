"""The linear algebra of the batched (submatrix) delayed updates, in numpy.

For a batch of link changes on disjoint supports S_j (T = their union), with
W = M^{-1} at the batch start, C = W[:, T], Y = W[T, :], G0 = W[T, T]:
  * every proposal's ratio is the bordered Pfaffian Pf([[D, -1], [1, G[S, S]]])
    of the current small matrix G, and equals Pf(M') / Pf(M);
  * on accept, G[F, F] -= G[F, S] Z G[S, F] for the later links F and
    X += P Z Q with P = E_S - X G0[:, S], Q = E_S^T - G0[S, :] X,
    Z = (1 + D G[S, S])^{-1} D;
  * after the batch the inverse is W - C X Y.
C must be the true columns of the stored W: reading it as -Y^T (equal for an
exactly antisymmetric W) makes the rounding error grow geometrically from
batch to batch (8x8 Z2 in FP32: 1e-2 after one sweep; 12x12: 8e3).
Pfaffians come from the oracle's Parlett-Reid routine; inverses from numpy.
"""
import numpy as np
import pytest

import ggf_inputs as gi
from oracle import pfaffian, weight


def _asym(rng, n, cplx):
    a = rng.normal(size=(n, n)) + (1j * rng.normal(size=(n, n)) if cplx else 0.0)
    return a - a.T


def _batch(W, M, T, r, deltas, accept, dt):
    """One batch on the small block; returns the new W, the new M and the ratios."""
    k = len(T) // r
    C = W[:, T].copy()
    Y = W[T, :].copy()
    G0 = C[T, :].copy()
    G = G0.copy()
    X = np.zeros((k * r, k * r), dtype=dt)
    rhos = []
    for j in range(k):
        sl = slice(j * r, (j + 1) * r)
        D = deltas[j]
        Wss = G[sl, sl].astype(complex if np.iscomplexobj(G) else float)
        rho = pfaffian.pfaffian(np.block([[D, -np.eye(r)], [np.eye(r), Wss]]))
        rhos.append(rho)
        if not accept(j, rho):
            continue
        Z = np.linalg.solve(np.eye(r) + D @ Wss, D).astype(dt)
        fut = slice((j + 1) * r, k * r)
        G[fut, fut] -= G[fut, sl] @ Z @ G[sl, fut]
        E = np.zeros((k * r, r), dtype=dt)
        E[sl, :] = np.eye(r)
        P = E - X @ G0[:, sl]
        Q = E.T - G0[sl, :] @ X
        X = X + P @ Z @ Q
        M = M.copy()
        M[np.ix_(T[sl], T[sl])] += D
    return W - C @ (X @ Y), M, rhos


@pytest.mark.parametrize("cplx", [False, True])
def test_batched_updates_reproduce_direct_inverse(cplx):
    rng = np.random.default_rng(7 + 2 * cplx)
    n, r, k = 48, 4, 6
    dt = complex if cplx else float
    M = _asym(rng, n, cplx) + 3.0 * np.kron(np.eye(n // 2), np.array([[0.0, -1.0], [1.0, 0.0]]))
    W = np.linalg.inv(M)
    T = rng.permutation(n)[: k * r]
    deltas = [0.4 * _asym(rng, r, cplx) for _ in range(k)]
    # ratios against Pf(M') / Pf(M) along the accepted path
    Mcur = M
    Wn, Mn, rhos = _batch(W, M, T, r, deltas, lambda j, rho: j % 3 != 1, dt)
    for j in range(k):
        S = T[j * r:(j + 1) * r]
        Mp = Mcur.copy()
        Mp[np.ix_(S, S)] += deltas[j]
        ref = pfaffian.pfaffian(Mp) / pfaffian.pfaffian(Mcur)
        assert abs(rhos[j] - ref) <= 1e-9 * abs(ref)
        if j % 3 != 1:
            Mcur = Mp
    exact = np.linalg.inv(Mn)
    assert np.abs(Wn - exact).max() <= 1e-10 * np.abs(exact).max()
    assert np.abs(Wn + Wn.T).max() <= 1e-10 * np.abs(exact).max()


def _reduced_z2(L):
    """The reduced (virtual-only) matrix D + O Gamma_X O^T of an L x L Z2 problem
    (n_v = 1, K = 1) at the cold configuration, built from the oracle's
    covariances, with each link's support and its r x r twisted block."""
    p = gi.make_problem(L, gi.Z2, 1, 1)
    GA = weight.gamma_A(p)
    GX = weight.BondData(p).embedded(0, 0).real
    virt = np.array([i for i in range(p.m_s * p.V) if i % p.m_s >= 2])
    pos = -np.ones(p.m_s * p.V, dtype=int)
    pos[virt] = np.arange(len(virt))
    S = [pos[np.array(ix)] for ix in weight.link_majoranas(p)]
    M = GA[np.ix_(virt, virt)] + GX[np.ix_(virt, virt)]

    def block(l, g):
        o = np.ones(len(S[l]))
        o[:2] = g                     # the source end carries the twist
        return o[:, None] * GX[np.ix_(virt, virt)][np.ix_(S[l], S[l])] * o[None, :]
    return p, M, S, block


def test_batched_sweep_stays_accurate_in_fp32():
    p, M, S, block = _reduced_z2(8)
    rng = np.random.default_rng(3)
    W = np.linalg.inv(M).astype(np.float32)
    links = np.ones(p.n_links)
    kb, r, accepted = 4, 4, 0
    for l0 in range(0, p.n_links, kb):
        ls = list(range(l0, l0 + kb))
        T = np.concatenate([S[l] for l in ls])
        deltas = [block(l, -links[l]) - block(l, links[l]) for l in ls]
        u = rng.random(kb)
        acc = lambda j, rho: rho.real > 0 and u[j] < rho.real
        W, M, rhos = _batch(W, M, T, r, deltas, acc, np.float32)
        for j, l in enumerate(ls):
            if acc(j, rhos[j]):
                links[l] = -links[l]
                accepted += 1
    exact = np.linalg.inv(M)
    assert accepted > p.n_links // 2
    assert np.abs(W - exact).max() <= 1e-4 * np.abs(exact).max()
