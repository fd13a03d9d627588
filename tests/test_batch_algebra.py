"""The linear algebra of the batched (submatrix) delayed updates, in FP64 numpy.

For a batch of link changes on disjoint supports S_j (T = their union), with
W = M^{-1} at the batch start, C = W[:, T], Y = W[T, :], G0 = W[T, T]:
  * every proposal's ratio is the bordered Pfaffian Pf([[D, -1], [1, G[S, S]]])
    of the current small matrix G, and equals Pf(M') / Pf(M);
  * on accept, G[F, F] -= G[F, S] Z G[S, F] for the later links F and
    X += P Z Q with P = E_S - X G0[:, S], Q = E_S^T - G0[S, :] X,
    Z = (1 + D G[S, S])^{-1} D;
  * after the batch the inverse is W - C X Y.
Pfaffians come from the oracle's Parlett-Reid routine; inverses from numpy.
"""
import numpy as np
import pytest

from oracle import pfaffian


def _asym(rng, n, cplx):
    a = rng.normal(size=(n, n)) + (1j * rng.normal(size=(n, n)) if cplx else 0.0)
    return a - a.T


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("upper", [False, True])
def test_batched_updates_reproduce_direct_inverse(cplx, upper):
    rng = np.random.default_rng(7 + 2 * cplx + upper)
    n, r, k = 48, 4, 6
    dt = complex if cplx else float
    M = _asym(rng, n, cplx) + 3.0 * np.kron(np.eye(n // 2), np.array([[0.0, -1.0], [1.0, 0.0]]))
    W = np.linalg.inv(M)
    T = rng.permutation(n)[: k * r]
    Y = W[T, :].copy()
    # upper-triangle reading: the columns are the negated rows (W antisymmetric)
    C = -Y.T.copy() if upper else W[:, T].copy()
    G0 = C[T, :].copy()
    G = G0.copy()
    X = np.zeros((k * r, k * r), dtype=dt)
    Mcur = M.copy()
    accepted = 0
    for j in range(k):
        sl = slice(j * r, (j + 1) * r)
        S = T[sl]
        D = 0.4 * _asym(rng, r, cplx)
        Wss = G[sl, sl]
        bord = np.block([[D, -np.eye(r)], [np.eye(r), Wss]])
        rho = pfaffian.pfaffian(bord)
        Mn = Mcur.copy()
        Mn[np.ix_(S, S)] += D
        ref = pfaffian.pfaffian(Mn) / pfaffian.pfaffian(Mcur)
        assert abs(rho - ref) <= 1e-9 * abs(ref)
        if j % 3 == 1:          # a rejected proposal leaves everything as it was
            continue
        accepted += 1
        Z = np.linalg.solve(np.eye(r) + D @ Wss, D)
        fut = slice((j + 1) * r, k * r)
        G[fut, fut] -= G[fut, sl] @ Z @ G[sl, fut]
        E = np.zeros((k * r, r))
        E[sl, :] = np.eye(r)
        P = E - X @ G0[:, sl]
        Q = E.T - G0[sl, :] @ X
        X = X + P @ Z @ Q
        Mcur = Mn
    assert accepted >= 3
    Wf = W - C @ X @ Y
    exact = np.linalg.inv(Mcur)
    assert np.abs(Wf - exact).max() <= 1e-10 * np.abs(exact).max()
    # the composed update keeps W antisymmetric
    assert np.abs(Wf + Wf.T).max() <= 1e-10 * np.abs(exact).max()
