"""Pin the oracle Pfaffian to closed forms and to numpy's determinant."""
import numpy as np
import pytest

from oracle.pfaffian import pfaffian, log_pfaffian


def antisym(rng, n, cplx=True):
    X = rng.normal(size=(n, n)) + (1j * rng.normal(size=(n, n)) if cplx else 0)
    return X - X.T


def matchings(idx):
    if not idx:
        yield 1, []
        return
    a = idx[0]
    for k in range(1, len(idx)):
        b = idx[k]
        rest = idx[1:k] + idx[k + 1:]
        for sgn, m in matchings(rest):
            yield sgn * (-1) ** (k - 1), [(a, b)] + m


def brute_pf(A):
    tot = 0
    for sgn, m in matchings(list(range(A.shape[0]))):
        tot += sgn * np.prod([A[i, j] for i, j in m])
    return tot


def test_2x2_and_J_blocks():
    A = np.array([[0, 3.5], [-3.5, 0]])
    assert pfaffian(A) == pytest.approx(3.5)
    J = np.kron(np.eye(5), np.array([[0, 1.0], [-1.0, 0]]))
    assert pfaffian(J) == pytest.approx(1.0)


def test_4x4_formula():
    rng = np.random.default_rng(0)
    A = antisym(rng, 4)
    want = A[0, 1] * A[2, 3] - A[0, 2] * A[1, 3] + A[0, 3] * A[1, 2]
    assert abs(pfaffian(A) - want) < 1e-13 * abs(want)


@pytest.mark.parametrize("cplx", [True, False])
def test_6x6_and_8x8_matchings(cplx):
    rng = np.random.default_rng(1)
    for n in (6, 8):
        A = antisym(rng, n, cplx)
        want = brute_pf(A)
        assert abs(pfaffian(A) - want) < 1e-12 * max(1, abs(want))


@pytest.mark.parametrize("n", [10, 24, 63 * 2])
def test_square_is_det(n):
    rng = np.random.default_rng(n)
    for cplx in (True, False):
        A = antisym(rng, n, cplx)
        pf = pfaffian(A)
        sd, ld = np.linalg.slogdet(A)
        la, _ = log_pfaffian(A)
        assert abs(2 * la - ld) < 1e-10
        assert abs(pf**2 / (sd * np.exp(ld)) - 1) < 1e-10


def test_congruence_and_blocks():
    rng = np.random.default_rng(3)
    A = antisym(rng, 8)
    B = rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8))
    assert abs(pfaffian(B @ A @ B.T) - np.linalg.det(B) * pfaffian(A)) < 1e-10 * abs(pfaffian(B @ A @ B.T))
    C = antisym(rng, 6)
    D = np.zeros((14, 14), dtype=complex)
    D[:8, :8], D[8:, 8:] = A, C
    assert abs(pfaffian(D) - pfaffian(A) * pfaffian(C)) < 1e-10 * abs(pfaffian(D))


def test_singular_and_odd():
    A = np.zeros((4, 4))
    assert pfaffian(A) == 0
    la, ph = log_pfaffian(np.zeros((3, 3)))
    assert la == -np.inf and ph == 0
