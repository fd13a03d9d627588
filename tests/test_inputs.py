"""The seeded input generator produces valid, symmetric Gaussian states."""
import numpy as np
import pytest

import ggf_inputs as gi


@pytest.mark.parametrize("grp,nv", [(gi.Z2, 1), (gi.U1, 1), (gi.U1, 2)])
def test_pure_and_symmetric(grp, nv):
    p = gi.make_problem(3, grp, nv, 3, site_mode="random", bond_mode="random", bond_scale=0.3)
    for s in range(p.V):
        G = p.gamma_site[s]
        assert np.allclose(G @ G.T, np.eye(p.m_s), atol=1e-13) and np.allclose(G, -G.T)
        if grp == gi.U1:
            R = gi._rotation(gi.site_charges(nv, int(p.q_phys[s])), 0.731)
            assert np.allclose(R @ G @ R.T, G, atol=1e-13)
    qb = np.concatenate([p.q_src, -p.q_src])
    for n in range(p.K):
        for l in range(p.n_links):
            B = p.gamma_bond[n, l]
            assert np.allclose(B @ B.T, np.eye(p.r), atol=1e-13)
            if grp == gi.U1:
                R = gi._rotation(qb, 1.234)
                assert np.allclose(R @ B @ R.T, B, atol=1e-13)
    assert abs(np.linalg.norm(p.lam) - 1) < 1e-14


def test_max_entangled_bond_reduced_state():
    for nv in (1, 2):
        B = gi.max_entangled_bond(nv)
        h = 2 * nv
        assert np.allclose(B[:h, :h], 0) and np.allclose(B[h:, h:], 0)


def test_seeded_reproducible():
    a = gi.make_problem(4, gi.U1, 2, 4)
    b = gi.make_problem(4, gi.U1, 2, 4)
    assert np.array_equal(a.gamma_site, b.gamma_site) and np.array_equal(a.lam, b.lam)
