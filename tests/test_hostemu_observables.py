"""The observable kernels' per-thread code (csrc/ggf_obs.cuh) and the SU(2)
proposal and twist helpers, built for the host by
tests/hostemu/emu_observables.cu, against the oracle -- on CPU.

The test lays out the device-side arrays as the library does (site blocks
D, A, B; bond blocks Gamma_X per pair; the chains' inverses of the reduced
matrix D + O Gamma_X O^T; log-weights per pair) and checks the electric
observable, the fermionic bilinears and the per-pair parts item by item
against oracle.electric, oracle.fermionic and oracle.variational.  This checks
the kernels' index arithmetic and data layout before a GPU runs them; the
GPU parity tests remain the parity claim.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import ggf_inputs as gi
from oracle import electric, fermionic, variational, weight

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("emu") / "libemu.so")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC", "-gencode",
                    "arch=compute_103a,code=sm_103a", "-o", out,
                    os.path.join(HERE, "hostemu", "emu_observables.cu")], check=True, capture_output=True)
    return ctypes.CDLL(out)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _cplx(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1))


class Layout:
    """Device-side arrays of one problem and a set of chain configurations."""

    def __init__(self, p, links):
        self.p = p
        V, B, nl, K = p.V, 8 * p.n_v, p.n_links, p.K
        self.q = np.array([int(p.q_src[0]), int(p.q_src[1]) if p.n_v > 1 else 1] if p.group == gi.U1 else [1, 1],
                          dtype=np.int32)
        self.D = np.ascontiguousarray(np.array([p.gamma_site[s][2:, 2:] for s in range(V)]))
        self.Ap = np.ascontiguousarray(np.array([p.gamma_site[s][:2, :2] for s in range(V)]))
        self.Bp = np.ascontiguousarray(np.array([p.gamma_site[s][:2, 2:] for s in range(V)]))
        bd = weight.BondData(p)
        pairs = [(n, n) for n in range(K)] + [(n, m) for n in range(K) for m in range(n + 1, K)]
        self.pairs = pairs
        self.Gr = np.ascontiguousarray(np.array([[bd.G[n, n, l].real for l in range(nl)] for n in range(K)]))
        cp = pairs[K:]
        self.Gc = _cplx(np.array([[bd.G[n, m, l] for l in range(nl)] for n, m in cp]) if cp
                        else np.zeros((1, nl, p.r, p.r)))
        lam = p.lam
        self.w = _cplx([abs(lam[n]) ** 2 if n == m else 2 * np.conj(lam[n]) * lam[m] for n, m in pairs])
        self.logc = _cplx(np.zeros(len(pairs)))
        W = weight.Weights(p)
        virt = np.array([i for i in range(p.m_s * V) if i % p.m_s >= 2])
        Dfull = np.zeros((B * V, B * V))
        for s in range(V):
            Dfull[s * B:(s + 1) * B, s * B:(s + 1) * B] = self.D[s]
        Wr, Wc, ell = [], [], []
        for G in links:
            Ov = weight.twist_matrix(p, G)[np.ix_(virt, virt)]
            lnm = W.log_n_matrix(G)
            inv = {nm: np.linalg.inv(Dfull + Ov @ W.GX[nm][np.ix_(virt, virt)] @ Ov.T) for nm in pairs}
            Wr.append([inv[(n, n)].real for n in range(K)])
            Wc.append([inv[nm] for nm in cp])
            ell.append([lnm[n, m] for n, m in pairs])
        self.Wr = np.ascontiguousarray(np.array(Wr))
        self.Wc = _cplx(np.array(Wc)) if cp else np.zeros(2)
        self.ell = _cplx(np.array(ell))
        self.links = np.ascontiguousarray(links)
        self.n = len(links)

    def common(self):
        p = self.p
        return [ctypes.c_int(p.L), ctypes.c_int(p.group), ctypes.c_int(p.n_v), _ptr(self.q), ctypes.c_int(p.K),
                _ptr(self.D), _ptr(self.Ap), _ptr(self.Bp), _ptr(self.Gr), _ptr(self.Gc), _ptr(self.logc),
                _ptr(self.w), ctypes.c_int(self.n)]


def _c(a):
    return a[..., 0] + 1j * a[..., 1]


CASES = [(3, gi.Z2, 1, 3), (2, gi.Z2, 2, 2), (3, gi.U1, 1, 2), (2, gi.U1, 2, 3), (2, gi.SU2, 2, 2),
         (1, gi.U1, 1, 2)]


@pytest.mark.parametrize("L,grp,n_v,K", CASES)
def test_electric_items_match_oracle(emu, L, grp, n_v, K):
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=13)
    lay = Layout(p, links)
    out = np.zeros((2, p.n_links, 2))
    pairs = np.zeros((2, p.n_links, K, K, 2))
    emu.emu_electric(*lay.common()[:-1], ctypes.c_int(2), _ptr(lay.links), _ptr(lay.Wr), _ptr(lay.Wc),
                     _ptr(lay.ell), _ptr(out), _ptr(pairs))
    el, lm = electric.Electric(p), variational.LocalMatrices(p)
    for c in range(2):
        ref = el.f_electric(links[c])
        assert np.abs(_c(out)[c] - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
        refp = lm(links[c])["electric"]
        assert np.abs(_c(pairs)[c] - refp).max() <= 1e-11 * max(1.0, np.abs(refp).max())


@pytest.mark.parametrize("L,grp,n_v,K", CASES)
def test_fermion_items_match_oracle(emu, L, grp, n_v, K):
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=14)
    lay = Layout(p, links)
    site = np.zeros((2, p.V, 2))
    link = np.zeros((2, p.n_links, 2, 2, 2))
    ps = np.zeros((2, p.V, K, K, 2))
    pl = np.zeros((2, p.n_links, 2, 2, K, K, 2))
    emu.emu_fermion(*lay.common(), _ptr(lay.Wr), _ptr(lay.Wc), _ptr(lay.ell), _ptr(site), _ptr(link),
                    _ptr(ps), _ptr(pl))
    fe, lm = fermionic.Fermionic(p), variational.LocalMatrices(p)
    for c in range(2):
        rs, rl = fe.bilinears(links[c])
        assert np.abs(_c(site)[c] - rs).max() <= 1e-11
        assert np.abs(_c(link)[c] - rl).max() <= 1e-11
        ref = lm(links[c])
        assert np.abs(_c(ps)[c] - ref["density"]).max() <= 1e-11 * max(1.0, np.abs(ref["density"]).max())
        Ge = fe.gamma_eff(links[c])
        for l in range(p.n_links):
            s, t = fermionic._link_sites(p, l)
            for a in range(2):
                for b in range(2):
                    i, j = 2 * s + a, 2 * t + b
                    want = np.array([[ref["norm"][n, m] * (1.0 if i == j else -1j * Ge[n, m][i, j])
                                      for m in range(K)] for n in range(K)])
                    assert np.abs(_c(pl)[c, l, a, b] - want).max() <= 1e-11 * max(1.0, np.abs(want).max())


def test_pair_norm_items_match_oracle(emu):
    p = gi.make_problem(2, gi.U1, 1, 3, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=15)
    lay = Layout(p, links)
    out = np.zeros((2, 3, 3, 2))
    emu.emu_pair_norm(ctypes.c_int(p.L), ctypes.c_int(p.group), ctypes.c_int(p.n_v), _ptr(lay.q),
                      ctypes.c_int(p.K), _ptr(lay.logc), _ptr(lay.w), ctypes.c_int(2), _ptr(lay.ell), _ptr(out))
    lm = variational.LocalMatrices(p)
    for c in range(2):
        assert np.abs(_c(out)[c] - lm(links[c])["norm"]).max() <= 1e-12


def test_su2_proposal_and_twist_match_oracle(emu):
    """The GPU's SU(2) move (Philox words -> quaternion) equals the oracle's
    proposal to rounding, so FP64 decisions can agree bit for bit; the
    doublet rotation and the twisted link block equal the oracle's."""
    from oracle import mcmc
    from oracle.philox import draws4
    emu.emu_draw_su2.restype = ctypes.c_double
    emu.emu_twisted_su2.restype = ctypes.c_double
    p = gi.make_problem(1, gi.SU2, 2, 1)
    rng = np.random.default_rng(4)
    for k in range(20):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        c, sweep, seed, width = k % 3, 5 + k, 1234 + k, 0.5 + 0.1 * k
        qn, Ro, Rn = np.zeros(4), np.zeros(16), np.zeros(16)
        u = emu.emu_draw_su2(ctypes.c_ulonglong(sweep), ctypes.c_uint64(seed), ctypes.c_int(c),
                             ctypes.c_double(width), _ptr(q), _ptr(qn), _ptr(Ro), _ptr(Rn))
        ua, up, uz, uf = draws4(seed, c, sweep, 0)
        assert u == ua
        want = mcmc.propose(gi.SU2, q, up, width, uz, uf)
        assert np.abs(qn - want).max() <= 4e-16
        assert np.abs(Ro.reshape(4, 4) - weight.doublet_rotation(weight.su2_matrix(q))).max() <= 1e-15
        assert np.abs(Rn.reshape(4, 4) - weight.doublet_rotation(weight.su2_matrix(want))).max() <= 1e-15
    # twisted block of one link against O Gamma O^T with the oracle's twist
    G = np.ascontiguousarray(p.gamma_bond[0, 0])
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    R = np.ascontiguousarray(weight.doublet_rotation(weight.su2_matrix(q)))
    O = np.eye(8)
    O[:4, :4] = R
    want = O @ G @ O.T
    got = np.array([[emu.emu_twisted_su2(_ptr(G), x, y, _ptr(R)) for y in range(8)] for x in range(8)])
    assert np.abs(got - want).max() <= 1e-15


@pytest.mark.parametrize("L,grp,n_v,K", [(3, gi.Z2, 1, 2), (2, gi.U1, 2, 2), (2, gi.SU2, 2, 2), (1, gi.SU2, 2, 2)])
def test_assembled_matrix_matches_reduced_matrix(emu, L, grp, n_v, K):
    """assemble_elem builds D + O(G) Gamma_X O(G)^T on the virtual modes, whose
    Pfaffian is the covariance route's full-space one up to a fixed sign."""
    from oracle.pfaffian import log_pfaffian
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=16)
    lay = Layout(p, links[:1])
    W = weight.Weights(p)
    virt = np.array([i for i in range(p.m_s * p.V) if i % p.m_s >= 2])
    Ov = weight.twist_matrix(p, links[0])[np.ix_(virt, virt)]
    N = 8 * p.n_v * p.V
    Dfull = np.zeros((N, N))
    B = 8 * p.n_v
    for s in range(p.V):
        Dfull[s * B:(s + 1) * B, s * B:(s + 1) * B] = lay.D[s]
    for k, (n, m) in enumerate(lay.pairs):
        cplx = k >= K
        M = np.zeros((N, N, 2)) if cplx else np.zeros((N, N))
        emu.emu_assemble(ctypes.c_int(p.L), ctypes.c_int(p.group), ctypes.c_int(p.n_v), _ptr(lay.q),
                         ctypes.c_int(K), _ptr(lay.D), _ptr(lay.Gr), _ptr(lay.Gc), _ptr(lay.links),
                         ctypes.c_int(k - K if cplx else k), ctypes.c_int(int(cplx)), _ptr(M))
        got = _c(M) if cplx else M
        want = Dfull + Ov @ W.GX[n, m][np.ix_(virt, virt)] @ Ov.T
        assert np.abs(got - want).max() <= 1e-14
        # and the full-space Pfaffian of the covariance route agrees with it up
        # to the sites' fixed sign prod_s sign(Gamma_s[0, 1])
        O = weight.twist_matrix(p, links[0])
        la, ph = log_pfaffian(O.T @ W.GA @ O + W.GX[n, m])
        lb, pb = log_pfaffian(got)
        sign = np.prod([np.sign(p.gamma_site[s][0, 1]) for s in range(p.V)])
        assert abs(np.exp((la + np.log(complex(ph))) - (lb + np.log(complex(pb)))) - sign) <= 1e-12


@pytest.mark.parametrize("L,grp,n_v,K", [(2, gi.Z2, 1, 2), (2, gi.U1, 2, 3), (2, gi.SU2, 2, 2)])
def test_score_items_match_oracle(emu, L, grp, n_v, K):
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=17)
    lay = Layout(p, links)
    B = 8 * n_v
    out = np.zeros((2, p.V, B, B))
    emu.emu_score(ctypes.c_int(p.L), ctypes.c_int(p.group), ctypes.c_int(p.n_v), _ptr(lay.q), ctypes.c_int(K),
                  _ptr(lay.logc), _ptr(lay.w), ctypes.c_int(2), _ptr(lay.Wr), _ptr(lay.Wc), _ptr(lay.ell), _ptr(out))
    for c in range(2):
        ref = variational.score_sites(p, links[c])
        assert np.abs(out[c] - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("L,grp,n_v,K", [(3, gi.Z2, 1, 3), (2, gi.U1, 2, 2), (3, gi.U1, 1, 2), (1, gi.Z2, 1, 2)])
def test_fermion4_items_match_oracle(emu, L, grp, n_v, K):
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=18)
    lay = Layout(p, links)
    out = np.zeros((2, p.n_links, 2))
    pairs = np.zeros((2, p.n_links, K, K, 2))
    emu.emu_fermion4(*lay.common(), _ptr(lay.Wr), _ptr(lay.Wc), _ptr(lay.ell), _ptr(out), _ptr(pairs))
    fe = fermionic.Fermionic(p)
    lm = variational.LocalMatrices(p)
    for c in range(2):
        for l in range(p.n_links):
            s_, t_ = fermionic._link_sites(p, l)
            want = -1.0 if s_ == t_ else fe.monomial(links[c], (2 * s_, 2 * s_ + 1, 2 * t_, 2 * t_ + 1))
            assert abs(_c(out)[c, l] - want) <= 1e-11
        ref = lm(links[c])["four"]
        assert np.abs(_c(pairs)[c] - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
        assert np.abs(np.einsum("n,lnm,m->l", np.conj(p.lam), ref, p.lam) - _c(out)[c]).max() <= 1e-11


def test_su2_plaquette_matches_oracle(emu):
    from oracle.observables import plaquette_mean
    emu.emu_plaquette_su2.restype = ctypes.c_double
    for L in (1, 2, 3):
        p = gi.make_problem(L, gi.SU2, 2, 1)
        for G in gi.random_links(p, 3, seed=19):
            G = np.ascontiguousarray(G)
            got = emu.emu_plaquette_su2(ctypes.c_int(L), _ptr(G))
            assert abs(got - plaquette_mean(gi.SU2, L, G)[0]) <= 1e-14


@pytest.mark.parametrize("L,grp,n_v,K", [(2, gi.Z2, 1, 2), (2, gi.U1, 2, 3), (3, gi.U1, 1, 2), (2, gi.SU2, 2, 2)])
def test_link_score_items_match_oracle(emu, L, grp, n_v, K):
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=20)
    lay = Layout(p, links)
    P = K * (K + 1) // 2
    out = np.zeros((2, P, p.n_links, p.r, p.r, 2))
    emu.emu_link_score(ctypes.c_int(p.L), ctypes.c_int(p.group), ctypes.c_int(p.n_v), _ptr(lay.q), ctypes.c_int(K),
                       _ptr(lay.D), _ptr(lay.Gr), _ptr(lay.Gc), _ptr(lay.logc), _ptr(lay.w), ctypes.c_int(2),
                       _ptr(lay.links), _ptr(lay.Wr), _ptr(lay.Wc), _ptr(lay.ell), _ptr(out))
    for c in range(2):
        ref = variational.score_links(p, links[c])
        assert np.abs(_c(out)[c] - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("grp", [gi.Z2, gi.U1, gi.SU2])
def test_loops_match_oracle(emu, grp):
    from oracle.observables import polyakov_values, wilson_loop_values
    for L in (1, 3, 4):
        p = gi.make_problem(L, grp, 2 if grp == gi.SU2 else 1, 1)
        G = np.ascontiguousarray(gi.random_links(p, 1, seed=21)[0])
        for R, T in ((1, 1), (1, 2), (2, 3), (L, 1), (L, L)):
            if R > L or T > L:
                continue
            out = np.zeros(p.V)
            emu.emu_loops(ctypes.c_int(L), ctypes.c_int(grp), _ptr(G), ctypes.c_int(R), ctypes.c_int(T),
                          ctypes.c_int(0), _ptr(out))
            assert np.abs(out - wilson_loop_values(grp, L, G, R, T)[0]).max() <= 1e-14
        out = np.zeros(L)
        emu.emu_loops(ctypes.c_int(L), ctypes.c_int(grp), _ptr(G), ctypes.c_int(0), ctypes.c_int(0),
                      ctypes.c_int(1), _ptr(out))
        assert np.abs(out - polyakov_values(grp, L, G)[0]).max() <= 1e-14


@pytest.mark.parametrize("L,n_v,K", [(3, 1, 2), (2, 2, 3), (1, 2, 2)])
def test_field_items_match_oracle(emu, L, n_v, K):
    p = gi.make_problem(L, gi.U1, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=22)
    lay = Layout(p, links)
    out = np.zeros((2, p.n_links, 2))
    pairs = np.zeros((2, p.n_links, K, K, 2))
    emu.emu_field(*lay.common()[:-1], ctypes.c_int(2), _ptr(lay.links), _ptr(lay.Wr), _ptr(lay.Wc), _ptr(lay.ell),
                  _ptr(out), _ptr(pairs))
    el = electric.Electric(p)
    lm = variational.LocalMatrices(p)
    for c in range(2):
        ref = el.field(links[c])
        assert np.abs(_c(out)[c] - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
        rp = lm(links[c])["field"]
        assert np.abs(_c(pairs)[c] - rp).max() <= 1e-11 * max(1.0, np.abs(rp).max())


@pytest.mark.parametrize("L,grp,n_v,K", [(2, gi.U1, 1, 2), (3, gi.U1, 1, 2), (2, gi.Z2, 2, 3), (1, gi.U1, 2, 2),
                                         (1, gi.Z2, 2, 1)])
def test_link_term_items_match_oracle(emu, L, grp, n_v, K):
    """The link-term item on the emulated fermion outputs (combined and per
    pair) against oracle.fermionic's link terms."""
    p = gi.make_problem(L, grp, n_v, K, bond_scale=0.3)
    links = gi.random_links(p, 2, seed=24)
    lay = Layout(p, links)
    site = np.zeros((2, p.V, 2))
    link = np.zeros((2, p.n_links, 2, 2, 2))
    ps = np.zeros((2, p.V, K, K, 2))
    pl = np.zeros((2, p.n_links, 2, 2, K, K, 2))
    emu.emu_fermion(*lay.common(), _ptr(lay.Wr), _ptr(lay.Wc), _ptr(lay.ell), _ptr(site), _ptr(link),
                    _ptr(ps), _ptr(pl))
    q = np.ascontiguousarray(p.q_phys, dtype=np.int32)
    out = np.zeros((2, p.n_links, 2))
    pout = np.zeros((2, p.n_links, K, K, 2))
    emu.emu_link_terms(ctypes.c_int(p.L), ctypes.c_int(p.group), ctypes.c_int(p.n_v), ctypes.c_int(K),
                       ctypes.c_int(2), _ptr(lay.links), _ptr(q), _ptr(link), _ptr(pl), _ptr(out), _ptr(pout))
    fe = fermionic.Fermionic(p)
    for c in range(2):
        ref = fe.link_terms(links[c])
        assert np.abs(ref).max() > 1e-3
        assert np.abs(_c(out)[c] - ref).max() <= 1e-11
        want = fermionic.link_terms_from_block(p, links[c], _c(pl)[c])
        assert np.abs(_c(pout)[c] - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
        lam = p.lam
        assert np.abs(np.einsum("n,lnm,m->l", np.conj(lam), _c(pout)[c], lam) - ref).max() <= 1e-11
