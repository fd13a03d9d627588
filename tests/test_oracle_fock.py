"""Pin the Fock-space machinery: Majorana conventions, Gaussian states,
fermionic reordering and contraction (App. C worked example)."""
import os

import numpy as np
import scipy.linalg

import ggf_inputs as gi
from oracle import fock
from oracle.pfaffian import pfaffian

GOLD = os.path.join(os.path.dirname(__file__), "golden", "appC_two_mode_contraction.txt")


def test_vacuum_covariance():
    vac = np.zeros(8, dtype=complex)
    vac[0] = 1
    G = fock.covariance_of(vac)
    assert np.allclose(G, gi.vacuum(3))


def test_majorana_algebra():
    cs = fock.majoranas(3)
    for a in range(6):
        for b in range(6):
            ac = (cs[a] @ cs[b] + cs[b] @ cs[a]).toarray()
            assert np.allclose(ac, 2 * (a == b) * np.eye(8))


def test_roundtrip_random_pure_states():
    p = gi.make_problem(1, gi.U1, 1, 1, site_mode="random")
    for G in (p.gamma_site[0], p.gamma_bond[0, 0], gi.vacuum(2)):
        psi = fock.state_from_covariance(G)
        assert np.allclose(fock.covariance_of(psi), G, atol=1e-12)


def test_overlap_pfaffian_formula():
    """|<a|b>|^2 = tr(rho_a rho_b) = 2^-n Pf(Ga) Pf(Ga + Gb) (Sec. 3.2)."""
    p = gi.make_problem(1, gi.Z2, 1, 1, site_mode="random")
    q = gi.make_problem(1, gi.Z2, 1, 1, seed=99, site_mode="random")
    Ga, Gb = p.gamma_site[0], q.gamma_site[0]
    a, b = fock.state_from_covariance(Ga), fock.state_from_covariance(Gb)
    n = Ga.shape[0] // 2
    want = abs(np.vdot(a, b)) ** 2
    got = 2.0**-n * pfaffian(Ga) * pfaffian(Ga + Gb)
    assert abs(got - want) < 1e-13
    # the positive square root of det((Ga + Gb) / 2) gives the same number
    assert abs(np.sqrt(np.linalg.det((Ga + Gb) / 2)) - want) < 1e-13


def test_reorder_matches_operator_products():
    n = 4
    ann, cre = fock.fermion_ops(n)
    vac = np.zeros(1 << n, dtype=complex)
    vac[0] = 1
    rng = np.random.default_rng(0)
    perm = [2, 0, 3, 1]
    for occ in ([0, 2], [1, 3], [0, 1, 2], [0, 1, 2, 3]):
        v = vac
        for m in reversed(occ):
            v = cre[m] @ v                      # psi_occ0^dag psi_occ1^dag ... |0>
        w = fock.reorder(v, perm)
        # same operator string written with new labels, then sorted
        newpos = {old: k for k, old in enumerate(perm)}
        lab = [newpos[m] for m in occ]
        sign = 1
        for i in range(len(lab)):
            for j in range(i + 1, len(lab)):
                if lab[i] > lab[j]:
                    sign = -sign
        u = vac
        for m in reversed(sorted(lab)):
            u = cre[m] @ u
        assert np.allclose(w, sign * u)
    del rng


def _read_golden():
    rows, sign = {}, None
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split(":", 1)
        if k == "sign_T13T24_canonical":
            sign = int(v)
        else:
            rows[k.strip()] = v.strip()
    return rows, sign


def test_appC_worked_contraction():
    rows, sign = _read_golden()
    n = 4
    ann, cre = fock.fermion_ops(n)
    rng = np.random.default_rng(5)
    T = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    T = T - T.T
    B12 = 0.7 - 0.2j
    # |T> = exp(1/2 sum_ij T_ij psi_i^dag psi_j^dag)|0>, modes 1..4 -> 0..3
    gen = sum(0.5 * T[i, j] * (cre[i] @ cre[j]) for i in range(4) for j in range(4) if i != j)
    vac = np.zeros(16, dtype=complex)
    vac[0] = 1
    Tstate = scipy.linalg.expm(gen.toarray()) @ vac
    # |B> = (1 + B12 psi1^dag psi2^dag)|0> on modes 1, 2 (2-mode register)
    annB, creB = fock.fermion_ops(2)
    vac2 = np.zeros(4, dtype=complex)
    vac2[0] = 1
    Bstate = vac2 + np.conj(B12) * (creB[0] @ creB[1] @ vac2)   # bra carries B12
    psi = fock.contract(Tstate, [2, 3], [0, 1], Bstate)
    env = {"B12": B12, "T12": T[0, 1], "T13": T[0, 2], "T14": T[0, 3], "T23": T[1, 2],
           "T24": T[1, 3], "T34": T[2, 3]}
    want00 = eval(rows["00"], {}, env)
    # printed 11 amplitude with the (13)(24) colouring read in canonical order
    printed11 = rows["11"].replace("B12*T13*T24", f"({sign})*B12*T13*T24")
    want11 = eval(printed11, {}, env)
    assert abs(psi[0] - want00) < 1e-12
    assert abs(psi[3] - want11) < 1e-12
    assert abs(psi[1]) < 1e-14 and abs(psi[2]) < 1e-14


def test_bond_phase_convention():
    p = gi.make_problem(2, gi.U1, 1, 3)
    bs = fock.bond_states(p.gamma_bond)
    for n in range(3):
        for l in range(p.n_links):
            ov = np.vdot(bs[n, l], bs[0, l])
            assert abs(ov.imag) < 1e-14 and ov.real > 0
