"""Pins of the oracle's fermionic pieces: JW (Eq. 15-16), the Hamiltonian (Eq. 1-2),
dUCC factors (Eq. 19), PQE (Eq. 23-26), ADAPT gradients (Eq. 21) and Tab. 1's
parameter and CNOT counts."""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import fermion, pauli
from workloads import integrals, amplitudes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("n", [1, 3, 6])
def test_jw_ladder_matches_bitstring_action(n):
    for p in range(n):
        for dag in (False, True):
            d = sum(c * fermion.letters_dense(s) for s, c in fermion.jw_ladder(n, p, dag).items())
            np.testing.assert_allclose(d, fermion.ladder_dense(n, p, dag), atol=1e-15)


def test_anticommutation():
    n = 4
    a = [fermion.ladder_dense(n, p, False) for p in range(n)]
    ad = [fermion.ladder_dense(n, p, True) for p in range(n)]
    for p, q in itertools.product(range(n), repeat=2):
        np.testing.assert_allclose(a[p] @ ad[q] + ad[q] @ a[p], np.eye(16) * (p == q), atol=1e-15)
        np.testing.assert_allclose(a[p] @ a[q] + a[q] @ a[p], 0, atol=1e-15)


def test_ladder_sign_closed_form():
    # a+_2 |q0=1,q1=1,q2=0> = (-1)^2 |111>;  a_1 |011> = (-1)^1 |001>
    n = 3
    v = np.zeros(8, dtype=complex); v[0b011] = 1
    assert fermion.create(v, n, 2)[0b111] == 1
    assert fermion.annihilate(v, n, 1)[0b001] == -1
    assert fermion.annihilate(v, n, 2).sum() == 0


def test_excitation_counts():
    # spin-conserving singles + doubles at the four molecular sizes
    expect = {(4, 4): (8, 18), (8, 8): (32, 328), (12, 12): (72, 1746), (2, 2): (2, 1)}
    for (no, ne), (ns, nd) in expect.items():
        ex = fermion.excitations(no, ne)
        assert sum(len(e[0]) == 1 for e in ex) == ns
        assert sum(len(e[0]) == 2 for e in ex) == nd


def test_excitation_order_is_ascending_determinant():
    ex = fermion.excitations(4, 4)
    ref = fermion.hf_det(4)
    dets = []
    for e in ex:
        v = np.zeros(256, dtype=complex); v[ref] = 1
        w = fermion.apply_string(v, 8, fermion.tau_string(e))
        nz = np.flatnonzero(w)
        assert len(nz) == 1 and abs(abs(w[nz[0]]) - 1) < 1e-15
        dets.append(int(nz[0]))
    assert dets == sorted(dets) and len(set(dets)) == len(dets)


@pytest.mark.parametrize("ex", [((1,), (3,)), ((0, 1), (2, 3)), ((0, 3), (4, 7)), ((2, 3), (4, 5))])
def test_ucc_factor_matches_expm_and_pauli_product(ex):
    n = 8
    rng = np.random.default_rng(0)
    psi = rng.normal(size=256) + 1j * rng.normal(size=256)
    t = 0.7
    K = fermion.kappa_dense(n, ex)
    np.testing.assert_allclose(K, -K.conj().T, atol=1e-15)
    ref = sl.expm(t * K) @ psi
    np.testing.assert_allclose(fermion.ucc_factor_apply(psi, n, ex, t), ref, atol=1e-12)
    # kappa = i sum_k c_k P_k and the commuting product of exp(-i(-c_k t)P_k)
    rots = fermion.jw_kappa_rotations(n, ex)
    np.testing.assert_allclose(1j * sum(c * pauli.dense(n, x, z) for x, z, c in rots), K, atol=1e-14)
    expected_count = 2 if len(ex[0]) == 1 else 8
    assert len(rots) == expected_count
    out = psi.copy()
    for x, z, c in rots:
        out = pauli.rotate(out, n, x, z, -c * t)
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_pqe_omega_identity():
    """Eq. 25: exp(pi/4 kappa)|Phi0> = (|Phi0> + |Phi_mu>)/sqrt2 with |Phi_mu> = tau|Phi0>."""
    n, ne = 8, 4
    ref = np.zeros(256, dtype=complex); ref[fermion.hf_det(ne)] = 1
    for ex in fermion.excitations(4, ne)[::5]:
        phimu = fermion.apply_string(ref, n, fermion.tau_string(ex))
        out = fermion.ucc_factor_apply(ref, n, ex, np.pi / 4)
        np.testing.assert_allclose(out, (ref + phimu) / np.sqrt(2), atol=1e-15)


def test_tab1_pduccd_cnot_count():
    """Tab. 1: the p-dUCCD ansatz for H4 (8 qubits, 4 electrons, 4 paired doubles)
    has 192 CNOTs; each JW string of weight w costs 2(w-1) CNOTs in the Fig. 4
    ladder, so this pins the number and weight of the JW strings."""
    gold = GOLD["pdUCCD_H4_NCNOT"]
    n, ne = gold["n_qubits"], gold["n_el"]
    nocc, nvir = ne // 2, (n - ne) // 2
    total = 0
    npar = 0
    for i in range(nocc):
        for a in range(nvir):
            ia, ib = 2 * i, 2 * i + 1
            aa, ab = 2 * nocc + 2 * a, 2 * nocc + 2 * a + 1
            # tau = a+_{a_b} a+_{a_a} a_{i_a} a_{i_b} as in the p-dUCCD factor
            tau = [("+", ab), ("+", aa), ("-", ia), ("-", ib)]
            taud = [("+", ib), ("+", ia), ("-", aa), ("-", ab)]
            k = fermion.jw_product(n, tau)
            for s, c in fermion.jw_product(n, taud).items():
                k[s] = k.get(s, 0) - c
            for s, c in k.items():
                if abs(c) > 1e-14:
                    w = sum(ch != "I" for ch in s)
                    total += 2 * (w - 1)
            npar += 1
    assert npar == gold["n_par"]
    assert total == gold["value"]


def test_tab1_duccsd_parameter_and_cnot_counts():
    """Tab. 1: dUCCSD for linear H4 (8 qubits, 4 electrons) has 14 parameters and
    736 CNOTs.  The chain's orbitals alternate sigma_g / sigma_u, so the
    totally symmetric excitations are those with an even number of sigma_u
    orbitals; each JW string of weight w costs 2(w-1) CNOTs (Fig. 4).  Checked
    for the oracle's strings and for host prep's ansatz."""
    from paper_2108_04413_gb300 import prep

    gold = GOLD["dUCCSD_H4"]
    n, ne = gold["n_qubits"], gold["n_el"]
    irrep = gold["orbital_symmetry"]
    exs = fermion.excitations(n // 2, ne)
    keep = [k for k, (occ, vir) in enumerate(exs) if sum(irrep[q // 2] for q in occ + vir) % 2 == 0]
    assert len(keep) == gold["n_par"]
    cnot = sum(2 * (bin(int(x) | int(z)).count("1") - 1)
               for k in keep for x, z, _ in fermion.jw_kappa_rotations(n, exs[k]))
    assert cnot == gold["n_cnot"]
    A, exs_p = prep.uccsd_ansatz(n // 2, ne)
    assert [tuple(map(tuple, e)) for e in exs_p] == [tuple(map(tuple, e)) for e in exs]
    rows = np.isin(A["param"], keep)
    w = np.array([bin(int(x) | int(z)).count("1") for x, z in zip(A["x"][rows], A["z"][rows])])
    assert int(np.sum(2 * (w - 1))) == gold["n_cnot"]


@pytest.mark.parametrize("n_orb", [2, 3])
def test_hamiltonian_three_ways(n_orb):
    h, g = integrals(n_orb, 11 + n_orb)
    n = 2 * n_orb
    Hf = fermion.hamiltonian_dense(n_orb, h, g)
    np.testing.assert_allclose(Hf, Hf.conj().T, atol=1e-14)
    Hp = pauli.dense_sum(n, fermion.jw_hamiltonian(n_orb, h, g))
    np.testing.assert_allclose(Hp, Hf, atol=1e-12)
    rng = np.random.default_rng(1)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    np.testing.assert_allclose(fermion.hamiltonian_apply(psi, n_orb, h, g), Hf @ psi, atol=1e-12)


def test_integral_symmetry():
    h, g = integrals(4, 0)
    np.testing.assert_array_equal(h, h.T)
    assert np.all(np.diag(h) <= 0) and np.all(np.diag(h) >= -2)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)]:
        np.testing.assert_array_equal(g, g.transpose(perm))


def test_hf_energy_slater_condon_and_variational_bound():
    n_orb, ne = 4, 4
    h, g = integrals(n_orb, 0)
    H = fermion.hamiltonian_dense(n_orb, h, g)
    det = fermion.hf_det(ne)
    e0 = fermion.hf_energy_closed_form(h, g, ne)
    assert abs(H[det, det].real - e0) < 1e-12
    exs = fermion.excitations(n_orb, ne)
    t = amplitudes(len(exs), 0, 0.1)
    assert abs(fermion.ucc_energy(n_orb, ne, h, g, np.zeros(len(exs)), exs) - e0) < 1e-12
    psi = fermion.ucc_state(n_orb, ne, t, exs)
    e = np.vdot(psi, H @ psi)
    assert abs(e.imag) < 1e-13
    # lowest eigenvalue in the 4-electron, S_z = 0 sector bounds E from below
    b = np.arange(256)
    na = np.array([bin(v & 0x55).count("1") for v in b]); nb = np.array([bin(v & 0xAA).count("1") for v in b])
    sec = np.flatnonzero((na == 2) & (nb == 2))
    efci = np.linalg.eigvalsh(H[np.ix_(sec, sec)].real)[0]
    assert e.real >= efci - 1e-12
    # state stays in the sector with unit norm
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    out = np.setdiff1d(b, sec)
    assert np.abs(psi[out]).max() < 1e-14


def test_ucc_adjoint_matches_fd():
    n_orb, ne = 3, 2
    h, g = integrals(n_orb, 5)
    exs = fermion.excitations(n_orb, ne)
    t = amplitudes(len(exs), 5, 0.3)
    e, grad = fermion.ucc_gradient_adjoint(n_orb, ne, h, g, t, exs)
    fd = fermion.ucc_gradient_fd(n_orb, ne, h, g, t, list(range(len(exs))), step=1e-5, exs=exs)
    np.testing.assert_allclose(grad, fd, atol=1e-8)


def test_ucc_pauli_route_equals_fermion_route():
    """The oracle's two routes to the dUCC state agree: fermionic closed-form
    factors vs the JW Pauli rotations (each excitation's strings, in order)."""
    n_orb, ne = 3, 2
    n = 6
    exs = fermion.excitations(n_orb, ne)
    t = amplitudes(len(exs), 9, 0.4)
    a = fermion.ucc_state(n_orb, ne, t, exs)
    psi = np.zeros(64, dtype=complex); psi[fermion.hf_det(ne)] = 1
    for ex, tm in zip(exs, t):
        for x, z, c in fermion.jw_kappa_rotations(n, ex):
            psi = pauli.rotate(psi, n, x, z, -c * tm)
    np.testing.assert_allclose(psi, a, atol=1e-13)


@pytest.mark.parametrize("n_orb,ne,seed", [(3, 2, 11), (4, 4, 12)])
def test_pqe_residuals_projection_equals_energy_form(n_orb, ne, seed):
    """Eq. 23 (projection of U^dagger H U Phi_0 on tau_mu Phi_0) and Eq. 24 (three
    energies with Omega_mu of Eq. 25) give the same residuals."""
    h, g = integrals(n_orb, seed)
    exs = fermion.excitations(n_orb, ne)
    t = amplitudes(len(exs), seed, 0.3)
    e, r = fermion.pqe_residuals(n_orb, ne, h, g, t, exs)
    assert np.abs(r.imag).max() < 1e-14
    np.testing.assert_allclose(r.real, fermion.pqe_residuals_from_energies(n_orb, ne, h, g, t, exs), atol=1e-12)
    assert abs(e - fermion.ucc_energy(n_orb, ne, h, g, t, exs)) < 1e-12


def test_pqe_residuals_at_reference_are_half_the_gradient_and_hamiltonian_elements():
    """At t = 0: r_mu = <Phi_mu|H|Phi_0> (a Hamiltonian matrix element), and
    dE/dt_mu = <Phi_0|[H, kappa_mu]|Phi_0> = 2 r_mu for real H."""
    n_orb, ne = 3, 2
    n = 2 * n_orb
    h, g = integrals(n_orb, 13)
    exs = fermion.excitations(n_orb, ne)
    t = np.zeros(len(exs))
    _, r = fermion.pqe_residuals(n_orb, ne, h, g, t, exs)
    _, grad = fermion.ucc_gradient_adjoint(n_orb, ne, h, g, t, exs)
    np.testing.assert_allclose(2 * r.real, grad, atol=1e-12)
    H = fermion.hamiltonian_dense(n_orb, h, g)
    ref = np.zeros(1 << n, dtype=complex)
    ref[fermion.hf_det(ne)] = 1.0
    for ex, rm in zip(exs, r):
        assert abs(rm - np.vdot(fermion.excited_state(n, ne, ex), H @ ref)) < 1e-12


def test_pqe_residuals_pauli_route_equals_fermion_route():
    """The Pauli route (JW rotations and Hamiltonian, residual read at the excited
    determinant's index times its fermionic sign) equals the fermionic route."""
    from paper_2108_04413_gb300 import prep

    n_orb, ne = 3, 2
    n = 2 * n_orb
    h, g = integrals(n_orb, 14)
    exs = fermion.excitations(n_orb, ne)
    t = amplitudes(len(exs), 14, 0.4)
    _, r_f = fermion.pqe_residuals(n_orb, ne, h, g, t, exs)
    A, exs_p = prep.uccsd_ansatz(n_orb, ne)
    T = prep.molecular_hamiltonian(h, g)
    assert [tuple(map(tuple, e)) for e in exs_p] == [tuple(map(tuple, e)) for e in exs]
    dets, signs = [], []
    for ex in exs:
        v = fermion.excited_state(n, ne, ex)
        b = int(np.flatnonzero(v)[0])
        dets.append(b)
        signs.append(v[b].real)
    arots = list(zip(A["x"], A["z"], A["coeff"], A["param"]))
    _, r_p = pauli.residuals(n, fermion.hf_det(ne), arots, t, list(zip(T["x"], T["z"], T["coeff"])), dets)
    np.testing.assert_allclose(np.array(signs) * r_p, r_f, atol=1e-12)


def test_prep_excited_determinants_match_ladder_action():
    """Host prep's excited determinants and signs against the oracle's tau_mu |Phi_0>."""
    from paper_2108_04413_gb300 import prep

    n_orb, ne = 4, 4
    n = 2 * n_orb
    exs = fermion.excitations(n_orb, ne)
    idx, sgn = prep.excited_determinants(exs, fermion.hf_det(ne))
    for ex, b, s in zip(exs, idx, sgn):
        v = fermion.excited_state(n, ne, ex)
        ref = np.zeros_like(v)
        ref[int(b)] = s
        np.testing.assert_array_equal(v, ref)


def test_adapt_gradients_dense_commutator_and_pauli_route():
    """Eq. 21: g_nu = <Psi|[H, kappa_nu]|Psi> against the dense commutator, against
    the Pauli route with the JW pool, and, for the ansatz's own operators at
    t = 0, against the dUCC gradient."""
    from paper_2108_04413_gb300 import prep

    n_orb, ne = 3, 2
    n = 2 * n_orb
    h, g = integrals(n_orb, 21)
    exs = fermion.excitations(n_orb, ne)
    t = amplitudes(len(exs), 21, 0.3)
    pool = exs[::-1]
    e, gp = fermion.adapt_gradients(n_orb, ne, h, g, t, exs, pool)
    psi = fermion.ucc_state(n_orb, ne, t, exs)
    H = fermion.hamiltonian_dense(n_orb, h, g)
    for ex, gv in zip(pool, gp):
        K = fermion.kappa_dense(n, ex)
        assert abs(np.vdot(psi, (H @ K - K @ H) @ psi) - gv) < 1e-12
    A, _ = prep.uccsd_ansatz(n_orb, ne)
    T = prep.molecular_hamiltonian(h, g)
    # the pool is the excitation list reversed: ansatz parameter p is pool operator len - 1 - p
    pool_rots = [(x, z, c, len(pool) - 1 - p) for x, z, c, p in zip(A["x"], A["z"], A["coeff"], A["param"])]
    e2, g2 = pauli.pool_gradients(n, fermion.hf_det(ne), list(zip(A["x"], A["z"], A["coeff"], A["param"])), t,
                                  list(zip(T["x"], T["z"], T["coeff"])), pool_rots, len(pool))
    assert abs(e - e2) < 1e-12
    np.testing.assert_allclose(g2, gp, atol=1e-12)
    _, g0 = fermion.adapt_gradients(n_orb, ne, h, g, np.zeros(len(exs)), exs, exs)
    _, gref = fermion.ucc_gradient_adjoint(n_orb, ne, h, g, np.zeros(len(exs)), exs)
    np.testing.assert_allclose(g0, gref, atol=1e-12)


def _gapped_integrals(n_orb, seed):
    """Seeded integrals with the orbitals relabelled by ascending h_pp, so that
    the determinant's occupied orbitals lie lowest (negative Moller-Plesset
    denominators, as for a Hartree-Fock reference)."""
    h, g = integrals(n_orb, seed)
    o = np.argsort(np.diag(h))
    return h[np.ix_(o, o)], g[np.ix_(o, o, o, o)]


def _sector_ground_energy(H, n_orb, ne):
    b = np.arange(1 << (2 * n_orb))
    na = np.array([bin(v & int("01" * n_orb, 2)).count("1") for v in b])
    nb = np.array([bin(v & int("10" * n_orb, 2)).count("1") for v in b])
    sec = np.flatnonzero((na == (ne + 1) // 2) & (nb == ne // 2))
    return np.linalg.eigvalsh(H[np.ix_(sec, sec)].real)[0]


def test_orbital_energies_koopmans():
    """The orbital energies of Eq. 26 against determinant energies of the dense
    fermionic Hamiltonian (frozen orbitals): taking occupied spin orbital i out
    of Phi_0 changes <Phi|H|Phi> by -eps_i, putting virtual a in changes it by
    +eps_a."""
    n_orb, ne = 4, 4
    h, g = integrals(n_orb, 0)
    H = fermion.hamiltonian_dense(n_orb, h, g)
    d0 = fermion.hf_det(ne)
    eps = fermion.orbital_energies(h, g, ne)
    for q in range(2 * n_orb):
        d = d0 ^ (1 << q)
        want = -eps[q] if q < ne else eps[q]
        assert abs((H[d, d] - H[d0, d0]).real - want) < 1e-12


def test_pqe_solve_two_electrons_reaches_the_exact_ground_state():
    """Two electrons: the singles and doubles span the whole sector, so at the
    fixed point of Eq. 26 (every residual of Eq. 23 zero) U Phi_0 is an
    eigenvector of H, here the lowest of the two-electron S_z = 0 block."""
    n_orb, ne = 3, 2
    h, g = _gapped_integrals(n_orb, 5)
    t, e, hist = fermion.pqe_solve(n_orb, ne, h, g, tol=1e-11)
    assert hist[-1][1] < 1e-11 and hist[-1][1] < hist[0][1]
    H = fermion.hamiltonian_dense(n_orb, h, g)
    assert abs(e - _sector_ground_energy(H, n_orb, ne)) < 1e-10


def test_pqe_solve_four_electrons_converges_above_the_ground_state():
    """Four electrons: the iteration converges (every |r_mu| < 1e-10) to a state
    whose energy, an expectation value, lies at or above the sector's lowest
    eigenvalue, and close to it (dUCCSD)."""
    n_orb, ne = 4, 4
    h, g = _gapped_integrals(n_orb, 0)
    t, e, hist = fermion.pqe_solve(n_orb, ne, h, g, tol=1e-10)
    assert hist[-1][1] < 1e-10
    efci = _sector_ground_energy(fermion.hamiltonian_dense(n_orb, h, g), n_orb, ne)
    assert efci - 1e-12 <= e < efci + 1e-6


@pytest.mark.parametrize("n_orb,ne,seed", [(4, 4, 0), (5, 6, 3), (4, 3, 7)])
def test_prep_orbital_energies_and_denominators_match_oracle(n_orb, ne, seed):
    """Host prep's orbital energies (vectorised) and denominators against the oracle's."""
    from paper_2108_04413_gb300 import prep

    h, g = integrals(n_orb, seed)
    eps = prep.orbital_energies(h, g, fermion.hf_det(ne))
    np.testing.assert_allclose(eps, fermion.orbital_energies(h, g, ne), rtol=0, atol=1e-14)
    exs = fermion.excitations(n_orb, ne)
    np.testing.assert_allclose(prep.mp_denominators(exs, eps), fermion.mp_denominators(eps, exs), rtol=0,
                               atol=1e-14)
