"""Pins of the oracle's Pauli-string exponential (Eq. 9, Eq. 11-13) and expectation (Eq. 18)."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import gates, pauli

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_single_qubit_closed_forms():
    th = 0.37
    c, s = np.cos(th), np.sin(th)
    zero = np.array([1, 0], dtype=complex)
    one = np.array([0, 1], dtype=complex)
    # exp(-i th X)|0> = c|0> - i s|1>
    np.testing.assert_allclose(pauli.rotate(zero, 1, 1, 0, th), [c, -1j * s], atol=1e-15)
    # exp(-i th Y)|0> = c|0> + s|1>   (Y|0> = i|1>)
    np.testing.assert_allclose(pauli.rotate(zero, 1, 1, 1, th), [c, s], atol=1e-15)
    # exp(-i th Z)|1> = e^{i th}|1>
    np.testing.assert_allclose(pauli.rotate(one, 1, 0, 1, th), [0, np.exp(1j * th)], atol=1e-15)
    # exp(-i th Z)|0> = e^{-i th}|0>
    np.testing.assert_allclose(pauli.rotate(zero, 1, 0, 1, th), [np.exp(-1j * th), 0], atol=1e-15)


def test_two_qubit_closed_form_bit_order():
    # P = X on qubit 0, Y on qubit 1 (x = 0b11, z = 0b10).  On |00>:
    # P|00> = X0 Y1 |q0=0,q1=0> = i |q0=1,q1=1>, so exp(-i th P)|00> = c|00> + s|11>.
    th = 0.81
    psi = np.zeros(4, dtype=complex); psi[0] = 1
    out = pauli.rotate(psi, 2, 0b11, 0b10, th)
    np.testing.assert_allclose(out, [np.cos(th), 0, 0, np.sin(th)], atol=1e-15)
    # Z on qubit 1 only: index 2 (q1 = 1) picks up the minus sign.
    psi = np.full(4, 0.5, dtype=complex)
    np.testing.assert_allclose(pauli.apply(psi, 2, 0, 0b10), [0.5, 0.5, -0.5, -0.5])


@pytest.mark.parametrize("n", [1, 2, 3])
def test_every_string_matches_expm(n):
    rng = np.random.default_rng(n)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    for x in range(1 << n):
        for z in range(1 << n):
            P = pauli.dense(n, x, z)
            np.testing.assert_allclose(P @ P, np.eye(1 << n), atol=1e-14)
            np.testing.assert_allclose(P, P.conj().T, atol=1e-15)
            th = rng.uniform(-np.pi, np.pi)
            np.testing.assert_allclose(pauli.rotate(psi, n, x, z, th), sl.expm(-1j * th * P) @ psi, atol=1e-12)


def test_random_strings_n8_match_expm():
    n = 8
    rng = np.random.default_rng(8)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    for _ in range(6):
        x, z = int(rng.integers(0, 256)), int(rng.integers(0, 256))
        th = rng.uniform(-np.pi, np.pi)
        ref = sl.expm(-1j * th * pauli.dense(n, x, z)) @ psi
        np.testing.assert_allclose(pauli.rotate(psi, n, x, z, th), ref, atol=1e-11)


def test_worked_example_fig4_identity():
    w = GOLD["worked_exponential"]
    n = 3
    ladder = gates.cnot(n, 0, 1), gates.cnot(n, 1, 2)
    u = (gates.hadamard(n, 2) @ ladder[0] @ ladder[1] @ gates.rz(n, 2, w["rz_angle"])
         @ ladder[1] @ ladder[0] @ gates.hadamard(n, 2))
    ref = sl.expm(-1j * w["theta"] * pauli.dense(n, w["x_mask"], w["z_mask"]))
    np.testing.assert_allclose(u, ref, atol=1e-14)
    # and the oracle's rotation reproduces every column
    for b in range(8):
        e = np.zeros(8, dtype=complex); e[b] = 1
        np.testing.assert_allclose(pauli.rotate(e, n, w["x_mask"], w["z_mask"], w["theta"]), u[:, b], atol=1e-14)
    # the opposite exponent sign does not match
    assert np.abs(sl.expm(+1j * w["theta"] * pauli.dense(n, w["x_mask"], w["z_mask"])) - u).max() > 0.1


def test_bell_state_and_expectation():
    g = GOLD
    psi = np.zeros(4, dtype=complex); psi[0] = 1
    # H_0 then the CNOT of Eq. 8 (control q0, target q1 in index terms)
    psi = gates.cnot(2, 0, 1) @ (gates.hadamard(2, 0) @ psi)
    np.testing.assert_allclose(psi, g["bell_state"]["value"], atol=1e-15)
    table = gates.cnot(2, 0, 1)
    for i, o in g["cnot_truth_table"]["value"]:
        assert table[o, i] == 1
    e = pauli.expectation(psi, 2, [(0b01, 0, 1.0), (0b10, 0, 1.0)])
    assert abs(e - g["bell_X0_plus_X1"]["value"]) < 1e-15
    # and <Z0 Z1> = 1, <X0 X1> = 1 for this Bell state
    assert abs(pauli.expectation(psi, 2, [(0, 0b11, 1.0)]) - 1) < 1e-15
    assert abs(pauli.expectation(psi, 2, [(0b11, 0, 1.0)]) - 1) < 1e-15


def test_expectation_matches_dense_and_is_real():
    n = 5
    rng = np.random.default_rng(5)
    psi = rng.normal(size=32) + 1j * rng.normal(size=32)
    psi /= np.linalg.norm(psi)
    terms = [(int(rng.integers(0, 32)), int(rng.integers(0, 32)), float(rng.normal())) for _ in range(40)]
    H = pauli.dense_sum(n, terms)
    e = pauli.expectation(psi, n, terms)
    np.testing.assert_allclose(e, psi.conj() @ H @ psi, atol=1e-13)
    assert abs(e.imag) < 1e-13


def test_rotations_preserve_norm():
    n = 10
    rng = np.random.default_rng(10)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    rots = [(int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n)), rng.uniform(-3, 3)) for _ in range(30)]
    out = pauli.apply_rotations(psi, n, rots)
    assert abs(np.linalg.norm(out) - 1) < 1e-13


def test_adjoint_gradient_matches_finite_differences():
    n = 6
    rng = np.random.default_rng(6)
    arots = [(int(rng.integers(1, 64)), int(rng.integers(0, 64)), float(rng.normal()), k % 5) for k in range(12)]
    t = rng.normal(size=5)
    terms = [(int(rng.integers(0, 64)), int(rng.integers(0, 64)), float(rng.normal())) for _ in range(20)]
    # make H Hermitian-real: drop terms whose string is imaginary-antisymmetric? all strings are Hermitian
    e, g, _ = pauli.adjoint_gradient(n, 0b000111, arots, t, terms)
    assert abs(e - pauli.energy(n, 0b000111, arots, t, terms)) < 1e-13
    fd = pauli.fd_gradient(n, 0b000111, arots, t, terms, list(range(5)), h=1e-5)
    np.testing.assert_allclose(g, fd, atol=1e-8)


def test_planted_sign_error_is_caught():
    """A rotation with the wrong exponent sign fails the closed form above."""
    th = 0.37
    zero = np.array([1, 0], dtype=complex)
    wrong = np.cos(th) * zero + 1j * np.sin(th) * pauli.apply(zero, 1, 1, 0)
    assert np.abs(wrong - np.array([np.cos(th), -1j * np.sin(th)])).max() > 0.5


def test_residuals_match_dense_transformed_hamiltonian():
    """<b|U^dagger H U|Phi> (Eq. 23 on basis determinants) against the dense
    matrices: U as the product of expm(-i theta P) built from Kronecker
    products, H as the dense Pauli sum."""
    n = 5
    rng = np.random.default_rng(23)
    arots = [(int(rng.integers(1, 32)), int(rng.integers(0, 32)), float(rng.normal()), k % 4) for k in range(10)]
    t = rng.normal(size=4)
    terms = [(int(rng.integers(0, 32)), int(rng.integers(0, 32)), float(rng.normal())) for _ in range(15)]
    det = 0b00101
    dets = list(range(32))
    e, r = pauli.residuals(n, det, arots, t, terms, dets)
    U = np.eye(32, dtype=complex)
    for (x, z, c, p) in arots:
        U = sl.expm(-1j * c * t[p] * pauli.dense(n, x, z)) @ U
    Hbar = U.conj().T @ pauli.dense_sum(n, terms) @ U
    np.testing.assert_allclose(r, Hbar[:, det], atol=1e-12)
    assert abs(e - Hbar[det, det].real) < 1e-12
    assert abs(e - pauli.energy(n, det, arots, t, terms)) < 1e-12


def test_pool_gradients_match_finite_differences_of_the_appended_block():
    """Eq. 21 on Pauli rotations: the pool gradient equals the derivative of the
    energy with the pool operator's rotations appended, at zero angle."""
    n = 5
    rng = np.random.default_rng(21)
    arots = [(int(rng.integers(1, 32)), int(rng.integers(0, 32)), float(rng.normal()), k % 3) for k in range(8)]
    t = rng.normal(size=3)
    terms = [(int(rng.integers(0, 32)), int(rng.integers(0, 32)), float(rng.normal())) for _ in range(15)]
    pool = [(int(rng.integers(1, 32)), int(rng.integers(0, 32)), float(rng.normal()), k % 4) for k in range(9)]
    det = 0b01011
    e, g = pauli.pool_gradients(n, det, arots, t, terms, pool, 4)
    assert abs(e - pauli.energy(n, det, arots, t, terms)) < 1e-13
    for p in range(4):
        block = [(x, z, c, 3) for (x, z, c, q) in pool if q == p]  # the pool operator as parameter 3 of an extension
        ext = list(arots) + block
        fd = []
        for s in (1e-5, -1e-5):
            tt = np.r_[t, s]
            fd.append(pauli.energy(n, det, ext, tt, terms))
        assert abs((fd[0] - fd[1]) / 2e-5 - g[p]) < 1e-8


def test_trotter_exact_for_commuting_terms():
    """Diagonal (Z-only) terms commute, so the Trotter product (Eq. 39) equals
    exp(-i t H) for every step count."""
    n = 4
    rng = np.random.default_rng(39)
    terms = [(0, int(z), float(rng.normal())) for z in rng.integers(0, 16, 8)]
    psi = rng.normal(size=16) + 1j * rng.normal(size=16)
    psi /= np.linalg.norm(psi)
    exact = sl.expm(-1j * 0.7 * pauli.dense_sum(n, terms)) @ psi
    for r in (1, 3):
        np.testing.assert_allclose(pauli.trotter(psi, n, terms, 0.7, r), exact, atol=1e-12)


def test_trotter_first_order_error_bound_and_rate():
    """Non-commuting terms: the first-order product error stays within
    (t^2 / 2r) sum_{j<k} ||[h_j P_j, h_k P_k]|| and halves when r doubles."""
    n = 4
    rng = np.random.default_rng(40)
    terms = [(int(rng.integers(0, 16)), int(rng.integers(0, 16)), float(rng.normal())) for _ in range(6)]
    psi = rng.normal(size=16) + 1j * rng.normal(size=16)
    psi /= np.linalg.norm(psi)
    t = 0.3
    exact = sl.expm(-1j * t * pauli.dense_sum(n, terms)) @ psi
    mats = [c * pauli.dense(n, x, z) for (x, z, c) in terms]
    comm = sum(np.linalg.norm(mats[j] @ mats[k] - mats[k] @ mats[j], 2)
               for j in range(len(mats)) for k in range(j + 1, len(mats)))
    errs = []
    for r in (8, 16, 32):
        err = np.linalg.norm(pauli.trotter(psi, n, terms, t, r) - exact)
        assert err <= t * t / (2 * r) * comm + 1e-12
        errs.append(err)
    assert 0.4 < errs[1] / errs[0] < 0.6 and 0.4 < errs[2] / errs[1] < 0.6
