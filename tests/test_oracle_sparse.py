"""Pins of the index-list oracle (oracle/sparse.py): closed forms on one and two
qubits, and the dense index-arithmetic routines of oracle.pauli (themselves
pinned to scipy.linalg.expm) on random circuits of 10 qubits."""
import numpy as np

from oracle import pauli, sparse
from workloads import random_angles, random_coefficients, random_pauli_masks


def test_closed_forms():
    th = 0.37
    # exp(-i th X)|0> = cos|0> - i sin|1>;  exp(-i th Y)|0> = cos|0> + sin|1>
    i, a = sparse.rotate(*sparse.basis(0), 1, 0, th)
    np.testing.assert_allclose(sparse.dense(i, a, 1), [np.cos(th), -1j * np.sin(th)], atol=1e-16)
    i, a = sparse.rotate(*sparse.basis(0), 1, 1, th)
    np.testing.assert_allclose(sparse.dense(i, a, 1), [np.cos(th), np.sin(th)], atol=1e-16)
    # exp(-i th Z)|1> = e^{i th}|1>
    i, a = sparse.rotate(*sparse.basis(1), 0, 1, th)
    np.testing.assert_allclose(sparse.dense(i, a, 1), [0, np.exp(1j * th)], atol=1e-16)
    # X0 Y1 on |00>: P|00> = i|11>, so exp(-i th P)|00> = cos|00> + sin|11>
    i, a = sparse.rotate(*sparse.basis(0), 0b11, 0b10, th)
    np.testing.assert_allclose(sparse.dense(i, a, 2), [np.cos(th), 0, 0, np.sin(th)], atol=1e-16)
    # <Y> on (|0> + i|1>)/sqrt2 is +1
    i = np.array([0, 1], dtype=np.uint64)
    a = np.array([1, 1j]) / np.sqrt(2)
    assert abs(sparse.expectation(i, a, [(1, 1, 1.0)]) - 1.0) < 1e-15


def test_random_circuit_matches_dense():
    n = 10
    x, z = random_pauli_masks(n, 14, 11)
    th = random_angles(14, 12)
    rots = list(zip(x, z, th))
    det = 0b1011001110
    i, a = sparse.apply_rotations(*sparse.basis(det), rots)
    ref = pauli.apply_rotations(pauli.basis_state(n, det), n, rots)
    np.testing.assert_allclose(sparse.dense(i, a, n), ref, atol=1e-14)
    assert abs(np.vdot(a, a).real - 1.0) < 1e-13
    tx, tz = random_pauli_masks(n, 40, 13)
    c = random_coefficients(40, 14)
    terms = list(zip(tx, tz, c))
    tx[:5] = 0  # diagonal terms too
    e = sparse.expectation(i, a, terms)
    e_ref = pauli.expectation(ref, n, terms)
    assert abs(e - e_ref) < 1e-14 and abs(e.imag) < 1e-15


def test_planted_phase_mistake_is_caught(monkeypatch):
    """Dropping the i^{popc(x&z)} factor (Y taken as XZ) must fail the dense check."""
    n = 6
    rots = [(0b000111, 0b000101, 0.3), (0b110000, 0b100001, -0.8)]
    ref = pauli.apply_rotations(pauli.basis_state(n, 5), n, rots)
    real = sparse.apply_pauli

    def no_y_phase(idx, amp, x, z, support):
        y = bin(x & z).count("1") % 4
        return real(idx, amp, x, z, support) / (1j) ** y

    monkeypatch.setattr(sparse, "apply_pauli", no_y_phase)
    i, a = sparse.apply_rotations(*sparse.basis(5), rots)
    assert np.abs(sparse.dense(i, a, n) - ref).max() > 1e-2
