"""Pauli-string exponentials on a state kept as its list of basis indices and
amplitudes (test infrastructure).

A state reached from one basis determinant by k rotations has at most 2^k
non-zero amplitudes, whatever the number of qubits.  Storing only those lets the
plain definition run on the full 28-qubit register for a prefix of a circuit:
* P|b> = i^{popc(x&z)} (-1)^{popc(z&b)} |b XOR x> (basis of Eq. 3, strings of
  Eq. 10, Y = both bits);
* exp(-i theta P) psi = cos(theta) psi - i sin(theta) P psi (Eq. 9 with the
  factor -i theta of Eq. 11-13);
* <psi|H|psi> = sum_l h_l <psi|P_l|psi>, term by term (Eq. 18).
A state is (idx, amp): idx ascending uint64 basis indices, amp complex128.  The
index list only grows (an amplitude that becomes exactly zero is kept).

Pinned (tests/test_oracle_sparse.py) against the dense routines of
`oracle.pauli` (which are pinned to scipy.linalg.expm) on 10 qubits, and
against closed forms on one and two qubits.
"""
from __future__ import annotations

import numpy as np


def _popcount(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, dtype=np.uint64)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    c = np.zeros(a.shape, dtype=np.int64)
    v = a.copy()
    while np.any(v):
        c += (v & np.uint64(1)).astype(np.int64)
        v >>= np.uint64(1)
    return c


def basis(det: int):
    return np.array([det], dtype=np.uint64), np.array([1.0 + 0j])


def _lookup(idx: np.ndarray, amp: np.ndarray, where: np.ndarray) -> np.ndarray:
    """amp at each index of `where` (0 where the index is not stored)."""
    j = np.searchsorted(idx, where)
    jc = np.minimum(j, len(idx) - 1)
    hit = (j < len(idx)) & (idx[jc] == where)
    out = np.zeros(len(where), dtype=complex)
    out[hit] = amp[jc[hit]]
    return out


def apply_pauli(idx: np.ndarray, amp: np.ndarray, x: int, z: int, support: np.ndarray) -> np.ndarray:
    """(P psi) at each index b of `support`: P psi has amplitude
    i^{popc(x&z)} (-1)^{popc(z & c)} psi[c] at b = c XOR x."""
    xs, zs = np.uint64(x), np.uint64(z)
    c = support ^ xs
    phase = (1j) ** (bin(x & z).count("1") % 4)
    sign = 1.0 - 2.0 * (_popcount(c & zs) & 1)
    return phase * sign * _lookup(idx, amp, c)


def rotate(idx: np.ndarray, amp: np.ndarray, x: int, z: int, theta: float):
    """exp(-i theta P(x, z)) applied to (idx, amp); returns the new (idx, amp)."""
    sup = np.union1d(idx, idx ^ np.uint64(x))
    psi = _lookup(idx, amp, sup)
    return sup, np.cos(theta) * psi - 1j * np.sin(theta) * apply_pauli(idx, amp, x, z, sup)


def apply_rotations(idx, amp, rots):
    """Apply (x, z, theta) triples in list order (element 0 first)."""
    for x, z, th in rots:
        idx, amp = rotate(idx, amp, int(x), int(z), float(th))
    return idx, amp


def expectation(idx: np.ndarray, amp: np.ndarray, terms) -> complex:
    """sum_l c_l <psi|P_l|psi> term by term, with no grouping."""
    e = 0.0 + 0.0j
    for x, z, c in terms:
        e += float(c) * np.vdot(amp, apply_pauli(idx, amp, int(x), int(z), idx))
    return e


def dense(idx: np.ndarray, amp: np.ndarray, n: int) -> np.ndarray:
    out = np.zeros(1 << n, dtype=complex)
    out[idx.astype(np.int64)] = amp
    return out
