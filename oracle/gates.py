"""Dense one- and two-qubit gate matrices (the "Gate class" section) used to pin
the Pauli-exponential convention against the circuit of Fig. 4 / Eq. 11-13."""
from __future__ import annotations

import numpy as np


def _embed1(n: int, q: int, m2: np.ndarray) -> np.ndarray:
    out = np.ones((1, 1), dtype=complex)
    for k in reversed(range(n)):
        out = np.kron(out, m2 if k == q else np.eye(2))
    return out


def hadamard(n: int, q: int) -> np.ndarray:
    """H|0> = (|0>+|1>)/sqrt2, H|1> = (|0>-|1>)/sqrt2 (Eq. 7)."""
    return _embed1(n, q, np.array([[1, 1], [1, -1]]) / np.sqrt(2.0))


def rz(n: int, q: int, phi: float) -> np.ndarray:
    """R_z(phi) = exp(-i phi Z / 2)."""
    return _embed1(n, q, np.diag([np.exp(-0.5j * phi), np.exp(0.5j * phi)]))


def cnot(n: int, control: int, target: int) -> np.ndarray:
    """Flip `target` where `control` is 1, built entry by entry on basis indices."""
    N = 1 << n
    m = np.zeros((N, N), dtype=complex)
    for b in range(N):
        c = b ^ (1 << target) if (b >> control) & 1 else b
        m[c, b] = 1.0
    return m
