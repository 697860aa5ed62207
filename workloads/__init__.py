"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no Jordan-Wigner transform, no excitation enumeration, no
rotation or expectation).  Both sides of every parity test call these
generators with the same seed and then build their own operators from the raw
draws.

Recipes (stand-ins for the paper's Psi4 molecular integrals, which are not
available; the workload shapes follow the hydrogen-chain timings of the
"Representative timings" section):

* one-electron integrals h_pq: real symmetric, diagonal ~ U(-2, 0), off-diagonal
  ~ N(0, 0.1);
* two-electron integrals (pq|rs) in chemists' notation: real, 8-fold symmetric,
  one draw per canonical quadruple, N(0, 0.05) * exp(-|p-q| - |r-s|);
* cluster amplitudes t_mu ~ N(0, sigma), drawn as a fixed-length stream so the
  first k values do not depend on how many a caller asks for;
* random Pauli strings: weight w ~ U{wmin..min(wmax, n)} distinct qubits, each letter
  uniform in {X, Y, Z}, returned as (x_mask, z_mask) with Y = both bits;
* random angles theta ~ U(-pi, pi); random Pauli-sum coefficients
  N(0, 1) / sqrt(count);
* Poisson request arrivals with exponential gaps.
"""
from __future__ import annotations

import numpy as np

_T_STREAM = 1 << 16


def integrals(n_orb: int, seed: int):
    """Return (h, g): h[p, q] and g[p, q, r, s] = (pq|rs), float64."""
    rng = np.random.default_rng(seed)
    h = np.zeros((n_orb, n_orb))
    for p in range(n_orb):
        h[p, p] = rng.uniform(-2.0, 0.0)
    for p in range(n_orb):
        for q in range(p + 1, n_orb):
            h[p, q] = h[q, p] = rng.normal(0.0, 0.1)
    g = np.zeros((n_orb,) * 4)
    for p in range(n_orb):
        for q in range(p + 1):
            for r in range(n_orb):
                for s in range(r + 1):
                    if (p * (p + 1) // 2 + q) < (r * (r + 1) // 2 + s):
                        continue
                    v = rng.normal(0.0, 0.05) * np.exp(-abs(p - q) - abs(r - s))
                    for (a, b, c, d) in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                                         (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
                        g[a, b, c, d] = v
    return h, g


def amplitudes(count: int, seed: int, sigma: float) -> np.ndarray:
    """First `count` values of a seeded N(0, sigma) stream."""
    if count > _T_STREAM:
        raise ValueError("too many amplitudes requested")
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, size=_T_STREAM)[:count].copy()


def random_pauli_masks(n_qubits: int, count: int, seed: int, wmin: int = 2, wmax: int = 8):
    """Random Pauli strings as uint64 (x_mask, z_mask) arrays."""
    rng = np.random.default_rng(seed)
    xs = np.zeros(count, dtype=np.uint64)
    zs = np.zeros(count, dtype=np.uint64)
    for k in range(count):
        w = int(rng.integers(min(wmin, n_qubits), min(wmax, n_qubits) + 1))
        qubits = rng.choice(n_qubits, size=w, replace=False)
        letters = rng.integers(0, 3, size=w)  # 0 = X, 1 = Y, 2 = Z
        x = 0
        z = 0
        for q, l in zip(qubits, letters):
            if l in (0, 1):
                x |= 1 << int(q)
            if l in (1, 2):
                z |= 1 << int(q)
        xs[k] = x
        zs[k] = z
    return xs, zs


def random_angles(count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi, np.pi, size=count)


def random_coefficients(count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0, size=count) / np.sqrt(count)


def random_state(n_qubits: int, seed: int) -> np.ndarray:
    """A normalised random complex128 state vector (for kernel-level tests)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << n_qubits) + 1j * rng.normal(size=1 << n_qubits)
    return v / np.linalg.norm(v)


def probe_vectors(count: int, length: int, seed: int) -> np.ndarray:
    """`count` seeded N(0, 1) vectors of the given length (random projections that
    compare two long vectors through a few numbers)."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=(count, length))


def sample_indices(length: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct seeded indices in [0, length), ascending."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(length, size=min(count, length), replace=False))


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def serving_choices(count: int, seed: int, qubit_counts=(10, 12, 14, 16, 18, 20, 22), pool_per_n: int = 2):
    """Per request: (qubit count, system index within that count's pool, amplitude seed)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(qubit_counts), size=count)
    sys_idx = rng.integers(0, pool_per_n, size=count)
    t_seeds = rng.integers(0, 2**31 - 1, size=count)
    return ns.astype(int), sys_idx.astype(int), t_seeds.astype(int)


# Sizes of the five workloads (qubits, spatial orbitals, electrons, seeds), by name.
WORKLOADS = {
    "ucc8": dict(name="8q UCCSD", n_qubits=8, n_orb=4, n_el=4, seed=0, t_sigma=0.1),
    "ucc16": dict(name="16q UCCSD", n_qubits=16, n_orb=8, n_el=8, seed=1, t_sigma=0.1),
    "ucc24": dict(name="24q UCCSD", n_qubits=24, n_orb=12, n_el=12, seed=2, t_sigma=0.05),
    "sweep28": dict(name="28q random Pauli exponentials", n_qubits=28, n_el=14, seed=3,
            n_rot=500, n_terms=20000),
    "serving": dict(name="serving", rate=200.0, qubit_counts=(10, 12, 14, 16, 18, 20, 22), seed=4),
}
