"""Pauli strings, their exponentials, expectation values and the adjoint gradient.

Conventions (readings of the paper, listed with their justification in the
design notes):

* Basis (Eq. 3): amplitude index b = sum_i q_i 2^i, so bit i is qubit q_i.
* A Pauli string is a pair of bit masks (x, z); qubit i carries X if only x_i is
  set, Z if only z_i is set and Y if both are set.  As an operator it is the
  Kronecker product of the single-qubit Paulis (qubit 0 is the least
  significant factor).  Acting on a basis state,
      P |b> = i^{popc(x & z)} (-1)^{popc(z & b)} |b XOR x>.
* Rotation (Eq. 9 with the worked example's factor -i*theta, Eq. 11-13):
      R(theta) = exp(-i theta P) = cos(theta) I - i sin(theta) P   (P^2 = I).
* A circuit is applied in list order: element 0 acts first.
"""
from __future__ import annotations

import numpy as np

_SIGMA = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def popcount(a: np.ndarray) -> np.ndarray:
    """Bit count of each element of an unsigned integer array."""
    a = np.asarray(a, dtype=np.uint64)
    c = np.zeros(a.shape, dtype=np.int64)
    v = a.copy()
    while np.any(v):
        c += (v & np.uint64(1)).astype(np.int64)
        v >>= np.uint64(1)
    return c


def letters(n: int, x: int, z: int) -> str:
    """Letter string of (x, z), qubit 0 first."""
    out = []
    for i in range(n):
        xi, zi = (x >> i) & 1, (z >> i) & 1
        out.append("Y" if (xi and zi) else "X" if xi else "Z" if zi else "I")
    return "".join(out)


def dense(n: int, x: int, z: int) -> np.ndarray:
    """Dense 2^n x 2^n matrix of the string, built as a Kronecker product of 2x2
    Pauli matrices (qubit n-1 is the most significant factor)."""
    m = np.ones((1, 1), dtype=complex)
    for ch in reversed(letters(n, x, z)):  # qubit n-1 first
        m = np.kron(m, _SIGMA[ch])
    return m


def apply(psi: np.ndarray, n: int, x: int, z: int) -> np.ndarray:
    """Return P psi by explicit index arithmetic over every basis index b."""
    N = 1 << n
    b = np.arange(N, dtype=np.uint64)
    y = bin(x & z).count("1")
    phase = (1j) ** y
    sign = 1.0 - 2.0 * (popcount(b & np.uint64(z)) & 1)
    out = np.zeros(N, dtype=complex)
    out[(b ^ np.uint64(x)).astype(np.int64)] = phase * sign * psi
    return out


def rotate(psi: np.ndarray, n: int, x: int, z: int, theta: float) -> np.ndarray:
    """exp(-i theta P) psi = cos(theta) psi - i sin(theta) P psi (Eq. 9, Eq. 11)."""
    return np.cos(theta) * psi - 1j * np.sin(theta) * apply(psi, n, x, z)


def apply_rotations(psi: np.ndarray, n: int, rots) -> np.ndarray:
    """Apply a list of (x, z, theta) in list order (element 0 first)."""
    for (x, z, th) in rots:
        psi = rotate(psi, n, int(x), int(z), float(th))
    return psi


def basis_state(n: int, det: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=complex)
    psi[det] = 1.0
    return psi


def expectation(psi: np.ndarray, n: int, terms) -> complex:
    """Exact operator averaging <psi|H|psi> = sum_l h_l <psi|P_l|psi> (Eq. 18),
    term by term with no grouping."""
    e = 0.0 + 0.0j
    for (x, z, c) in terms:
        e += c * np.vdot(psi, apply(psi, n, int(x), int(z)))
    return e


def apply_sum(psi: np.ndarray, n: int, terms) -> np.ndarray:
    """H psi for H = sum_l h_l P_l, term by term."""
    out = np.zeros_like(psi)
    for (x, z, c) in terms:
        out += c * apply(psi, n, int(x), int(z))
    return out


def dense_sum(n: int, terms) -> np.ndarray:
    m = np.zeros((1 << n, 1 << n), dtype=complex)
    for (x, z, c) in terms:
        m += c * dense(n, int(x), int(z))
    return m


def energy(n: int, det: int, arots, t, terms) -> float:
    """E(t) = <Phi|U(t)^dagger H U(t)|Phi> (Eq. 17) with U the product of
    exp(-i coeff_k t[param_k] P_k) in list order."""
    psi = basis_state(n, det)
    for (x, z, coeff, param) in arots:
        psi = rotate(psi, n, int(x), int(z), coeff * t[param])
    return expectation(psi, n, terms).real


def adjoint_gradient(n: int, det: int, arots, t, terms):
    """Energy and gradient of E(t) by the reverse-sweep (adjoint) recurrence.

    With psi_k = R_k ... R_1 Phi and lambda_K = H psi_K,
        dE/dtheta_k = 2 Im <lambda_k | P_k | psi_k>,
        psi_{k-1} = exp(+i theta_k P_k) psi_k,  lambda_{k-1} = exp(+i theta_k P_k) lambda_k,
    and the chain rule dE/dt_mu = sum_{k in mu} coeff_k dE/dtheta_k.
    Returns (E, dE/dt, dE/dtheta).
    """
    psi = basis_state(n, det)
    thetas = [coeff * t[param] for (_, _, coeff, param) in arots]
    for (x, z, _, _), th in zip(arots, thetas):
        psi = rotate(psi, n, int(x), int(z), th)
    lam = apply_sum(psi, n, terms)
    e = np.vdot(psi, lam).real
    g_theta = np.zeros(len(arots))
    for k in range(len(arots) - 1, -1, -1):
        x, z, coeff, param = arots[k]
        g_theta[k] = 2.0 * np.vdot(lam, apply(psi, n, int(x), int(z))).imag
        psi = rotate(psi, n, int(x), int(z), -thetas[k])
        lam = rotate(lam, n, int(x), int(z), -thetas[k])
    g = np.zeros(len(t))
    for (x, z, coeff, param), gk in zip(arots, g_theta):
        g[param] += coeff * gk
    return e, g, g_theta


def residuals(n: int, det: int, arots, t, terms, dets):
    """<b|U(t)^dagger H U(t)|Phi> for each basis index b in dets, with E(t).

    These are the projective residuals of Eq. 23 (Sec. PQE) on basis
    determinants; the residual of an excited determinant tau_mu|Phi> carries its
    fermionic sign on top.  Plainly: psi = U Phi, sigma = H psi, then U^dagger
    applied as the inverse rotations in reverse order, and sigma read at b.
    Returns (E, complex array over dets)."""
    psi = basis_state(n, det)
    thetas = [coeff * t[param] for (_, _, coeff, param) in arots]
    for (x, z, _, _), th in zip(arots, thetas):
        psi = rotate(psi, n, int(x), int(z), th)
    sig = apply_sum(psi, n, terms)
    e = np.vdot(psi, sig).real
    for k in range(len(arots) - 1, -1, -1):
        x, z, _, _ = arots[k]
        sig = rotate(sig, n, int(x), int(z), -thetas[k])
    return e, np.array([sig[int(b)] for b in dets], dtype=complex)


def pool_gradients(n: int, det: int, arots, t, terms, pool, n_pool: int):
    """Gradients of a pool of operators at the state U(t)|Phi> (Eq. 21, Sec.
    ADAPT): appending the pool's rotations exp(-i coeff_k s_p P_k) at s = 0,
        dE/ds_p = sum_{k in p} coeff_k * 2 Im <H psi | P_k | psi>.
    pool lists (x, z, coeff, param) with param in [0, n_pool).  Returns (E, g)."""
    psi = basis_state(n, det)
    for (x, z, coeff, param) in arots:
        psi = rotate(psi, n, int(x), int(z), coeff * t[param])
    lam = apply_sum(psi, n, terms)
    g = np.zeros(n_pool)
    for (x, z, coeff, param) in pool:
        g[param] += coeff * 2.0 * np.vdot(lam, apply(psi, n, int(x), int(z))).imag
    return np.vdot(psi, lam).real, g


def trotter(psi: np.ndarray, n: int, terms, time: float, steps: int) -> np.ndarray:
    """Trotterized time evolution (Eq. 39): (prod_l exp(-i time c_l P_l / r))^r psi
    with r = steps, the terms applied in list order within each step."""
    for _ in range(steps):
        for (x, z, c) in terms:
            psi = rotate(psi, n, int(x), int(z), c * time / steps)
    return psi


def fd_gradient(n: int, det: int, arots, t, terms, params, h: float = 1e-4):
    """Central finite differences of E(t) for the listed parameter indices."""
    t = np.asarray(t, dtype=float)
    out = np.zeros(len(params))
    for i, p in enumerate(params):
        tp = t.copy(); tp[p] += h
        tm = t.copy(); tm[p] -= h
        out[i] = (energy(n, det, arots, tp, terms) - energy(n, det, arots, tm, terms)) / (2 * h)
    return out
