"""Host-side problem preparation for the GPU path.

* Jordan-Wigner images (Eq. 15-16) of the molecular Hamiltonian (Eq. 1 -> Eq. 2)
  and of the dUCC generators kappa_mu = tau_mu - tau_mu^dagger (Eq. 19), computed
  with bit-mask Pauli algebra vectorised over all terms.
* The dUCCSD excitation list (spin-conserving singles and doubles) in the order
  of the excited determinant's integer value.
* Random Pauli-exponential circuits and random Hermitian Pauli sums built from
  the seeded draws of `workloads`.
* The excited determinants of PQE's residuals (Eq. 23) and the Moller-Plesset
  denominators of its quasi-Newton update (Eq. 26).

Pauli algebra used here: an operator is sum c X^x Z^z ("raw" form, Z applied
first), with (X^x1 Z^z1)(X^x2 Z^z2) = (-1)^{popc(z1 & x2)} X^{x1^x2} Z^{z1^z2}.
The Hermitian string of the C ABI is P(x, z) = i^{popc(x&z)} X^x Z^z, so a raw
coefficient c becomes c * (-i)^{popc(x&z)} on P(x, z).

a_p = (X_p + i Y_p)/2 Z_{<p} = 1/2 X^{e_p} Z^{e_p - 1} - 1/2 X^{e_p} Z^{2 e_p - 1}
a+_p                       = 1/2 X^{e_p} Z^{e_p - 1} + 1/2 X^{e_p} Z^{2 e_p - 1}
"""
from __future__ import annotations

import numpy as np

from .abi import as_arots, as_rots, as_terms

_U = np.uint64


def _popc(a: np.ndarray) -> np.ndarray:
    a = a.astype(np.uint64)
    a = a - ((a >> _U(1)) & _U(0x5555555555555555))
    a = (a & _U(0x3333333333333333)) + ((a >> _U(2)) & _U(0x3333333333333333))
    a = (a + (a >> _U(4))) & _U(0x0F0F0F0F0F0F0F0F)
    return ((a * _U(0x0101010101010101)) >> _U(56)).astype(np.int64)


def ladder_product(ops: np.ndarray, dagger: np.ndarray, coeff: np.ndarray):
    """JW image of products of ladder operators, vectorised over rows.

    ops: (T, k) spin-orbital indices, left to right; dagger: (k,) bools (same
    pattern for every row); coeff: (T,) complex.  Returns raw-form arrays
    (x, z, c) with T * 2^k rows (zero rows included)."""
    T, k = ops.shape
    xs, zs, cs = [], [], []
    for combo in range(1 << k):
        x = np.zeros(T, dtype=np.uint64)
        z = np.zeros(T, dtype=np.uint64)
        c = coeff.astype(np.complex128).copy()
        for f in range(k):
            p = ops[:, f].astype(np.uint64)
            e = np.left_shift(np.ones(T, dtype=np.uint64), p)
            second = (combo >> f) & 1
            fz = (e - _U(1)) | (e if second else _U(0))
            fx = e
            w = 0.5 if (dagger[f] or not second) else -0.5
            # (X^x Z^z)(X^fx Z^fz) = (-1)^{popc(z & fx)} X^{x^fx} Z^{z^fz}
            sgn = 1.0 - 2.0 * (_popc(z & fx) & 1)
            c = c * (w * sgn)
            x = x ^ fx
            z = z ^ fz
        xs.append(x)
        zs.append(z)
        cs.append(c)
    return np.concatenate(xs), np.concatenate(zs), np.concatenate(cs)


def _merge_to_hermitian(x, z, c, n: int, drop: float = 1e-14):
    """Sum duplicate raw strings, convert to P(x, z) coefficients, drop zeros."""
    if n > 32:
        raise ValueError("prep supports at most 32 qubits")
    key = (x << _U(32)) | z
    uk, inv = np.unique(key, return_inverse=True)
    acc = np.zeros(len(uk), dtype=np.complex128)
    np.add.at(acc, inv, c)
    ux = uk >> _U(32)
    uz = uk & _U(0xFFFFFFFF)
    y = _popc(ux & uz) & 3
    acc = acc * ((-1j) ** y)
    keep = np.abs(acc) > drop
    return ux[keep], uz[keep], acc[keep]


def molecular_hamiltonian(h: np.ndarray, g: np.ndarray):
    """Pauli sum of H = sum_{pq,s} h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs
    (spin orbitals interleaved: 2p alpha, 2p+1 beta).  Returns a TERM_DTYPE array."""
    no = h.shape[0]
    n = 2 * no
    # one-body
    p, q, s = np.meshgrid(np.arange(no), np.arange(no), np.arange(2), indexing="ij")
    p, q, s = p.ravel(), q.ravel(), s.ravel()
    c1 = h[p, q]
    ops1 = np.stack([2 * p + s, 2 * q + s], axis=1)
    x1, z1, cc1 = ladder_product(ops1, np.array([True, False]), c1)
    # two-body
    p, q, r, s_, sg, tg = np.meshgrid(*(np.arange(no),) * 4, np.arange(2), np.arange(2), indexing="ij")
    p, q, r, s_, sg, tg = (a.ravel() for a in (p, q, r, s_, sg, tg))
    P, Q, R, S = 2 * p + sg, 2 * q + sg, 2 * r + tg, 2 * s_ + tg
    v = 0.5 * g[p, q, r, s_]
    keep = (P != R) & (Q != S) & (v != 0.0)
    ops2 = np.stack([P[keep], R[keep], S[keep], Q[keep]], axis=1)
    x2, z2, cc2 = ladder_product(ops2, np.array([True, True, False, False]), v[keep])
    x, z, c = _merge_to_hermitian(np.concatenate([x1, x2]), np.concatenate([z1, z2]), np.concatenate([cc1, cc2]), n)
    if np.abs(c.imag).max(initial=0.0) > 1e-10:
        raise ValueError("Hamiltonian has non-real Pauli coefficients")
    return as_terms(x, z, c.real)


def uccsd_excitations(n_orb: int, n_el: int):
    """Spin-conserving particle-hole singles and doubles (occupied i<j, virtual
    a<b, spin orbitals interleaved), ordered by the integer value of the excited
    determinant (ascending)."""
    n = 2 * n_orb
    occ = np.arange(n_el)
    vir = np.arange(n_el, n)
    ref = (1 << n_el) - 1
    ex = []
    for i in occ:
        for a in vir:
            if i % 2 == a % 2:
                ex.append(((int(i),), (int(a),)))
    for ii, i in enumerate(occ):
        for j in occ[ii + 1:]:
            for aa, a in enumerate(vir):
                for b in vir[aa + 1:]:
                    if (i % 2) + (j % 2) == (a % 2) + (b % 2):
                        ex.append(((int(i), int(j)), (int(a), int(b))))
    dets = []
    for o, v in ex:
        d = ref
        for i in o:
            d &= ~(1 << i)
        for a in v:
            d |= 1 << a
        dets.append(d)
    order = np.argsort(np.array(dets, dtype=np.uint64), kind="stable")
    return [ex[k] for k in order]


def kappa_strings(n: int, ex):
    """JW image of kappa = tau - tau^+ for tau = a+_a a+_b ... a_j a_i:
    kappa = i sum_k c_k P_k; returns (x, z, c) sorted by (x, z)."""
    occ, vir = ex
    tau = list(vir) + list(reversed(occ))
    tau_dag = list(occ) + list(reversed(vir))
    k = len(tau)
    dag_t = np.array([True] * len(vir) + [False] * len(occ))
    dag_d = np.array([True] * len(occ) + [False] * len(vir))
    x1, z1, c1 = ladder_product(np.array([tau]), dag_t, np.array([1.0 + 0j]))
    x2, z2, c2 = ladder_product(np.array([tau_dag]), dag_d, np.array([-1.0 + 0j]))
    x, z, c = _merge_to_hermitian(np.concatenate([x1, x2]), np.concatenate([z1, z2]), np.concatenate([c1, c2]), n)
    ck = c / 1j
    if np.abs(ck.imag).max(initial=0.0) > 1e-12:
        raise ValueError("kappa image is not i * real")
    del k
    return x, z, ck.real


def uccsd_ansatz(n_orb: int, n_el: int):
    """dUCCSD rotations: exp(t_mu kappa_mu) = prod_k exp(-i theta_k P_k) with
    theta_k = -c_k t_mu (the strings of one excitation commute).  Returns
    (AROT_DTYPE array, excitation list)."""
    n = 2 * n_orb
    exs = uccsd_excitations(n_orb, n_el)
    xs, zs, cs, ps = [], [], [], []
    for mu, ex in enumerate(exs):
        x, z, c = kappa_strings(n, ex)
        xs.append(x)
        zs.append(z)
        cs.append(-c)
        ps.append(np.full(len(x), mu, dtype=np.int32))
    return as_arots(np.concatenate(xs), np.concatenate(zs), np.concatenate(cs), np.concatenate(ps)), exs


def excited_determinants(excitations, det: int):
    """The excited determinants tau_mu |det> of the PQE residuals (Eq. 23) as
    (basis indices, signs): tau = a+_a a+_b a_j a_i acts right to left, each
    ladder operator on spin orbital p contributing (-1)^{(occupied orbitals
    below p)} (Eq. 15-16).  r_mu = sign_mu * <index_mu| U^dagger H U |det>."""
    idx = np.zeros(len(excitations), dtype=np.uint64)
    sgn = np.zeros(len(excitations))
    for k, (occ, vir) in enumerate(excitations):
        d, s = int(det), 1.0
        ops = [(True, a) for a in vir] + [(False, i) for i in reversed(occ)]  # left to right
        for create, p in reversed(ops):
            occupied = (d >> p) & 1
            if occupied == create:
                raise ValueError("excitation does not act on this determinant")
            if bin(d & ((1 << p) - 1)).count("1") & 1:
                s = -s
            d ^= 1 << p
        idx[k] = d
        sgn[k] = s
    return idx, sgn


def orbital_energies(h: np.ndarray, g: np.ndarray, det: int) -> np.ndarray:
    """Diagonal Fock elements of the determinant det, one per spin orbital
    (qubit 2p is alpha, 2p + 1 beta of spatial orbital p):
        eps[2p + s] = h_pp + sum over occupied J of (pp|jj) - sum over occupied J
                      of spin s of (pj|jp).
    These are the Hartree-Fock orbital energies of the Moller-Plesset
    denominators in PQE's quasi-Newton update (Eq. 26)."""
    n_orb = h.shape[0]
    occ = np.array([q for q in range(2 * n_orb) if (int(det) >> q) & 1], dtype=np.int64)
    j, sj = occ // 2, occ % 2
    p = np.arange(n_orb)
    coulomb = g[p[:, None], p[:, None], j[None, :], j[None, :]].sum(axis=1)
    exch = g[p[:, None], j[None, :], j[None, :], p[:, None]]
    eps = np.empty(2 * n_orb)
    for s in (0, 1):
        eps[s::2] = np.diag(h) + coulomb - exch[:, sj == s].sum(axis=1)
    return eps


def mp_denominators(excitations, eps: np.ndarray) -> np.ndarray:
    """Moller-Plesset denominators Delta_mu = (sum of eps over the excitation's
    occupied spin orbitals) - (sum over its virtual ones), Eq. 26."""
    return np.array([float(np.sum(eps[list(occ)]) - np.sum(eps[list(vir)])) for occ, vir in excitations])


def bind_thetas(ansatz: np.ndarray, t) -> np.ndarray:
    """Plain rotation list (ROT_DTYPE) for parameters t."""
    t = np.asarray(t, dtype=np.float64)
    return as_rots(ansatz["x"], ansatz["z"], ansatz["coeff"] * t[ansatz["param"]])


def random_circuit(n: int, count: int, seed: int):
    """Random Pauli exponentials from the seeded masks and angles."""
    from workloads import random_angles, random_pauli_masks
    x, z = random_pauli_masks(n, count, seed)
    th = random_angles(count, seed + 1000)
    return as_rots(x, z, th)


def random_hamiltonian(n: int, count: int, seed: int):
    from workloads import random_coefficients, random_pauli_masks
    x, z = random_pauli_masks(n, count, seed + 2000)
    c = random_coefficients(count, seed + 3000)
    return as_terms(x, z, c)
