"""Fermionic operators on the qubit basis, the molecular Hamiltonian and the dUCC ansatz.

* Occupation: spin orbital p <-> qubit p; occupied = bit 1 (Eq. 15: a_p lowers
  |1>_p to |0>_p).
* Jordan-Wigner sign (Eq. 15-16): a_p |n> = (-1)^{sum_{q<p} n_q} |n - e_p> if n_p = 1,
      a_p^dagger |n> = (-1)^{sum_{q<p} n_q} |n + e_p> if n_p = 0.
* Spin orbitals are interleaved: 2p is alpha, 2p+1 is beta of spatial orbital p
  (the p-dUCCD example in the "Developing new algorithms" section); the
  Hartree-Fock determinant fills the lowest n_el spin orbitals.
* Molecular Hamiltonian (Eq. 1) from chemists'-notation spatial integrals:
      H = sum_{pq,s} h_pq a+_{ps} a_{qs}
        + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}.
* dUCC (Eq. 19): tau = a+_a a+_b ... a_j a_i with i<j occupied and a<b virtual,
  kappa = tau - tau^dagger, U = prod_mu exp(t_mu kappa_mu); operators are ordered
  by the integer value of the excited determinant tau_mu |Phi_HF> (ascending),
  the first one acting first on the reference.
* The Jordan-Wigner image is built here by multiplying single-qubit Pauli
  letters (a route independent of the bit-mask algebra used elsewhere).
* PQE: the residuals of Eq. 23, their three-energy form (Eq. 24-25), and the
  quasi-Newton iteration of Eq. 26 with Moller-Plesset denominators from the
  determinant's Fock diagonal; ADAPT operator gradients (Eq. 21).
"""
from __future__ import annotations

import itertools

import numpy as np

# ----------------------------------------------------------------------------
# fermion action on state vectors (vectorised over the basis; columns allowed)


def _below_parity(n: int, p: int) -> np.ndarray:
    b = np.arange(1 << n)
    mask = (1 << p) - 1
    c = np.zeros(1 << n, dtype=np.int64)
    v = b & mask
    while np.any(v):
        c += v & 1
        v >>= 1
    return 1.0 - 2.0 * (c & 1)


def annihilate(psi: np.ndarray, n: int, p: int) -> np.ndarray:
    """a_p psi (psi may be a vector or a matrix whose rows are basis indices)."""
    b = np.arange(1 << n)
    occ = ((b >> p) & 1) == 1
    sgn = _below_parity(n, p)
    out = np.zeros_like(psi)
    src = b[occ]
    if psi.ndim == 1:
        out[src ^ (1 << p)] = sgn[src] * psi[src]
    else:
        out[src ^ (1 << p)] = sgn[src][:, None] * psi[src]
    return out


def create(psi: np.ndarray, n: int, p: int) -> np.ndarray:
    """a_p^dagger psi."""
    b = np.arange(1 << n)
    emp = ((b >> p) & 1) == 0
    sgn = _below_parity(n, p)
    out = np.zeros_like(psi)
    src = b[emp]
    if psi.ndim == 1:
        out[src | (1 << p)] = sgn[src] * psi[src]
    else:
        out[src | (1 << p)] = sgn[src][:, None] * psi[src]
    return out


def apply_string(psi: np.ndarray, n: int, ops) -> np.ndarray:
    """Apply a product of ladder operators written left to right, e.g.
    [('+', a), ('+', b), ('-', j), ('-', i)] is a+_a a+_b a_j a_i; the rightmost
    acts first."""
    for kind, p in reversed(list(ops)):
        psi = create(psi, n, p) if kind == "+" else annihilate(psi, n, p)
    return psi


def ladder_dense(n: int, p: int, dagger: bool) -> np.ndarray:
    eye = np.eye(1 << n, dtype=complex)
    return create(eye, n, p) if dagger else annihilate(eye, n, p)


# ----------------------------------------------------------------------------
# Hamiltonian


def hamiltonian_apply_direct(psi: np.ndarray, n_orb: int, h: np.ndarray, g: np.ndarray) -> np.ndarray:
    """H psi with every spin-orbital term applied by the ladder action (slow, plain)."""
    n = 2 * n_orb
    out = np.zeros_like(psi)
    for p in range(n_orb):
        for q in range(n_orb):
            for s in range(2):
                out += h[p, q] * apply_string(psi, n, [("+", 2 * p + s), ("-", 2 * q + s)])
    for p, q, r, s_ in itertools.product(range(n_orb), repeat=4):
        v = g[p, q, r, s_]
        if v == 0.0:
            continue
        for sg in range(2):
            for tg in range(2):
                P, Q, R, S = 2 * p + sg, 2 * q + sg, 2 * r + tg, 2 * s_ + tg
                out += 0.5 * v * apply_string(psi, n, [("+", P), ("+", R), ("-", S), ("-", Q)])
    return out


def _E(psi: np.ndarray, n_orb: int, p: int, q: int) -> np.ndarray:
    """Spin-summed excitation E_pq = sum_s a+_{ps} a_{qs}."""
    n = 2 * n_orb
    out = apply_string(psi, n, [("+", 2 * p), ("-", 2 * q)])
    out += apply_string(psi, n, [("+", 2 * p + 1), ("-", 2 * q + 1)])
    return out


def hamiltonian_apply(psi: np.ndarray, n_orb: int, h: np.ndarray, g: np.ndarray) -> np.ndarray:
    """H psi through spin-summed excitations, using the anticommutation identity
    a+_{ps} a+_{rt} a_{st} a_{qs} summed over spins = E_pq E_rs - delta_qr E_ps.
    Pinned against hamiltonian_apply_direct for small systems."""
    phi = {}
    for r in range(n_orb):
        for s in range(n_orb):
            phi[r, s] = _E(psi, n_orb, r, s)
    out = np.zeros_like(psi)
    for p in range(n_orb):
        for q in range(n_orb):
            chi = h[p, q] * psi
            for r in range(n_orb):
                for s in range(n_orb):
                    if g[p, q, r, s] != 0.0:
                        chi = chi + 0.5 * g[p, q, r, s] * phi[r, s]
            out += _E(chi, n_orb, p, q)
            # -1/2 sum_r (pr|rq) E_pq psi
            k = 0.5 * sum(g[p, r, r, q] for r in range(n_orb))
            if k != 0.0:
                out -= k * phi[p, q]
    return out


def hamiltonian_dense(n_orb: int, h: np.ndarray, g: np.ndarray) -> np.ndarray:
    n = 2 * n_orb
    return hamiltonian_apply_direct(np.eye(1 << n, dtype=complex), n_orb, h, g)


def hf_det(n_el: int) -> int:
    return (1 << n_el) - 1


def hf_energy_closed_form(h: np.ndarray, g: np.ndarray, n_el: int) -> float:
    """Slater-Condon energy of the determinant filling spin orbitals 0..n_el-1:
    E = sum_i h_ii + 1/2 sum_{ij} [(ii|jj) - delta_{s_i s_j} (ij|ji)] over
    occupied spin orbitals."""
    occ = list(range(n_el))
    e = 0.0
    for i in occ:
        e += h[i // 2, i // 2]
    for i in occ:
        for j in occ:
            pi, pj = i // 2, j // 2
            e += 0.5 * g[pi, pi, pj, pj]
            if i % 2 == j % 2:
                e -= 0.5 * g[pi, pj, pj, pi]
    return e


# ----------------------------------------------------------------------------
# dUCC ansatz


def excitations(n_orb: int, n_el: int):
    """Spin-conserving particle-hole singles and doubles, each as (occ tuple,
    vir tuple), sorted by the integer value of tau_mu |Phi_HF>."""
    n = 2 * n_orb
    occ = list(range(n_el))
    vir = list(range(n_el, n))
    ref = hf_det(n_el)
    out = []
    for i in occ:
        for a in vir:
            if i % 2 == a % 2:
                out.append(((i,), (a,)))
    for i, j in itertools.combinations(occ, 2):
        for a, b in itertools.combinations(vir, 2):
            if (i % 2) + (j % 2) == (a % 2) + (b % 2):
                out.append(((i, j), (a, b)))

    def det(ex):
        d = ref
        for i in ex[0]:
            d ^= 1 << i
        for a in ex[1]:
            d |= 1 << a
        return d

    out.sort(key=det)
    return out


def tau_string(ex):
    """tau = a+_a a+_b ... a_j a_i as a left-to-right ladder list."""
    occ, vir = ex
    ops = [("+", a) for a in vir] + [("-", i) for i in reversed(occ)]
    return ops


def tau_dagger_string(ex):
    occ, vir = ex
    ops = [("+", i) for i in occ] + [("-", a) for a in reversed(vir)]
    return ops


def kappa_apply(psi: np.ndarray, n: int, ex) -> np.ndarray:
    return apply_string(psi, n, tau_string(ex)) - apply_string(psi, n, tau_dagger_string(ex))


def kappa_dense(n: int, ex) -> np.ndarray:
    return kappa_apply(np.eye(1 << n, dtype=complex), n, ex)


def ucc_factor_apply(psi: np.ndarray, n: int, ex, t: float) -> np.ndarray:
    """exp(t kappa) psi = psi + sin(t) kappa psi + (1 - cos t) kappa^2 psi,
    which follows from kappa^3 = -kappa for a single excitation generator."""
    k1 = kappa_apply(psi, n, ex)
    k2 = kappa_apply(k1, n, ex)
    return psi + np.sin(t) * k1 + (1.0 - np.cos(t)) * k2


def ucc_state(n_orb: int, n_el: int, t, exs=None) -> np.ndarray:
    """U_dUCC(t) |Phi_HF> (Eq. 19), first operator in the sorted order acting first."""
    n = 2 * n_orb
    if exs is None:
        exs = excitations(n_orb, n_el)
    psi = np.zeros(1 << n, dtype=complex)
    psi[hf_det(n_el)] = 1.0
    for ex, tm in zip(exs, t):
        psi = ucc_factor_apply(psi, n, ex, float(tm))
    return psi


def ucc_energy(n_orb, n_el, h, g, t, exs=None) -> float:
    psi = ucc_state(n_orb, n_el, t, exs)
    return np.vdot(psi, hamiltonian_apply(psi, n_orb, h, g)).real


def ucc_gradient_fd(n_orb, n_el, h, g, t, params, step=1e-4, exs=None):
    t = np.asarray(t, dtype=float)
    out = np.zeros(len(params))
    for k, p in enumerate(params):
        tp = t.copy(); tp[p] += step
        tm = t.copy(); tm[p] -= step
        out[k] = (ucc_energy(n_orb, n_el, h, g, tp, exs) - ucc_energy(n_orb, n_el, h, g, tm, exs)) / (2 * step)
    return out


def ucc_gradient_adjoint(n_orb, n_el, h, g, t, exs=None):
    """dE/dt_mu = 2 Re <lambda_mu| kappa_mu |psi_mu> by a plain reverse sweep over
    the excitation factors (psi_mu, lambda_mu taken after factor mu)."""
    n = 2 * n_orb
    if exs is None:
        exs = excitations(n_orb, n_el)
    psi = ucc_state(n_orb, n_el, t, exs)
    lam = hamiltonian_apply(psi, n_orb, h, g)
    e = np.vdot(psi, lam).real
    grad = np.zeros(len(exs))
    for mu in range(len(exs) - 1, -1, -1):
        ex = exs[mu]
        grad[mu] = 2.0 * np.vdot(lam, kappa_apply(psi, n, ex)).real
        psi = ucc_factor_apply(psi, n, ex, -float(t[mu]))
        lam = ucc_factor_apply(lam, n, ex, -float(t[mu]))
    return e, grad


def adapt_gradients(n_orb, n_el, h, g, t, exs, pool):
    """g_nu = <Psi| [H, kappa_nu] |Psi> (Eq. 21) = 2 Re <H Psi| kappa_nu Psi> for
    each pool excitation, with Psi the dUCC state of exs and t.  Returns (E, g)."""
    n = 2 * n_orb
    psi = ucc_state(n_orb, n_el, t, exs)
    lam = hamiltonian_apply(psi, n_orb, h, g)
    out = np.array([2.0 * np.vdot(lam, kappa_apply(psi, n, ex)).real for ex in pool])
    return np.vdot(psi, lam).real, out


def excited_state(n: int, n_el: int, ex) -> np.ndarray:
    """|Phi_mu> = tau_mu |Phi_HF> (with its fermionic sign)."""
    phi = np.zeros(1 << n, dtype=complex)
    phi[hf_det(n_el)] = 1.0
    return apply_string(phi, n, tau_string(ex))


def pqe_residuals(n_orb, n_el, h, g, t, exs=None):
    """r_mu(t) = <Phi_mu| U^dagger(t) H U(t) |Phi_0> (Eq. 23) for every excitation:
    sigma = H U Phi_0 (direct fermionic action), U^dagger applied factor by factor
    in reverse order, then projected on tau_mu Phi_0.  Returns (E, r)."""
    n = 2 * n_orb
    if exs is None:
        exs = excitations(n_orb, n_el)
    psi = ucc_state(n_orb, n_el, t, exs)
    sig = hamiltonian_apply(psi, n_orb, h, g)
    e = np.vdot(psi, sig).real
    for mu in range(len(exs) - 1, -1, -1):
        sig = ucc_factor_apply(sig, n, exs[mu], -float(t[mu]))
    r = np.array([np.vdot(excited_state(n, n_el, ex), sig) for ex in exs])
    return e, r


def pqe_residuals_from_energies(n_orb, n_el, h, g, t, exs=None):
    """The same residuals from three energies each (Eq. 24): with
    Omega_mu = exp(pi/4 kappa_mu) Phi_0 (Eq. 25),
        r_mu = <Omega_mu|Ubar|Omega_mu> - <Phi_0|Ubar|Phi_0>/2 - <Phi_mu|Ubar|Phi_mu>/2,
    Ubar = U^dagger H U; valid for real H and real amplitudes."""
    n = 2 * n_orb
    if exs is None:
        exs = excitations(n_orb, n_el)

    def ubar_energy(start):
        psi = start
        for ex, tm in zip(exs, t):
            psi = ucc_factor_apply(psi, n, ex, float(tm))
        return np.vdot(psi, hamiltonian_apply(psi, n_orb, h, g)).real

    phi0 = np.zeros(1 << n, dtype=complex)
    phi0[hf_det(n_el)] = 1.0
    e0 = ubar_energy(phi0)
    out = []
    for ex in exs:
        omega = ucc_factor_apply(phi0, n, ex, np.pi / 4)
        out.append(ubar_energy(omega) - 0.5 * e0 - 0.5 * ubar_energy(excited_state(n, n_el, ex)))
    return np.array(out)


def orbital_energies(h, g, n_el):
    """Hartree-Fock orbital energies of the determinant filling spin orbitals
    0..n_el-1, one per spin orbital P (spatial p = P // 2, spin P % 2): the
    diagonal Fock element
        eps_P = h_pp + sum over occupied J of [(pp|jj) - delta_{s_P s_J} (pj|jp)],
    whose differences form the Moller-Plesset denominators of Eq. 26."""
    n = 2 * h.shape[0]
    eps = np.zeros(n)
    for P in range(n):
        p = P // 2
        e = h[p, p]
        for J in range(n_el):
            j = J // 2
            e += g[p, p, j, j]
            if P % 2 == J % 2:
                e -= g[p, j, j, p]
        eps[P] = e
    return eps


def mp_denominators(eps, exs):
    """Delta_mu = eps_i + eps_j + ... - eps_a - eps_b - ... (Eq. 26)."""
    return np.array([sum(eps[i] for i in occ) - sum(eps[a] for a in vir) for occ, vir in exs])


def pqe_solve(n_orb, n_el, h, g, exs=None, t0=None, tol=1e-10, max_iter=200):
    """PQE by the quasi-Newton iteration of Eq. 26,
        t_mu <- t_mu + r_mu(t) / Delta_mu,
    with the residuals of Eq. 23 (`pqe_residuals`) and the denominators of the
    Hartree-Fock orbital energies, from t0 (zeros by default) until every
    |r_mu| < tol.  Returns (t, E, history): history lists (E, max |r|) at each
    evaluated t, and E and t are those of the last evaluation."""
    if exs is None:
        exs = excitations(n_orb, n_el)
    delta = mp_denominators(orbital_energies(h, g, n_el), exs)
    t = np.zeros(len(exs)) if t0 is None else np.array(t0, dtype=float)
    history = []
    for _ in range(max_iter):
        e, r = pqe_residuals(n_orb, n_el, h, g, t, exs)
        r = r.real
        history.append((e, float(np.abs(r).max())))
        if history[-1][1] < tol:
            break
        t = t + r / delta
    return t, e, history


# ----------------------------------------------------------------------------
# Jordan-Wigner by Pauli-letter multiplication

# single-qubit products: (a, b) -> (phase, c) with a b = phase c
_MUL = {
    ("I", "I"): (1, "I"), ("I", "X"): (1, "X"), ("I", "Y"): (1, "Y"), ("I", "Z"): (1, "Z"),
    ("X", "I"): (1, "X"), ("X", "X"): (1, "I"), ("X", "Y"): (1j, "Z"), ("X", "Z"): (-1j, "Y"),
    ("Y", "I"): (1, "Y"), ("Y", "X"): (-1j, "Z"), ("Y", "Y"): (1, "I"), ("Y", "Z"): (1j, "X"),
    ("Z", "I"): (1, "Z"), ("Z", "X"): (1j, "Y"), ("Z", "Y"): (-1j, "X"), ("Z", "Z"): (1, "I"),
}


def _mul_strings(sa: str, sb: str):
    phase = 1 + 0j
    out = []
    for a, b in zip(sa, sb):
        ph, c = _MUL[(a, b)]
        phase *= ph
        out.append(c)
    return phase, "".join(out)


def jw_ladder(n: int, p: int, dagger: bool):
    """Eq. 15-16: a_p = (X_p + i Y_p)/2 Z_{p-1}...Z_0, a+_p = (X_p - i Y_p)/2 Z..."""
    base = ["Z"] * p + ["I"] * (n - p)
    sx = base.copy(); sx[p] = "X"
    sy = base.copy(); sy[p] = "Y"
    s = -0.5j if dagger else 0.5j
    return {"".join(sx): 0.5 + 0j, "".join(sy): s}


def jw_product(n: int, ops):
    """JW image of a product of ladder operators (left to right) as {letters: coeff}."""
    acc = {"I" * n: 1 + 0j}
    for kind, p in ops:
        f = jw_ladder(n, p, kind == "+")
        nxt = {}
        for sa, ca in acc.items():
            for sb, cb in f.items():
                ph, sc = _mul_strings(sa, sb)
                nxt[sc] = nxt.get(sc, 0) + ca * cb * ph
        acc = {k: v for k, v in nxt.items() if abs(v) > 1e-15}
    return acc


def letters_to_masks(s: str):
    x = z = 0
    for i, ch in enumerate(s):
        if ch in "XY":
            x |= 1 << i
        if ch in "YZ":
            z |= 1 << i
    return x, z


def letters_dense(s: str) -> np.ndarray:
    mats = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
            "Z": np.array([[1, 0], [0, -1]])}
    m = np.ones((1, 1), dtype=complex)
    for ch in reversed(s):
        m = np.kron(m, mats[ch])
    return m


def jw_kappa_rotations(n: int, ex):
    """kappa = tau - tau+ = i sum_k c_k P_k (real c_k); returns [(x, z, c_k)].
    Then exp(t kappa) = prod_k exp(-i theta_k P_k) with theta_k = -c_k t because
    the strings commute."""
    a = jw_product(n, tau_string(ex))
    b = jw_product(n, tau_dagger_string(ex))
    k = dict(a)
    for s, c in b.items():
        k[s] = k.get(s, 0) - c
    out = []
    for s in sorted(k):
        c = k[s]
        if abs(c) < 1e-14:
            continue
        ck = c / 1j
        assert abs(ck.imag) < 1e-12
        x, z = letters_to_masks(s)
        out.append((x, z, ck.real))
    return out


def jw_hamiltonian(n_orb: int, h: np.ndarray, g: np.ndarray):
    """Qubit Hamiltonian (Eq. 2) from the letter-product JW of every term."""
    n = 2 * n_orb
    acc = {}

    def add(ops, coeff):
        for s, c in jw_product(n, ops).items():
            acc[s] = acc.get(s, 0) + coeff * c

    for p in range(n_orb):
        for q in range(n_orb):
            for s in range(2):
                if h[p, q] != 0.0:
                    add([("+", 2 * p + s), ("-", 2 * q + s)], h[p, q])
    for p, q, r, s_ in itertools.product(range(n_orb), repeat=4):
        v = g[p, q, r, s_]
        if v == 0.0:
            continue
        for sg in range(2):
            for tg in range(2):
                P, Q, R, S = 2 * p + sg, 2 * q + sg, 2 * r + tg, 2 * s_ + tg
                if P == R or Q == S:
                    continue
                add([("+", P), ("+", R), ("-", S), ("-", Q)], 0.5 * v)
    out = []
    for s in sorted(acc):
        c = acc[s]
        if abs(c) < 1e-14:
            continue
        assert abs(c.imag) < 1e-10
        x, z = letters_to_masks(s)
        out.append((x, z, c.real))
    return out
