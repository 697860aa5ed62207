"""The fermionic oracle restated on one particle-number sector (test infrastructure).

Every operator in the dUCC energy keeps the number of occupied alpha (even) and
beta (odd) spin orbitals: the molecular Hamiltonian of Eq. 1 is a sum of
spin-conserving a+_p a_q and a+_p a+_r a_s a_q, and each generator
kappa_mu = tau_mu - tau_mu^dagger of Eq. 19 moves electrons between orbitals of
the same spin.  A state that starts as a determinant therefore has non-zero
amplitudes only on the determinants with the same (N_alpha, N_beta), and this
module stores exactly those: entry k of a sector vector is the amplitude of
the k-th such determinant in ascending integer order.  The paper's conclusion
names this restriction as the way to larger systems; here it only makes the
plain computation fit in host memory at 20-24 qubits.

The arithmetic is the plain definition, as in `fermion`:
* ladder operators act on determinants as in Eq. 15-16 (sign = parity of the
  occupied orbitals below p);
* exp(t kappa) = 1 + sin(t) kappa + (1 - cos t) kappa^2 (kappa^3 = -kappa for a
  single excitation generator);
* H psi through spin-summed excitations E_pq, with
  sum over spins of a+_ps a+_rt a_st a_qs = E_pq E_rs - delta_qr E_ps;
* the gradient dE/dt_mu = 2 Re <lambda_mu| kappa_mu |psi_mu> by a reverse sweep
  (psi_mu, lambda_mu taken after factor mu), the PQE residuals of Eq. 23 read
  from U^dagger H U |Phi_0> at the excited determinants, and the ADAPT operator
  gradients of Eq. 21 as 2 Re <H psi| kappa_nu psi>.

Pinned (tests/test_oracle_sector.py) against the dense full-space routes at
n <= 12: the state against products of scipy.linalg.expm of the dense kappa
matrices, H against the dense ladder-matrix Hamiltonian, the energy and
gradient against central differences of the dense energy, and the variational
bound against the sector's lowest eigenvalue.
"""
from __future__ import annotations

import itertools

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


def sector_dets(n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """All determinants with n_alpha occupied alpha (qubit 2p) and n_beta occupied
    beta (qubit 2p+1) spin orbitals, ascending, as uint64."""
    alpha = [sum(1 << (2 * p) for p in c) for c in itertools.combinations(range(n_orb), n_alpha)]
    beta = [sum(1 << (2 * p + 1) for p in c) for c in itertools.combinations(range(n_orb), n_beta)]
    a = np.array(alpha, dtype=np.uint64)
    b = np.array(beta, dtype=np.uint64)
    return np.sort((a[:, None] | b[None, :]).ravel())


def counts_of(det: int):
    """(N_alpha, N_beta) of a determinant."""
    na = sum((det >> q) & 1 for q in range(0, 64, 2))
    nb = sum((det >> q) & 1 for q in range(1, 64, 2))
    return na, nb


def embed(vec: np.ndarray, dets: np.ndarray, n: int) -> np.ndarray:
    """The full 2^n vector of a sector vector."""
    out = np.zeros(1 << n, dtype=complex)
    out[dets.astype(np.int64)] = vec
    return out


class LadderMap:
    """A product of ladder operators restricted to a sector: for each column k
    in `src` it sends |dets[src[k]]> to sgn[k] |dets[dst[k]]>; every other
    determinant goes to zero.  ops lists (kind, p) left to right ('+' creates,
    '-' annihilates); the rightmost acts first (Eq. 15-16)."""

    def __init__(self, dets: np.ndarray, ops):
        d = dets.copy()
        src = np.arange(len(dets), dtype=np.int64)
        sgn = np.ones(len(dets), dtype=np.int8)
        for kind, p in reversed(list(ops)):
            bit = np.uint64(1) << np.uint64(p)
            occ = (d & bit) != 0
            keep = occ if kind == "-" else ~occ
            d, src, sgn = d[keep], src[keep], sgn[keep]
            below = _popcount(d & (bit - np.uint64(1))) & 1
            sgn = np.where(below == 1, -sgn, sgn).astype(np.int8)
            d = d ^ bit
        dst = np.searchsorted(dets, d)
        ok = (dst < len(dets))
        if not np.all(ok) or not np.all(dets[np.minimum(dst, len(dets) - 1)] == d):
            raise ValueError("the operator leaves the sector")
        self.src = src
        self.dst = dst.astype(np.int64)
        self.sgn = sgn.astype(np.float64)
        # each ladder operator toggles one fixed bit of the determinants it keeps,
        # so distinct sources have distinct images
        if len(np.unique(self.dst)) != len(self.dst):
            raise AssertionError("ladder map is not one-to-one")

    def apply(self, vec: np.ndarray) -> np.ndarray:
        out = np.zeros_like(vec)
        out[self.dst] = self.sgn * vec[self.src]
        return out


def _tau_ops(ex):
    occ, vir = ex
    return [("+", a) for a in vir] + [("-", i) for i in reversed(occ)]


def _tau_dagger_ops(ex):
    occ, vir = ex
    return [("+", i) for i in occ] + [("-", a) for a in reversed(vir)]


class Kappa:
    """kappa_mu = tau_mu - tau_mu^dagger on the sector (Eq. 19)."""

    def __init__(self, dets: np.ndarray, ex):
        self.tau = LadderMap(dets, _tau_ops(ex))
        self.tau_dag = LadderMap(dets, _tau_dagger_ops(ex))

    def apply(self, vec: np.ndarray) -> np.ndarray:
        return self.tau.apply(vec) - self.tau_dag.apply(vec)

    def factor(self, vec: np.ndarray, t: float) -> np.ndarray:
        """exp(t kappa) vec = vec + sin(t) kappa vec + (1 - cos t) kappa^2 vec."""
        k1 = self.apply(vec)
        k2 = self.apply(k1)
        return vec + np.sin(t) * k1 + (1.0 - np.cos(t)) * k2


class Hamiltonian:
    """The molecular Hamiltonian of Eq. 1 from chemists'-notation spatial integrals,
        H = sum_{pq,s} h_pq a+_ps a_qs + 1/2 sum_{pqrs,s,t} (pq|rs) a+_ps a+_rt a_st a_qs,
    acting on one sector through the spin-summed E_pq = sum_s a+_ps a_qs."""

    def __init__(self, dets: np.ndarray, n_orb: int, h: np.ndarray, g: np.ndarray):
        self.n_orb = n_orb
        self.h = np.asarray(h, dtype=float)
        self.g = np.asarray(g, dtype=float)
        self.E = {}
        for p in range(n_orb):
            for q in range(n_orb):
                self.E[p, q] = (LadderMap(dets, [("+", 2 * p), ("-", 2 * q)]),
                                LadderMap(dets, [("+", 2 * p + 1), ("-", 2 * q + 1)]))

    def _E(self, p: int, q: int, vec: np.ndarray) -> np.ndarray:
        a, b = self.E[p, q]
        return a.apply(vec) + b.apply(vec)

    def apply(self, psi: np.ndarray) -> np.ndarray:
        """H psi = sum_pq E_pq (h_pq psi + 1/2 sum_rs (pq|rs) E_rs psi)
                   - 1/2 sum_pq (sum_r (pr|rq)) E_pq psi."""
        no = self.n_orb
        phi = np.stack([self._E(r, s, psi) for r in range(no) for s in range(no)])  # (no*no, M)
        gm = self.g.reshape(no * no, no * no)
        out = np.zeros_like(psi)
        for p in range(no):
            for q in range(no):
                chi = self.h[p, q] * psi + 0.5 * (gm[p * no + q] @ phi)
                out += self._E(p, q, chi)
                k = 0.5 * sum(self.g[p, r, r, q] for r in range(no))
                if k != 0.0:
                    out -= k * phi[p * no + q]
        return out


def reference_vector(dets: np.ndarray, det: int) -> np.ndarray:
    """|Phi_0> = |det> as a sector vector."""
    k = int(np.searchsorted(dets, np.uint64(det)))
    if k >= len(dets) or int(dets[k]) != int(det):
        raise ValueError("determinant is not in the sector")
    v = np.zeros(len(dets), dtype=complex)
    v[k] = 1.0
    return v


class UCC:
    """dUCC (Eq. 19) from the determinant det of n_el electrons filling the
    lowest spin orbitals: U(t) = prod_mu exp(t_mu kappa_mu), the first excitation
    of the list acting first."""

    def __init__(self, n_orb: int, n_el: int, h, g, exs):
        self.n_orb = n_orb
        self.n = 2 * n_orb
        self.det = (1 << n_el) - 1
        na, nb = counts_of(self.det)
        self.dets = sector_dets(n_orb, na, nb)
        self.exs = list(exs)
        self.kappas = [Kappa(self.dets, ex) for ex in self.exs]
        self.H = Hamiltonian(self.dets, n_orb, h, g)

    def state(self, t) -> np.ndarray:
        psi = reference_vector(self.dets, self.det)
        for k, tm in zip(self.kappas, t):
            psi = k.factor(psi, float(tm))
        return psi

    def energy(self, t) -> float:
        psi = self.state(t)
        return float(np.vdot(psi, self.H.apply(psi)).real)

    def evaluate(self, t):
        """One forward pass, H psi and one reverse sweep.  Returns a dict with
        the energy E, the final state psi, the gradient dE/dt_mu (adjoint), the
        ADAPT gradients of the ansatz's own operators at psi,
        2 Re <H psi|kappa_mu psi> (Eq. 21), and sigma = U^dagger H U |Phi_0>,
        whose entries at the excited determinants give the PQE residuals
        (Eq. 23)."""
        psi = self.state(t)
        lam = self.H.apply(psi)
        e = float(np.vdot(psi, lam).real)
        pool = np.array([2.0 * np.vdot(lam, k.apply(psi)).real for k in self.kappas])
        grad = np.zeros(len(self.kappas))
        p, l = psi, lam
        for mu in range(len(self.kappas) - 1, -1, -1):
            k = self.kappas[mu]
            grad[mu] = 2.0 * np.vdot(l, k.apply(p)).real
            p = k.factor(p, -float(t[mu]))
            l = k.factor(l, -float(t[mu]))
        return dict(energy=e, psi=psi, grad=grad, pool=pool, sigma=l)

    def residuals(self, sigma: np.ndarray) -> np.ndarray:
        """r_mu = <Phi_mu| U^dagger H U |Phi_0> with |Phi_mu> = tau_mu |Phi_0>
        (its fermionic sign included)."""
        ref = reference_vector(self.dets, self.det)
        return np.array([np.vdot(k.tau.apply(ref), sigma) for k in self.kappas])
