"""The PQE driver's host loop (Eq. 26) on the CPU, with the oracle's Pauli route
standing in for the library's residual call."""
import numpy as np
import pytest

from oracle import fermion, pauli
from paper_2108_04413_gb300 import pqe, prep
from workloads import integrals


class _OracleState:
    """Answers `residuals` like qf.State, from the oracle's Pauli route."""

    def __init__(self, n):
        self.n = n
        self.calls = 0

    def residuals(self, det, ansatz, t, terms, dets):
        self.calls += 1
        arots = list(zip(ansatz["x"], ansatz["z"], ansatz["coeff"], ansatz["param"]))
        return pauli.residuals(self.n, det, arots, t, list(zip(terms["x"], terms["z"], terms["coeff"])),
                               [int(d) for d in dets])


def _problem(n_orb, ne, seed):
    h, g = integrals(n_orb, seed)
    o = np.argsort(np.diag(h))  # occupied orbitals lowest: negative denominators
    h, g = h[np.ix_(o, o)], g[np.ix_(o, o, o, o)]
    A, exs = prep.uccsd_ansatz(n_orb, ne)
    T = prep.molecular_hamiltonian(h, g)
    det = (1 << ne) - 1
    delta = prep.mp_denominators(exs, prep.orbital_energies(h, g, det))
    return h, g, A, exs, T, det, delta


def test_solve_follows_the_oracle_iteration():
    n_orb, ne = 3, 2
    h, g, A, exs, T, det, delta = _problem(n_orb, ne, 5)
    st = _OracleState(2 * n_orb)
    res = pqe.solve(st, det, A, exs, T, delta, tol=1e-10)
    t_o, e_o, hist_o = fermion.pqe_solve(n_orb, ne, h, g, tol=1e-10)
    assert res.converged and st.calls == len(hist_o) == len(res.history)
    np.testing.assert_allclose(res.t, t_o, rtol=0, atol=1e-10)
    assert abs(res.energy - e_o) < 1e-11
    np.testing.assert_allclose([m for _, m in res.history], [m for _, m in hist_o], rtol=1e-6, atol=1e-13)


def test_solve_stops_at_max_iter_with_the_last_evaluated_point():
    n_orb, ne = 3, 2
    h, g, A, exs, T, det, delta = _problem(n_orb, ne, 5)
    res = pqe.solve(_OracleState(2 * n_orb), det, A, exs, T, delta, tol=1e-14, max_iter=2)
    assert not res.converged and len(res.history) == 2
    # the reported point is the second evaluation: one update from zero
    _, r0 = fermion.pqe_residuals(n_orb, ne, h, g, np.zeros(len(exs)))
    np.testing.assert_allclose(res.t, r0.real / delta, rtol=0, atol=1e-12)
    assert abs(res.energy - fermion.ucc_energy(n_orb, ne, h, g, res.t)) < 1e-12


def test_solve_rejects_bad_denominators():
    n_orb, ne = 3, 2
    h, g, A, exs, T, det, delta = _problem(n_orb, ne, 5)
    with pytest.raises(ValueError):
        pqe.solve(_OracleState(6), det, A, exs, T, delta[:-1])
    d0 = delta.copy()
    d0[0] = 0.0
    with pytest.raises(ValueError):
        pqe.solve(_OracleState(6), det, A, exs, T, d0)
