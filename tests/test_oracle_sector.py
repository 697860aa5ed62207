"""Pins of the determinant-space oracle (oracle/sector.py).

Every check goes through matrices built independently of the module's ladder
maps: Jordan-Wigner images of Eq. 15-16 as Kronecker products of 2x2 Pauli
matrices, the qubit Hamiltonian of Eq. 2 from the letter-product JW, products of
scipy.linalg.expm of the dense generators, central differences of the dense
energy, and numpy's eigenvalues.  A planted sign mistake in the ladder action
must fail them."""
import functools
import itertools
from math import comb

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import fermion, pauli, sector
from workloads import amplitudes, integrals


def _jw_dense(n, ops):
    """Dense matrix of a ladder-operator product (left to right) from the
    Kronecker-product JW images a_p = (X_p + i Y_p)/2 Z_{<p}."""
    m = np.eye(1 << n, dtype=complex)
    for kind, p in ops:
        f = sum(c * fermion.letters_dense(s) for s, c in fermion.jw_ladder(n, p, kind == "+").items())
        m = m @ f
    return m


@functools.lru_cache(maxsize=None)
def _dense_h(n_orb, seed):
    """Dense qubit Hamiltonian (Eq. 2) of the seeded integrals, from the
    letter-product JW and Kronecker-product strings."""
    h, g = integrals(n_orb, seed)
    return pauli.dense_sum(2 * n_orb, fermion.jw_hamiltonian(n_orb, h, g))


def _sector_block(m, dets):
    i = dets.astype(np.int64)
    return m[np.ix_(i, i)]


@pytest.mark.parametrize("n_orb,na,nb", [(3, 1, 1), (4, 2, 2), (4, 3, 1), (5, 3, 2)])
def test_sector_dets_brute_force(n_orb, na, nb):
    d = sector.sector_dets(n_orb, na, nb)
    n = 2 * n_orb
    brute = [b for b in range(1 << n)
             if bin(b & int("01" * n_orb, 2)).count("1") == na and bin(b & int("10" * n_orb, 2)).count("1") == nb]
    assert d.tolist() == brute
    assert len(d) == comb(n_orb, na) * comb(n_orb, nb)
    assert sector.counts_of(int(d[0])) == (na, nb)


def test_ladder_maps_match_kronecker_jw():
    n_orb, n = 3, 6
    dets = sector.sector_dets(n_orb, 2, 1)
    rng = np.random.default_rng(5)
    v = rng.normal(size=len(dets)) + 1j * rng.normal(size=len(dets))
    full = sector.embed(v, dets, n)
    # spin-conserving strings: one-body, same-spin and opposite-spin two-body
    for ops in ([("+", 4), ("-", 0)], [("+", 1), ("-", 3)], [("+", 2), ("+", 4), ("-", 0), ("-", 2)],
                [("+", 4), ("+", 5), ("-", 1), ("-", 0)], [("+", 0), ("-", 0)]):
        got = sector.LadderMap(dets, ops).apply(v)
        ref = _jw_dense(n, ops) @ full
        np.testing.assert_allclose(sector.embed(got, dets, n), ref, atol=1e-15)


def test_ladder_map_rejects_operators_leaving_the_sector():
    dets = sector.sector_dets(3, 1, 1)
    with pytest.raises(ValueError):
        sector.LadderMap(dets, [("+", 2), ("-", 1)])  # beta -> alpha


@pytest.mark.parametrize("ex", [((1,), (3,)), ((0, 1), (4, 7)), ((0, 2), (4, 6)), ((2, 3), (4, 5))])
def test_kappa_factor_matches_expm(ex):
    n_orb, n = 4, 8
    dets = sector.sector_dets(n_orb, 2, 2)
    k = sector.Kappa(dets, ex)
    K = _jw_dense(n, [("+", a) for a in ex[1]] + [("-", i) for i in reversed(ex[0])])
    K = K - K.conj().T
    rng = np.random.default_rng(1)
    v = rng.normal(size=len(dets)) + 1j * rng.normal(size=len(dets))
    for t in (0.3, -1.1):
        ref = sl.expm(t * _sector_block(K, dets)) @ v
        np.testing.assert_allclose(k.factor(v, t), ref, atol=1e-13)


@pytest.mark.parametrize("n_orb,n_el,seed", [(3, 3, 7), (4, 4, 0), (5, 5, 3)])
def test_hamiltonian_matches_letter_product_jw(n_orb, n_el, seed):
    n = 2 * n_orb
    h, g = integrals(n_orb, seed)
    na, nb = sector.counts_of((1 << n_el) - 1)
    dets = sector.sector_dets(n_orb, na, nb)
    H = sector.Hamiltonian(dets, n_orb, h, g)
    Hd = _dense_h(n_orb, seed)
    rng = np.random.default_rng(seed)
    v = rng.normal(size=len(dets)) + 1j * rng.normal(size=len(dets))
    np.testing.assert_allclose(H.apply(v), _sector_block(Hd, dets) @ v, atol=1e-12)
    # H maps the sector into itself: nothing of Hd v lands outside it
    out = Hd @ sector.embed(v, dets, n)
    mask = np.ones(1 << n, dtype=bool)
    mask[dets.astype(np.int64)] = False
    assert np.abs(out[mask]).max() < 1e-13


def _dense_kappas(n, exs):
    out = []
    for ex in exs:
        K = _jw_dense(n, [("+", a) for a in ex[1]] + [("-", i) for i in reversed(ex[0])])
        out.append(K - K.conj().T)
    return out


def _dense_ucc(n, n_el, Hd, Ks, t):
    """State and energy of the dense route: product of expm(t kappa) on |HF>."""
    psi = np.zeros(1 << n, dtype=complex)
    psi[(1 << n_el) - 1] = 1.0
    for K, tm in zip(Ks, t):
        psi = sl.expm(tm * K) @ psi
    return psi, float(np.vdot(psi, Hd @ psi).real)


def test_ucc_evaluation_matches_dense_route():
    n_orb, n_el = 4, 4
    n = 2 * n_orb
    h, g = integrals(n_orb, 0)
    exs = fermion.excitations(n_orb, n_el)
    t = amplitudes(len(exs), 0, 0.3)
    u = sector.UCC(n_orb, n_el, h, g, exs)
    r = u.evaluate(t)
    Hd, Ks = _dense_h(n_orb, 0), _dense_kappas(n, exs)
    psi_d, e_d = _dense_ucc(n, n_el, Hd, Ks, t)
    np.testing.assert_allclose(sector.embed(r["psi"], u.dets, n), psi_d, atol=1e-13)
    assert abs(r["energy"] - e_d) < 1e-12
    # gradient: central differences of the dense energy, on the sector blocks of
    # the Kronecker matrices (they map the sector into itself, checked above)
    Hb, Kb = _sector_block(Hd, u.dets), [_sector_block(K, u.dets) for K in Ks]
    v0 = np.zeros(len(u.dets), dtype=complex)
    v0[np.searchsorted(u.dets, np.uint64((1 << n_el) - 1))] = 1.0

    def e_block(tt):
        v = v0
        for K, tm in zip(Kb, tt):
            v = sl.expm(tm * K) @ v
        return float(np.vdot(v, Hb @ v).real)

    step = 1e-5
    for mu in (0, 3, 9, len(exs) - 1):
        tp, tm = t.copy(), t.copy()
        tp[mu] += step
        tm[mu] -= step
        fd = (e_block(tp) - e_block(tm)) / (2 * step)
        assert abs(fd - r["grad"][mu]) < 1e-8
    # ADAPT gradients of the ansatz's own operators: <psi|[H, kappa]|psi>
    for mu in (0, 5, 20):
        c = Hd @ Ks[mu] - Ks[mu] @ Hd
        assert abs(np.vdot(psi_d, c @ psi_d).real - r["pool"][mu]) < 1e-12
    # PQE residuals: <Phi_mu| U^+ H U |Phi_0> with the dense U
    U = np.eye(1 << n, dtype=complex)
    for K, tm in zip(Ks, t):
        U = sl.expm(tm * K) @ U
    ref = np.zeros(1 << n, dtype=complex)
    ref[(1 << n_el) - 1] = 1.0
    ubar = U.conj().T @ Hd @ U @ ref
    res = u.residuals(r["sigma"])
    for mu, ex in enumerate(exs):
        phi_mu = _jw_dense(n, [("+", a) for a in ex[1]] + [("-", i) for i in reversed(ex[0])]) @ ref
        assert abs(np.vdot(phi_mu, ubar) - res[mu]) < 1e-12


def test_ucc_norm_and_variational_bound_odd_electrons():
    n_orb, n_el = 5, 5  # 3 alpha, 2 beta
    h, g = integrals(n_orb, 3)
    exs = fermion.excitations(n_orb, n_el)
    t = amplitudes(len(exs), 3, 0.2)
    u = sector.UCC(n_orb, n_el, h, g, exs)
    psi = u.state(t)
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13
    Hd = _dense_h(n_orb, 3)
    e_min = np.linalg.eigvalsh(_sector_block(Hd, u.dets)).min()
    assert u.energy(t) >= e_min - 1e-12
    # the full-space state of the vectorised fermionic route agrees
    np.testing.assert_allclose(sector.embed(psi, u.dets, 2 * n_orb), fermion.ucc_state(n_orb, n_el, t, exs),
                               atol=1e-13)


def test_planted_parity_mistake_is_caught(monkeypatch):
    """Counting only the alpha orbitals below p in the ladder sign (a plausible
    slip with interleaved spin orbitals) must fail the expm comparison."""
    n_orb, n = 4, 8
    dets = sector.sector_dets(n_orb, 2, 2)
    ex = ((0, 3), (4, 7))
    K = _jw_dense(n, [("+", a) for a in ex[1]] + [("-", i) for i in reversed(ex[0])])
    K = K - K.conj().T
    rng = np.random.default_rng(2)
    v = rng.normal(size=len(dets)) + 0j
    ref = sl.expm(0.4 * _sector_block(K, dets)) @ v
    real_pc = sector._popcount
    monkeypatch.setattr(sector, "_popcount",
                        lambda a: real_pc(np.asarray(a, dtype=np.uint64) & np.uint64(0x5555555555555555)))
    bad = sector.Kappa(dets, ex).factor(v, 0.4)
    assert np.abs(bad - ref).max() > 1e-3


def test_excitation_lists_agree_with_host_prep():
    from paper_2108_04413_gb300 import prep
    for no, ne in ((4, 4), (5, 5), (6, 6)):
        assert fermion.excitations(no, ne) == prep.uccsd_excitations(no, ne)
    assert len(list(itertools.islice(fermion.excitations(12, 12), 5000))) == 1818
