"""Host-side checks that need no GPU: the library loads and exports every call
declared in include/qf.h; the product-side host preparation matches the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qf_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_call():
    from paper_2108_04413_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "qf_apply_pauli_exp" in names and "qf_energy_grad" in names
    for name in names:
        assert hasattr(lib, name), name
    from paper_2108_04413_gb300 import qf

    assert sorted(qf.EXPORTED) == names


def test_prep_hamiltonian_matches_oracle_fermion_matrix():
    from oracle import fermion, pauli
    from paper_2108_04413_gb300 import prep
    from workloads import integrals

    for no, seed in ((2, 3), (3, 4), (4, 0)):
        h, g = integrals(no, seed)
        T = prep.molecular_hamiltonian(h, g)
        Hp = pauli.dense_sum(2 * no, list(zip(T["x"], T["z"], T["coeff"])))
        np.testing.assert_allclose(Hp, fermion.hamiltonian_dense(no, h, g), atol=1e-12)


def test_prep_ansatz_matches_oracle_ucc_state():
    from oracle import fermion, pauli
    from paper_2108_04413_gb300 import prep
    from workloads import amplitudes

    for no, ne in ((3, 2), (4, 4), (3, 3)):
        A, exs = prep.uccsd_ansatz(no, ne)
        assert exs == fermion.excitations(no, ne)
        t = amplitudes(len(exs), 1, 0.3)
        R = prep.bind_thetas(A, t)
        n = 2 * no
        psi = pauli.apply_rotations(pauli.basis_state(n, (1 << ne) - 1), n, list(zip(R["x"], R["z"], R["theta"])))
        np.testing.assert_allclose(psi, fermion.ucc_state(no, ne, t, exs), atol=1e-13)


def test_workload_counts():
    from paper_2108_04413_gb300 import prep

    A, exs = prep.uccsd_ansatz(4, 4)
    assert (len(exs), len(A)) == (26, 160)
    A, exs = prep.uccsd_ansatz(8, 8)
    assert (len(exs), len(A)) == (360, 2688)
