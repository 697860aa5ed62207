"""GPU against the oracle at 20, 24 and 28 qubits, through the C ABI.

* 20 qubits (10 spatial orbitals, 10 electrons, 875 excitations, 63,504 sector
  members): the determinant-space oracle runs here, in seconds.  Compared: the
  energy, every gradient component, every PQE residual and ADAPT pool gradient
  of the compact sector path, and the whole state of qf_apply_circuit (the
  full-layout sector sweep, which runs on several CTAs with grid barriers at
  this size).
* 24 qubits (the benchmarked dUCCSD evaluation): the same quantities against
  tests/golden/ucc24_oracle.json, written by tests/golden/make_ucc_golden.py
  from the oracle alone; the state through its sampled amplitudes and seeded
  random projections.
* 28 qubits (the random Pauli-exponential workload): the first 20 rotations
  and the first 200 terms of the 20000-term sum, with the index-list oracle on
  the full register (5 of the 20 strings have their highest X bit at 24-27).

Tolerances as in test_gpu_parity.py: complex128 amplitudes 1e-12, energies and
gradient components 1e-10; complex64 energies 1e-5 Eh, gradients 1e-4
relative in the 2-norm, amplitudes 2e-5.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()

from oracle import fermion, sector, sparse  # noqa: E402
from paper_2108_04413_gb300 import prep, qf  # noqa: E402
from workloads import (WORKLOADS, amplitudes, integrals, probe_vectors, random_angles,  # noqa: E402
                       random_coefficients, random_pauli_masks)

TOL_AMP = {"c128": 1e-12, "c64": 2e-5}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ucc24_oracle.json")


def _close_vec(got, ref, dtype, what):
    if dtype == "c128":
        err = float(np.abs(got - ref).max())
        assert err < 1e-10, (what, err)
    else:
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert err < 1e-4, (what, err)


@pytest.fixture(scope="module")
def ucc20():
    n_orb, n_el, seed = 10, 10, 20
    h, g = integrals(n_orb, seed)
    exs = fermion.excitations(n_orb, n_el)
    t = amplitudes(len(exs), seed, 0.1)
    u = sector.UCC(n_orb, n_el, h, g, exs)
    ref = u.evaluate(t)
    ref["residuals"] = u.residuals(ref["sigma"])
    T = prep.molecular_hamiltonian(h, g)
    A, exs_p = prep.uccsd_ansatz(n_orb, n_el)
    assert exs_p == exs
    return dict(n=2 * n_orb, det=(1 << n_el) - 1, t=t, T=T, A=A, exs=exs, u=u, ref=ref)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ucc20_evaluation_matches_oracle(ucc20, dtype):
    p, ref = ucc20, ucc20["ref"]
    st = qf.State(p["n"], dtype)
    e, grad = st.energy_grad(p["det"], p["A"], p["t"], p["T"])
    assert abs(e - ref["energy"]) < (1e-10 if dtype == "c128" else 1e-5)
    _close_vec(grad, ref["grad"], dtype, "gradient")
    idx, sgn = prep.excited_determinants(p["exs"], p["det"])
    e_r, r = st.residuals(p["det"], p["A"], p["t"], p["T"], idx)
    assert abs(e_r - ref["energy"]) < (1e-10 if dtype == "c128" else 1e-5)
    _close_vec(sgn * r.real, ref["residuals"].real, dtype, "residuals")
    assert np.abs(r.imag).max() == 0.0
    e_p, gp = st.pool_gradients(p["det"], p["A"], p["t"], p["T"], p["A"], len(p["exs"]))
    _close_vec(gp, ref["pool"], dtype, "pool gradients")
    st.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ucc20_apply_circuit_state_matches_oracle(ucc20, dtype):
    """qf_apply_circuit on a sector state: the full-layout sweep kernel over all
    875 excitation blocks, several CTAs with bounded grid barriers."""
    p, ref = ucc20, ucc20["ref"]
    st = qf.State(p["n"], dtype)
    st.set_basis(p["det"])
    st.apply_circuit(prep.bind_thetas(p["A"], p["t"]))
    psi = st.to_numpy()
    members = p["u"].dets.astype(np.int64)
    err = float(np.abs(psi[members] - ref["psi"]).max())
    assert err < TOL_AMP[dtype], err
    outside = np.ones(len(psi), dtype=bool)
    outside[members] = False
    assert np.count_nonzero(psi[outside]) == 0
    e, im = st.expectation(p["T"])
    assert abs(e - ref["energy"]) < (1e-10 if dtype == "c128" else 1e-5) and im == 0.0
    st.close()


@pytest.fixture(scope="module")
def ucc24():
    gold = json.load(open(GOLDEN))
    cfg = WORKLOADS["ucc24"]
    assert (gold["n_orb"], gold["n_el"], gold["seed"], gold["t_sigma"]) == \
        (cfg["n_orb"], cfg["n_el"], cfg["seed"], cfg["t_sigma"])
    h, g = integrals(cfg["n_orb"], cfg["seed"])
    T = prep.molecular_hamiltonian(h, g)
    A, exs = prep.uccsd_ansatz(cfg["n_orb"], cfg["n_el"])
    t = amplitudes(len(exs), cfg["seed"], cfg["t_sigma"])
    return dict(gold=gold, n=cfg["n_qubits"], det=(1 << cfg["n_el"]) - 1, T=T, A=A, exs=exs, t=t)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ucc24_evaluation_matches_oracle_golden(ucc24, dtype):
    """The benchmarked evaluation: energy and all 1818 gradient components, the
    1818 PQE residuals and the 1818 ADAPT gradients of the ansatz's operators."""
    p, gold = ucc24, ucc24["gold"]
    st = qf.State(p["n"], dtype)
    e, grad = st.energy_grad(p["det"], p["A"], p["t"], p["T"])
    assert abs(e - gold["energy"]) < (1e-10 if dtype == "c128" else 1e-5)
    _close_vec(grad, np.array(gold["grad"]), dtype, "gradient")
    idx, sgn = prep.excited_determinants(p["exs"], p["det"])
    _, r = st.residuals(p["det"], p["A"], p["t"], p["T"], idx)
    _close_vec(sgn * r.real, np.array(gold["residuals"]), dtype, "residuals")
    _, gp = st.pool_gradients(p["det"], p["A"], p["t"], p["T"], p["A"], len(p["exs"]))
    _close_vec(gp, np.array(gold["pool"]), dtype, "pool gradients")
    st.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ucc24_apply_circuit_state_matches_oracle_golden(ucc24, dtype):
    p, gold = ucc24, ucc24["gold"]
    st = qf.State(p["n"], dtype)
    st.set_basis(p["det"])
    st.apply_circuit(prep.bind_thetas(p["A"], p["t"]))
    psi = st.to_numpy()
    st.close()
    dets = np.array(gold["sample_dets"], dtype=np.int64)
    err = float(np.abs(psi[dets] - np.array(gold["sample_amps"])).max())
    assert err < TOL_AMP[dtype], err
    members = sector.sector_dets(12, 6, 6).astype(np.int64)
    assert len(members) == gold["n_members"]
    v = psi[members]
    assert abs(np.vdot(v, v).real - gold["norm2"]) < (1e-12 if dtype == "c128" else 1e-5)
    proj = probe_vectors(4, len(members), gold["probe_seed"]) @ v
    tol = 1e-9 if dtype == "c128" else 2e-3
    assert np.abs(proj - np.array(gold["probes"])).max() < tol
    assert np.abs(proj.imag).max() == 0.0


def _sweep28_prefix(k_rot, k_terms):
    """The first rotations and terms of the 28-qubit random workload, drawn from
    the seeded generators with the seeds the library-side helpers use."""
    n, seed = 28, WORKLOADS["sweep28"]["seed"]
    x, z = random_pauli_masks(n, 500, seed)
    th = random_angles(500, seed + 1000)
    tx, tz = random_pauli_masks(n, 20000, seed + 2000)
    c = random_coefficients(20000, seed + 3000)
    return list(zip(x[:k_rot], z[:k_rot], th[:k_rot])), list(zip(tx[:k_terms], tz[:k_terms], c[:k_terms]))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_sweep28_prefix_matches_oracle(dtype):
    n, det = 28, (1 << 14) - 1
    rots, terms = _sweep28_prefix(20, 200)
    idx, amp = sparse.apply_rotations(*sparse.basis(det), rots)
    e_ref = sparse.expectation(idx, amp, terms)
    R = prep.random_circuit(n, 500, WORKLOADS["sweep28"]["seed"])[:20]
    T = prep.random_hamiltonian(n, 20000, WORKLOADS["sweep28"]["seed"])[:200]
    assert [(int(a), int(b)) for a, b, _ in rots] == list(zip(R["x"].tolist(), R["z"].tolist()))
    f = torch.float64 if dtype == "c128" else torch.float32
    ref = torch.zeros(1 << n, dtype=torch.complex128 if dtype == "c128" else torch.complex64, device="cuda")
    ref[torch.from_numpy(idx.astype(np.int64)).cuda()] = torch.from_numpy(amp).to(ref.dtype).cuda()
    for fused in (True, False):
        buf = torch.empty(2 << n, dtype=f, device="cuda")
        st = qf.State(n, dtype, buffer=buf)
        st.set_basis(det)
        if fused:
            st.apply_circuit(R)
        else:
            for r in R:
                st.apply_pauli_exp(int(r["x"]), int(r["z"]), float(r["theta"]))
        torch.cuda.synchronize()
        st.fold_scale()
        torch.cuda.synchronize()
        v = torch.view_as_complex(buf.view(-1, 2))
        err = float((v - ref).abs().max())
        assert err < TOL_AMP[dtype], (fused, err)
        e, im = st.expectation(T)
        assert im == 0.0 and abs(e - e_ref.real) < (1e-10 if dtype == "c128" else 1e-5), (fused, e, e_ref)
        st.close()
        del buf, v
    del ref
    torch.cuda.empty_cache()
