"""Properties at the benchmark sizes (24 and 28 qubits) that hold at any size:
unit norm, nothing outside the particle-number sector, the two H|psi>
arithmetic modes and the two precisions agreeing, central differences of the
energy on 50 parameters, fused against unfused sweeps, and the t = 0 identities
of the residuals and pool gradients.  The oracle comparisons at these sizes
are in test_gpu_oracle_large.py.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()

from oracle import fermion, pauli  # noqa: E402
from paper_2108_04413_gb300 import prep, qf  # noqa: E402
from workloads import WORKLOADS, amplitudes, integrals  # noqa: E402


@pytest.fixture(scope="module")
def ucc24():
    cfg = WORKLOADS["ucc24"]
    h, g = integrals(cfg["n_orb"], cfg["seed"])
    T = prep.molecular_hamiltonian(h, g)
    A, exs = prep.uccsd_ansatz(cfg["n_orb"], cfg["n_el"])
    t = amplitudes(len(exs), cfg["seed"], cfg["t_sigma"])
    return cfg, h, g, T, A, exs, t


def _view(st, buf):
    torch.cuda.synchronize()
    st.fold_scale()
    torch.cuda.synchronize()
    return torch.view_as_complex(buf.view(-1, 2))


def test_ucc24_prefix_and_sampled_terms_match_oracle(ucc24):
    cfg, h, g, T, A, exs, t = ucc24
    n, det = cfg["n_qubits"], (1 << cfg["n_el"]) - 1
    k = 2  # first two excitations (a single and a double in determinant order)
    sel = A["param"] < k
    st = qf.State(n, "c128")
    st.set_basis(det)
    st.apply_circuit(prep.bind_thetas(A[sel], t))
    psi = st.to_numpy()
    ref = np.zeros(1 << n, dtype=complex)
    ref[det] = 1.0
    for ex, tm in zip(exs[:k], t[:k]):
        ref = fermion.ucc_factor_apply(ref, n, ex, float(tm))
    assert np.abs(psi - ref).max() < 1e-12
    rng = np.random.default_rng(24)
    pick = rng.choice(len(T), 4, replace=False)
    for i in pick:
        term = T[i:i + 1]
        e, _ = st.expectation(term)
        e_ref = pauli.expectation(ref, n, [(int(term["x"][0]), int(term["z"][0]), float(term["coeff"][0]))])
        assert abs(e - e_ref.real) < 1e-12


def test_ucc24_full_evaluation_properties(ucc24):
    cfg, h, g, T, A, exs, t = ucc24
    n, det = cfg["n_qubits"], (1 << cfg["n_el"]) - 1
    buf = torch.empty(2 << n, dtype=torch.float64, device="cuda")
    st = qf.State(n, "c128", buffer=buf)
    e, grad = st.energy_grad(det, A, t, T)
    # the forward state: unit norm, nothing outside the (6, 6) sector
    st.set_basis(det)
    st.apply_circuit(prep.bind_thetas(A, t))
    v = _view(st, buf)
    assert abs(float((v.abs() ** 2).sum()) - 1.0) < 1e-12
    idx = torch.arange(1 << n, device="cuda", dtype=torch.int64)
    na = torch.zeros_like(idx)
    nb = torch.zeros_like(idx)
    for q in range(0, n, 2):
        na += (idx >> q) & 1
        nb += (idx >> (q + 1)) & 1
    outside = (na != 6) | (nb != 6)
    assert float(v[outside].abs().max()) == 0.0
    e_fwd, im = st.expectation(T)
    assert abs(e_fwd - e) < 1e-10 and im == 0.0
    # the H|psi> arithmetic mode and the complex64 state agree within their tolerances
    s2 = qf.State(n, "c128")
    s2.set_hpsi_mode(qf.QF_HPSI_FP64)
    e2, g2 = s2.energy_grad(det, A, t, T)
    assert abs(e2 - e) < 1e-10 and np.abs(g2 - grad).max() < 1e-10
    s3 = qf.State(n, "c64")
    e3, g3 = s3.energy_grad(det, A, t, T)
    assert abs(e3 - e) < 1e-5 and np.linalg.norm(g3 - grad) / np.linalg.norm(grad) < 1e-4
    # central differences (h = 1e-4) on 50 seeded parameters
    rng = np.random.default_rng(2)
    for p in rng.choice(len(t), 50, replace=False):
        vals = []
        for sgn in (1, -1):
            tt = t.copy()
            tt[p] += sgn * 1e-4
            st.set_basis(det)
            st.apply_circuit(prep.bind_thetas(A, tt))
            vals.append(st.expectation(T)[0])
        fd = (vals[0] - vals[1]) / 2e-4
        assert abs(fd - grad[p]) < 1e-6 * max(1.0, abs(grad[p]))


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 2e-5)])
def test_sweep28_fused_equals_unfused(dtype, tol):
    n = 28
    R = prep.random_circuit(n, 60, 3)
    det = (1 << 14) - 1
    f = torch.float64 if dtype == "c128" else torch.float32
    b1 = torch.empty(2 << n, dtype=f, device="cuda")
    b2 = torch.empty(2 << n, dtype=f, device="cuda")
    s1 = qf.State(n, dtype, buffer=b1)
    s2 = qf.State(n, dtype, buffer=b2)
    s1.set_basis(det)
    s1.apply_circuit(R)
    s2.set_basis(det)
    for r in R:
        s2.apply_pauli_exp(int(r["x"]), int(r["z"]), float(r["theta"]))
    v1 = _view(s1, b1)
    v2 = _view(s2, b2)
    assert float((v1 - v2).abs().max()) < tol
    assert abs(float((v1.abs().double() ** 2).sum()) - 1.0) < (1e-11 if dtype == "c128" else 1e-4)
    Tm = prep.random_hamiltonian(n, 20000, 3)[:64]
    e1, im1 = s1.expectation(Tm)
    e2, _ = s2.expectation(Tm)
    assert im1 == 0.0 and abs(e1 - e2) < (1e-11 if dtype == "c128" else 1e-5)
    s1.close()
    s2.close()


def test_ucc24_residuals_at_reference_are_half_the_gradient(ucc24):
    """At t = 0, dE/dt_mu = <Phi_0|[H, kappa_mu]|Phi_0> = 2 r_mu for every one of
    the 1818 excitations (a property that holds at any size; the oracle pins it
    at small sizes)."""
    cfg, h, g, T, A, exs, t = ucc24
    det = (1 << cfg["n_el"]) - 1
    idx, sgn = prep.excited_determinants(exs, det)
    t0 = np.zeros(len(exs))
    st = qf.State(cfg["n_qubits"], "c128")
    e, r, grad = st.residuals(det, A, t0, T, idx, grad=True)
    assert np.abs(r.imag).max() == 0.0
    assert np.abs(2 * sgn * r.real - grad).max() < 1e-10
    e1, r1 = st.residuals(det, A, t, T, idx)
    assert abs(e1 - st.energy_grad(det, A, t, T)[0]) < 1e-12
    assert np.isfinite(r1).all()


def test_ucc24_pool_gradients_of_the_ansatz_at_reference_equal_the_gradient(ucc24):
    """With the ansatz's own operators as the pool and t = 0 the pool gradients are
    the energy gradient (both are <Phi_0|[H, kappa_mu]|Phi_0>), for all 1818."""
    cfg, h, g, T, A, exs, t = ucc24
    det = (1 << cfg["n_el"]) - 1
    t0 = np.zeros(len(exs))
    st = qf.State(cfg["n_qubits"], "c128")
    e, gp = st.pool_gradients(det, A, t0, T, A, len(exs))
    e2, grad = st.energy_grad(det, A, t0, T)
    assert abs(e - e2) < 1e-12
    assert np.abs(gp - grad).max() < 1e-10
