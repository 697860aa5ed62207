"""GPU vs oracle parity through the C ABI (libqf).

Tolerances (from the accuracy targets of the method's precision options):
complex128 amplitudes 1e-12 max abs, complex128 energies 1e-10 Eh, complex64
energies 1e-5 Eh, complex64 gradients 1e-4 relative (in the 2-norm).
"""
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
from workloads import WORKLOADS, amplitudes, integrals, random_state  # noqa: E402

TOL_AMP_C128 = 1e-12
TOL_E_C128 = 1e-10
TOL_AMP_C64 = 2e-5
TOL_E_C64 = 1e-5
TOL_G_C64 = 1e-4


def _rots_list(R):
    return list(zip(R["x"], R["z"], R["theta"]))


def _terms_list(T):
    return list(zip(T["x"], T["z"], T["coeff"]))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_every_pauli_string_n3(dtype):
    n = 3
    tol = TOL_AMP_C128 if dtype == "c128" else TOL_AMP_C64
    st = qf.State(n, dtype)
    psi0 = random_state(n, 3)
    for x in range(8):
        for z in range(8):
            th = 0.1 + 0.37 * x - 0.21 * z
            st.from_numpy(psi0)
            st.apply_pauli_exp(x, z, th)
            ref = pauli.rotate(psi0, n, x, z, th)
            assert np.abs(st.to_numpy() - ref).max() < tol, (x, z)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_unfused_rotations_random(n, dtype):
    rng = np.random.default_rng(n)
    tol = TOL_AMP_C128 if dtype == "c128" else TOL_AMP_C64 * 4
    st = qf.State(n, dtype)
    psi = random_state(n, 10 + n)
    st.from_numpy(psi)
    for k in range(40):
        x = int(rng.integers(0, 1 << n)) if k % 5 else (1 if k % 10 else 0)
        z = int(rng.integers(0, 1 << n))
        th = float(rng.uniform(-np.pi, np.pi))
        st.apply_pauli_exp(x, z, th)
        psi = pauli.rotate(psi, n, x, z, th)
    assert np.abs(st.to_numpy() - psi).max() < tol


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [6, 13, 16])
def test_circuit_fused_random(n, dtype):
    """Random weight-2..8 exponentials: exercises tile fusion, diagonal and x=1 cases."""
    R = prep.random_circuit(n, 120, seed=n)
    psi0 = np.zeros(1 << n, dtype=complex)
    psi0[(1 << (n // 2)) - 1] = 1
    st = qf.State(n, dtype)
    st.set_basis((1 << (n // 2)) - 1)
    st.apply_circuit(R)
    ref = pauli.apply_rotations(psi0, n, _rots_list(R))
    tol = TOL_AMP_C128 if dtype == "c128" else 1e-4
    assert np.abs(st.to_numpy() - ref).max() < tol


def test_scale_renormalisation_long_circuit():
    """Many large-angle rotations drive the kept scale through the fold-back path."""
    n = 7
    rng = np.random.default_rng(77)
    R = qf.as_rots(rng.integers(0, 128, 3000), rng.integers(0, 128, 3000), rng.uniform(0.6, 0.97, 3000))
    st = qf.State(n, "c128")
    st.set_basis(5)
    st.apply_circuit(R)
    ref = pauli.apply_rotations(pauli.basis_state(n, 5), n, _rots_list(R))
    out = st.to_numpy()
    assert abs(np.linalg.norm(out) - 1) < 1e-12
    assert np.abs(out - ref).max() < 1e-11


def _ucc_problem(name):
    cfg = WORKLOADS[name]
    h, g = integrals(cfg["n_orb"], cfg["seed"])
    T = prep.molecular_hamiltonian(h, g)
    A, exs = prep.uccsd_ansatz(cfg["n_orb"], cfg["n_el"])
    t = amplitudes(len(exs), cfg["seed"], cfg["t_sigma"])
    return cfg, h, g, T, A, exs, t


@pytest.mark.parametrize("workload", ["ucc8", "ucc16"])
def test_ucc_state_and_energy_c128(workload):
    cfg, h, g, T, A, exs, t = _ucc_problem(workload)
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], "c128")
    st.set_basis(det)
    st.apply_circuit(prep.bind_thetas(A, t))
    e, im = st.expectation(T)
    psi = st.to_numpy()
    ref = fermion.ucc_state(cfg["n_orb"], cfg["n_el"], t, exs)
    assert np.abs(psi - ref).max() < TOL_AMP_C128
    e_ref = np.vdot(ref, fermion.hamiltonian_apply(ref, cfg["n_orb"], h, g)).real
    assert abs(e - e_ref) < TOL_E_C128
    assert im == 0.0


@pytest.mark.parametrize("workload", ["ucc8", "ucc16"])
def test_ucc_energy_c64(workload):
    cfg, h, g, T, A, exs, t = _ucc_problem(workload)
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], "c64")
    st.set_basis(det)
    st.apply_circuit(prep.bind_thetas(A, t))
    e, _ = st.expectation(T)
    ref = fermion.ucc_state(cfg["n_orb"], cfg["n_el"], t, exs)
    e_ref = np.vdot(ref, fermion.hamiltonian_apply(ref, cfg["n_orb"], h, g)).real
    assert abs(e - e_ref) < TOL_E_C64


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_ucc_general_sparse_path_unknown_sector(dtype):
    """A determinant loaded from the host has no tracked sector, so the dUCC
    blocks run on the general sparse kernels; same state and energy as the oracle."""
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc16")
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], dtype)
    st.from_numpy(pauli.basis_state(cfg["n_qubits"], det))
    st.apply_circuit(prep.bind_thetas(A, t))
    e, _ = st.expectation(T)
    ref = fermion.ucc_state(cfg["n_orb"], cfg["n_el"], t, exs)
    e_ref = np.vdot(ref, fermion.hamiltonian_apply(ref, cfg["n_orb"], h, g)).real
    if dtype == "c128":
        assert np.abs(st.to_numpy() - ref).max() < TOL_AMP_C128
        assert abs(e - e_ref) < TOL_E_C128
    else:
        assert abs(e - e_ref) < TOL_E_C64


def test_energy_grad_particle_changing_blocks():
    """Pair-creation blocks kappa = a+_a a+_b - h.c. are sparse but change the
    particle number, so they take the general sparse adjoint path."""
    n = 10
    rows = []
    pairs = [(0, 5), (2, 7), (1, 3), (4, 9), (6, 8)]
    for mu, (a, b) in enumerate(pairs):
        k = fermion.jw_product(n, [("+", a), ("+", b)])
        for s_, c in fermion.jw_product(n, [("-", b), ("-", a)]).items():
            k[s_] = k.get(s_, 0) - c
        for s_, c in sorted(k.items()):
            if abs(c) > 1e-14:
                x, z = fermion.letters_to_masks(s_)
                rows.append((x, z, -(c / 1j).real, mu))
    A = qf.as_arots([r[0] for r in rows], [r[1] for r in rows], [r[2] for r in rows], [r[3] for r in rows])
    t = np.array([0.3, -0.2, 0.5, 0.1, -0.4])
    rng = np.random.default_rng(3)
    T = qf.as_terms(rng.integers(0, 1 << n, 80), rng.integers(0, 1 << n, 80), rng.normal(size=80))
    det = 0b0000110011
    st = qf.State(n, "c128")
    e, grad = st.energy_grad(det, A, t, T)
    arots = list(zip(A["x"], A["z"], A["coeff"], A["param"]))
    e_ref, g_ref, _ = pauli.adjoint_gradient(n, det, arots, t, _terms_list(T))
    assert abs(e - e_ref) < TOL_E_C128
    assert np.abs(grad - g_ref).max() < 1e-10


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_expectation_random_terms_mixed(dtype):
    """Duplicated terms, x = 0 terms, odd and even Y counts, many groups."""
    n = 11
    rng = np.random.default_rng(11)
    psi = random_state(n, 5)
    xs = rng.integers(0, 1 << n, 300)
    xs[:40] = 0
    xs[40:60] = xs[60:80]
    zs = rng.integers(0, 1 << n, 300)
    cs = rng.normal(size=300)
    T = qf.as_terms(xs, zs, cs)
    st = qf.State(n, dtype)
    st.from_numpy(psi)
    e, _ = st.expectation(T)
    ref = pauli.expectation(psi, n, _terms_list(T))
    assert abs(ref.imag) < 1e-12
    tol = 1e-11 if dtype == "c128" else 1e-5
    assert abs(e - ref.real) < tol


def test_energy_grad_ucc_c128_matches_oracle_adjoint():
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc8")
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], "c128")
    e, grad = st.energy_grad(det, A, t, T)
    e_ref, g_ref = fermion.ucc_gradient_adjoint(cfg["n_orb"], cfg["n_el"], h, g, t, exs)
    assert abs(e - e_ref) < TOL_E_C128
    assert np.abs(grad - g_ref).max() < 1e-10
    # the sector path leaves exactly the reference determinant (lambda, kept in
    # psi's imaginary slots for a real Hamiltonian, is cleared)
    out = st.to_numpy()
    ref = np.zeros_like(out)
    ref[det] = 1.0
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_energy_grad_repeated_calls_new_angles(dtype):
    """The ansatz structure is planned once per handle; later calls refill the
    composites for new angles.  Each call must match the oracle."""
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc8")
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], dtype)
    for k, tt in enumerate((t, 3 * t[::-1].copy(), amplitudes(len(exs), 99, 0.4))):
        e, grad = st.energy_grad(det, A, tt, T)
        e_ref, g_ref = fermion.ucc_gradient_adjoint(cfg["n_orb"], cfg["n_el"], h, g, tt, exs)
        if dtype == "c128":
            assert abs(e - e_ref) < TOL_E_C128, k
            assert np.abs(grad - g_ref).max() < 1e-10, k
        else:
            assert abs(e - e_ref) < TOL_E_C64, k
            assert np.linalg.norm(grad - g_ref) / np.linalg.norm(g_ref) < TOL_G_C64, k
        out = st.to_numpy()
        assert out[det] == 1.0 and np.count_nonzero(out) == 1, k


@pytest.mark.parametrize("mode", ["fp64", "ds"])
def test_energy_grad_ucc_16q_matches_oracle_both_hpsi_modes(mode):
    """16-qubit dUCCSD energy and full gradient with the H|psi> step in FP64 and
    in double-single arithmetic, against the oracle's fermionic adjoint."""
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc16")
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], "c128")
    st.set_hpsi_mode(qf.QF_HPSI_FP64 if mode == "fp64" else qf.QF_HPSI_DS)
    e, grad = st.energy_grad(det, A, t, T)
    e_ref, g_ref = fermion.ucc_gradient_adjoint(cfg["n_orb"], cfg["n_el"], h, g, t, exs)
    assert abs(e - e_ref) < TOL_E_C128
    assert np.abs(grad - g_ref).max() < 1e-10


def test_energy_grad_ucc_16q_fd():
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc16")
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], "c128")
    e, grad = st.energy_grad(det, A, t, T)
    rng = np.random.default_rng(1)
    params = rng.choice(len(t), 20, replace=False)
    hstep = 1e-4
    for p in params:
        tp = t.copy(); tp[p] += hstep
        tm = t.copy(); tm[p] -= hstep
        st.set_basis(det); st.apply_circuit(prep.bind_thetas(A, tp)); ep, _ = st.expectation(T)
        st.set_basis(det); st.apply_circuit(prep.bind_thetas(A, tm)); em, _ = st.expectation(T)
        fd = (ep - em) / (2 * hstep)
        assert abs(fd - grad[p]) < 1e-6 * max(1.0, abs(grad[p])), (p, fd, grad[p])


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_energy_grad_same_ansatz_across_sectors(dtype):
    """One handle evaluates one dUCC ansatz from determinants in different
    (alpha, beta) sectors and back: the cached part-local run plan of each
    sector must be rebuilt or reused correctly (oracle: plain Pauli adjoint)."""
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc8")
    n = cfg["n_qubits"]
    hf = (1 << cfg["n_el"]) - 1
    # sectors (2, 2); (3, 2) and (1, 2), where the alpha-alpha doubles touch no
    # member (identity blocks); (2, 2) from another determinant; (2, 2) again
    dets = [hf, hf | 0b10000, hf ^ 0b11 ^ 0b1100000, hf ^ 0b1, hf]
    st = qf.State(n, dtype)
    arots = list(zip(A["x"], A["z"], A["coeff"], A["param"]))
    for k, det in enumerate(dets):
        tt = t * (1 + 0.3 * k)
        e, grad = st.energy_grad(det, A, tt, T)
        e_ref, g_ref, _ = pauli.adjoint_gradient(n, det, arots, tt, _terms_list(T))
        if dtype == "c128":
            assert abs(e - e_ref) < TOL_E_C128, k
            assert np.abs(grad - g_ref).max() < 1e-10, k
        else:
            assert abs(e - e_ref) < TOL_E_C64, k
            assert np.linalg.norm(grad - g_ref) <= TOL_G_C64 * max(1.0, np.linalg.norm(g_ref)), k
        out = st.to_numpy()  # the sector path leaves exactly |det>
        assert out[det] == 1.0 and np.count_nonzero(out) == 1, k


def test_energy_grad_generic_ansatz_matches_oracle():
    """Non-commuting rotations sharing parameters: the unfused adjoint path."""
    n = 8
    rng = np.random.default_rng(8)
    m, npar = 40, 9
    A = qf.as_arots(rng.integers(0, 256, m), rng.integers(0, 256, m), rng.normal(size=m), rng.integers(0, npar, m))
    t = rng.normal(size=npar)
    T = qf.as_terms(rng.integers(0, 256, 60), rng.integers(0, 256, 60), rng.normal(size=60))
    det = 0b00110101
    st = qf.State(n, "c128")
    e, grad = st.energy_grad(det, A, t, T)
    arots = list(zip(A["x"], A["z"], A["coeff"], A["param"]))
    e_ref, g_ref, _ = pauli.adjoint_gradient(n, det, arots, t, _terms_list(T))
    assert abs(e - e_ref) < TOL_E_C128
    assert np.abs(grad - g_ref).max() < 1e-10


@pytest.mark.parametrize("n,dtype", [(12, "c128"), (13, "c128"), (12, "c64")])
def test_energy_grad_generic_complex_tiled(n, dtype):
    """Complex state and odd-Y terms at n >= 10: the tiled H|psi> kernel's complex path."""
    rng = np.random.default_rng(n)
    m, npar = 30, 7
    A = qf.as_arots(rng.integers(0, 1 << n, m), rng.integers(0, 1 << n, m), rng.normal(size=m),
                    rng.integers(0, npar, m))
    t = rng.normal(size=npar)
    xs = rng.integers(0, 1 << n, 400)
    xs[:50] = xs[50:100] ^ 1
    xs[100:110] = 0
    T = qf.as_terms(xs, rng.integers(0, 1 << n, 400), rng.normal(size=400) / 20)
    det = (1 << (n // 2)) - 1
    st = qf.State(n, dtype)
    e, grad = st.energy_grad(det, A, t, T)
    arots = list(zip(A["x"], A["z"], A["coeff"], A["param"]))
    e_ref, g_ref, _ = pauli.adjoint_gradient(n, det, arots, t, _terms_list(T))
    if dtype == "c128":
        assert abs(e - e_ref) < TOL_E_C128
        assert np.abs(grad - g_ref).max() < 1e-10
    else:
        assert abs(e - e_ref) < TOL_E_C64
        assert np.linalg.norm(grad - g_ref) / np.linalg.norm(g_ref) < TOL_G_C64


def test_energy_grad_c64_relative():
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc16")
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], "c64")
    e, grad = st.energy_grad(det, A, t, T)
    ref = qf.State(cfg["n_qubits"], "c128")
    e_ref, g_ref = ref.energy_grad(det, A, t, T)
    assert abs(e - e_ref) < TOL_E_C64
    assert np.linalg.norm(grad - g_ref) / np.linalg.norm(g_ref) < TOL_G_C64


def test_invalid_arguments_rejected():
    st = qf.State(4, "c128")
    with pytest.raises(qf.QFError) as ei:
        st.apply_pauli_exp(1 << 4, 0, 0.1)
    assert ei.value.status == qf.QF_EINVAL
    with pytest.raises(qf.QFError):
        st.set_basis(1 << 5)
    with pytest.raises(qf.QFError):
        st.expectation(qf.as_terms([0], [1 << 4], [1.0]))
    A = qf.as_arots([1], [0], [1.0], [3])
    with pytest.raises(qf.QFError):
        st.energy_grad(0, A, np.zeros(2), qf.as_terms([0], [1], [1.0]))
    with pytest.raises(qf.QFError):
        qf.State(0, "c128")
    # the state is unchanged by rejected calls
    st.set_basis(3)
    assert np.abs(st.to_numpy() - pauli.basis_state(4, 3)).max() == 0


def test_empty_inputs():
    st = qf.State(5, "c128")
    st.set_basis(7)
    st.apply_circuit(qf.as_rots([], [], []))
    assert st.expectation(qf.as_terms([], [], []))[0] == 0.0
    e, g = st.energy_grad(7, qf.as_arots([], [], [], []), np.zeros(0), qf.as_terms([0], [0], [2.5]))
    assert abs(e - 2.5) < 1e-15 and len(g) == 0


def test_torch_owned_buffer():
    n = 10
    buf = torch.empty(2 << n, dtype=torch.float64, device="cuda")
    st = qf.State(n, "c128", buffer=buf)
    st.set_basis(3)
    st.apply_pauli_exp(0b1010, 0b0110, 0.3)
    st.fold_scale()
    torch.cuda.synchronize()
    v = torch.view_as_complex(buf.view(-1, 2)).cpu().numpy()
    ref = pauli.rotate(pauli.basis_state(n, 3), n, 0b1010, 0b0110, 0.3)
    assert np.abs(v - ref).max() < 1e-15


def test_bounded_wait_times_out_and_context_survives():
    """A device wait on a word that nothing sets gives up after its limit and the
    host reads QF_ETIMEOUT; the context keeps working afterwards."""
    import time

    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    assert qf.selftest_bounded_wait(stream, 0.25) == qf.QF_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    st = qf.State(6, "c128")
    st.set_basis(3)
    st.apply_pauli_exp(0b101, 0b010, 0.4)
    ref = pauli.rotate(pauli.basis_state(6, 3), 6, 0b101, 0b010, 0.4)
    assert np.abs(st.to_numpy() - ref).max() < 1e-15


@pytest.mark.parametrize("workload,dtype", [("ucc8", "c128"), ("ucc16", "c128"), ("ucc8", "c64"), ("ucc16", "c64")])
def test_pqe_residuals_match_oracle(workload, dtype):
    """PQE residuals r_mu = <Phi_mu|U^dagger H U|Phi_0> (Eq. 23) of every dUCCSD
    excitation, through qf_residuals on the compact sector path, against the
    oracle's fermionic route; the energy and gradient that come along match
    qf_energy_grad."""
    cfg, h, g, T, A, exs, t = _ucc_problem(workload)
    det = (1 << cfg["n_el"]) - 1
    idx, sgn = prep.excited_determinants(exs, det)
    st = qf.State(cfg["n_qubits"], dtype)
    e, r, gr = st.residuals(det, A, t, T, idx, grad=True)
    e_ref, r_ref = fermion.pqe_residuals(cfg["n_orb"], cfg["n_el"], h, g, t, exs)
    tol = TOL_E_C128 if dtype == "c128" else TOL_E_C64
    assert abs(e - e_ref) < tol
    assert np.abs(sgn * r - r_ref).max() < tol
    e2, g2 = st.energy_grad(det, A, t, T)
    assert e2 == e and np.array_equal(g2, gr)
    out = st.to_numpy()  # the sector path leaves exactly |det>
    assert out[det] == 1.0 and np.count_nonzero(out) == 1


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_residuals_general_path_match_oracle(dtype):
    """Determinants outside the reference's sector send qf_residuals down the
    general path (H may connect sectors); a non-commuting generic ansatz always
    takes it.  Every basis index of 8 qubits, against the Pauli oracle."""
    n = 8
    rng = np.random.default_rng(31)
    T = qf.as_terms(rng.integers(0, 256, 50), rng.integers(0, 256, 50), rng.normal(size=50))
    terms = _terms_list(T)
    cfg, h, g, Tu, A, exs, t = _ucc_problem("ucc8")
    det = (1 << cfg["n_el"]) - 1
    dets = np.arange(256, dtype=np.uint64)
    tol = 1e-10 if dtype == "c128" else 1e-5
    st = qf.State(n, dtype)
    for ans, tt in ((A, t), (qf.as_arots(rng.integers(0, 256, 30), rng.integers(0, 256, 30), rng.normal(size=30),
                                          rng.integers(0, 7, 30)), rng.normal(size=7))):
        e, r = st.residuals(det, ans, tt, T, dets)
        arots = list(zip(ans["x"], ans["z"], ans["coeff"], ans["param"]))
        e_ref, r_ref = pauli.residuals(n, det, arots, tt, terms, dets)
        assert abs(e - e_ref) < tol
        assert np.abs(r - r_ref).max() < tol


def test_residuals_invalid_determinant_rejected():
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc8")
    st = qf.State(cfg["n_qubits"], "c128")
    with pytest.raises(qf.QFError):
        st.residuals(15, A, t, T, np.array([1 << cfg["n_qubits"]], dtype=np.uint64))


@pytest.mark.parametrize("dtype,tol,etol", [("c128", 1e-10, 1e-10), ("c64", 1e-5, 5e-5)])
def test_pqe_solve_matches_oracle(dtype, tol, etol):
    """PQE's quasi-Newton iteration (Eq. 26), each step one qf_residuals call,
    reaches the oracle iteration's fixed point (8 qubits, orbitals ordered so
    that the denominators are negative).  complex64 stops at max |r| < 1e-5; its
    energy then carries that convergence error on top of its rounding."""
    from paper_2108_04413_gb300 import pqe

    n_orb, ne = 4, 4
    h, g = integrals(n_orb, 0)
    o = np.argsort(np.diag(h))
    h, g = h[np.ix_(o, o)], g[np.ix_(o, o, o, o)]
    A, exs = prep.uccsd_ansatz(n_orb, ne)
    T = prep.molecular_hamiltonian(h, g)
    det = (1 << ne) - 1
    delta = prep.mp_denominators(exs, prep.orbital_energies(h, g, det))
    st = qf.State(2 * n_orb, dtype)
    res = pqe.solve(st, det, A, exs, T, delta, tol=tol, max_iter=200)
    t_o, e_o, hist_o = fermion.pqe_solve(n_orb, ne, h, g, tol=1e-10)
    assert res.converged and hist_o[-1][1] < 1e-10
    assert abs(res.energy - e_o) < etol
    if dtype == "c128":
        np.testing.assert_allclose(res.t, t_o, rtol=0, atol=1e-8)


@pytest.mark.parametrize("workload,dtype", [("ucc8", "c128"), ("ucc16", "c128"), ("ucc8", "c64"), ("ucc16", "c64")])
def test_pool_gradients_match_oracle(workload, dtype):
    """ADAPT pool gradients (Eq. 21) of every spin-conserving single and double
    excitation at the dUCCSD state: the overlap pass on the compact sector path,
    against the oracle's fermionic commutator route."""
    cfg, h, g, T, A, exs, t = _ucc_problem(workload)
    det = (1 << cfg["n_el"]) - 1
    pool = A.copy()
    pool["param"] = len(exs) - 1 - A["param"]  # operators numbered in reverse
    st = qf.State(cfg["n_qubits"], dtype)
    e, gp = st.pool_gradients(det, A, t, T, pool, len(exs))
    e_ref, g_ref = fermion.adapt_gradients(cfg["n_orb"], cfg["n_el"], h, g, t, exs, exs[::-1])
    if dtype == "c128":
        assert abs(e - e_ref) < TOL_E_C128
        assert np.abs(gp - g_ref).max() < 1e-10
    else:
        assert abs(e - e_ref) < TOL_E_C64
        assert np.linalg.norm(gp - g_ref) <= TOL_G_C64 * np.linalg.norm(g_ref)
    # a second call reuses the pool plan
    e2, gp2 = st.pool_gradients(det, A, 1.5 * t, T, pool, len(exs))
    e_ref2, g_ref2 = fermion.adapt_gradients(cfg["n_orb"], cfg["n_el"], h, g, 1.5 * t, exs, exs[::-1])
    tol = 1e-10 if dtype == "c128" else TOL_G_C64 * np.linalg.norm(g_ref2)
    assert np.abs(gp2 - g_ref2).max() < tol


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_pool_gradients_general_route_match_oracle(dtype):
    """A pool of arbitrary Pauli rotations (not sector blocks) and a Hamiltonian
    with odd-Y terms go through the appended-at-zero route; against the Pauli oracle."""
    n = 8
    rng = np.random.default_rng(41)
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc8")
    det = (1 << cfg["n_el"]) - 1
    pool = qf.as_arots(rng.integers(1, 256, 12), rng.integers(0, 256, 12), rng.normal(size=12), rng.integers(0, 5, 12))
    arots = list(zip(A["x"], A["z"], A["coeff"], A["param"]))
    pr = list(zip(pool["x"], pool["z"], pool["coeff"], pool["param"]))
    Tr = qf.as_terms(rng.integers(0, 256, 40), rng.integers(0, 256, 40), rng.normal(size=40))
    tol = 1e-10 if dtype == "c128" else 1e-5
    st = qf.State(n, dtype)
    for TT in (T, Tr):
        e, gp = st.pool_gradients(det, A, t, TT, pool, 5)
        e_ref, g_ref = pauli.pool_gradients(n, det, arots, t, _terms_list(TT), pr, 5)
        assert abs(e - e_ref) < tol
        assert np.abs(gp - g_ref).max() < (tol if dtype == "c128" else 1e-4 * max(1.0, np.abs(g_ref).max()))


@pytest.mark.parametrize("n,dtype", [(10, "c128"), (13, "c128"), (10, "c64")])
def test_trotter_matches_oracle(n, dtype):
    """Trotterized time evolution (Eq. 39) of a random Pauli Hamiltonian from a
    random state, through qf_trotter, against the oracle's product."""
    rng = np.random.default_rng(100 + n)
    T = qf.as_terms(rng.integers(0, 1 << n, 120), rng.integers(0, 1 << n, 120), rng.normal(size=120) / 5)
    psi0 = random_state(n, n)
    st = qf.State(n, dtype)
    st.from_numpy(psi0.astype(np.complex128 if dtype == "c128" else np.complex64))
    st.trotter(T, 0.8, 3)
    ref = pauli.trotter(psi0, n, _terms_list(T), 0.8, 3)
    tol = TOL_AMP_C128 if dtype == "c128" else TOL_AMP_C64
    assert np.abs(st.to_numpy() - ref).max() < tol


def test_trotter_molecular_hamiltonian_from_reference():
    """The molecular Hamiltonian's evolution of the Hartree-Fock determinant (the
    time-evolved basis states of the quantum Krylov method): against the oracle,
    and the energy is conserved up to the Trotter error."""
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc8")
    n = cfg["n_qubits"]
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(n, "c128")
    st.set_basis(det)
    st.trotter(T, 0.5, 4)
    ref = pauli.trotter(pauli.basis_state(n, det), n, _terms_list(T), 0.5, 4)
    assert np.abs(st.to_numpy() - ref).max() < TOL_AMP_C128
    with pytest.raises(qf.QFError):
        st.trotter(T, 0.5, 0)


def test_pool_gradients_different_pools_across_clear_plans():
    """Two different pools on one handle, with the plans cleared in between: each
    call must use its own pool's descriptors (oracle: fermionic commutators)."""
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc8")
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], "c128")
    doubles = [k for k, ex in enumerate(exs) if len(ex[0]) == 2]
    sub = np.isin(A["param"], doubles)
    pool2 = A[sub].copy()
    remap = {p: k for k, p in enumerate(doubles)}
    pool2["param"] = [remap[int(p)] for p in pool2["param"]]
    for pool, pexs in ((A, exs), (pool2, [exs[k] for k in doubles])):
        _, gp = st.pool_gradients(det, A, t, T, pool, len(pexs))
        _, g_ref = fermion.adapt_gradients(cfg["n_orb"], cfg["n_el"], h, g, t, exs, pexs)
        assert np.abs(gp - g_ref).max() < 1e-10
        st.clear_plans()


def test_plan_caches_evict_and_stay_correct():
    """One handle sees twelve Hamiltonians and twelve ansatz orders (more than the
    eight plans per cache it keeps), then the first pair again: every result
    matches the oracle, and the first pair's result is bit-identical after its
    plans were dropped and rebuilt."""
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc8")
    n, det = cfg["n_qubits"], (1 << cfg["n_el"]) - 1
    rng = np.random.default_rng(77)
    st = qf.State(n, "c128")
    first = None
    for k in range(12):
        Tk = T.copy()
        Tk["coeff"] = T["coeff"] * (1.0 + 0.05 * k)
        order = rng.permutation(len(exs)) if k else np.arange(len(exs))
        Ak = np.concatenate([A[A["param"] == p] for p in order])
        e, grad = st.energy_grad(det, Ak, t, Tk)
        arots = list(zip(Ak["x"], Ak["z"], Ak["coeff"], Ak["param"]))
        e_ref, g_ref, _ = pauli.adjoint_gradient(n, det, arots, t, _terms_list(Tk))
        assert abs(e - e_ref) < TOL_E_C128 and np.abs(grad - g_ref).max() < 1e-10, k
        if k == 0:
            first = (Ak, Tk, e, grad)
    Ak, Tk, e0, g0 = first
    e, grad = st.energy_grad(det, Ak, t, Tk)
    assert e == e0 and np.array_equal(grad, g0)
    st.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_sector_hpsi_chunk_tables_for_non_molecular_terms(dtype):
    """A real Hamiltonian outside the molecular form (here a Z string of weight
    three and a double flip with extra Z letters) keeps the chunk-table sector
    H|psi>; the molecular part alone takes the direct tables.  Both against the
    oracle's adjoint gradient."""
    cfg, h, g, T, A, exs, t = _ucc_problem("ucc8")
    n, det = cfg["n_qubits"], (1 << cfg["n_el"]) - 1
    extra = qf.as_terms(np.array([0, 0b00110011], dtype=np.uint64), np.array([0b10101, 0b10000000], dtype=np.uint64),
                        np.array([0.11, -0.07]))
    arots = list(zip(A["x"], A["z"], A["coeff"], A["param"]))
    st = qf.State(n, dtype)
    for TT in (T, np.concatenate([T, extra])):
        e, grad = st.energy_grad(det, A, t, TT)
        e_ref, g_ref, _ = pauli.adjoint_gradient(n, det, arots, t, _terms_list(TT))
        if dtype == "c128":
            assert abs(e - e_ref) < TOL_E_C128 and np.abs(grad - g_ref).max() < 1e-10
        else:
            assert abs(e - e_ref) < TOL_E_C64
            assert np.linalg.norm(grad - g_ref) <= TOL_G_C64 * np.linalg.norm(g_ref)
    st.close()


def test_fp64_peak_probe():
    """The roofline probe returns the FP64 FMA rate of the CUDA cores within a
    plausible range for this part (2 FMA per clock per SM, nominal 1.26 TFLOP/s
    at 2070 MHz on 152 SMs) and a positive FP64 MMA rate."""
    fma, dmma = qf.probe_fp64_peaks(torch.cuda.current_stream().cuda_stream)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 2 * 2 * 2.1e9
    assert 0.2 * nominal < fma < 1.2 * nominal, (fma, nominal)
    assert dmma > 0.0


def test_sweep_run_items_count_the_sector_pairs():
    """The part-local sweep's per-run item counts (the units its traffic and flops
    are scaled by) add up to the brute-force count of (determinant, excitation)
    pairs: the sector determinants with the excitation's occupied orbitals filled
    and its virtual orbitals empty (Eq. 19's factors act on exactly these)."""
    from oracle import sector

    cfg, h, g, T, A, exs, t = _ucc_problem("ucc16")
    det = (1 << cfg["n_el"]) - 1
    st = qf.State(cfg["n_qubits"], "c128")
    with pytest.raises(qf.QFError):
        st.sweep_run_items()
    st.energy_grad(det, A, t, T)
    items = st.sweep_run_items()
    na, nb = sector.counts_of(det)
    dets = sector.sector_dets(cfg["n_orb"], na, nb)
    expect = 0
    for occ, vir in exs:
        om = sum(1 << q for q in occ)
        vm = sum(1 << q for q in vir)
        expect += int(np.count_nonzero(((dets & np.uint64(om)) == np.uint64(om)) & ((dets & np.uint64(vm)) == 0)))
    assert len(items) >= 1 and (items > 0).all()
    assert int(items.sum()) == expect
    st.close()
