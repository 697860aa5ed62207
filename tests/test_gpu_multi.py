"""qf_energy_grad_multi: several parameter vectors of one system in one call.
Small sectors run every row in one kernel launch (one CTA per row, the state in
shared memory); each row must give what qf_energy_grad gives for it, and what the
oracle's fermionic adjoint gives.  Larger systems fall back to one
qf_energy_grad per row with the same results."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()

from oracle import fermion  # noqa: E402
from paper_2108_04413_gb300 import prep, qf  # noqa: E402
from workloads import amplitudes, integrals  # noqa: E402

TOL = {"c128": (1e-11, 1e-10), "c64": (2e-5, 1e-4)}  # energy (Eh), gradient (abs for c128, rel for c64)


def _system(n_orb, n_el, seed):
    h, g = integrals(n_orb, seed)
    A, exs = prep.uccsd_ansatz(n_orb, n_el)
    return h, g, A, exs, prep.molecular_hamiltonian(h, g), (1 << n_el) - 1


def _rows(n_par, count, seed):
    return np.stack([amplitudes(n_par, seed + k, 0.15) for k in range(count)])


def _close(dtype, e, g, e_ref, g_ref):
    te, tg = TOL[dtype]
    assert abs(e - e_ref) < te
    if dtype == "c128":
        assert np.abs(g - g_ref).max() < tg
    else:
        assert np.linalg.norm(g - g_ref) <= tg * max(np.linalg.norm(g_ref), 1e-12)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n_orb,n_el", [(4, 4), (5, 5), (7, 7), (8, 8)])
def test_multi_rows_match_single_calls(n_orb, n_el, dtype):
    h, g, A, exs, T, det = _system(n_orb, n_el, 40 + n_orb)
    t = _rows(len(exs), 9, 1000 + n_orb)
    st = qf.State(2 * n_orb, dtype)
    e_m, g_m = st.energy_grad_multi(det, A, t, T)  # first call: row 0 plans through qf_energy_grad
    e_m2, g_m2 = st.energy_grad_multi(det, A, t, T)  # planned: every row in one launch
    ref = qf.State(2 * n_orb, dtype)
    for k in range(len(t)):
        e1, g1 = ref.energy_grad(det, A, t[k], T)
        _close(dtype, e_m[k], g_m[k], e1, g1)
        _close(dtype, e_m2[k], g_m2[k], e1, g1)
    out = st.to_numpy()
    assert out[det] == 1.0 and np.count_nonzero(out) == 1
    st.close()
    ref.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_multi_rows_match_oracle(dtype):
    n_orb, n_el = 4, 4
    h, g, A, exs, T, det = _system(n_orb, n_el, 7)
    t = _rows(len(exs), 3, 77)
    st = qf.State(2 * n_orb, dtype)
    st.energy_grad(det, A, t[0], T)  # plans
    e_m, g_m = st.energy_grad_multi(det, A, t, T)
    for k in range(len(t)):
        e_ref, g_ref = fermion.ucc_gradient_adjoint(n_orb, n_el, h, g, t[k], exs)
        _close(dtype, e_m[k], g_m[k], e_ref, g_ref)
    st.close()


def test_multi_largest_sector_in_shared_memory_is_one_launch():
    """16 qubits at half filling (4900 members, psi and lambda 78 KB in complex128)
    is the largest sector a CTA holds: its rows still take one launch."""
    h, g, A, exs, T, det = _system(8, 8, 21)
    t = _rows(len(exs), 4, 31)
    st = qf.State(16, "c128")
    st.energy_grad_multi(det, A, t[:1], T)
    qf.kernel_launches(reset=True)
    e, gr = st.energy_grad_multi(det, A, t, T)
    assert qf.kernel_launches(reset=True) == 2
    ref = qf.State(16, "c128")
    for k in range(len(t)):
        e1, g1 = ref.energy_grad(det, A, t[k], T)
        _close("c128", e[k], gr[k], e1, g1)
    st.close()
    ref.close()


def test_multi_is_one_launch_for_all_rows():
    """After planning, 32 rows of a 14-qubit system take two kernel launches: the
    evaluation of all rows and the reset of the handle's state to |det>."""
    h, g, A, exs, T, det = _system(7, 7, 3)
    t = _rows(len(exs), 32, 5)
    st = qf.State(14, "c64")
    st.energy_grad_multi(det, A, t[:2], T)
    qf.kernel_launches(reset=True)
    e, gr = st.energy_grad_multi(det, A, t, T)
    assert qf.kernel_launches(reset=True) == 2
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(gr))
    st.close()


def test_multi_falls_back_for_large_sectors():
    """An 18-qubit sector (15876 members) does not fit one CTA's shared memory in
    complex128: the rows run through qf_energy_grad, with the same results."""
    h, g, A, exs, T, det = _system(9, 9, 11)
    t = _rows(len(exs), 3, 9)
    st = qf.State(18, "c128")
    e_m, g_m = st.energy_grad_multi(det, A, t, T)
    ref = qf.State(18, "c128")
    for k in range(len(t)):
        e1, g1 = ref.energy_grad(det, A, t[k], T)
        assert e_m[k] == e1 and np.array_equal(g_m[k], g1)
    st.close()
    ref.close()


def test_multi_rejects_bad_parameters():
    h, g, A, exs, T, det = _system(4, 4, 2)
    st = qf.State(8, "c128")
    t = _rows(len(exs), 3, 1)
    st.energy_grad_multi(det, A, t, T)
    bad = t.copy()
    bad[2, 0] = np.inf
    with pytest.raises(qf.QFError):
        st.energy_grad_multi(det, A, bad, T)
    with pytest.raises(qf.QFError):
        st.energy_grad_multi(det, A, t[:, :-1], T)  # a parameter index past the row length
    e, _ = st.energy_grad_multi(det, A, t, T)  # the handle still works
    assert np.all(np.isfinite(e))
    st.close()
