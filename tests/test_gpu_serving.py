"""Serving on the GPU: each energy+gradient result is the same when the request
runs alone and when it runs in a concurrent mix of systems of different sizes
(complex64 state, FP64 reductions; tolerance 1e-5 Eh and 1e-4 relative).  Also
the torch.autograd.Function wrapper."""
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
from paper_2108_04413_gb300.autograd import energy  # noqa: E402
from paper_2108_04413_gb300.serving import GpuExecutor, Request, Server, System, latency_stats, replay  # noqa: E402
from workloads import amplitudes, integrals  # noqa: E402


def _system(n, seed):
    no, ne = n // 2, n // 2
    h, g = integrals(no, seed)
    A, exs = prep.uccsd_ansatz(no, ne)
    return System(f"n{n}s{seed}", n, (1 << ne) - 1, A, prep.molecular_hamiltonian(h, g)), len(exs)


def test_results_same_alone_and_in_mix():
    systems, npar = {}, {}
    for n, seed in ((8, 0), (10, 1), (12, 2), (12, 3)):
        s, k = _system(n, seed)
        systems[s.key] = s
        npar[s.key] = k
    rng = np.random.default_rng(5)
    keys = sorted(systems)
    reqs = []
    for i in range(24):
        key = keys[i % len(keys)]
        reqs.append(Request(i, key, rng.normal(0, 0.1, npar[key]), 0.0))
    alone = {}
    for r in reqs:
        st = qf.State(systems[r.system].n, "c64")
        alone[r.rid] = st.energy_grad(systems[r.system].det, systems[r.system].ansatz, r.t, systems[r.system].terms)
        st.close()
    srv = Server(systems, GpuExecutor("c64"), workers=4, hbm_budget=1 << 30, dtype="c64")
    done = replay(srv, reqs, realtime=False)
    srv.close()
    assert len(done) == len(reqs) and all(r.error is None for r in done)
    assert srv.max_concurrent > 1
    for r in done:
        e, g = alone[r.rid]
        assert abs(r.energy - e) < 1e-5
        assert np.linalg.norm(r.grad - g) <= 1e-4 * max(np.linalg.norm(g), 1e-12)
    st = latency_stats(done)
    assert st["failed"] == 0


def test_autograd_energy_matches_oracle():
    no, ne = 4, 4
    h, g = integrals(no, 0)
    A, exs = prep.uccsd_ansatz(no, ne)
    T = prep.molecular_hamiltonian(h, g)
    t0 = amplitudes(len(exs), 0, 0.1)
    st = qf.State(2 * no, "c128")
    t = torch.tensor(t0, dtype=torch.float64, requires_grad=True)
    e = energy(t, st, (1 << ne) - 1, A, T)
    (2.0 * e).backward()
    e_ref, g_ref = fermion.ucc_gradient_adjoint(no, ne, h, g, t0, exs)
    assert abs(e.item() - e_ref) < 1e-10
    assert np.abs(t.grad.numpy() - 2.0 * g_ref).max() < 1e-10
