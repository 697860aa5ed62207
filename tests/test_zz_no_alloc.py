"""qf_expectation_noalloc: the allocation-free expectation entry point.

It serves callers that cannot allocate device memory (their GPU memory is
reserved by another allocator, or they must avoid cudaMalloc's implicit
synchronisation); it keeps its scratch in a static device array instead.  Here
it is called through the C ABI on amplitudes that a torch tensor owns and
compared with qf_expectation (which allocates through its state handle) and
with the oracle's term-by-term expectation, on two calls in a row with
different Hamiltonians, so a stale scratch would show.  The device's free
memory must not change across a call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()

from oracle import pauli  # noqa: E402
from paper_2108_04413_gb300 import qf  # noqa: E402
from workloads import random_state  # noqa: E402


def _terms(n, count, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 1 << n, count)
    x[: count // 8] = 0
    return qf.as_terms(x, rng.integers(0, 1 << n, count), rng.normal(size=count))


@pytest.mark.parametrize("dtype,tol,otol", [("c128", 1e-11, 1e-10), ("c64", 1e-11, 1e-5)])
def test_noalloc_matches_expectation_twice(dtype, tol, otol):
    n = 14
    psi = random_state(n, 21)
    # the oracle sees the amplitudes the GPU holds (complex64 rounding included)
    held = psi.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi
    buf = torch.empty(2 << n, dtype=torch.float64 if dtype == "c128" else torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    st = qf.State(n, dtype, stream=stream, buffer=buf)
    st.from_numpy(psi)
    for call, (count, seed) in enumerate(((600, 1), (2048, 2))):
        T = _terms(n, count, seed)
        ref, _ = st.expectation(T)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        got, im = qf.expectation_noalloc(buf.data_ptr(), n, dtype, stream.cuda_stream, T)
        assert torch.cuda.mem_get_info()[0] == free0, "the call changed the device's free memory"
        assert im == 0.0
        assert abs(got - ref) < tol * max(1.0, abs(ref)), (call, got, ref)
        e_or = pauli.expectation(held, n, list(zip(T["x"], T["z"], T["coeff"])))
        assert abs(got - e_or.real) < otol, (call, got, e_or)
    st.close()


def test_noalloc_rejects_too_many_terms():
    n = 10
    buf = torch.zeros(2 << n, dtype=torch.float64, device="cuda")
    T = _terms(n, qf.QF_NOALLOC_MAX_TERMS + 1, 3)
    with pytest.raises(qf.QFError) as ei:
        qf.expectation_noalloc(buf.data_ptr(), n, "c128", torch.cuda.current_stream().cuda_stream, T)
    assert ei.value.status == qf.QF_EINVAL
    assert "QF_NOALLOC_MAX_TERMS" in str(ei.value)
