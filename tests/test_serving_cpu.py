"""Serving scheduler logic without a GPU (fake executor): every request
completes, admission never exceeds the HBM budget, idle systems are evicted
least-recently-used first, work overlaps, and results do not depend on the mix."""
import threading
import time

import numpy as np

from paper_2108_04413_gb300.serving import Request, Server, System, footprint_bytes, latency_stats, replay


class FakeExecutor:
    def __init__(self, budget, dtype):
        self.budget = budget
        self.dtype = dtype
        self.used = 0
        self.max_used = 0
        self.active = 0
        self.max_active = 0
        self.lock = threading.Lock()
        self.created = []

    def create(self, sysm):
        with self.lock:
            self.used += footprint_bytes(sysm.n, self.dtype)
            self.max_used = max(self.max_used, self.used)
            self.created.append(sysm.key)
        return {"key": sysm.key, "n": sysm.n}

    def run(self, handle, sysm, t):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
        time.sleep(0.002 * (sysm.n - 6))
        with self.lock:
            self.active -= 1
        e = float(np.sum(np.sin(t)) + sysm.n)
        return e, np.cos(t)

    def release(self, handle):
        with self.lock:
            self.used -= footprint_bytes(handle["n"], self.dtype)


def _systems():
    out = {}
    for n in (8, 10, 12):
        for k in range(2):
            key = f"n{n}-{k}"
            out[key] = System(key, n, (1 << (n // 2)) - 1, np.zeros(0), np.zeros(0))
    return out


def _requests(systems, count, seed):
    rng = np.random.default_rng(seed)
    keys = sorted(systems)
    arr = np.cumsum(rng.exponential(1 / 400.0, count))
    return [Request(i, keys[int(rng.integers(0, len(keys)))], rng.normal(size=5), float(arr[i])) for i in range(count)]


def test_all_complete_and_match_sequential():
    systems = _systems()
    reqs = _requests(systems, 60, 1)
    ex = FakeExecutor(1 << 30, "c64")
    srv = Server(systems, ex, workers=4, hbm_budget=1 << 30)
    done = replay(srv, reqs)
    srv.close()
    assert len(done) == 60 and all(r.error is None for r in done)
    for r in done:
        e, g = FakeExecutor(0, "c64").run(None, systems[r.system], r.t)
        assert r.energy == e and np.array_equal(r.grad, g)
        assert r.done >= r.start >= r.arrival - 1e-9
    assert ex.max_active > 1  # requests overlapped
    st = latency_stats(done)
    assert st["failed"] == 0 and st["p99_ms"] >= st["p50_ms"] > 0


def test_budget_respected_with_eviction():
    systems = _systems()
    reqs = _requests(systems, 50, 2)
    budget = footprint_bytes(12, "c64") + footprint_bytes(10, "c64")  # two systems at most
    ex = FakeExecutor(budget, "c64")
    srv = Server(systems, ex, workers=3, hbm_budget=budget)
    done = replay(srv, reqs, realtime=False)
    srv.close()
    assert len(done) == 50 and all(r.error is None for r in done)
    assert ex.max_used <= budget
    assert srv.evictions > 0
    assert ex.used == 0  # everything released at close


def test_oversized_system_fails_alone():
    systems = _systems()
    reqs = _requests(systems, 10, 3)
    systems["big"] = System("big", 30, 0, np.zeros(0), np.zeros(0))
    reqs.append(Request(99, "big", np.zeros(5), 0.0))
    ex = FakeExecutor(1 << 26, "c64")
    srv = Server(systems, ex, workers=2, hbm_budget=1 << 26)
    done = replay(srv, reqs, realtime=False)
    srv.close()
    big = [r for r in done if r.rid == 99][0]
    assert big.error is not None
    assert sum(r.error is None for r in done) == 10


def test_footprint_counts_sector_log_items_by_brute_force():
    """The sector part of footprint_bytes: 2 * members amplitudes for the compact
    copy, one amplitude pair per (member pair, excitation) for the forward log and
    one map word per pair, plus the run descriptors.  A pair is a sector member
    carrying the excitation's annihilated orbitals on its support; count those
    directly."""
    from paper_2108_04413_gb300 import prep

    n_orb, n_el = 4, 4
    n = 2 * n_orb
    A, exs = prep.uccsd_ansatz(n_orb, n_el)
    det = (1 << n_el) - 1
    even = sum(1 << q for q in range(0, n, 2))
    na, nb = bin(det & even).count("1"), bin(det & ~even).count("1")
    members = [c for c in range(1 << n) if bin(c & even).count("1") == na and bin(c & ~even).count("1") == nb]
    items = 0
    for occ, vir in exs:
        p0 = sum(1 << q for q in occ)
        sup = p0 | sum(1 << q for q in vir)
        items += sum(1 for c in members if c & sup == p0)
    from paper_2108_04413_gb300 import serving

    for dtype, size in (("c128", 16), ("c64", 8)):
        base = footprint_bytes(n, dtype)
        assert base == 2 * (size << n) + serving.FIXED_BYTES
        assert footprint_bytes(n, dtype, n_terms=100) == base + 100 * serving.TABLE_BYTES_PER_TERM
        got = footprint_bytes(n, dtype, det, A) - base
        assert got == (2 * len(members) * size + items * size + items * 4 +
                       len(exs) * serving.RUN_BYTES_PER_EXCITATION)


class BatchingExecutor(FakeExecutor):
    """FakeExecutor with a multi-request call (one call serves a group)."""

    def __init__(self, budget, dtype):
        super().__init__(budget, dtype)
        self.groups = []

    def run_multi(self, handle, sysm, ts):
        with self.lock:
            self.groups.append((sysm.key, len(ts)))
        time.sleep(0.002 * (sysm.n - 6))
        return [(float(np.sum(np.sin(t)) + sysm.n), np.cos(t)) for t in ts]


def test_small_systems_batched_and_results_unchanged():
    """A closed-loop burst: requests of one small system are served together (at
    most `batch` per call); larger systems never are; every result equals the
    one-at-a-time result."""
    systems = _systems()
    systems["n20"] = System("n20", 20, (1 << 10) - 1, np.zeros(0), np.zeros(0))
    reqs = _requests(systems, 80, 4)
    ex = BatchingExecutor(1 << 34, "c64")
    srv = Server(systems, ex, workers=2, hbm_budget=1 << 34, batch=6, batch_qubits=12)
    done = replay(srv, reqs, realtime=False)
    srv.close()
    assert len(done) == 80 and all(r.error is None for r in done)
    for r in done:
        e, g = FakeExecutor(0, "c64").run(None, systems[r.system], r.t)
        assert r.energy == e and np.array_equal(r.grad, g)
    assert srv.batches > 0 and ex.groups
    assert all(2 <= k <= 6 and systems[key].n <= 12 for key, k in ex.groups)
    assert sum(k for _, k in ex.groups) <= 80


def test_no_batching_without_multi_call():
    systems = _systems()
    reqs = _requests(systems, 30, 5)
    ex = FakeExecutor(1 << 30, "c64")
    srv = Server(systems, ex, workers=2, hbm_budget=1 << 30, batch=8)
    done = replay(srv, reqs, realtime=False)
    srv.close()
    assert len(done) == 30 and all(r.error is None for r in done)
    assert srv.batches == 0


def test_replicas_run_one_system_side_by_side():
    """One system, a burst of requests: with three replicas its requests overlap
    on three handles (each charged against the budget), results unchanged; with
    one they run one at a time."""
    systems = {"n12": System("n12", 12, (1 << 6) - 1, np.zeros(0), np.zeros(0))}
    rng = np.random.default_rng(6)
    reqs = [Request(i, "n12", rng.normal(size=5), 0.0) for i in range(24)]
    fp = footprint_bytes(12, "c64")
    for replicas, expect_overlap in ((3, True), (1, False)):
        ex = FakeExecutor(1 << 30, "c64")
        srv = Server(systems, ex, workers=4, hbm_budget=3 * fp, replicas=replicas)
        done = replay(srv, [Request(r.rid, r.system, r.t, 0.0) for r in reqs], realtime=False)
        srv.close()
        assert len(done) == 24 and all(r.error is None for r in done)
        for r in done:
            e, g = FakeExecutor(0, "c64").run(None, systems[r.system], r.t)
            assert r.energy == e and np.array_equal(r.grad, g)
        assert (ex.max_active > 1) == expect_overlap
        assert len(ex.created) == replicas and ex.max_used <= 3 * fp and ex.used == 0
