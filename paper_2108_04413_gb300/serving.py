"""Continuous-batching server for energy + gradient requests.

Requests (system, parameters) arrive over time.  A dispatcher admits them as
worker slots free up and as device memory allows: every system keeps its state
resident (psi, lambda or the sector path's compact copy and forward log, plus its
cached plans; see footprint_bytes) so repeated-parameter requests skip all
planning, and admission charges each resident handle's footprint against an HBM
budget, evicting idle handles (least recently used first) when a new one does
not fit.  A system may hold up to `replicas` handles, so requests of one busy
system can run side by side; one handle is never used by two threads at once.
Admitted requests run on worker threads, each call on its handle's own CUDA
stream; libqf calls release the GIL, so the device work of several requests
overlaps.

Small systems are also batched: when a worker takes a request for a system of
at most `batch_qubits` qubits, it takes up to `batch` - 1 more pending requests
for the same system and runs them all in one qf_energy_grad_multi call (one
kernel launch, one CTA per request, each request's sector state in shared
memory).  Latency = completion time - arrival time; the server reports
throughput and p50/p99 latency.  The executor is pluggable so the scheduling
logic can be tested without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class System:
    key: str
    n: int
    det: int
    ansatz: np.ndarray
    terms: np.ndarray


@dataclasses.dataclass
class Request:
    rid: int
    system: str
    t: np.ndarray
    arrival: float  # seconds on the server clock
    start: float = 0.0
    done: float = 0.0
    energy: float = 0.0
    grad: Optional[np.ndarray] = None
    error: Optional[str] = None


def _popc(v: int) -> int:
    return bin(v).count("1")


# Per-handle device memory beyond the amplitudes (upper bounds of what the
# library allocates): work buffers, Pauli-sum plan tables per term, sweep
# descriptors per excitation, and the limits of the forward log and item maps.
FIXED_BYTES = 128 << 10
TABLE_BYTES_PER_TERM = 512
RUN_BYTES_PER_EXCITATION = 1536
LOG_MAX_BYTES = 16 << 30
MAP_MAX_BYTES = 1 << 30


def footprint_bytes(n: int, dtype: str, det: Optional[int] = None, ansatz: Optional[np.ndarray] = None,
                    n_terms: int = 0) -> int:
    """Device bytes a resident system holds, an upper bound: psi and lambda
    (2 * 2^n amplitudes), the handle's work buffers and its Pauli-sum plan tables
    (n_terms terms).  Given the determinant and the ansatz, also the sector
    path's compact copy (2 * members amplitudes), its forward log (one amplitude
    pair per (member pair, excitation) item, at most 16 GB), its item maps (at
    most one 4-byte word per item, at most 1 GB) and its run descriptors: an
    excitation whose flips cover sa alpha and sb beta spin orbitals, half of each
    occupied, moves C(ne - sa, na - sa/2) * C(no - sb, nb - sb/2) items."""
    from math import comb

    size = 16 if dtype == "c128" else 8
    total = 2 * (size << n) + FIXED_BYTES + TABLE_BYTES_PER_TERM * int(n_terms)
    if det is None or ansatz is None or len(ansatz) == 0:
        return total
    ne, no = (n + 1) // 2, n // 2
    even = sum(1 << q for q in range(0, n, 2))
    na, nb = _popc(det & even), _popc(det & ~even)
    members = comb(ne, na) * comb(no, nb)
    flips = {}
    for x, p in zip(ansatz["x"].tolist(), ansatz["param"].tolist()):
        flips.setdefault(int(p), int(x))
    items = 0
    for x in flips.values():
        sa, sb = _popc(x & even), _popc(x & ~even)
        ka, kb = na - sa // 2, nb - sb // 2
        if 0 <= ka <= ne - sa and 0 <= kb <= no - sb:
            items += comb(ne - sa, ka) * comb(no - sb, kb)
    return (total + 2 * members * size + min(items * size, LOG_MAX_BYTES) + min(items * 4, MAP_MAX_BYTES) +
            RUN_BYTES_PER_EXCITATION * len(flips))


class GpuExecutor:
    """Runs qf_energy_grad on resident libqf states, one CUDA stream per state."""

    def __init__(self, dtype: str = "c64", device: int = 0):
        import torch

        from . import qf

        self.qf = qf
        self.torch = torch
        self.dtype = dtype
        self.device = device

    def create(self, sysm: System):
        self.torch.cuda.set_device(self.device)
        stream = self.torch.cuda.Stream()
        return self.qf.State(sysm.n, self.dtype, stream=stream)

    def run(self, handle, sysm: System, t: np.ndarray):
        self.torch.cuda.set_device(self.device)
        return handle.energy_grad(sysm.det, sysm.ansatz, t, sysm.terms)

    def run_multi(self, handle, sysm: System, ts: List[np.ndarray]):
        """Several requests of one system in one qf_energy_grad_multi call."""
        self.torch.cuda.set_device(self.device)
        e, g = handle.energy_grad_multi(sysm.det, sysm.ansatz, np.stack(ts), sysm.terms)
        return [(float(e[k]), g[k]) for k in range(len(ts))]

    def release(self, handle):
        handle.close()


class Server:
    def __init__(self, systems: Dict[str, System], executor, workers: int = 4, hbm_budget: int = 8 << 30,
                 dtype: str = "c64", clock: Callable[[], float] = time.perf_counter, batch: int = 1,
                 batch_qubits: int = 16, replicas: int = 1):
        self.systems = systems
        self.ex = executor
        self.batch = batch if hasattr(executor, "run_multi") else 1
        self.batch_qubits = batch_qubits
        self.batches = 0  # calls that served more than one request
        # resident handles a system may hold at once (each charged its footprint):
        # requests of one busy system run side by side on different handles
        self.replicas = max(1, replicas)
        self.workers = workers
        self.budget = hbm_budget
        self.dtype = dtype
        self.clock = clock
        self._lock = threading.Condition()
        self._pending: collections.deque = collections.deque()
        # (system, slot) -> handle, least recently used first; busy or idle
        self._resident: "collections.OrderedDict[tuple, object]" = collections.OrderedDict()
        self._busy: Dict[tuple, bool] = {}
        self._slots: Dict[str, int] = {}  # handles of each system (resident or being created)
        self._next_slot = 0
        self._used = 0
        self._active = 0
        self._closed = False
        self.done: List[Request] = []
        self.evictions = 0
        self.max_concurrent = 0
        self._fp: Dict[str, int] = {}
        self._threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(workers)]
        self.t0 = self.clock()
        for th in self._threads:
            th.start()

    def now(self) -> float:
        return self.clock() - self.t0

    def _footprint(self, key: str) -> int:
        """Device bytes charged for a resident handle of a system (cached per system)."""
        fp = self._fp.get(key)
        if fp is None:
            sysm = self.systems[key]
            fp = self._fp[key] = footprint_bytes(sysm.n, self.dtype, sysm.det, sysm.ansatz, len(sysm.terms))
        return fp

    # -- submission
    def submit(self, req: Request):
        with self._lock:
            self._pending.append(req)
            self._lock.notify_all()

    def close(self):
        with self._lock:
            self._closed = True
            self._lock.notify_all()
        for th in self._threads:
            th.join()
        for h in list(self._resident.values()):
            self.ex.release(h)
        self._resident.clear()

    # -- admission (called with the lock held): the first pending request that has
    # an idle resident handle of its system, or room for a new one (within the
    # system's replica count and, after evicting idle handles least recently used
    # first, the HBM budget)
    def _admit(self):
        for i, req in enumerate(self._pending):
            key = req.system
            idle = next((rk for rk in self._resident if rk[0] == key and not self._busy.get(rk)), None)
            if idle is not None:
                del self._pending[i]
                self._resident.move_to_end(idle)
                return self._group(req), self._resident[idle], False, idle
            if self._slots.get(key, 0) >= self.replicas:
                continue  # wait for one of its handles
            need = self._footprint(key)
            if need > self.budget:
                del self._pending[i]
                req.error = "system does not fit the HBM budget"
                req.done = self.now()
                self.done.append(req)
                return None
            victims = []
            free = self.budget - self._used
            for rk in self._resident:  # least recently used first
                if free >= need:
                    break
                if not self._busy.get(rk):
                    victims.append(rk)
                    free += self._footprint(rk[0])
            if free < need:
                continue  # wait for a busy handle to finish
            for rk in victims:
                h = self._resident.pop(rk)
                self._busy.pop(rk, None)
                self._slots[rk[0]] -= 1
                self._used -= self._footprint(rk[0])
                self.evictions += 1
                self.ex.release(h)
            del self._pending[i]
            self._used += need
            self._slots[key] = self._slots.get(key, 0) + 1
            rk = (key, self._next_slot)
            self._next_slot += 1
            return self._group(req), None, True, rk
        return None

    def _group(self, req: Request) -> List[Request]:
        """req and, for a small system, up to batch - 1 more pending requests of
        the same system (earliest first), taken off the queue (lock held)."""
        group = [req]
        if self.batch > 1 and self.systems[req.system].n <= self.batch_qubits:
            rest = collections.deque()
            while self._pending:
                r = self._pending.popleft()
                if r.system == req.system and len(group) < self.batch:
                    group.append(r)
                else:
                    rest.append(r)
            self._pending = rest
        return group

    def _worker(self):
        while True:
            with self._lock:
                while True:
                    got = self._admit() if self._pending else None
                    if got is not None:
                        break
                    if self._closed and not self._pending:
                        return
                    self._lock.wait(timeout=0.05)
                group, handle, fresh, rk = got
                key = rk[0]
                self._busy[rk] = True
                self._active += 1
                self.max_concurrent = max(self.max_concurrent, self._active)
                if len(group) > 1:
                    self.batches += 1
            sysm = self.systems[key]
            try:
                if fresh:
                    handle = self.ex.create(sysm)
                t0 = self.now()
                for req in group:
                    req.start = t0
                if len(group) > 1:
                    results = self.ex.run_multi(handle, sysm, [req.t for req in group])
                else:
                    results = [self.ex.run(handle, sysm, group[0].t)]
                for req, (e, g) in zip(group, results):
                    req.energy, req.grad = float(e), np.asarray(g)
            except Exception as exc:  # the requests fail, the server keeps going
                for req in group:
                    req.error = repr(exc)
            t1 = self.now()
            for req in group:
                req.done = t1
            with self._lock:
                if fresh and handle is not None:
                    self._resident[rk] = handle
                    self._resident.move_to_end(rk)
                elif fresh:  # the handle was never created
                    self._used -= self._footprint(key)
                    self._slots[key] -= 1
                self._busy[rk] = False
                self._active -= 1
                self.done.extend(group)
                self._lock.notify_all()


def replay(server: Server, requests: List[Request], realtime: bool = True) -> List[Request]:
    """Submit requests at their arrival times (server clock), wait for all."""
    for req in sorted(requests, key=lambda r: r.arrival):
        if realtime:
            delay = req.arrival - server.now()
            if delay > 0:
                time.sleep(delay)
        server.submit(req)
    while True:
        with server._lock:
            if len(server.done) >= len(requests):
                break
        time.sleep(0.002)
    return server.done


def latency_stats(done: List[Request]) -> dict:
    ok = [r for r in done if r.error is None]
    lat = np.array([r.done - r.arrival for r in ok])
    span = max(r.done for r in ok) - min(r.arrival for r in ok) if ok else 0.0
    return {"requests": len(done), "failed": len(done) - len(ok),
            "throughput_rps": len(ok) / span if span > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None}
