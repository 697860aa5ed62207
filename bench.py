#!/usr/bin/env python
"""Benchmark of the Pauli-exponential state-vector hot path on GB300.

Default workload (one "step" = one energy + full adjoint-gradient evaluation,
every row of the hot path): 24 qubits (12 spatial orbitals, 12 electrons),
seeded synthetic molecular integrals -> Jordan-Wigner Hamiltonian (29737 Pauli
terms in 5479 X-mask groups), dUCCSD ansatz of 1818 excitations (14112 Pauli
exponentials), t ~ N(0, 0.05), complex128.  Each step rewrites the handle's
256 MiB state and streams the 2 GB sweep log, more than the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload ucc24|ucc16|sweep28] [--dtype c128|c64]

Under torchrun each rank evaluates its own copy of the workload (independent
problems, no collective); the value is the evaluations of all ranks divided by
the slowest rank's time.  `--impl reference` times the CPU oracle (the
plain restatement of the paper's definitions that the tests compare against) on
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FP64_FMA_PER_CLK_PER_SM = 2  # GB300 CUDA cores: 2 FP64 FMA per clock per SM (nominal, for context)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ucc24", choices=["ucc24", "ucc16", "sweep28"])
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--no-extras", action="store_true", help="skip the c64 / end-to-end / CPU-baseline legs")
    return ap.parse_args()


_FP64 = {}  # FP64 peaks measured once per process by the library's probe


def peaks():
    """Roofline denominators: HBM and bf16 from MEASURED_PEAKS.json (else the
    fallback figures); FP64 FMA and FP64 MMA measured in this process on this GPU
    (qf_probe_fp64_peaks), with the derived nominal FMA figure for context."""
    p = {"hbm_gbs": 6782.8, "bf16_tflops": 1939.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        p.update({k: m[k] for k in ("hbm_gbs", "bf16_tflops", "sm_max_mhz") if k in m})
        p["source"] = "measured"
    if not _FP64:
        import torch

        from paper_2108_04413_gb300 import qf
        fma, dmma = qf.probe_fp64_peaks(torch.cuda.current_stream().cuda_stream)
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        _FP64.update({"fma_tflops": fma / 1e12, "dmma_tflops": dmma / 1e12, "sms": sms,
                      "nominal_fma_tflops": sms * FP64_FMA_PER_CLK_PER_SM * 2 * p["sm_max_mhz"] * 1e6 / 1e12})
    p["fp64_tflops"] = _FP64["fma_tflops"]
    p["fp64"] = dict(_FP64)
    return p


FP64_NOTE = ("FP64 FMA throughput measured in this run by qf_probe_fp64_peaks (independent FMA chains on every "
             "SM, CUDA events)")


# ----------------------------------------------------------------------------- workloads


def ucc_workload(n_orb: int, n_el: int, seed: int, sigma: float):
    from paper_2108_04413_gb300 import prep
    from workloads import amplitudes, integrals

    h, g = integrals(n_orb, seed)
    terms = prep.molecular_hamiltonian(h, g)
    ansatz, exs = prep.uccsd_ansatz(n_orb, n_el)
    t = amplitudes(len(exs), seed, sigma)
    return dict(n=2 * n_orb, det=(1 << n_el) - 1, terms=terms, ansatz=ansatz, exs=exs, t=t, h=h, g=g,
                n_orb=n_orb, n_el=n_el)


def group_stats(terms, n):
    """Per X-mask group: (terms, chunks of four, has odd-Y terms)."""
    x = terms["x"]
    z = terms["z"]
    y = np.array([bin(int(a) & int(b)).count("1") for a, b in zip(x, z)])
    order = np.argsort(x, kind="stable")
    xs = x[order]
    ys = y[order]
    starts = np.flatnonzero(np.r_[True, xs[1:] != xs[:-1]])
    ends = np.r_[starts[1:], len(xs)]
    out = []
    for s, e in zip(starts, ends):
        cnt = e - s
        out.append((int(cnt), int((cnt + 3) // 4), bool(np.any(ys[s:e] & 1))))
    return out


def sector_pairs(terms, n: int, na: int, nb: int):
    """Connected (sector member c, X group g) pairs of the sector H|psi>: group x
    links c to c ^ x inside the sector iff x flips as many occupied as empty even
    qubits of c, and likewise odd ones.  Counted in closed form per group."""
    from math import comb

    ne, no = (n + 1) // 2, n // 2
    ev = int(sum(1 << q for q in range(0, n, 2)))
    total = 0
    for x in np.unique(terms["x"]):
        x = int(x)
        xe, xo = bin(x & ev).count("1"), bin(x & ~ev).count("1")
        if xe % 2 or xo % 2:
            continue
        total += (comb(xe, xe // 2) * comb(ne - xe, na - xe // 2) * comb(xo, xo // 2) * comb(no - xo, nb - xo // 2))
    return total, comb(ne, na) * comb(no, nb)


def measured_traffic(kernel: str, run_items=None):
    """(DRAM bytes per roofline unit, how they were taken) from the committed ncu summary
    (profiles/traffic.json), or None when the kernel's source changed since the
    capture.  A sweep's record holds the bytes of a few of its run launches and
    their run indices; it is scaled to the whole sweep by the items the runs
    process (run_items, from the library's plan), since the forward log that
    dominates the traffic grows with the items."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["sha256_prefix"]:
        return None
    if "runs" not in rec:
        return rec["bytes"], "one ncu capture of one launch, cold caches"
    if run_items is None or len(run_items) != rec.get("n_runs") or max(rec["runs"]) >= len(run_items):
        return None
    sampled = sum(int(run_items[r]) for r in rec["runs"])
    total = int(sum(int(v) for v in run_items))
    if not sampled or sampled != rec.get("items", sampled):  # the plan's runs changed since the capture
        return None
    return rec["bytes"] * total / sampled, (
        f"ncu DRAM bytes of runs {rec['runs']} ({sampled} items, cold caches) scaled to the sweep's {total} items")


def hpsi_flops(stats, n, real: bool):
    """Algorithmic FP64 flops of one H|psi> over the grouped Pauli sum: one
    multiply-add D_g(b) * psi[b] per (X group, amplitude) -- 2 flops when the
    state and every D are real, 8 when complex -- plus the energy and norm
    accumulations (4 or 8 flops per amplitude)."""
    N = 1 << n
    per = 2 if real else 8
    return N * (per * len(stats) + (4 if real else 8))


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
            os.unlink(self.path)
            return
        # nvidia-smi takes a moment to start: wait (at most 3 s) for its first
        # sample, so that the sampling covers the timed region from its start
        deadline = time.time() + 3.0
        while time.time() < deadline and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [c.strip() for c in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax = float(p[2])
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- distributed


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        backend = "nccl"
        import torch

        if not torch.cuda.is_available():
            backend = "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def aggregate(pg, units_per_rank: float, ms: float):
    """Whole-job throughput: the units all ranks processed divided by the slowest
    rank's time (ms).  Returns (value per second, slowest ms)."""
    ms_max = max_over_ranks(pg, ms)
    world = pg.get_world_size() if pg is not None else 1
    return world * units_per_rank / (ms_max / 1e3), ms_max


def max_over_ranks(pg, v: float) -> float:
    if pg is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- CPU oracle sample


def oracle_sample_ucc(w, budget_s: float = 15.0):
    """Time the oracle on a bounded sample of one energy+gradient evaluation:
    a few rotations and a few Hamiltonian terms on the full state, then scale by
    the counts of one evaluation (forward rotations, reverse rotations on two
    states with one overlap each, and one H|psi> term application per term)."""
    from oracle import pauli

    n = w["n"]
    psi = pauli.basis_state(n, w["det"])
    A = w["ansatz"]
    T = w["terms"]
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    nrot = 0
    while True:
        k = int(rng.integers(0, len(A)))
        psi = pauli.rotate(psi, n, int(A["x"][k]), int(A["z"][k]), 0.01)
        nrot += 1
        if time.perf_counter() - t0 > budget_s / 2 or nrot >= 16:
            break
    t_rot = (time.perf_counter() - t0) / nrot
    t1 = time.perf_counter()
    nterm = 0
    acc = np.zeros_like(psi)
    while True:
        k = int(rng.integers(0, len(T)))
        acc += T["coeff"][k] * pauli.apply(psi, n, int(T["x"][k]), int(T["z"][k]))
        nterm += 1
        if time.perf_counter() - t1 > budget_s / 2 or nterm >= 16:
            break
    t_term = (time.perf_counter() - t1) / nterm
    K = len(A)
    t_eval = t_rot * (K + 2 * K) + t_term * (len(T) + K)
    sample = (f"{nrot} Pauli exponentials and {nterm} Hamiltonian terms of the {n}-qubit workload on the full "
              f"state, scaled to one evaluation ({K} forward + {2 * K} reverse rotations, {K} overlaps, "
              f"{len(T)} terms)")
    return t_eval, sample


# ----------------------------------------------------------------------------- GPU arm


def run_gpu(args, rank, world, local, pg):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2108_04413_gb300 import prep, qf

    torch.cuda.set_device(local)
    pk = peaks()
    if args.workload == "sweep28":
        return run_sweep28(args, rank, world, local, pg, pk)
    cfg = {"ucc24": (12, 12, 2, 0.05), "ucc16": (8, 8, 1, 0.1)}[args.workload]
    w = ucc_workload(*cfg)
    n = w["n"]
    stream = torch.cuda.Stream()
    st = qf.State(n, args.dtype, stream=stream)
    S = 16 if args.dtype == "c128" else 8
    N = 1 << n
    for _ in range(args.warmup):
        st.energy_grad(w["det"], w["ansatz"], w["t"], w["terms"])
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    qf.profile_begin(qf.K_ALL)
    qf.kernel_launches(reset=True)
    barrier(pg)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    energies = []
    for _ in range(args.steps):
        e, g = st.energy_grad(w["det"], w["ansatz"], w["t"], w["terms"])
        energies.append(e)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    ms = e0.elapsed_time(e1)
    launches = qf.kernel_launches(reset=True)
    per_kind = {}
    for kbit, name in qf.KIND_NAMES.items():
        cnt, kms = qf.profile_read(kbit)
        if cnt:
            per_kind[name] = {"launches": cnt, "ms": kms}
    qf.profile_end()
    clk = clocks.stop()
    value, ms_max = aggregate(pg, args.steps, ms)
    step_ms = ms_max / args.steps

    # roofline of the dominant kernel
    dom = max(per_kind.items(), key=lambda kv: kv[1]["ms"])[0]
    stats = group_stats(w["terms"], n)
    roof = roofline_for(dom, per_kind[dom], w, stats, n, S, pk, args.dtype)
    if dom in ("sparse", "adj_sparse"):
        # part-local sector sweeps: every excitation rotates the two active
        # amplitudes of each sector member pair it touches (a real 2x2 rotation,
        # 4 multiply-adds), for psi and, in reverse, lambda, plus the gradient
        # overlap (2 multiply-adds).  The compact sector state is L2-resident, so
        # the bound is the FP64 pipe.
        from math import comb

        ev = int(sum(1 << q for q in range(0, n, 2)))
        na = bin(w["det"] & ev).count("1")
        nb_ = bin(w["det"]).count("1") - na
        ne, no = (n + 1) // 2, n // 2
        items = 0
        for occ, vir in w["exs"]:
            sup = list(occ) + list(vir)
            ea = sum(1 for q in occ if q % 2 == 0)
            eb = len(occ) - ea
            ce = sum(1 for q in sup if q % 2 == 0)
            items += comb(ne - ce, na - ea) * comb(no - (len(sup) - ce), nb_ - eb)
        rev = dom == "adj_sparse"
        # reverse: psi after each block comes back from the forward log, so its work
        # is lambda's rotation and the overlap
        fl = items * (2 * (4 + 2) if rev else 2 * 4)
        avg_s = per_kind[dom]["ms"] / per_kind[dom]["launches"] / 1e3
        roof = {"kernel": "k_sector_run (" + ("reverse" if rev else "forward") + ")", "bound": "alu",
                "achieved": fl / avg_s / 1e12, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
                "frac": fl / avg_s / 1e12 / pk["fp64_tflops"], "traffic": None,
                "algorithmic": (f"{fl:.4g} FP64 flop per sweep: {items} (member pair, excitation) items x "
                                + ("(4 multiply-adds rotating lambda + 2 for the overlap; psi read from the "
                                   "forward log)" if rev else "4 multiply-adds rotating psi") + " x 2 flop"),
                "peak_note": FP64_NOTE,
                "note": "one launch per run of excitations; the compact sector state stays in L2"}
    if dom == "hpsi":
        # the dUCC state stays in one (alpha, beta) sector, where H|psi> runs on members only
        na = bin(w["det"] & int(sum(1 << q for q in range(0, n, 2)))).count("1")
        pairs, members = sector_pairs(w["terms"], n, na, bin(w["det"]).count("1") - na)
        avg_s = per_kind[dom]["ms"] / per_kind[dom]["launches"] / 1e3
        fl = 2 * pairs + 4 * members
        roof = {"kernel": "k_sector_hpsi_direct", "bound": "alu", "achieved": fl / avg_s / 1e12,
                "peak": pk["fp64_tflops"],
                "unit": "TFLOP/s", "frac": fl / avg_s / 1e12 / pk["fp64_tflops"], "traffic": None,
                "algorithmic": (f"{fl:.4g} FP64 flop per launch: one multiply-add per connected (sector member, "
                                f"X group) pair ({pairs} pairs, {members} members)"),
                "peak_note": FP64_NOTE + (("; in the default double-single mode the pair products run on the FP32 "
                                           "pipe, so frac compares with the native-FP64 roofline of the same work")
                                          if args.dtype == "c128" else "")}

    try:
        run_items = st.sweep_run_items()
    except qf.QFError:
        run_items = None
    mt = measured_traffic(roof.get("kernel", ""), run_items)
    roof["traffic"] = mt[0] if mt else None
    if mt:
        roof["traffic_note"] = mt[1]
    out = {
        "metric": "energy+grad evals/s",
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f64 (amplitudes, rotations, reductions; sector H|psi> pair products in double-single, "
                  "about 48-bit, on the FP32 pipe: the library's default QF_HPSI_DS mode; hpsi_fp64_mode times "
                  "FP64 products)" if args.dtype == "c128" else "f32 state, f64 reductions"),
        "data": "synthetic (seeded integrals, dUCCSD amplitudes)",
        "config": {
            "workload": f"{n}-qubit dUCCSD energy + adjoint gradient ({args.workload})",
            "qubits": n, "state": args.dtype, "excitations": len(w["exs"]), "rotations": int(len(w["ansatz"])),
            "pauli_terms": int(len(w["terms"])), "xmask_groups": len(stats),
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": (f"no explicit flush: every step rewrites the {N * S >> 20} MiB state (reset to |det>) and "
                   "streams the 2 GB sweep log, more than the 129 MB L2; the 13.7 MB compact sector state "
                   "is L2-resident within a step"),
        },
        "energy": float(energies[-1]),
        "kernels": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps} for k, v in per_kind.items()},
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clk,
        "fp64_peaks": pk["fp64"],
    }
    if rank == 0 and not args.no_extras:
        out["e2e"] = e2e_leg(st, w, args, stats, stream)
        if args.dtype == "c128":
            out["c64"] = c64_leg(w, args, value, float(energies[-1]), g)
            out["hpsi_fp64_mode"] = fp64_mode_leg(w, args, value, float(energies[-1]), g)
            out["pqe"] = pqe_leg(w, args, value, g)
            out["adapt"] = adapt_leg(w, args, value)
        out["serving"] = serving_leg(args)
        out["sweep28"] = sweep28_leg()
        out["trotter"] = trotter_leg()
        t_eval, sample = oracle_sample_ucc(w)
        out["cpu_baseline"] = {"value": 1.0 / t_eval, "unit": "evals/s", "cores": 1, "kind": "oracle",
                               "sample": sample}
    st.close()
    return out


def roofline_for(kind, rec, w, stats, n, S, pk, dtype):
    N = 1 << n
    avg_s = rec["ms"] / rec["launches"] / 1e3
    if kind in ("hpsi",) and dtype == "c128":
        real = not any(odd for _, _, odd in stats)  # dUCC states are real; H real iff no odd-Y term
        fl = hpsi_flops(stats, n, real)
        ach = fl / avg_s / 1e12
        return {"kernel": "k_hpsi", "bound": "alu", "achieved": ach, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
                "frac": ach / pk["fp64_tflops"], "traffic": None,
                "algorithmic": f"{fl:.4g} FP64-equivalent flop per launch (one multiply-add per X group and amplitude)",
                "peak_note": (FP64_NOTE + "; the default double-single kernel runs these multiply-adds on the FP32 "
                              "pipe, so frac is measured against the native-FP64 roofline of the same work")}
    if kind in ("hpsi",):
        by = (len(stats) + 2) * N * S
        ach = by / avg_s / 1e9
        return {"kernel": "k_hpsi", "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None}
    if kind in ("sparse", "adj_sparse"):
        # each UCC block touches the active rows only: 2 of 16 support patterns (doubles), 2 of 4 (singles)
        frac_rows = sum((2 / 16 if len(e[0]) == 2 else 2 / 4) for e in w["exs"]) / len(w["exs"])
        nst = 2 if kind == "adj_sparse" else 1
        by = 2 * nst * N * S * frac_rows
        ach = by / avg_s / 1e9
        return {"kernel": "k_" + kind, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None}
    by = 2 * N * S
    ach = by / avg_s / 1e9
    return {"kernel": "k_" + kind, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": ach / pk["hbm_gbs"], "traffic": None}


def e2e_leg(st, w, args, stats, stream):
    """Through the public call with host buffers: every step starts from a handle
    with no cached plans, so the call groups and uploads the Hamiltonian, plans
    the ansatz blocks, copies the parameters in and reads energy and gradient
    back.  The byte counts are the library's own transfer counters."""
    import torch

    from paper_2108_04413_gb300 import qf

    steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    qf.transfer_bytes(reset=True)
    t0 = time.perf_counter()
    for _ in range(steps):
        st.clear_plans()
        st.energy_grad(w["det"], w["ansatz"], w["t"], w["terms"])
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    h2d, d2h = qf.transfer_bytes(reset=True)
    # the same call as a VQE loop makes it: plans kept (found again by comparing the
    # term and rotation arrays), new parameters and composites uploaded every step
    st.energy_grad(w["det"], w["ansatz"], w["t"], w["terms"])
    torch.cuda.synchronize()
    qf.transfer_bytes(reset=True)
    wsteps = max(3, args.steps)
    t0 = time.perf_counter()
    for k in range(wsteps):
        st.energy_grad(w["det"], w["ansatz"], w["t"] * (1.0 + 1e-3 * k), w["terms"])
    torch.cuda.synchronize()
    dtw = (time.perf_counter() - t0) / wsteps
    h2dw, d2hw = qf.transfer_bytes(reset=True)
    return {"value": 1.0 / dt, "unit": "evals/s", "h2d_bytes_per_step": h2d // steps,
            "d2h_bytes_per_step": d2h // steps, "steps": steps,
            "note": "cold plans every step (Hamiltonian grouping and tables, ansatz block structure)",
            "warm_plans": {"value": 1.0 / dtw, "unit": "evals/s", "h2d_bytes_per_step": h2dw // wsteps,
                           "d2h_bytes_per_step": d2hw // wsteps, "steps": wsteps,
                           "note": "plans kept across steps, as in a VQE loop; new parameters every step"}}


def serving_systems(qubit_counts=(10, 12, 14, 16, 18, 20, 22)):
    from paper_2108_04413_gb300 import prep
    from paper_2108_04413_gb300.serving import System
    from workloads import integrals

    systems, npar = {}, {}
    for n in qubit_counts:
        no, ne = n // 2, n // 2
        h, g = integrals(no, 100 + n)
        A, exs = prep.uccsd_ansatz(no, ne)
        key = f"n{n}"
        systems[key] = System(key, n, (1 << ne) - 1, A, prep.molecular_hamiltonian(h, g))
        npar[key] = len(exs)
    return systems, npar


def serving_leg(args, count: int = 240, rate: float = 200.0, saturate: int = 960):
    """Poisson stream (seeded, `rate` requests/s) of energy+gradient requests with
    qubit counts uniform in {10,...,22}, t ~ N(0, 0.1), served three ways: the
    complex64 continuous-batching server (8 workers, up to 4 resident handles per
    system, HBM-budget admission), the same with small systems (<= 16 qubits)
    grouped up to 32 requests per qf_energy_grad_multi call (one launch, one CTA
    per request), and one-at-a-time complex128 solves (one worker, one handle per
    system).  Each mode is also driven
    closed-loop -- `saturate` requests of the same mix all queued at once -- for
    its saturated throughput; throughput_multiple compares the best complex64
    mode with one-at-a-time complex128.  A second closed-loop stream of small
    systems only ({10, 12, 14} qubits) isolates the grouped launch."""
    from paper_2108_04413_gb300.serving import GpuExecutor, Request, Server, latency_stats, replay
    from workloads import poisson_arrivals

    systems, npar = serving_systems()
    keys = sorted(systems)
    rng = np.random.default_rng(4)
    arrivals = poisson_arrivals(rate, count, 4)
    picks = rng.integers(0, len(keys), max(count, saturate))
    ts = [rng.normal(0.0, 0.1, npar[keys[k]]) for k in picks]

    def stream(m, timed):
        return [Request(i, keys[picks[i]], ts[i], float(arrivals[i]) if timed else 0.0) for i in range(m)]

    def serve(dtype, workers, batch, reqs_timed, reqs_sat, warm_keys, replicas=1):
        srv = Server(systems, GpuExecutor(dtype), workers=workers, hbm_budget=32 << 30, dtype=dtype,
                     batch=batch, batch_qubits=16, replicas=replicas)
        replay(srv, [Request(-1 - i, k, np.zeros(npar[k]), 0.0) for i, k in enumerate(warm_keys)], realtime=False)
        srv.done.clear()  # warm-up: one request per system plans and allocates its state
        st = {}
        if reqs_timed:
            srv.t0 = srv.clock()
            st = latency_stats(replay(srv, reqs_timed))
            st["max_concurrent"] = srv.max_concurrent
            srv.done.clear()
        srv.t0 = srv.clock()
        sat = latency_stats(replay(srv, reqs_sat, realtime=False))
        st["saturated_throughput_rps"] = sat["throughput_rps"]
        st["saturated_failed"] = sat["failed"]
        st["grouped_calls"] = srv.batches
        srv.close()
        return st

    out = {"requests": count, "arrival_rate_rps": rate, "qubits": "uniform in {10,...,22}",
           "saturated_requests": saturate}
    for label, dtype, workers, batch, replicas in (("continuous_batching_c64", "c64", 8, 1, 4),
                                                   ("grouped_small_c64", "c64", 8, 32, 4),
                                                   ("one_at_a_time_c128", "c128", 1, 1, 1)):
        out[label] = serve(dtype, workers, batch, stream(count, True), stream(saturate, False), keys, replicas)
        out[label]["server"] = {"workers": workers, "replicas": replicas, "group": batch}
    b = out["one_at_a_time_c128"]["saturated_throughput_rps"]
    best = max(out["continuous_batching_c64"]["saturated_throughput_rps"],
               out["grouped_small_c64"]["saturated_throughput_rps"])
    out["throughput_multiple"] = best / b if b else None
    out["throughput_multiple_note"] = ("best complex64 mode over one-at-a-time complex128, saturated (closed-loop) "
                                       "throughputs; at 200 req/s every mode keeps up")
    # small systems only: the grouped launch against one call per request
    small = [k for k in keys if systems[k].n <= 14]
    spick = rng.integers(0, len(small), saturate)
    tsmall = [rng.normal(0.0, 0.1, npar[small[k]]) for k in spick]
    sreqs = lambda: [Request(i, small[spick[i]], tsmall[i], 0.0) for i in range(saturate)]  # noqa: E731
    one = serve("c64", 8, 1, None, sreqs(), small, 4)
    grp = serve("c64", 8, 32, None, sreqs(), small, 4)
    out["small_systems"] = {"qubits": sorted({systems[k].n for k in small}), "requests": saturate,
                            "per_request_calls_rps": one["saturated_throughput_rps"],
                            "grouped_calls_rps": grp["saturated_throughput_rps"],
                            "grouped_calls": grp["grouped_calls"],
                            "grouped_multiple": (grp["saturated_throughput_rps"] / one["saturated_throughput_rps"]
                                                 if one["saturated_throughput_rps"] else None)}
    return out


def sweep28_leg(n: int = 28, n_rot: int = 500, n_terms: int = 20000):
    """28-qubit random Pauli exponentials (weight 2..8, theta ~ U(-pi, pi)):
    fused circuit vs one launch per rotation, complex128 and complex64, and the
    grouped expectation of the 20000-term random Hermitian sum.  Times are the
    library's CUDA-event records of its own kernels.  A fused pass is one launch
    that reads and writes the state once; the expectation reads the state once
    per X group."""
    import torch

    from paper_2108_04413_gb300 import prep, qf

    R = prep.random_circuit(n, n_rot, 3)
    T = prep.random_hamiltonian(n, 20000, 3)[:n_terms]
    groups = len(np.unique(T["x"]))
    N = 1 << n
    det = (1 << 14) - 1
    pk = peaks()
    out = {"qubits": n, "rotations": n_rot, "terms": n_terms, "x_groups": groups}
    sweep_kinds = qf.K_ROT | qf.K_TILE | qf.K_SPARSE
    for dtype in ("c128", "c64"):
        S = 16 if dtype == "c128" else 8
        stream = torch.cuda.Stream()
        st = qf.State(n, dtype, stream=stream)
        res = {}
        for label in ("fused", "unfused"):
            def run():
                st.set_basis(det)
                if label == "fused":
                    st.apply_circuit(R)
                else:
                    for r in R:
                        st.apply_pauli_exp(int(r["x"]), int(r["z"]), float(r["theta"]))
            run()
            torch.cuda.synchronize()
            qf.profile_begin(sweep_kinds)
            run()
            torch.cuda.synchronize()
            passes, ms = qf.profile_read(sweep_kinds)
            qf.profile_end()
            s_ = ms / 1e3
            gbs = passes * 2 * N * S / s_ / 1e9
            res[label] = {"ms": ms, "passes": passes, "rotations_amplitudes_per_s": n_rot * N / s_,
                          "hbm_gbs_per_pass": gbs, "frac_of_measured_hbm": gbs / pk["hbm_gbs"]}
        st.expectation(T)  # plans the groups and tables
        torch.cuda.synchronize()
        qf.profile_begin(qf.K_EXPECT)
        t0 = time.perf_counter()
        e, _ = st.expectation(T)
        wall = time.perf_counter() - t0
        _, ms = qf.profile_read(qf.K_EXPECT)
        qf.profile_end()
        s_ = ms / 1e3
        gbs = groups * N * S / s_ / 1e9
        ex = {"terms": n_terms, "x_groups": groups, "ms": ms, "wall_ms": wall * 1e3, "energy": e,
              "terms_amplitudes_per_s": n_terms * N / s_, "hbm_gbs": gbs, "frac_of_measured_hbm": gbs / pk["hbm_gbs"]}
        if dtype == "c128":
            # FP64 operations per amplitude pair and group (2^(n-1) pairs a group): one term, 2
            # (signed real or imaginary part of conj(u) v); several terms of one Y parity, 3 (that
            # part, then its table weight); both parities, 6
            ops = 0
            ys = np.array([bin(int(a) & int(b)).count("1") & 1 for a, b in zip(T["x"], T["z"])])
            for xv in np.unique(T["x"]):
                sel = T["x"] == xv
                par = set(ys[sel].tolist())
                ops += 2 if sel.sum() == 1 else (6 if len(par) == 2 else 3)
            fl = ops * (N // 2) * 2
            ex["fp64_ops_per_pair_avg"] = ops / groups
            ex["fp64_tflops"] = fl / s_ / 1e12
            ex["frac_of_measured_fp64"] = fl / s_ / 1e12 / pk["fp64_tflops"]
        res["expectation"] = ex
        out[dtype] = res
        st.close()
    return out


def fp64_mode_leg(w, args, value_ds, e_ds, g_ds):
    """The same c128 evaluation with H|psi> in plain FP64 multiply-adds: its
    throughput, and how far the default double-single result is from it."""
    import torch

    from paper_2108_04413_gb300 import qf

    stream = torch.cuda.Stream()
    st = qf.State(w["n"], "c128", stream=stream)
    st.set_hpsi_mode(qf.QF_HPSI_FP64)
    st.energy_grad(w["det"], w["ansatz"], w["t"], w["terms"])
    torch.cuda.synchronize()
    steps = max(2, min(args.steps, 3))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        e, g = st.energy_grad(w["det"], w["ansatz"], w["t"], w["terms"])
    e1.record(stream)
    torch.cuda.synchronize()
    v = steps / (e0.elapsed_time(e1) / 1e3)
    st.close()
    return {"value": v, "unit": "evals/s", "default_speedup": value_ds / v,
            "default_energy_diff": abs(e - e_ds), "default_grad_max_diff": float(np.abs(g - g_ds).max())}



def c64_leg(w, args, value128, e128, g128):
    import torch

    from paper_2108_04413_gb300 import qf

    stream = torch.cuda.Stream()
    st = qf.State(w["n"], "c64", stream=stream)
    for _ in range(2):
        st.energy_grad(w["det"], w["ansatz"], w["t"], w["terms"])
    torch.cuda.synchronize()
    steps = max(2, args.steps)
    qf.profile_begin(qf.K_ALL)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        e, g = st.energy_grad(w["det"], w["ansatz"], w["t"], w["terms"])
    e1.record(stream)
    torch.cuda.synchronize()
    v = steps / (e0.elapsed_time(e1) / 1e3)
    kernels = {}
    for kbit, name in qf.KIND_NAMES.items():
        cnt, kms = qf.profile_read(kbit)
        if cnt:
            kernels[name] = {"launches": cnt, "ms_per_step": kms / steps}
    qf.profile_end()
    st.close()
    return {"value": v, "unit": "evals/s", "speedup_vs_c128": v / value128, "energy_err_vs_c128": abs(e - e128),
            "grad_rel_err_vs_c128": float(np.linalg.norm(g - g128) / np.linalg.norm(g128)), "kernels": kernels}


def pqe_leg(w, args, value128, g128):
    """PQE residuals (Eq. 23) of every excitation with the same pass's energy and
    gradient: qf_residuals on the 24-qubit workload, complex128."""
    import torch

    from paper_2108_04413_gb300 import prep, qf

    idx, sgn = prep.excited_determinants(w["exs"], w["det"])
    stream = torch.cuda.Stream()
    st = qf.State(w["n"], "c128", stream=stream)
    for _ in range(2):
        st.residuals(w["det"], w["ansatz"], w["t"], w["terms"], idx, grad=True)
    torch.cuda.synchronize()
    steps = max(2, args.steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        e, r, g = st.residuals(w["det"], w["ansatz"], w["t"], w["terms"], idx, grad=True)
    e1.record(stream)
    torch.cuda.synchronize()
    v = steps / (e0.elapsed_time(e1) / 1e3)
    st.close()
    rr = sgn * r.real
    return {"value": v, "unit": "residual evals/s (1818 residuals + energy + gradient each)",
            "relative_to_energy_grad": v / value128, "max_abs_residual": float(np.abs(rr).max()),
            "grad_same_as_energy_grad": bool(np.array_equal(g, g128))}


def adapt_leg(w, args, value128):
    """ADAPT pool gradients (Eq. 21) of the full spin-conserving singles-and-doubles
    pool (1818 operators) at the 24-qubit dUCCSD state, complex128."""
    import torch

    from paper_2108_04413_gb300 import qf

    pool = w["ansatz"].copy()
    npool = len(w["exs"])
    stream = torch.cuda.Stream()
    st = qf.State(w["n"], "c128", stream=stream)
    for _ in range(2):
        st.pool_gradients(w["det"], w["ansatz"], w["t"], w["terms"], pool, npool)
    torch.cuda.synchronize()
    steps = max(2, args.steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        e, gp = st.pool_gradients(w["det"], w["ansatz"], w["t"], w["terms"], pool, npool)
    e1.record(stream)
    torch.cuda.synchronize()
    v = steps / (e0.elapsed_time(e1) / 1e3)
    st.close()
    return {"value": v, "unit": f"pool-gradient evals/s ({npool} operators + energy each)",
            "relative_to_energy_grad": v / value128, "max_abs_pool_gradient": float(np.abs(gp).max())}


def trotter_leg():
    """Trotterized time evolution (Eq. 39) of the 24-qubit molecular Hamiltonian
    (29737 terms, one rotation each per step) from the Hartree-Fock determinant,
    complex128, one step: rotations * amplitudes / s and the equivalent HBM rate
    of one read and one write of the state per rotation."""
    import torch

    from paper_2108_04413_gb300 import prep, qf
    from workloads import integrals

    n_orb, n_el = 12, 12
    n = 2 * n_orb
    h, g = integrals(n_orb, 2)
    T = prep.molecular_hamiltonian(h, g)
    stream = torch.cuda.Stream()
    st = qf.State(n, "c128", stream=stream)
    st.set_basis((1 << n_el) - 1)
    st.trotter(T, 0.05, 1)  # warm-up (plans)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st.trotter(T, 0.05, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    norm = float(np.linalg.norm(st.to_numpy()))
    st.close()
    ra = len(T) * (1 << n) / (ms / 1e3)
    return {"qubits": n, "terms": int(len(T)), "steps": 1, "ms_per_step": ms, "rotations_amplitudes_per_s": ra,
            "unfused_equivalent_gbs": ra * 2 * 16 / 1e9, "norm_after": norm}


def run_sweep28(args, rank, world, local, pg, pk):
    """28-qubit random Pauli exponentials (500, weight 2..8, theta ~ U(-pi, pi)):
    fused circuit application, rotations*amplitudes/s."""
    import torch

    from paper_2108_04413_gb300 import prep, qf

    n = 28
    R = prep.random_circuit(n, 500, 3)
    stream = torch.cuda.Stream()
    st = qf.State(n, args.dtype, stream=stream)
    S = 16 if args.dtype == "c128" else 8
    N = 1 << n
    det = (1 << 14) - 1
    for _ in range(args.warmup):
        st.set_basis(det)
        st.apply_circuit(R)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    qf.profile_begin(qf.K_ALL)
    qf.kernel_launches(reset=True)
    barrier(pg)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st.set_basis(det)
        st.apply_circuit(R)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    ms = max_over_ranks(pg, e0.elapsed_time(e1))
    launches = qf.kernel_launches(reset=True)
    per_kind = {}
    for kbit, name in qf.KIND_NAMES.items():
        cnt, kms = qf.profile_read(kbit)
        if cnt:
            per_kind[name] = {"launches": cnt, "ms": kms}
    qf.profile_end()
    clk = clocks.stop()
    value = world * args.steps * len(R) * N / (ms / 1e3)
    dom = max(per_kind.items(), key=lambda kv: kv[1]["ms"])[0]
    rec = per_kind[dom]
    avg_s = rec["ms"] / rec["launches"] / 1e3
    by = 2 * N * S
    roof = {"kernel": "k_" + dom, "bound": "hbm", "achieved": by / avg_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": by / avg_s / 1e9 / pk["hbm_gbs"], "traffic": None}
    out = {"metric": "rotations·amplitudes/s", "value": value, "unit": "rotation·amplitudes/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.dtype == "c128" else "f32",
           "data": "synthetic (seeded random Pauli strings)",
           "config": {"workload": "28-qubit 500 random Pauli exponentials (sweep28)", "qubits": n,
                      "state": args.dtype, "l2": f"state {N * S >> 20} MiB > L2"},
           "kernels": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps} for k, v in
                       per_kind.items()},
           "roofline": roof, "gpu_launches": int(launches), "clocks": clk}
    st.close()
    return out


# ----------------------------------------------------------------------------- reference arm


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cfg = {"ucc24": (12, 12, 2, 0.05), "ucc16": (8, 8, 1, 0.1), "sweep28": None}[args.workload]
    if cfg is None:
        return {"impl": "reference", "unavailable": "the oracle needs hours per 28-qubit step; use ucc24"}
    w = ucc_workload(*cfg)
    times, walls = [], []
    sample = ""
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        t_eval, sample = oracle_sample_ucc(w, budget_s=4.0)
        if i >= args.warmup:
            times.append(t_eval)
            walls.append(time.perf_counter() - t0)
    v = 1.0 / statistics.mean(times)
    return {"impl": "reference", "metric": "energy+grad evals/s", "value": v, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded integrals, dUCCSD amplitudes)",
            "config": {"workload": f"{w['n']}-qubit dUCCSD energy + adjoint gradient ({args.workload})"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": v, "unit": "evals/s"},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_wall_s_per_step": statistics.mean(walls),
            "note": ("each step times a bounded sample of one evaluation (the cpu_baseline sample) and scales it to "
                     "a whole evaluation: ms_per_step is that extrapolated evaluation time, "
                     "sample_wall_s_per_step the wall time a step took")}


def main():
    args = parse_args()
    rank, world, local, pg = dist_setup()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_gpu(args, rank, world, local, pg)
    if rank == 0 and out is not None:
        print(json.dumps(out, default=lambda o: o.item() if hasattr(o, "item") else str(o)))
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
