"""Write the oracle's values for the 24-qubit dUCCSD workload to ucc24_oracle.json.

Calls only the oracle (oracle/sector.py, oracle/fermion.py) and the seeded input
generators (workloads): 12 spatial orbitals, 12 electrons, every spin-conserving
single and double (1818 excitations in ascending excited-determinant order),
integrals of seed 2, amplitudes t ~ N(0, 0.05) of seed 2.  Stored:
* E(t) (Eq. 17-18) and the gradient dE/dt for all 1818 amplitudes (adjoint);
* the ADAPT gradients of the ansatz's own operators at U(t)|Phi_0> (Eq. 21);
* the PQE residuals of all excitations (Eq. 23), fermionic sign included;
* the state U(t)|Phi_0> through its norm, 512 sampled amplitudes (the 256
  largest in magnitude and 256 seeded members) and four seeded random
  projections <v_k|psi> over the 853,776 sector members.
Runs in about 8 minutes and 10 GB of host memory:
    python tests/golden/make_ucc_golden.py
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import fermion, sector  # noqa: E402
from workloads import WORKLOADS, amplitudes, integrals, probe_vectors, sample_indices  # noqa: E402

PROBE_SEED = 2024
SAMPLE_SEED = 2025


def main(out=os.path.join(HERE, "ucc24_oracle.json")):
    cfg = WORKLOADS["ucc24"]
    t0 = time.time()
    h, g = integrals(cfg["n_orb"], cfg["seed"])
    exs = fermion.excitations(cfg["n_orb"], cfg["n_el"])
    t = amplitudes(len(exs), cfg["seed"], cfg["t_sigma"])
    u = sector.UCC(cfg["n_orb"], cfg["n_el"], h, g, exs)
    r = u.evaluate(t)
    res = u.residuals(r["sigma"])
    psi = r["psi"]
    assert np.abs(res.imag).max() < 1e-14 and np.abs(psi.imag).max() == 0.0
    big = np.argsort(-np.abs(psi), kind="stable")[:256]
    pick = np.unique(np.concatenate([big, sample_indices(len(psi), 256, SAMPLE_SEED)]))
    probes = probe_vectors(4, len(psi), PROBE_SEED)
    doc = {
        "_about": "Oracle values (oracle/sector.py) for the 24-qubit dUCCSD workload: 12 spatial orbitals, "
                  "12 electrons, integrals and amplitudes of seed 2 (t ~ N(0, 0.05)), all 1818 "
                  "spin-conserving singles and doubles. Written by make_ucc_golden.py, which calls only "
                  "the oracle and the seeded generators.",
        "n_orb": cfg["n_orb"], "n_el": cfg["n_el"], "seed": cfg["seed"], "t_sigma": cfg["t_sigma"],
        "n_members": int(len(psi)),
        "energy": r["energy"],
        "grad": r["grad"].tolist(),
        "pool": r["pool"].tolist(),
        "residuals": res.real.tolist(),
        "norm2": float(np.vdot(psi, psi).real),
        "sample_dets": [int(d) for d in u.dets[pick]],
        "sample_amps": psi.real[pick].tolist(),
        "probe_seed": PROBE_SEED,
        "probes": (probes @ psi.real).tolist(),
        "seconds": round(time.time() - t0, 1),
    }
    with open(out, "w") as f:
        json.dump(doc, f, indent=0)
    print(f"E = {r['energy']:.15f}  |g| = {np.linalg.norm(r['grad']):.6e}  {doc['seconds']} s -> {out}")


if __name__ == "__main__":
    main()
