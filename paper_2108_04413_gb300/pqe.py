"""Projective quantum eigensolver (PQE) on the engine.

PQE drives every residual r_mu(t) = <Phi_mu| U^dagger(t) H U(t) |Phi_0>
(Eq. 23) to zero by the quasi-Newton update of Eq. 26,

    t_mu <- t_mu + r_mu(t) / Delta_mu,

with Delta_mu the Moller-Plesset denominator of excitation mu (`prep.mp_denominators`).
Each iteration is one `qf_residuals` call: the forward sweep, H|psi>, the
reverse sweep and the gather of all residuals run on the GPU; the update of the
n_par amplitudes is host arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import prep


@dataclass
class PQEResult:
    t: np.ndarray                # amplitudes of the last evaluation
    energy: float                # E(t) of the last evaluation
    converged: bool              # every |r_mu| < tol at t
    history: list = field(default_factory=list)  # (E, max |r_mu|) per evaluation


def solve(state, det: int, ansatz: np.ndarray, excitations, terms: np.ndarray, delta, t0=None,
          tol: float = 1e-8, max_iter: int = 100) -> PQEResult:
    """Iterates Eq. 26 from t0 (zeros by default) until max |r_mu| < tol or
    max_iter evaluations.  `ansatz` and `excitations` are `prep.uccsd_ansatz`'s
    rotation list and excitation list (parameter mu of the ansatz is
    excitation mu), `delta` the denominators, `state` a `qf.State`."""
    delta = np.asarray(delta, dtype=np.float64)
    if len(delta) != len(excitations):
        raise ValueError("one denominator per excitation")
    if np.any(delta == 0.0):
        raise ValueError("zero Moller-Plesset denominator")
    idx, sgn = prep.excited_determinants(excitations, det)
    t = np.zeros(len(excitations)) if t0 is None else np.array(t0, dtype=np.float64)
    history = []
    for k in range(max(1, int(max_iter))):
        e, r = state.residuals(det, ansatz, t, terms, idx)
        r_mu = sgn * r.real  # r_mu = sign_mu <index_mu| U^dagger H U |det>
        rmax = float(np.abs(r_mu).max()) if len(r_mu) else 0.0
        history.append((float(e), rmax))
        if rmax < tol or k + 1 == max(1, int(max_iter)):
            return PQEResult(t, float(e), rmax < tol, history)
        t = t + r_mu / delta
