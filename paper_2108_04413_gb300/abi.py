"""NumPy layouts of the C ABI's structs (include/qf.h); no library access."""
from __future__ import annotations

import numpy as np

ROT_DTYPE = np.dtype([("x", "<u8"), ("z", "<u8"), ("theta", "<f8")])            # qf_rot
TERM_DTYPE = np.dtype([("x", "<u8"), ("z", "<u8"), ("coeff", "<f8")])           # qf_term
AROT_DTYPE = np.dtype([("x", "<u8"), ("z", "<u8"), ("coeff", "<f8"),            # qf_arot
                       ("param", "<i4"), ("reserved", "<i4")])


def as_rots(x, z, theta) -> np.ndarray:
    a = np.zeros(len(x), dtype=ROT_DTYPE)
    a["x"], a["z"], a["theta"] = x, z, theta
    return a


def as_terms(x, z, coeff) -> np.ndarray:
    a = np.zeros(len(x), dtype=TERM_DTYPE)
    a["x"], a["z"], a["coeff"] = x, z, coeff
    return a


def as_arots(x, z, coeff, param) -> np.ndarray:
    a = np.zeros(len(x), dtype=AROT_DTYPE)
    a["x"], a["z"], a["coeff"], a["param"] = x, z, coeff, param
    return a
