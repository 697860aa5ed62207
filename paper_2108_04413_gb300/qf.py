"""ctypes binding of libqf (include/qf.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python / NumPy
/ torch arguments into the C structs and pointers the ABI takes.  Importing it
fails loudly when libqf.so has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqf.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libqf.so is not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = ctypes.CDLL(LIB_PATH)

QF_OK, QF_EINVAL, QF_ENOMEM, QF_ECUDA, QF_ETIMEOUT = range(5)
QF_C128, QF_C64 = 0, 1
QF_HPSI_FP64, QF_HPSI_DS = 0, 1
QF_MAX_QUBITS = 34

from .abi import AROT_DTYPE, ROT_DTYPE, TERM_DTYPE, as_arots, as_rots, as_terms  # noqa: F401

_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_sz = ctypes.c_size_t
_d = ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "qf_state_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "qf_state_destroy": (ctypes.c_int, [_vp]),
    "qf_set_basis": (ctypes.c_int, [_vp, _u64]),
    "qf_apply_pauli_exp": (ctypes.c_int, [_vp, _u64, _u64, _d]),
    "qf_apply_circuit": (ctypes.c_int, [_vp, _vp, _sz]),
    "qf_expectation": (ctypes.c_int, [_vp, _vp, _sz, _dp, _dp]),
    "qf_energy_grad": (ctypes.c_int, [_vp, _u64, _vp, _sz, _vp, _sz, _vp, _sz, _dp, _vp]),
    "qf_energy_grad_multi": (ctypes.c_int, [_vp, _u64, _vp, _sz, _vp, _sz, _sz, _vp, _sz, _vp, _vp]),
    "qf_residuals": (ctypes.c_int, [_vp, _u64, _vp, _sz, _vp, _sz, _vp, _sz, _vp, _sz, _dp, _vp, _vp]),
    "qf_pool_gradients": (ctypes.c_int, [_vp, _u64, _vp, _sz, _vp, _sz, _vp, _sz, _vp, _sz, _sz, _dp, _vp]),
    "qf_trotter": (ctypes.c_int, [_vp, _vp, _sz, _d, ctypes.c_int]),
    "qf_state_copy_to_host": (ctypes.c_int, [_vp, _vp, _sz]),
    "qf_state_copy_from_host": (ctypes.c_int, [_vp, _vp, _sz]),
    "qf_state_fold_scale": (ctypes.c_int, [_vp]),
    "qf_state_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(_vp), _dp]),
    "qf_state_clear_plans": (ctypes.c_int, [_vp]),
    "qf_state_set_hpsi_mode": (ctypes.c_int, [_vp, ctypes.c_int]),
    "qf_kernel_launches": (ctypes.c_uint64, [ctypes.c_int]),
    "qf_transfer_bytes": (None, [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "qf_profile_begin": (ctypes.c_int, [ctypes.c_uint]),
    "qf_profile_read": (ctypes.c_int, [ctypes.c_uint, ctypes.POINTER(ctypes.c_uint64), _dp]),
    "qf_profile_end": (ctypes.c_int, []),
    "qf_sweep_run_items": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64), _sz, ctypes.POINTER(_sz)]),
    "qf_expectation_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _sz, _dp, _dp]),
    "qf_selftest_bounded_wait": (ctypes.c_int, [_vp, ctypes.c_double]),
    "qf_probe_fp64_peaks": (ctypes.c_int, [_vp, _dp, _dp]),
    "qf_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class QFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libqf status {status}: {msg}")
        self.status = status


def _check(status: int) -> None:
    if status != QF_OK:
        raise QFError(status, _lib.qf_last_error().decode(errors="replace"))


def transfer_bytes(reset: bool = False):
    """(host-to-device, device-to-host) bytes copied by this thread's calls."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _lib.qf_transfer_bytes(1 if reset else 0, ctypes.byref(a), ctypes.byref(b))
    return int(a.value), int(b.value)


QF_NOALLOC_MAX_TERMS = 2048


def expectation_noalloc(amplitudes_ptr: int, n: int, dtype: str, stream_ptr: int, terms: np.ndarray):
    """<psi|H|psi> from caller-owned device amplitudes without any device
    allocation (qf_expectation_noalloc); returns (re, im)."""
    terms = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
    re, im = _d(), _d()
    _check(_lib.qf_expectation_noalloc(_vp(amplitudes_ptr), int(n), QF_C128 if dtype == "c128" else QF_C64,
                                       _vp(stream_ptr), _ptr(terms), len(terms), ctypes.byref(re), ctypes.byref(im)))
    return re.value, im.value


def kernel_launches(reset: bool = False) -> int:
    return int(_lib.qf_kernel_launches(1 if reset else 0))


K_SET, K_ROT, K_TILE, K_SPARSE, K_EXPECT, K_HPSI, K_ADJ_ROT, K_ADJ_SPARSE = (1 << i for i in range(8))
K_ALL = 255
KIND_NAMES = {K_SET: "set", K_ROT: "rot", K_TILE: "tile", K_SPARSE: "sparse", K_EXPECT: "expect",
              K_HPSI: "hpsi", K_ADJ_ROT: "adj_rot", K_ADJ_SPARSE: "adj_sparse"}


def selftest_bounded_wait(stream_ptr: int, limit_s: float) -> int:
    """Runs the bounded-wait self-test; returns the status (QF_ETIMEOUT expected)."""
    return int(_lib.qf_selftest_bounded_wait(_vp(stream_ptr), float(limit_s)))


def probe_fp64_peaks(stream_ptr: int):
    """(FP64 FMA flop/s, FP64 MMA flop/s) measured on the current device."""
    a, b = _d(), _d()
    _check(_lib.qf_probe_fp64_peaks(_vp(stream_ptr), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def profile_begin(mask: int = K_ALL) -> None:
    _check(_lib.qf_profile_begin(mask))


def profile_read(mask: int):
    n, ms = ctypes.c_uint64(), _d()
    _check(_lib.qf_profile_read(mask, ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def profile_end() -> None:
    _check(_lib.qf_profile_end())


def _ptr(a: np.ndarray):
    return a.ctypes.data if a is not None and len(a) else None


class State:
    """A device state vector behind a qf_state handle.

    stream: a torch.cuda.Stream (or None for the current torch stream).
    buffer: optional torch tensor (on the GPU) providing the amplitudes' memory.
    """

    def __init__(self, n: int, dtype: str = "c128", stream=None, buffer=None):
        import torch

        self.n = int(n)
        self.dtype = dtype
        self._dt = QF_C128 if dtype == "c128" else QF_C64
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._buffer = buffer
        h = _vp()
        if buffer is not None:
            _check(_lib.qf_state_create(self.n, self._dt, _vp(stream.cuda_stream), _vp(buffer.data_ptr()),
                                        buffer.numel() * buffer.element_size(), ctypes.byref(h)))
        else:
            _check(_lib.qf_state_create(self.n, self._dt, _vp(stream.cuda_stream), None, 0, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def nbytes(self) -> int:
        return (16 if self._dt == QF_C128 else 8) << self.n

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(_lib.qf_state_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_basis(self, det: int):
        _check(_lib.qf_set_basis(self._h, int(det)))

    def apply_pauli_exp(self, x: int, z: int, theta: float):
        _check(_lib.qf_apply_pauli_exp(self._h, int(x), int(z), float(theta)))

    def apply_circuit(self, rots: np.ndarray):
        rots = np.ascontiguousarray(rots, dtype=ROT_DTYPE)
        _check(_lib.qf_apply_circuit(self._h, _ptr(rots), len(rots)))

    def expectation(self, terms: np.ndarray):
        terms = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
        re, im = _d(), _d()
        _check(_lib.qf_expectation(self._h, _ptr(terms), len(terms), ctypes.byref(re), ctypes.byref(im)))
        return re.value, im.value

    def energy_grad(self, det: int, ansatz: np.ndarray, t, terms: np.ndarray):
        ansatz = np.ascontiguousarray(ansatz, dtype=AROT_DTYPE)
        terms = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
        t = np.ascontiguousarray(t, dtype=np.float64)
        grad = np.zeros(len(t), dtype=np.float64)
        e = _d()
        _check(_lib.qf_energy_grad(self._h, int(det), _ptr(ansatz), len(ansatz), _ptr(t), len(t), _ptr(terms),
                                   len(terms), ctypes.byref(e), _ptr(grad)))
        return e.value, grad

    def energy_grad_multi(self, det: int, ansatz: np.ndarray, t, terms: np.ndarray):
        """Energy and gradient for each row of t (n_req x n_par): qf_energy_grad_multi,
        one launch for all rows when the system is small enough."""
        ansatz = np.ascontiguousarray(ansatz, dtype=AROT_DTYPE)
        terms = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
        t = np.ascontiguousarray(np.atleast_2d(t), dtype=np.float64)
        n_req, n_par = t.shape
        energies = np.zeros(n_req, dtype=np.float64)
        grads = np.zeros((n_req, n_par), dtype=np.float64)
        _check(_lib.qf_energy_grad_multi(self._h, int(det), _ptr(ansatz), len(ansatz), _ptr(t), n_par, n_req,
                                         _ptr(terms), len(terms), _ptr(energies), _ptr(grads)))
        return energies, grads

    def residuals(self, det: int, ansatz: np.ndarray, t, terms: np.ndarray, dets, grad: bool = False):
        """PQE residuals <b|U^dagger H U|det> for the basis indices dets (complex
        array), with the energy and, if grad, the gradient."""
        ansatz = np.ascontiguousarray(ansatz, dtype=AROT_DTYPE)
        terms = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
        t = np.ascontiguousarray(t, dtype=np.float64)
        dets = np.ascontiguousarray(dets, dtype=np.uint64)
        res = np.zeros(2 * len(dets), dtype=np.float64)
        g = np.zeros(len(t), dtype=np.float64) if grad else None
        e = _d()
        _check(_lib.qf_residuals(self._h, int(det), _ptr(ansatz), len(ansatz), _ptr(t), len(t), _ptr(terms),
                                 len(terms), _ptr(dets), len(dets), ctypes.byref(e),
                                 _ptr(g) if grad else None, _ptr(res)))
        r = res[0::2] + 1j * res[1::2]
        return (e.value, r, g) if grad else (e.value, r)

    def pool_gradients(self, det: int, ansatz: np.ndarray, t, terms: np.ndarray, pool: np.ndarray, n_pool: int):
        """Gradients of a pool of operators at U(t)|det> (ADAPT, Eq. 21); pool is an
        ansatz-style rotation list whose params index the n_pool operators."""
        ansatz = np.ascontiguousarray(ansatz, dtype=AROT_DTYPE)
        terms = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
        pool = np.ascontiguousarray(pool, dtype=AROT_DTYPE)
        t = np.ascontiguousarray(t, dtype=np.float64)
        g = np.zeros(int(n_pool), dtype=np.float64)
        e = _d()
        _check(_lib.qf_pool_gradients(self._h, int(det), _ptr(ansatz), len(ansatz), _ptr(t), len(t), _ptr(terms),
                                      len(terms), _ptr(pool), len(pool), int(n_pool), ctypes.byref(e), _ptr(g)))
        return e.value, g

    def trotter(self, terms: np.ndarray, time: float, steps: int):
        """Trotterized exp(-i time H) with the given number of steps (Eq. 39)."""
        terms = np.ascontiguousarray(terms, dtype=TERM_DTYPE)
        _check(_lib.qf_trotter(self._h, _ptr(terms), len(terms), float(time), int(steps)))

    def set_hpsi_mode(self, mode: int):
        _check(_lib.qf_state_set_hpsi_mode(self._h, int(mode)))

    def clear_plans(self):
        _check(_lib.qf_state_clear_plans(self._h))

    def sweep_run_items(self) -> np.ndarray:
        """Items of each part-local run of the last sector sweep, in plan order (the
        forward sweep's launch order; the reverse launches them last to first)."""
        n = _sz()
        _check(_lib.qf_sweep_run_items(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, dtype=np.uint64)
        _check(_lib.qf_sweep_run_items(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n.value,
                                       ctypes.byref(n)))
        return out

    def fold_scale(self):
        _check(_lib.qf_state_fold_scale(self._h))

    def info(self):
        n, dt, p, s = ctypes.c_int(), ctypes.c_int(), _vp(), _d()
        _check(_lib.qf_state_info(self._h, ctypes.byref(n), ctypes.byref(dt), ctypes.byref(p), ctypes.byref(s)))
        return n.value, dt.value, p.value, s.value

    def to_numpy(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex128 if self._dt == QF_C128 else np.complex64)
        _check(_lib.qf_state_copy_to_host(self._h, out.ctypes.data, out.nbytes))
        return out

    def from_numpy(self, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.complex128 if self._dt == QF_C128 else np.complex64)
        _check(_lib.qf_state_copy_from_host(self._h, a.ctypes.data, a.nbytes))
