"""ctypes wrapper around the plain-C index-loop oracle (qd_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, smoke() and the CPU-baseline legs of
bench.py.  The C file applies one gate per call in FP64; gate matrices come
from :mod:`oracle.qudit_oracle`, so both oracle modes share the gate
definitions and nothing else.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import qudit_oracle as qo

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qd_oracle.c")
_LIB = os.path.join(_HERE, "libqd_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile qd_oracle.c with gcc (OpenMP) into oracle/libqd_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        dp = ctypes.POINTER(ctypes.c_double)
        L.qo_apply.argtypes = [dp, ctypes.c_int32, i32p, dp, ctypes.c_int32, i32p,
                               ctypes.c_int32, i32p, i32p, ctypes.c_int32]
        L.qo_apply.restype = ctypes.c_int
        L.qo_norm2.argtypes = [dp, ctypes.c_int64]
        L.qo_norm2.restype = ctypes.c_double
        L.qo_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _i32(xs):
    a = np.ascontiguousarray(np.array(list(xs) if len(xs) else [0], dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def apply(psi: np.ndarray, dims, gate, nthreads: int = 0) -> None:
    """Apply one gate record to ``psi`` (complex128, C-contiguous) in place."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    g = np.ascontiguousarray(qo.target_matrix(gate, dims), dtype=np.complex128)
    ctrls, lv = qo._levels(gate, dims)
    d_a, d_p = _i32(dims)
    t_a, t_p = _i32(list(gate.targets))
    c_a, c_p = _i32(ctrls)
    l_a, l_p = _i32(lv)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().qo_apply(psi.ctypes.data_as(dp), len(dims), d_p, g.ctypes.data_as(dp),
                        len(gate.targets), t_p, len(ctrls), c_p, l_p, int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the gate")


def run_circuit(dims, gates, init_levels=None, nthreads: int = 0, psi0=None) -> np.ndarray:
    """Gates in order; a "MEASURE" record ends the circuit (Sec. 3.4: gates
    after the Measurement Gate are ignored)."""
    psi = qo.basis_state(dims, init_levels) if psi0 is None else np.array(psi0, dtype=np.complex128)
    for g in gates:
        if getattr(g, "kind", None) == "MEASURE":
            break
        apply(psi, dims, g, nthreads)
    return psi


def max_threads() -> int:
    return int(lib().qo_max_threads())
