"""ctypes binding of libqudit (include/qudit.h).

Argument marshalling only: every call goes straight to the C ABI of the CUDA
library, under the same name; failures raise :class:`QuditError` with the
library's message.  There is no other implementation behind these names: if
libqudit.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from .build import LIB_PATH

# ---- constants mirrored from include/qudit.h ----------------------------
QD_OK = 0
QD_C64, QD_C128 = 1, 2
QD_HOST, QD_DEVICE = 0, 1
QD_GATE_X, QD_GATE_Z, QD_GATE_H, QD_GATE_U, QD_GATE_DIAG, QD_GATE_MEASURE = 1, 2, 3, 4, 5, 6
QD_OUT_AMPLITUDE, QD_OUT_PROBABILITY = 0, 1
QD_PLAN_NONE, QD_PLAN_GREEDY, QD_PLAN_LEARNED, QD_PLAN_EXHAUSTIVE = 0, 1, 2, 3
QD_MAX_TARGETS, QD_MAX_CONTROLS = 6, 8
QD_TUNE_TILE_STRIDE, QD_TUNE_FUSE_KMAX, QD_TUNE_FUSE_DMAX, QD_TUNE_TC_MIN_D, QD_TUNE_INDEX64 = 1, 2, 3, 4, 5
# kernel forms of one launch (launch feature 10)
QD_FORM_MONO, QD_FORM_DENSE, QD_FORM_BLOCK, QD_FORM_BLOCK_TC, QD_FORM_DIAG_RUN, QD_FORM_DENSE_RUN = range(6)
QD_MODEL_FEATURES, QD_MODEL_PARAMS = 12, 9217
QD_BATCH_TILE_AMPS, QD_BATCH_CTAS_PER_SM, QD_BATCH_SMALL_AMPS, QD_BATCH_GROUP_AMPS = 1, 2, 3, 4
QD_BATCH_TILES_PER_ITEM, QD_BATCH_POLL_LIMIT = 5, 6
ERRORS = {-1: "QD_ERR_ARG", -2: "QD_ERR_DIM", -3: "QD_ERR_OVERLAP", -4: "QD_ERR_OOM", -5: "QD_ERR_CUDA",
          -6: "QD_ERR_TIMEOUT", -7: "QD_ERR_DEVICE", -8: "QD_ERR_UNSUPPORTED"}

_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p


class QdGate(ctypes.Structure):
    _fields_ = [("kind", _i32), ("k", _i32), ("targets", _i32 * QD_MAX_TARGETS), ("nc", _i32),
                ("controls", _i32 * QD_MAX_CONTROLS), ("ctrl_levels", _i32 * QD_MAX_CONTROLS),
                ("param", _i32), ("reserved", _i32), ("matrix", _dp)]


class QuditError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None

# (name, argtypes) for every exported call; restype is int unless noted
_SIGS = {
    "qd_create": [_i32p, _i32, _i32p, _i32, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)],
    "qd_destroy": [_vp],
    "qd_reset": [_vp, _i32p],
    "qd_info": [_vp, _i64p, _i32p, ctypes.POINTER(_vp), _i32p],
    "qd_set_stream": [_vp, _vp],
    "qd_set_tuning": [_vp, _i32, _i64],
    "qd_apply": [_vp, _dp, _i32p, _i32, _i32p, _i32p, _i32],
    "qd_apply_diag": [_vp, _dp, _i32p, _i32, _i32p, _i32p, _i32],
    "qd_apply_x": [_vp, _i32, _i32],
    "qd_apply_z": [_vp, _i32, _i32],
    "qd_apply_h": [_vp, _i32],
    "qd_apply_cx": [_vp, _i32, _i32, _i32, _i32],
    "qd_apply_mct": [_vp, _i32p, _i32p, _i32, _i32, _i32],
    "qd_apply_gate": [_vp, ctypes.POINTER(QdGate)],
    "qd_plan_create": [_vp, ctypes.POINTER(QdGate), _i32, _i32, ctypes.POINTER(_vp)],
    "qd_plan_run": [_vp],
    "qd_plan_info": [_vp, _i32p, _i32p],
    "qd_plan_destroy": [_vp],
    "qd_plan_profile": [_vp, _i32],
    "qd_plan_timings": [_vp, ctypes.POINTER(ctypes.c_float), _dp, _i32p],
    "qd_run_circuit": [_vp, ctypes.POINTER(QdGate), _i32, _i32],
    "qd_norm": [_vp, _dp],
    "qd_probabilities": [_vp, _dp, _i32],
    "qd_marginal": [_vp, _i32, _dp],
    "qd_overlap": [_vp, _vp, _dp, _dp],
    "qd_cdf": [_vp, _dp, _i32],
    "qd_sample": [_vp, ctypes.c_uint64, _i64, _i64p],
    "qd_sample_u": [_vp, _dp, _i64, _i64p],
    "qd_get_amplitudes": [_vp, _vp, _i32],
    "qd_set_amplitudes": [_vp, _vp, _i32],
    "qd_sync": [_vp, _i32p],
    "qd_cdf_noalloc": [_vp, _i64, _i32, _dp, _vp],
    "qd_model_create": [ctypes.POINTER(_vp)],
    "qd_model_destroy": [_vp],
    "qd_model_set": [_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                     ctypes.POINTER(ctypes.c_float), ctypes.c_float, ctypes.c_float],
    "qd_model_get": [_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                     ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
    "qd_model_train": [_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _i32, _i32, _i32,
                       ctypes.c_float, ctypes.c_uint64, _dp],
    "qd_model_predict": [_vp, ctypes.POINTER(ctypes.c_float), _i32, ctypes.POINTER(ctypes.c_float)],
    "qd_model_forward_raw": [_vp, ctypes.POINTER(ctypes.c_float), _i32, ctypes.POINTER(ctypes.c_float), _i32],
    "qd_model_grad_raw": [_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _i32, _dp,
                          ctypes.POINTER(ctypes.c_float)],
    "qd_set_cost_model": [_vp, _vp],
    "qd_segment_features": [_vp, ctypes.POINTER(QdGate), _i32, _i32, _i32, ctypes.POINTER(ctypes.c_float)],
    "qd_plan_create_segmented": [_vp, ctypes.POINTER(QdGate), _i32, _i32p, _i32p, _i32, ctypes.POINTER(_vp)],
    "qd_plan_create_forms": [_vp, ctypes.POINTER(QdGate), _i32, _i32p, _i32p, _i32p, _i32, ctypes.POINTER(_vp)],
    "qd_segment_forms": [_vp, ctypes.POINTER(QdGate), _i32, _i32, _i32, _i32p, ctypes.POINTER(ctypes.c_float), _i32, _i32p],
    "qd_batch_create": [_i32, _i32p, _i32p, _vp, ctypes.POINTER(_vp)],
    "qd_batch_set_circuit": [_vp, _i32, ctypes.POINTER(QdGate), _i32],
    "qd_batch_tune": [_vp, _i32, _i64],
    "qd_batch_run": [_vp],
    "qd_batch_probabilities": [_vp, _i32, _dp],
    "qd_batch_get_amplitudes": [_vp, _i32, _vp],
    "qd_batch_info": [_vp, _i64p, _i32p, _i32p, _i32p],
    "qd_batch_profile": [_vp, _i32],
    "qd_batch_timings": [_vp, ctypes.POINTER(ctypes.c_float), _dp],
    "qd_batch_autotune": [_vp, _i32, _i64p, ctypes.POINTER(ctypes.c_float)],
    "qd_batch_destroy": [_vp],
    "qd_batch_sync": [_vp, _i32p],
    "qd_measure_all": [_vp],
    "qd_is_measured": [_vp, _i32p],
    "qd_toffoli_gates": [_i32p, _i32, _i32, _i32, _i32, _i32, ctypes.POINTER(QdGate)],
    "qd_apply_toffoli": [_vp, _i32, _i32, _i32, _i32],
    "qd_mct_tree_gates": [_i32p, _i32, _i32p, _i32p, _i32, _i32, _i32, ctypes.POINTER(QdGate), _i32, _i32p, _i32p],
    "qd_apply_mct_tree": [_vp, _i32p, _i32p, _i32, _i32, _i32],
    "qd_ket_list": [_vp, _i32, ctypes.c_double, _i64, _i64p, _dp, _i64p],
    "qd_ket_label": [_i32p, _i32, _i64, ctypes.c_char_p, _i32],
    "qd_qasm_parse": [ctypes.c_char_p, _i32p, _i32, _i32p, ctypes.POINTER(QdGate), _i32, _i32p, _i32p],
    "qd_run_moments": [_vp, ctypes.POINTER(QdGate), _i32, _i32p],
    "qd_moment_packing": [_i32p, _i32, ctypes.POINTER(QdGate), _i32, _i32p, _i32p],
}


def exported_names() -> list[str]:
    return list(_SIGS) + ["qd_strerror", "qd_last_error"]


def load(path: Optional[str] = None):
    """Load libqudit.so (raises if it is not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise QuditError(-5, f"libqudit.so is not built at {p}; run __graft_entry__.build()")
    L = ctypes.CDLL(p)
    for name, args in _SIGS.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.qd_strerror.argtypes = [ctypes.c_int]
    L.qd_strerror.restype = ctypes.c_char_p
    L.qd_last_error.argtypes = []
    L.qd_last_error.restype = ctypes.c_char_p
    if path is None:
        _lib = L
    return L


def _check(rc: int):
    if rc != QD_OK:
        raise QuditError(rc, load().qd_last_error().decode(errors="replace"))


def _arr_i32(xs):
    a = np.ascontiguousarray(np.asarray(list(xs), dtype=np.int32))
    return a, (a.ctypes.data_as(_i32p) if a.size else None)


def _cplx(m) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(m, dtype=np.complex128))


# ---- register ------------------------------------------------------------

def qd_create(dims: Sequence[int], init_levels: Optional[Sequence[int]] = None, precision: int = QD_C64,
              dev_buf: int = 0, dev_buf_bytes: int = 0, stream: int = 0) -> int:
    d, dp = _arr_i32(dims)
    lv, lp = _arr_i32(init_levels) if init_levels is not None else (None, None)
    out = _vp()
    _check(load().qd_create(dp, len(d), lp, precision, _vp(dev_buf or None), dev_buf_bytes, _vp(stream or None),
                            ctypes.byref(out)))
    return out.value


def qd_destroy(reg: int) -> None:
    _check(load().qd_destroy(_vp(reg)))


def qd_reset(reg: int, init_levels: Optional[Sequence[int]] = None) -> None:
    lv, lp = _arr_i32(init_levels) if init_levels is not None else (None, None)
    _check(load().qd_reset(_vp(reg), lp))


def qd_info(reg: int) -> dict:
    N, n, st, pr = _i64(), _i32(), _vp(), _i32()
    _check(load().qd_info(_vp(reg), ctypes.byref(N), ctypes.byref(n), ctypes.byref(st), ctypes.byref(pr)))
    return {"N": N.value, "n": n.value, "state": st.value, "precision": pr.value}


def qd_set_stream(reg: int, stream: int) -> None:
    _check(load().qd_set_stream(_vp(reg), _vp(stream or None)))


def qd_set_tuning(reg: int, key: int, value: int) -> None:
    _check(load().qd_set_tuning(_vp(reg), key, value))


# ---- gates ------------------------------------------------------------------

def qd_apply(reg: int, matrix, targets, controls=(), ctrl_levels=None) -> None:
    m = _cplx(matrix)
    t, tp = _arr_i32(targets)
    c, cp = _arr_i32(controls)
    lv, lp = _arr_i32(ctrl_levels) if ctrl_levels is not None else (None, None)
    _check(load().qd_apply(_vp(reg), m.ctypes.data_as(_dp), tp, len(t), cp, lp, len(c)))


def qd_apply_diag(reg: int, diag, targets, controls=(), ctrl_levels=None) -> None:
    m = _cplx(diag)
    t, tp = _arr_i32(targets)
    c, cp = _arr_i32(controls)
    lv, lp = _arr_i32(ctrl_levels) if ctrl_levels is not None else (None, None)
    _check(load().qd_apply_diag(_vp(reg), m.ctypes.data_as(_dp), tp, len(t), cp, lp, len(c)))


def qd_apply_x(reg: int, t: int, shift: int = 1) -> None:
    _check(load().qd_apply_x(_vp(reg), t, shift))


def qd_apply_z(reg: int, t: int, power: int = 1) -> None:
    _check(load().qd_apply_z(_vp(reg), t, power))


def qd_apply_h(reg: int, t: int) -> None:
    _check(load().qd_apply_h(_vp(reg), t))


def qd_apply_cx(reg: int, c: int, t: int, shift: int = 1, ctrl_level: int = -1) -> None:
    _check(load().qd_apply_cx(_vp(reg), c, t, shift, ctrl_level))


def qd_apply_mct(reg: int, controls, t: int, shift: int = 1, ctrl_levels=None) -> None:
    c, cp = _arr_i32(controls)
    lv, lp = _arr_i32(ctrl_levels) if ctrl_levels is not None else (None, None)
    _check(load().qd_apply_mct(_vp(reg), cp, lp, len(c), t, shift))


_KIND = {"X": QD_GATE_X, "Z": QD_GATE_Z, "H": QD_GATE_H, "U": QD_GATE_U, "DIAG": QD_GATE_DIAG,
         "MEASURE": QD_GATE_MEASURE}
_KIND_NAME = {v: k for k, v in _KIND.items()}


class GateArray:
    """A C array of qd_gate built from gate records (objects with ``kind``,
    ``targets``, ``controls``, ``levels``, ``param``, ``matrix``); it keeps
    the matrix buffers alive while the array is in use."""

    def __init__(self, gates):
        self.n = len(gates)
        self.arr = (QdGate * max(1, self.n))()
        self._keep = []
        for i, g in enumerate(gates):
            s = self.arr[i]
            s.kind = _KIND[g.kind]
            s.k = len(g.targets)
            for j, t in enumerate(g.targets):
                s.targets[j] = int(t)
            ctrls = tuple(g.controls or ())
            s.nc = len(ctrls)
            lv = g.levels if g.levels is not None else [-1] * len(ctrls)
            for j, (c, l) in enumerate(zip(ctrls, lv)):
                s.controls[j] = int(c)
                s.ctrl_levels[j] = -1 if l is None else int(l)
            s.param = int(g.param or 0)
            if g.matrix is not None:
                m = _cplx(g.matrix)
                self._keep.append(m)
                s.matrix = m.ctypes.data_as(_dp)
            else:
                s.matrix = None
        self.ptr = ctypes.cast(self.arr, ctypes.POINTER(QdGate))

    def matrix_bytes(self) -> int:
        return int(sum(m.nbytes for m in self._keep))


def qd_apply_gate(reg: int, gate) -> None:
    ga = GateArray([gate])
    _check(load().qd_apply_gate(_vp(reg), ga.ptr))


def qd_plan_create(reg: int, gates, plan_kind: int = QD_PLAN_NONE) -> int:
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    out = _vp()
    _check(load().qd_plan_create(_vp(reg), ga.ptr, ga.n, plan_kind, ctypes.byref(out)))
    return out.value


def qd_plan_run(plan: int) -> None:
    _check(load().qd_plan_run(_vp(plan)))


def qd_plan_info(plan: int) -> dict:
    la, bl = _i32(), _i32()
    _check(load().qd_plan_info(_vp(plan), ctypes.byref(la), ctypes.byref(bl)))
    return {"launches": la.value, "blocks": bl.value}


def qd_plan_profile(plan: int, enable: bool = True) -> None:
    _check(load().qd_plan_profile(_vp(plan), 1 if enable else 0))


KCLASS_NAMES = {0: "dense_direct", 1: "dense_tile", 2: "mono_direct", 3: "mono_tile", 4: "tensor_block",
                5: "diag_table", 6: "dense_table"}


def qd_plan_timings(plan: int, with_times: bool = True):
    """(ms[launches] or None, alg_bytes[launches], kclass[launches])."""
    n = qd_plan_info(plan)["launches"]
    ms = np.zeros(max(n, 1), dtype=np.float32)
    ab = np.zeros(max(n, 1), dtype=np.float64)
    kc = np.zeros(max(n, 1), dtype=np.int32)
    _check(load().qd_plan_timings(_vp(plan), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if with_times else None,
                                  ab.ctypes.data_as(_dp), kc.ctypes.data_as(_i32p)))
    return (ms[:n] if with_times else None), ab[:n], kc[:n]


def kclass_name(c: int) -> str:
    return f"{KCLASS_NAMES[c & 0xff]}_D{c >> 8}"


def qd_plan_destroy(plan: int) -> None:
    _check(load().qd_plan_destroy(_vp(plan)))


def qd_run_circuit(reg: int, gates, plan_kind: int = QD_PLAN_NONE) -> None:
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    _check(load().qd_run_circuit(_vp(reg), ga.ptr, ga.n, plan_kind))


# ---- readout -----------------------------------------------------------------

def qd_norm(reg: int) -> float:
    out = ctypes.c_double()
    _check(load().qd_norm(_vp(reg), ctypes.byref(out)))
    return out.value


def _n(reg):
    return qd_info(reg)["N"]


def qd_probabilities(reg: int, out: Optional[np.ndarray] = None, where: int = QD_HOST, dev_ptr: int = 0):
    if where == QD_DEVICE:
        _check(load().qd_probabilities(_vp(reg), ctypes.cast(_vp(dev_ptr), _dp), QD_DEVICE))
        return None
    if out is None:
        out = np.empty(_n(reg), dtype=np.float64)
    _check(load().qd_probabilities(_vp(reg), out.ctypes.data_as(_dp), QD_HOST))
    return out


def qd_overlap(a: int, b: int) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(load().qd_overlap(_vp(a), _vp(b), ctypes.byref(re), ctypes.byref(im)))
    return complex(re.value, im.value)


def qd_marginal(reg: int, q: int, d: int) -> np.ndarray:
    out = np.empty(d, dtype=np.float64)
    _check(load().qd_marginal(_vp(reg), q, out.ctypes.data_as(_dp)))
    return out


def qd_cdf(reg: int, out: Optional[np.ndarray] = None, where: int = QD_HOST, dev_ptr: int = 0):
    if where == QD_DEVICE:
        _check(load().qd_cdf(_vp(reg), ctypes.cast(_vp(dev_ptr), _dp), QD_DEVICE))
        return None
    if out is None:
        out = np.empty(_n(reg), dtype=np.float64)
    _check(load().qd_cdf(_vp(reg), out.ctypes.data_as(_dp), QD_HOST))
    return out


def qd_sample(reg: int, seed: int, shots: int) -> np.ndarray:
    out = np.empty(shots, dtype=np.int64)
    _check(load().qd_sample(_vp(reg), ctypes.c_uint64(seed), shots, out.ctypes.data_as(_i64p)))
    return out


def qd_sample_u(reg: int, u) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    out = np.empty(len(u), dtype=np.int64)
    _check(load().qd_sample_u(_vp(reg), u.ctypes.data_as(_dp), len(u), out.ctypes.data_as(_i64p)))
    return out


def qd_cdf_noalloc(state_ptr: int, n_amplitudes: int, precision: int, cdf_out_ptr: int, stream: int = 0) -> None:
    """Prefix sums into a caller-provided device buffer; allocates nothing."""
    _check(load().qd_cdf_noalloc(_vp(state_ptr), n_amplitudes, precision, ctypes.cast(_vp(cdf_out_ptr), _dp),
                                 _vp(stream or None)))


def qd_get_amplitudes(reg: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    info = qd_info(reg)
    dt = np.complex64 if info["precision"] == QD_C64 else np.complex128
    if out is None:
        out = np.empty(info["N"], dtype=dt)
    assert out.dtype == dt and out.size == info["N"] and out.flags.c_contiguous
    _check(load().qd_get_amplitudes(_vp(reg), _vp(out.ctypes.data), QD_HOST))
    return out


def qd_set_amplitudes(reg: int, src, where: int = QD_HOST) -> None:
    if where == QD_DEVICE:
        _check(load().qd_set_amplitudes(_vp(reg), _vp(int(src)), QD_DEVICE))
        return
    info = qd_info(reg)
    dt = np.complex64 if info["precision"] == QD_C64 else np.complex128
    a = np.ascontiguousarray(np.asarray(src, dtype=dt))
    assert a.size == info["N"]
    _check(load().qd_set_amplitudes(_vp(reg), _vp(a.ctypes.data), QD_HOST))


def qd_sync(reg: int) -> int:
    err = _i32()
    rc = load().qd_sync(_vp(reg), ctypes.byref(err))
    _check(rc)
    return err.value


def qd_strerror(code: int) -> str:
    return load().qd_strerror(code).decode()


def qd_last_error() -> str:
    return load().qd_last_error().decode(errors="replace")


class Register:
    """Owns one qd_reg handle (convenience wrapper, marshalling only)."""

    def __init__(self, dims, init_levels=None, precision=QD_C64, dev_buf=0, dev_buf_bytes=0, stream=0,
                 tile_stride=None):
        self.dims = [int(d) for d in dims]
        self.precision = precision
        self.h = qd_create(self.dims, init_levels, precision, dev_buf, dev_buf_bytes, stream)
        if tile_stride is not None:
            qd_set_tuning(self.h, QD_TUNE_TILE_STRIDE, tile_stride)

    def close(self):
        if self.h:
            qd_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, gates, plan_kind=QD_PLAN_NONE):
        qd_run_circuit(self.h, gates, plan_kind)

    def amplitudes(self):
        return qd_get_amplitudes(self.h)


# ---- host-only planner inspection (include/qudit_debug.h) ------------------

def qd_debug_gate_members(dims: Sequence[int], gate, cap: int = 1 << 20, tile_stride: int = -1):
    """Replay the planned kernel's index arithmetic on the host.

    Returns (members[groups, D] int64, info dict); see include/qudit_debug.h."""
    L = load()
    fn = L.qd_debug_gate_members_tuned
    fn.argtypes = [_i32p, _i32, ctypes.POINTER(QdGate), _i64, _i64p, _i64, _i64p]
    fn.restype = ctypes.c_int
    d, dp = _arr_i32(dims)
    ga = GateArray([gate])
    out = np.zeros(cap, dtype=np.int64)
    info = np.zeros(7, dtype=np.int64)
    _check(fn(dp, len(d), ga.ptr, tile_stride, out.ctypes.data_as(_i64p), cap, info.ctypes.data_as(_i64p)))
    keys = ["mode", "D", "groups", "kind", "active", "B", "noop"]
    inf = {k: int(v) for k, v in zip(keys, info)}
    if inf["noop"]:
        return np.zeros((0, 0), dtype=np.int64), inf
    n = inf["groups"] * inf["D"]
    assert n <= cap
    return out[:n].reshape(inf["groups"], inf["D"]), inf


def qd_debug_gate_members_tuned(dims: Sequence[int], gate, tile_stride: int, cap: int = 1 << 20):
    return qd_debug_gate_members(dims, gate, cap, tile_stride)


def qd_debug_batch_emulate(circuits, tile_amps: int = -1, small_amps: int = -1, group_amps: int = -1,
                           tiles_per_item: int = -1):
    """Host replay of a batched run (see include/qudit_debug.h): returns the
    final FP64 states (one array per circuit) and the info dict."""
    L = load()
    fn = L.qd_debug_batch_emulate
    fn.argtypes = [_i32, _i32p, _i32p, ctypes.POINTER(QdGate), _i32p, _i64p, _dp, _i64p]
    fn.restype = ctypes.c_int
    nq, nqp = _arr_i32([len(d) for d, _ in circuits])
    dc, dcp = _arr_i32([int(x) for d, _ in circuits for x in d])
    ng, ngp = _arr_i32([len(g) for _, g in circuits])
    allg = [g for _, gs in circuits for g in gs]
    ga = GateArray(allg)
    tune = np.array([tile_amps, small_amps, group_amps, tiles_per_item], dtype=np.int64)
    Ns = [int(np.prod(d)) for d, _ in circuits]
    amps = np.zeros(2 * sum(Ns), dtype=np.float64)
    info = np.zeros(5, dtype=np.int64)
    _check(fn(len(circuits), nqp, dcp, ga.ptr if allg else None, ngp, tune.ctypes.data_as(_i64p),
              amps.ctypes.data_as(_dp), info.ctypes.data_as(_i64p)))
    z = amps.view(np.complex128)
    out, o = [], 0
    for n in Ns:
        out.append(z[o:o + n].copy())
        o += n
    keys = ["segments", "items", "max_tile", "alg_bytes", "errors"]
    return out, {k: int(v) for k, v in zip(keys, info)}


def qd_debug_fuse_plan(dims, gates, plan_kind, precision=QD_C64, kmax=3, dmax=32):
    """(segments [(first, last)], model cost) chosen by the host planner."""
    L = load()
    fn = L.qd_debug_fuse_plan
    fn.argtypes = [_i32p, _i32, _i32, ctypes.POINTER(QdGate), _i32, _i32, _i32, _i32, _i32p, _i32p, _i32, _i32p, _dp]
    fn.restype = ctypes.c_int
    d, dp = _arr_i32(dims)
    ga = GateArray(gates)
    cap = max(1, ga.n)
    f = np.zeros(cap, np.int32)
    l = np.zeros(cap, np.int32)
    ns = _i32()
    c = ctypes.c_double()
    _check(fn(dp, len(d), precision, ga.ptr, ga.n, plan_kind, kmax, dmax, f.ctypes.data_as(_i32p),
              l.ctypes.data_as(_i32p), cap, ctypes.byref(ns), ctypes.byref(c)))
    return list(zip(f[:ns.value].tolist(), l[:ns.value].tolist())), c.value


def qd_debug_segment_cost(dims, gates, first, last, precision=QD_C64):
    L = load()
    fn = L.qd_debug_segment_cost
    fn.argtypes = [_i32p, _i32, _i32, ctypes.POINTER(QdGate), _i32, _i32, _i32, _dp]
    fn.restype = ctypes.c_int
    d, dp = _arr_i32(dims)
    ga = GateArray(gates)
    c = ctypes.c_double()
    _check(fn(dp, len(d), precision, ga.ptr, ga.n, first, last, ctypes.byref(c)))
    return c.value


def qd_debug_segment_forms(dims, gates, first, last, precision=QD_C64):
    """[(kernel form, 12 features)] of every feasible form of a segment (host only)."""
    L = load()
    fn = L.qd_debug_segment_forms
    fn.argtypes = [_i32p, _i32, _i32, ctypes.POINTER(QdGate), _i32, _i32, _i32, _i32p,
                   ctypes.POINTER(ctypes.c_float), _i32, _i32p]
    fn.restype = ctypes.c_int
    d, dp = _arr_i32(dims)
    ga = GateArray(gates)
    k, kp = _arr_i32([0] * 4)
    feats = np.zeros((4, QD_MODEL_FEATURES), np.float32)
    n = _i32(0)
    _check(fn(dp, len(d), precision, ga.ptr, ga.n, first, last, kp, feats.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
              4, ctypes.byref(n)))
    return [(int(k[i]), feats[i].copy()) for i in range(n.value)]


def qd_debug_fuse_block(dims, gates, first, last):
    """(qudits, D x D complex matrix) of the fused block of gates[first..last]."""
    L = load()
    fn = L.qd_debug_fuse_block
    fn.argtypes = [_i32p, _i32, ctypes.POINTER(QdGate), _i32, _i32, _i32, _i32p, _i32p, _i32p, _dp, _i64]
    fn.restype = ctypes.c_int
    d, dp = _arr_i32(dims)
    ga = GateArray(gates)
    qs = np.zeros(6, np.int32)
    k, D = _i32(), _i32()
    cap = 2 * 1024 * 1024
    m = np.zeros(cap, np.float64)
    _check(fn(dp, len(d), ga.ptr, ga.n, first, last, qs.ctypes.data_as(_i32p), ctypes.byref(k), ctypes.byref(D),
              m.ctypes.data_as(_dp), cap))
    Dv = D.value
    M = m[:2 * Dv * Dv].view(np.complex128).reshape(Dv, Dv).copy()
    return qs[:k.value].tolist(), M


# ---- learned cost model ------------------------------------------------------

_fp = ctypes.POINTER(ctypes.c_float)


def _f32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a, a.ctypes.data_as(_fp)


def qd_model_create() -> int:
    out = _vp()
    _check(load().qd_model_create(ctypes.byref(out)))
    return out.value


def qd_model_destroy(model: int) -> None:
    _check(load().qd_model_destroy(_vp(model)))


def qd_model_set(model: int, params, feat_mean=None, feat_std=None, y_mean: float = 0.0, y_std: float = 1.0) -> None:
    p, pp = _f32(params)
    assert p.size == QD_MODEL_PARAMS
    m, mp = _f32(feat_mean) if feat_mean is not None else (None, None)
    sd, sp = _f32(feat_std) if feat_std is not None else (None, None)
    _check(load().qd_model_set(_vp(model), pp, mp, sp, y_mean, y_std))


def qd_model_get(model: int) -> dict:
    p = np.zeros(QD_MODEL_PARAMS, np.float32)
    m = np.zeros(QD_MODEL_FEATURES, np.float32)
    sd = np.zeros(QD_MODEL_FEATURES, np.float32)
    ym, ys = ctypes.c_float(), ctypes.c_float()
    _check(load().qd_model_get(_vp(model), p.ctypes.data_as(_fp), m.ctypes.data_as(_fp), sd.ctypes.data_as(_fp),
                               ctypes.byref(ym), ctypes.byref(ys)))
    return {"params": p, "feat_mean": m, "feat_std": sd, "y_mean": ym.value, "y_std": ys.value}


def qd_model_train(model: int, X, y, epochs: int = 60, batch: int = 256, lr: float = 2e-3, seed: int = 0) -> float:
    Xa, Xp = _f32(X)
    ya, yp = _f32(y)
    loss = ctypes.c_double()
    _check(load().qd_model_train(_vp(model), Xp, yp, len(ya), epochs, batch, lr, ctypes.c_uint64(seed),
                                 ctypes.byref(loss)))
    return loss.value


def qd_model_predict(model: int, X) -> np.ndarray:
    Xa, Xp = _f32(X)
    n = Xa.shape[0]
    out = np.zeros(n, np.float32)
    _check(load().qd_model_predict(_vp(model), Xp, n, out.ctypes.data_as(_fp)))
    return out


def qd_model_forward_raw(model: int, Xn, fp16: bool = False) -> np.ndarray:
    Xa, Xp = _f32(Xn)
    n = Xa.shape[0]
    out = np.zeros(n, np.float32)
    _check(load().qd_model_forward_raw(_vp(model), Xp, n, out.ctypes.data_as(_fp), 1 if fp16 else 0))
    return out


def qd_model_grad_raw(model: int, Xn, t):
    Xa, Xp = _f32(Xn)
    ta, tp = _f32(t)
    g = np.zeros(QD_MODEL_PARAMS, np.float32)
    loss = ctypes.c_double()
    _check(load().qd_model_grad_raw(_vp(model), Xp, tp, len(ta), ctypes.byref(loss), g.ctypes.data_as(_fp)))
    return loss.value, g


def qd_set_cost_model(reg: int, model: int) -> None:
    _check(load().qd_set_cost_model(_vp(reg), _vp(model or None)))


def qd_segment_features(reg: int, gates, first: int, last: int) -> np.ndarray:
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    out = np.zeros(QD_MODEL_FEATURES, np.float32)
    _check(load().qd_segment_features(_vp(reg), ga.ptr, ga.n, first, last, out.ctypes.data_as(_fp)))
    return out


def qd_plan_create_segmented(reg: int, gates, segments, kinds=None) -> int:
    """Plan from explicit (first, last) segments; kinds: the kernel class of
    each segment (-1: the cost model's choice), None: all chosen."""
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    f, fp = _arr_i32([a for a, _ in segments])
    l, lp = _arr_i32([b for _, b in segments])
    out = _vp()
    if kinds is None:
        _check(load().qd_plan_create_segmented(_vp(reg), ga.ptr, ga.n, fp, lp, len(segments), ctypes.byref(out)))
    else:
        k, kp = _arr_i32([int(x) for x in kinds])
        _check(load().qd_plan_create_forms(_vp(reg), ga.ptr, ga.n, fp, lp, kp, len(segments), ctypes.byref(out)))
    return out.value


def qd_plan_create_forms(reg: int, gates, segments, kinds) -> int:
    """Plan from explicit segments with the kernel form of each given."""
    return qd_plan_create_segmented(reg, gates, segments, list(kinds))


def qd_segment_forms(reg: int, gates, first: int, last: int):
    """[(kernel class, 12 features)] of every feasible form of one segment."""
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    k, kp = _arr_i32([0] * 4)
    feats = np.zeros((4, QD_MODEL_FEATURES), np.float32)
    n = _i32(0)
    _check(load().qd_segment_forms(_vp(reg), ga.ptr, ga.n, first, last, kp, feats.ctypes.data_as(_fp), 4,
                                   ctypes.byref(n)))
    return [(int(k[i]), feats[i].copy()) for i in range(n.value)]


# ---- batched persistent execution -----------------------------------------

def qd_batch_create(registers: Sequence[Sequence[int]], stream: int = 0) -> int:
    """One batch of independent registers (one dims list per circuit)."""
    nq, nqp = _arr_i32([len(r) for r in registers])
    dc, dcp = _arr_i32([int(d) for r in registers for d in r])
    out = _vp()
    _check(load().qd_batch_create(len(nq), nqp, dcp, _vp(stream or None), ctypes.byref(out)))
    return out.value


def qd_batch_set_circuit(batch: int, c: int, gates) -> None:
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    _check(load().qd_batch_set_circuit(_vp(batch), c, ga.ptr if ga.n else None, ga.n))


def qd_batch_tune(batch: int, key: int, value: int) -> None:
    _check(load().qd_batch_tune(_vp(batch), key, int(value)))


def qd_batch_run(batch: int) -> None:
    _check(load().qd_batch_run(_vp(batch)))


def qd_batch_info(batch: int, with_error: bool = False) -> dict:
    t, it, la, er = _i64(), _i32(), _i32(), _i32()
    _check(load().qd_batch_info(_vp(batch), ctypes.byref(t), ctypes.byref(it), ctypes.byref(la),
                                ctypes.byref(er) if with_error else None))
    d = {"total": t.value, "items": it.value, "launches": la.value}
    if with_error:
        d["device_error"] = er.value
    return d


def qd_batch_probabilities(batch: int, c: int, n: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    """FP64 probabilities of circuit c (n amplitudes) into ``out`` (float64,
    at least n entries) or a new array."""
    if out is None:
        out = np.empty(n, np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.size >= n
    _check(load().qd_batch_probabilities(_vp(batch), c, out.ctypes.data_as(_dp)))
    return out


def qd_batch_get_amplitudes(batch: int, c: int, n: int) -> np.ndarray:
    out = np.empty(n, np.complex64)
    _check(load().qd_batch_get_amplitudes(_vp(batch), c, _vp(out.ctypes.data)))
    return out


def qd_batch_profile(batch: int, enable: bool = True) -> None:
    _check(load().qd_batch_profile(_vp(batch), int(bool(enable))))


def qd_batch_timings(batch: int, with_time: bool = True):
    """(persistent-kernel ms of the last profiled run or None, algorithmic bytes)."""
    ms, ab = ctypes.c_float(), ctypes.c_double()
    _check(load().qd_batch_timings(_vp(batch), ctypes.byref(ms) if with_time else None, ctypes.byref(ab)))
    return (ms.value if with_time else None), ab.value


def qd_batch_autotune(batch: int, reps: int = 2) -> dict:
    """Pick the fastest launch shape (see include/qudit.h); returns it."""
    ch = np.zeros(4, dtype=np.int64)
    ms = ctypes.c_float()
    _check(load().qd_batch_autotune(_vp(batch), reps, ch.ctypes.data_as(_i64p), ctypes.byref(ms)))
    return {"tile_amps": int(ch[0]), "small_amps": int(ch[1]), "ctas_per_sm": int(ch[2]),
            "tiles_per_item": int(ch[3]), "kernel_ms": ms.value}


def qd_batch_destroy(batch: int) -> None:
    _check(load().qd_batch_destroy(_vp(batch)))


# ---- circuit layer: measurement flag, Toffoli / MCT decompositions, ket
# readout, QuDiet QASM, the paper's moment execution model -----------------

def _gate_from_struct(st):
    """A workloads.Gate view of one qd_gate record (named gates only)."""
    from .workloads import Gate
    ctrls = tuple(int(st.controls[i]) for i in range(st.nc))
    levels = tuple(int(st.ctrl_levels[i]) for i in range(st.nc)) if st.nc else None
    return Gate(_KIND_NAME[int(st.kind)], tuple(int(st.targets[i]) for i in range(st.k)), ctrls, levels,
                int(st.param))


def qd_measure_all(reg: int) -> None:
    _check(load().qd_measure_all(_vp(reg)))


def qd_is_measured(reg: int) -> bool:
    v = _i32()
    _check(load().qd_is_measured(_vp(reg), ctypes.byref(v)))
    return bool(v.value)


def qd_toffoli_gates(dims: Sequence[int], c1: int, carrier: int, t: int, shift: int = 1) -> list:
    d, dp = _arr_i32(dims)
    out = (QdGate * 3)()
    _check(load().qd_toffoli_gates(dp, len(d), c1, carrier, t, shift, out))
    return [_gate_from_struct(out[i]) for i in range(3)]


def qd_apply_toffoli(reg: int, c1: int, carrier: int, t: int, shift: int = 1) -> None:
    _check(load().qd_apply_toffoli(_vp(reg), c1, carrier, t, shift))


def qd_mct_tree_gates(dims: Sequence[int], controls, t: int, shift: int = 1, ctrl_levels=None):
    """(gate list, depth) of the logarithmic-depth MCT decomposition."""
    d, dp = _arr_i32(dims)
    c, cp = _arr_i32(controls)
    lv, lp = _arr_i32(ctrl_levels) if ctrl_levels is not None else (None, None)
    cnt, depth = _i32(), _i32()
    _check(load().qd_mct_tree_gates(dp, len(d), cp, lp, len(c), t, shift, None, 0, ctypes.byref(cnt), None))
    out = (QdGate * max(1, cnt.value))()
    _check(load().qd_mct_tree_gates(dp, len(d), cp, lp, len(c), t, shift, out, cnt.value, ctypes.byref(cnt),
                                    ctypes.byref(depth)))
    return [_gate_from_struct(out[i]) for i in range(cnt.value)], depth.value


def qd_apply_mct_tree(reg: int, controls, t: int, shift: int = 1, ctrl_levels=None) -> None:
    c, cp = _arr_i32(controls)
    lv, lp = _arr_i32(ctrl_levels) if ctrl_levels is not None else (None, None)
    _check(load().qd_apply_mct_tree(_vp(reg), cp, lp, len(c), t, shift))


def qd_ket_list(reg: int, method: int = QD_OUT_AMPLITUDE, threshold: float = 1e-14, cap: Optional[int] = None):
    """(indices int64[m], values) of the basis states with |psi_i|^2 > threshold,
    ascending; values complex128[m] (amplitudes) or float64[m] (probabilities);
    m = min(total, cap); also returns the total."""
    if cap is None:
        cnt = _i64()
        _check(load().qd_ket_list(_vp(reg), method, threshold, 0, None, None, ctypes.byref(cnt)))
        cap = cnt.value
    idx = np.zeros(max(cap, 1), dtype=np.int64)
    per = 2 if method == QD_OUT_AMPLITUDE else 1
    val = np.zeros(max(cap, 1) * per, dtype=np.float64)
    cnt = _i64()
    _check(load().qd_ket_list(_vp(reg), method, threshold, cap, idx.ctypes.data_as(_i64p), val.ctypes.data_as(_dp),
                              ctypes.byref(cnt)))
    m = min(cnt.value, cap)
    vals = val[: 2 * m].view(np.complex128) if per == 2 else val[:m]
    return idx[:m], vals.copy(), cnt.value


def qd_ket_label(dims: Sequence[int], index: int) -> str:
    d, dp = _arr_i32(dims)
    buf = ctypes.create_string_buffer(4 * len(d) + 8)
    _check(load().qd_ket_label(dp, len(d), int(index), buf, len(buf)))
    return buf.value.decode()


def ket_dict(reg: int, dims: Sequence[int], method: int = QD_OUT_AMPLITUDE, threshold: float = 1e-14) -> dict:
    """OutputType.print: {ket label: amplitude or probability} of the kept
    basis states (labels qudit 0 first), from qd_ket_list / qd_ket_label."""
    idx, vals, _ = qd_ket_list(reg, method, threshold)
    return {qd_ket_label(dims, int(i)): (complex(v) if method == QD_OUT_AMPLITUDE else float(v))
            for i, v in zip(idx, vals)}


def output(reg: int, dims: Sequence[int], output_type: str = "print", method: str = "probability"):
    """The paper's OutputType ("print": ket dict; "state": the raw state
    array) and OutputMethod ("amplitude" or "probability")."""
    m = QD_OUT_AMPLITUDE if method == "amplitude" else QD_OUT_PROBABILITY
    if output_type == "state":
        return qd_get_amplitudes(reg) if m == QD_OUT_AMPLITUDE else qd_probabilities(reg)
    return ket_dict(reg, dims, m)


def qd_qasm_parse(text: str):
    """(dims, gate list) of a QuDiet QASM program; raises QuditError with the
    line number on a syntax error."""
    src = text.encode()
    n, ng, line = _i32(), _i32(), _i32()
    rc = load().qd_qasm_parse(src, None, 0, ctypes.byref(n), None, 0, ctypes.byref(ng), ctypes.byref(line))
    if rc != QD_OK:
        err = QuditError(rc, load().qd_last_error().decode(errors="replace"))
        err.line = line.value
        raise err
    dims = np.zeros(max(n.value, 1), dtype=np.int32)
    arr = (QdGate * max(ng.value, 1))()
    _check(load().qd_qasm_parse(src, dims.ctypes.data_as(_i32p), n.value, ctypes.byref(n), arr, ng.value,
                                ctypes.byref(ng), ctypes.byref(line)))
    return [int(x) for x in dims[: n.value]], [_gate_from_struct(arr[i]) for i in range(ng.value)]


def qd_run_moments(reg: int, gates) -> int:
    """Apply the gates through the paper's moment / Kronecker / GEMM-chain
    execution model; returns the moment count."""
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    nm = _i32()
    _check(load().qd_run_moments(_vp(reg), ga.ptr, ga.n, ctypes.byref(nm)))
    return nm.value


def qd_moment_packing(dims: Sequence[int], gates):
    d, dp = _arr_i32(dims)
    ga = gates if isinstance(gates, GateArray) else GateArray(gates)
    m = np.zeros(max(ga.n, 1), dtype=np.int32)
    nm = _i32()
    _check(load().qd_moment_packing(dp, len(d), ga.ptr, ga.n, m.ctypes.data_as(_i32p), ctypes.byref(nm)))
    return m[: ga.n], nm.value


class Circuit:
    """Circuit builder over the C ABI (the paper's qc.h / qc.x / qc.cx /
    qc.Toffoli / measure_all calls, Sec. 3.4 and 3.6): collects gate records;
    the decompositions come from the library (qd_toffoli_gates,
    qd_mct_tree_gates); run() prepares and runs them on a register."""

    def __init__(self, dims: Sequence[int]):
        from .workloads import Gate
        self._Gate = Gate
        self.dims = [int(d) for d in dims]
        self.gates = []

    def x(self, q, plus=1):
        self.gates.append(self._Gate("X", (q,), param=plus))
        return self

    def z(self, q, power=1):
        self.gates.append(self._Gate("Z", (q,), param=power))
        return self

    def h(self, q):
        self.gates.append(self._Gate("H", (q,)))
        return self

    def cx(self, qs, plus=1, level=None):
        c, t = qs
        self.gates.append(self._Gate("X", (t,), (c,), None if level is None else (level,), plus))
        return self

    def unitary(self, targets, matrix, controls=(), levels=None):
        self.gates.append(self._Gate("U", tuple(targets), tuple(controls), levels, 0, np.asarray(matrix)))
        return self

    def toffoli(self, qs, plus=1):
        c1, carrier, t = qs
        self.gates.extend(qd_toffoli_gates(self.dims, c1, carrier, t, plus))
        return self

    def mct(self, controls, t, plus=1, levels=None):
        self.gates.extend(qd_mct_tree_gates(self.dims, controls, t, plus, levels)[0])
        return self

    def measure_all(self):
        self.gates.append(self._Gate("MEASURE", ()))
        return self

    def run(self, reg: int, plan_kind: int = QD_PLAN_NONE) -> None:
        qd_run_circuit(reg, self.gates, plan_kind)


def qd_batch_sync(batch: int) -> int:
    """The last run's device error word; raises QuditError (QD_ERR_TIMEOUT for
    an expired wait) when it is set."""
    err = _i32()
    rc = load().qd_batch_sync(_vp(batch), ctypes.byref(err))
    if rc != QD_OK:
        e = QuditError(rc, load().qd_last_error().decode(errors="replace"))
        e.device_error = err.value
        raise e
    return err.value
