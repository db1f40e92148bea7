"""ctypes binding of libqt.so: the C ABI of include/qt.h under the same names.

Argument marshalling only -- every step of the trajectory path runs in the
library's CUDA kernels.  There is no fallback: if libqt.so cannot be loaded
the import fails.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

QT_OK = 0
QT_ERR_INVALID_ARG = -1
QT_ERR_NOT_CPTP = -2
QT_ERR_OUT_OF_MEMORY = -3
QT_ERR_CUDA = -4
QT_ERR_TIMEOUT = -5
QT_ERR_UNSUPPORTED = -6
QT_ERR_INTERNAL = -7

QT_OP_GATE, QT_OP_KRAUS, QT_OP_MIXTURE = 0, 1, 2
QT_DELAYED, QT_EAGER = 0, 1
QT_FP32, QT_TF32X3 = 0, 1
QT_FLAG_TIME_KERNELS = 1
QT_FLAG_MULTI_GATE = 2
QT_FLAG_SHARE_PREFIX = 4


class QtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"qt status {status}: {msg}")
        self.status = status


class qt_op(C.Structure):
    _fields_ = [("kind", C.c_int32), ("moment", C.c_uint32), ("num_qubits", C.c_uint32),
                ("qubits", C.c_uint32 * 6), ("num_ops", C.c_uint32),
                ("probs", C.c_void_p), ("mats", C.c_void_p)]


class qt_run_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("first_traj", C.c_uint64), ("num_traj", C.c_uint32),
                ("mode", C.c_uint32), ("precision", C.c_uint32), ("samples_per_traj", C.c_uint32),
                ("num_z_masks", C.c_uint32), ("z_masks", C.c_void_p), ("keep_states", C.c_uint32),
                ("flags", C.c_uint32), ("stream", C.c_void_p), ("timeout_ns", C.c_uint64),
                ("readout_error", C.c_void_p)]


class qt_run_stats_t(C.Structure):
    _fields_ = [("num_traj", C.c_uint32), ("num_channels", C.c_uint32),
                ("fused_passes", C.c_uint64), ("prob_passes", C.c_uint64),
                ("gate_ops", C.c_uint64), ("flushes", C.c_uint64),
                ("device_ms", C.c_double), ("apply_ms", C.c_double),
                ("apply_bytes", C.c_uint64), ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64),
                ("kernel_launches", C.c_uint64), ("fused_pieces", C.c_uint64),
                ("passes_by_width", C.c_uint64 * 8), ("apply_ms_by_width", C.c_double * 8),
                ("folded_pieces", C.c_uint64), ("fold_split", C.c_uint32), ("pad", C.c_uint32),
                ("prefix_copies", C.c_uint64), ("prefix_ops", C.c_uint64), ("merged_pieces", C.c_uint64)]


class qt_fused_info_t(C.Structure):
    _fields_ = [("num_fused", C.c_uint32), ("max_width", C.c_uint32),
                ("num_ops", C.c_uint32), ("num_channels", C.c_uint32)]


class qt_batch_params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("first_traj", C.c_uint64), ("samples_per_traj", C.c_uint32),
                ("keep_states", C.c_uint32), ("use_graph", C.c_uint32), ("threads", C.c_uint32),
                ("stream", C.c_void_p), ("threads_global", C.c_uint32)]


class qt_batch_stats_t(C.Structure):
    _fields_ = [("num_traj", C.c_uint32), ("num_channels", C.c_uint32), ("total_amps", C.c_uint64),
                ("fused_gates", C.c_uint64), ("gate_ops", C.c_uint64), ("flushes", C.c_uint64),
                ("device_ms", C.c_double), ("folded_pieces", C.c_uint64)]


class qt_server_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("max_slots", C.c_uint32), ("small_n_max", C.c_uint32),
                ("flags", C.c_uint32)]


class qt_server_request(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("first_traj", C.c_uint64), ("num_traj", C.c_uint32),
                ("samples_per_traj", C.c_uint32)]


class qt_server_req_info(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("attempts", C.c_uint32), ("worker", C.c_int32),
                ("batched", C.c_uint32), ("num_traj", C.c_uint32), ("samples_per_traj", C.c_uint32),
                ("pad", C.c_uint32), ("bytes", C.c_uint64), ("flushes", C.c_uint64),
                ("queued_s", C.c_double), ("latency_s", C.c_double)]


class qt_server_stats_t(C.Structure):
    _fields_ = [("budget", C.c_uint64), ("inflight_bytes", C.c_uint64), ("peak_inflight_bytes", C.c_uint64),
                ("queued", C.c_uint32), ("running", C.c_uint32), ("done", C.c_uint32), ("failed", C.c_uint32),
                ("workers_alive", C.c_uint32), ("requeued", C.c_uint32), ("deferred", C.c_uint32),
                ("pad", C.c_uint32), ("lane_bytes", C.c_uint64), ("lane_launches", C.c_uint64),
                ("lane_trajectories", C.c_uint64)]


QT_SERVER_DRY_RUN = 1
QT_SERVER_NO_SHARED_PREFIX = 2
QT_FAULT_WORKER_EXIT, QT_FAULT_ALLOC = 1, 2


# qt_op as a numpy record (56 bytes, C layout) for vectorized marshalling
QT_OP_DTYPE = np.dtype({"names": ["kind", "moment", "num_qubits", "qubits", "num_ops", "probs", "mats"],
                        "formats": ["<i4", "<u4", "<u4", ("<u4", 6), "<u4", "<u8", "<u8"],
                        "offsets": [0, 4, 8, 12, 36, 40, 48], "itemsize": 56})


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

# every exported symbol of include/qt.h
EXPORTS = [
    "qt_circuit_create", "qt_fuse", "qt_run_trajectories", "qt_sample", "qt_expectation",
    "qt_run_kraus_indices", "qt_run_stats", "qt_run_state", "qt_run_norms", "qt_set_allocator",
    "qt_circuit_destroy", "qt_fused_destroy", "qt_run_destroy", "qt_last_error",
    "qt_fused_info", "qt_fused_gate", "qt_channel_lower_bounds", "qt_kernel_arch",
    "qt_state_apply", "qt_state_reduced_density", "qt_state_sample", "qt_state_expect_z",
    "qt_state_cdf", "qt_state_kraus_probabilities", "qt_state_reduced_density_noalloc",
    "qt_fuse_many", "qt_batch_create", "qt_batch_run", "qt_batch_samples", "qt_batch_kraus_indices",
    "qt_batch_state", "qt_batch_stats", "qt_batch_destroy", "qt_batch_autotune",
    "qt_server_create", "qt_server_submit", "qt_server_poll", "qt_server_wait", "qt_server_cancel",
    "qt_server_result", "qt_server_release", "qt_server_stats", "qt_server_inject", "qt_server_destroy",
]

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqt.so (building it first if needed).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libqt.so missing at {_build.LIB}: the CUDA library is required")
        lib = C.CDLL(_build.LIB)
        P = C.c_void_p
        u32, u64 = C.c_uint32, C.c_uint64
        sig = {
            "qt_circuit_create": [u32, u32, P, P],
            "qt_fuse": [P, u32, P],
            "qt_run_trajectories": [P, P, P],
            "qt_sample": [P, u32, P],
            "qt_expectation": [P, u32, P, P],
            "qt_run_kraus_indices": [P, P, P, C.c_size_t],
            "qt_run_stats": [P, P],
            "qt_run_state": [P, u32, P, C.c_size_t],
            "qt_run_norms": [P, P],
            "qt_set_allocator": [P, P, P],
            "qt_fused_info": [P, P],
            "qt_fused_gate": [P, u32, P, P, P, P, C.c_size_t, P],
            "qt_channel_lower_bounds": [P, u32, P, C.c_size_t, P],
            "qt_kernel_arch": [P, P],
            "qt_state_apply": [P, u32, u32, P, P, u32, P],
            "qt_state_reduced_density": [P, u32, u32, P, P, P],
            "qt_state_sample": [P, u32, u64, u64, u32, P, P, P],
            "qt_state_expect_z": [P, u32, u32, P, P, P],
            "qt_state_cdf": [P, u32, P, P],
            "qt_state_kraus_probabilities": [P, u32, u32, P, u32, P, P, P, P],
            "qt_state_reduced_density_noalloc": [P, u32, u32, P, P, P],
            "qt_fuse_many": [u32, P, u32, u32, P],
            "qt_batch_create": [u32, P, P],
            "qt_batch_run": [P, P],
            "qt_batch_samples": [P, P, C.c_size_t],
            "qt_batch_kraus_indices": [P, u32, P, P, C.c_size_t, P],
            "qt_batch_state": [P, u32, P, C.c_size_t],
            "qt_batch_stats": [P, P],
            "qt_batch_autotune": [u32, P, u32, u32, u32, P, P, P],
            "qt_server_create": [P, P],
            "qt_server_submit": [P, P, P, P],
            "qt_server_poll": [P, u64, P],
            "qt_server_wait": [P, u64, u64],
            "qt_server_cancel": [P, u64],
            "qt_server_result": [P, u64, P, C.c_size_t, P],
            "qt_server_release": [P, u64],
            "qt_server_stats": [P, P],
            "qt_server_inject": [P, u32, u32],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        for name in ("qt_circuit_destroy", "qt_fused_destroy", "qt_run_destroy", "qt_batch_destroy",
                     "qt_server_destroy"):
            fn = getattr(lib, name)
            fn.argtypes = [P]
            fn.restype = None
        lib.qt_last_error.restype = C.c_char_p
        lib.qt_last_error.argtypes = []
        _lib = lib
        return lib


def _check(status):
    if status != QT_OK:
        msg = load().qt_last_error().decode(errors="replace")
        raise QtError(status, msg)


def _ptr(a):
    return None if a is None else a.ctypes.data


# ----------------------------------------------------------------------------
# torch plumbing: device memory from torch's caching allocator, torch streams
# ----------------------------------------------------------------------------
_alloc_refs = None


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through torch's caching allocator."""
    global _alloc_refs
    lib = load()
    if not enable:
        _check(lib.qt_set_allocator(None, None, None))
        _alloc_refs = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:  # noqa: BLE001 -- reported to the library as NULL
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _alloc_refs = (a, f)
    _check(lib.qt_set_allocator(C.cast(a, C.c_void_p), C.cast(f, C.c_void_p), None))


def current_stream_handle():
    import torch
    return torch.cuda.current_stream().cuda_stream


# ----------------------------------------------------------------------------
# handles
# ----------------------------------------------------------------------------
class Circuit:
    """qt_circuit built from a list of ops (qtsynth.Op-like objects)."""

    def __init__(self, num_qubits, ops):
        lib = load()
        self.num_qubits = int(num_qubits)
        arr = (qt_op * max(len(ops), 1))()
        self._keep = []
        for i, o in enumerate(ops):
            mats = np.ascontiguousarray(np.asarray(o.mats, dtype=np.complex128)).view(np.float64).ravel()
            self._keep.append(mats)
            arr[i].kind = int(o.kind)
            arr[i].moment = int(o.moment)
            arr[i].num_qubits = len(o.qubits)
            for b, q in enumerate(o.qubits):
                arr[i].qubits[b] = int(q)
            arr[i].num_ops = int(np.asarray(o.mats).shape[0])
            arr[i].mats = mats.ctypes.data
            if o.probs is not None:
                pr = np.ascontiguousarray(o.probs, dtype=np.float64)
                self._keep.append(pr)
                arr[i].probs = pr.ctypes.data
        self.h = C.c_void_p()
        _check(lib.qt_circuit_create(self.num_qubits, len(ops), C.cast(arr, C.c_void_p), C.byref(self.h)))
        self.num_channels = sum(1 for o in ops if o.kind != QT_OP_GATE)
        self.num_ops = len(ops)
        self._keep = None

    @classmethod
    def from_synth(cls, circ):
        if hasattr(circ, "table_id"):
            return cls.from_compact(circ)
        return cls(circ.num_qubits, circ.ops)

    @classmethod
    def from_compact(cls, cc):
        """From a qtsynth.CompactCircuit: the qt_op array is built in one
        vectorized pass, every op pointing at its shared operator table entry."""
        lib = load()
        self = cls.__new__(cls)
        self.num_qubits = int(cc.num_qubits)
        mats_tab, probs_tab = [], []
        mptr = np.zeros(len(cc.table), np.uint64)
        pptr = np.zeros(len(cc.table), np.uint64)
        nops = np.zeros(len(cc.table), np.uint32)
        for t, (kind, mats, probs) in enumerate(cc.table):
            m = np.ascontiguousarray(np.asarray(mats, np.complex128)).view(np.float64).ravel()
            mats_tab.append(m)
            mptr[t] = m.ctypes.data
            nops[t] = np.asarray(mats).shape[0]
            if probs is not None:
                pr = np.ascontiguousarray(probs, np.float64)
                probs_tab.append(pr)
                pptr[t] = pr.ctypes.data
        arr = np.zeros(cc.num_ops, QT_OP_DTYPE)
        arr["kind"] = cc.kind
        arr["moment"] = cc.moment
        arr["num_qubits"] = cc.nq
        arr["qubits"][:, :2] = cc.qubits
        arr["num_ops"] = nops[cc.table_id]
        arr["probs"] = pptr[cc.table_id]
        arr["mats"] = mptr[cc.table_id]
        self.h = C.c_void_p()
        _check(lib.qt_circuit_create(self.num_qubits, cc.num_ops, arr.ctypes.data, C.byref(self.h)))
        self.num_channels = cc.num_channels
        self.num_ops = cc.num_ops
        self._keep = None
        return self

    def lower_bounds(self, channel):
        lib = load()
        out = np.zeros(64)
        k = C.c_uint32()
        _check(lib.qt_channel_lower_bounds(self.h, channel, _ptr(out), 64, C.byref(k)))
        return out[:k.value].copy()

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.qt_circuit_destroy(self.h)
            self.h = None


class Fused:
    def __init__(self, circuit: Circuit, max_fused_qubits: int = 0):
        lib = load()
        self.circuit = circuit           # the circuit must outlive the fused handle
        self.h = C.c_void_p()
        _check(lib.qt_fuse(circuit.h, int(max_fused_qubits), C.byref(self.h)))

    def info(self):
        i = qt_fused_info_t()
        _check(load().qt_fused_info(self.h, C.byref(i)))
        return dict(num_fused=i.num_fused, max_width=i.max_width, num_ops=i.num_ops,
                    num_channels=i.num_channels)

    def gate(self, g):
        lib = load()
        w = C.c_uint32()
        tg = np.zeros(8, dtype=np.uint32)
        nm = C.c_uint32()
        _check(lib.qt_fused_gate(self.h, g, C.byref(w), _ptr(tg), C.byref(nm), None, 0, None))
        mem = np.zeros(max(nm.value, 1), dtype=np.uint32)
        mat = np.zeros((1 << w.value) ** 2, dtype=np.complex128)
        _check(lib.qt_fused_gate(self.h, g, None, None, None, _ptr(mem), len(mem), _ptr(mat)))
        D = 1 << w.value
        return dict(targets=tg[:w.value].copy(), members=mem[:nm.value].copy(),
                    matrix=mat.reshape(D, D))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.qt_fused_destroy(self.h)
            self.h = None


class Run:
    def __init__(self, fused: Fused, num_traj, *, seed=0, first_traj=0, mode=QT_DELAYED,
                 precision=QT_FP32, samples_per_traj=0, z_masks=(), keep_states=False,
                 time_kernels=False, grouping=False, share_prefix=False, readout_error=None, stream=None):
        """readout_error: None, or [n, 2] readout error probabilities per qubit,
        (P(read 1 | 0), P(read 0 | 1)), applied to the samples (Sec. V.A).
        share_prefix: trajectories share the state along the default-choice prefix
        (QT_FLAG_SHARE_PREFIX, delayed mode)."""
        lib = load()
        self.fused = fused
        self.masks = np.ascontiguousarray(np.asarray(z_masks, dtype=np.uint64))
        n = fused.circuit.num_qubits
        self._ro = (None if readout_error is None else
                    np.ascontiguousarray(np.asarray(readout_error, np.float64).reshape(n, 2)))
        p = qt_run_params()
        p.seed, p.first_traj, p.num_traj = seed, first_traj, num_traj
        p.mode, p.precision, p.samples_per_traj = mode, precision, samples_per_traj
        p.num_z_masks = len(self.masks)
        p.z_masks = self.masks.ctypes.data if len(self.masks) else None
        p.keep_states = 1 if keep_states else 0
        p.flags = ((QT_FLAG_TIME_KERNELS if time_kernels else 0) | (QT_FLAG_MULTI_GATE if grouping else 0) |
                   (QT_FLAG_SHARE_PREFIX if share_prefix else 0))
        p.stream = stream
        p.readout_error = self._ro.ctypes.data if self._ro is not None else None
        self.params = p
        self.num_traj = num_traj
        self.S = samples_per_traj
        self.h = C.c_void_p()
        _check(lib.qt_run_trajectories(fused.h, C.byref(p), C.byref(self.h)))

    def samples(self, S=None):
        S = self.S if S is None else S
        out = np.zeros(max(self.num_traj * S, 1), dtype=np.uint64)
        _check(load().qt_sample(self.h, S, _ptr(out)))
        return out[:self.num_traj * S].reshape(self.num_traj, S)

    def expectation(self, masks=None):
        m = self.masks if masks is None else np.ascontiguousarray(np.asarray(masks, dtype=np.uint64))
        out = np.zeros(max(self.num_traj * len(m), 1))
        _check(load().qt_expectation(self.h, len(m), _ptr(m) if len(m) else None, _ptr(out)))
        return out[:self.num_traj * len(m)].reshape(self.num_traj, len(m))

    def kraus_indices(self):
        nch = self.fused.circuit.num_channels
        k = np.zeros(max(self.num_traj * nch, 1), dtype=np.int32)
        s = np.zeros_like(k)
        _check(load().qt_run_kraus_indices(self.h, _ptr(k), _ptr(s), len(k)))
        n = self.num_traj * nch
        return k[:n].reshape(self.num_traj, nch), s[:n].reshape(self.num_traj, nch)

    def stats(self):
        s = qt_run_stats_t()
        _check(load().qt_run_stats(self.h, C.byref(s)))
        out = {f: getattr(s, f) for f, _ in qt_run_stats_t._fields_}
        for f in ("passes_by_width", "apply_ms_by_width"):
            out[f] = list(out[f])
        return out

    def norms(self):
        out = np.zeros(max(self.num_traj, 1))
        _check(load().qt_run_norms(self.h, _ptr(out)))
        return out[:self.num_traj]

    def state(self, t):
        n = self.fused.circuit.num_qubits
        out = np.zeros(1 << n, dtype=np.complex64)
        _check(load().qt_run_state(self.h, t, _ptr(out), out.nbytes))
        return out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.qt_run_destroy(self.h)
            self.h = None


# ----------------------------------------------------------------------------
# state-level calls on a device pointer (e.g. a torch tensor's data_ptr())
# ----------------------------------------------------------------------------
def qt_state_apply(state_ptr, n, qubits, U, precision=QT_FP32, stream=None):
    q = np.ascontiguousarray(qubits, dtype=np.uint32)
    Um = np.ascontiguousarray(np.asarray(U, dtype=np.complex128)).view(np.float64)
    _check(load().qt_state_apply(state_ptr, n, len(q), _ptr(q), _ptr(Um), precision, stream))


def qt_state_reduced_density(state_ptr, n, qubits, stream=None):
    q = np.ascontiguousarray(qubits, dtype=np.uint32)
    D = 1 << len(q)
    out = np.zeros(D * D, dtype=np.complex128)
    _check(load().qt_state_reduced_density(state_ptr, n, len(q), _ptr(q), _ptr(out), stream))
    return out.reshape(D, D)


def qt_state_sample(state_ptr, n, seed, traj, S, readout_error=None, stream=None):
    """readout_error: None, or [n, 2] probabilities (P(read 1 | 0), P(read 0 | 1)) per qubit."""
    out = np.zeros(max(S, 1), dtype=np.uint64)
    ro = None if readout_error is None else np.ascontiguousarray(np.asarray(readout_error, np.float64).reshape(n, 2))
    _check(load().qt_state_sample(state_ptr, n, seed, traj, S, _ptr(out), _ptr(ro) if ro is not None else None,
                                  stream))
    return out[:S]


def qt_state_kraus_probabilities(state_ptr, n, qubits, Ks, stream=None):
    """(P[num_ops], N): P_i = <psi|K_i^dag K_i|psi> of the Kraus operators Ks
    (complex [num_ops, 2^q, 2^q]) on qubits, and N = <psi|psi>."""
    q = np.ascontiguousarray(qubits, dtype=np.uint32)
    K = np.ascontiguousarray(np.asarray(Ks, dtype=np.complex128)).view(np.float64)
    P = np.zeros(len(Ks))
    N = C.c_double()
    _check(load().qt_state_kraus_probabilities(state_ptr, n, len(q), _ptr(q), len(Ks), _ptr(K), _ptr(P),
                                               C.byref(N), stream))
    return P, N.value


def kernel_arch():
    """(binaryVersion, ptxVersion) of the library's kernels on the current device."""
    b, p = C.c_int32(0), C.c_int32(0)
    _check(load().qt_kernel_arch(C.byref(b), C.byref(p)))
    return b.value, p.value


def qt_state_cdf(state_ptr, n, stream=None):
    """The sampler's cumulative distribution C(x) of every x (2^n doubles)."""
    out = np.zeros(1 << n, dtype=np.float64)
    _check(load().qt_state_cdf(state_ptr, n, _ptr(out), stream))
    return out


def qt_state_expect_z(state_ptr, n, masks, stream=None):
    m = np.ascontiguousarray(masks, dtype=np.uint64)
    out = np.zeros(max(len(m), 1))
    _check(load().qt_state_expect_z(state_ptr, n, len(m), _ptr(m), _ptr(out), stream))
    return out[:len(m)]


# ----------------------------------------------------------------------------
# batched form
# ----------------------------------------------------------------------------
def fuse_many(circuits, max_fused_qubits=0, threads=0):
    """qt_fuse_many: fuse every circuit on host threads; returns Fused handles."""
    lib = load()
    n = len(circuits)
    hs = (C.c_void_p * n)(*[c.h for c in circuits])
    out = (C.c_void_p * n)()
    _check(lib.qt_fuse_many(n, C.cast(hs, C.c_void_p), int(max_fused_qubits), int(threads),
                            C.cast(out, C.c_void_p)))
    res = []
    for c, h in zip(circuits, out):
        f = Fused.__new__(Fused)
        f.circuit = c
        f.h = C.c_void_p(h)
        res.append(f)
    return res


class Batch:
    """qt_batch: one trajectory of each fused circuit per run, in one persistent launch."""

    def __init__(self, fused_list):
        lib = load()
        self.fused = list(fused_list)
        n = len(self.fused)
        hs = (C.c_void_p * n)(*[f.h for f in self.fused])
        self.h = C.c_void_p()
        _check(lib.qt_batch_create(n, C.cast(hs, C.c_void_p), C.byref(self.h)))
        self.num = n
        self.S = 0

    def run(self, seed=0, first_traj=0, samples_per_traj=0, keep_states=False, use_graph=False,
            threads=0, threads_global=0, stream=None):
        """threads: CTA size for states in shared memory (n <= 14); threads_global:
        for larger states (0 = threads)."""
        p = qt_batch_params()
        p.seed, p.first_traj, p.samples_per_traj = seed, first_traj, samples_per_traj
        p.keep_states = 1 if keep_states else 0
        p.use_graph = 1 if use_graph else 0
        p.threads = threads
        p.threads_global = threads_global
        p.stream = stream
        _check(load().qt_batch_run(self.h, C.byref(p)))
        self.S = samples_per_traj
        return self

    def samples(self):
        out = np.zeros(max(self.num * self.S, 1), dtype=np.uint64)
        _check(load().qt_batch_samples(self.h, _ptr(out), len(out)))
        return out[:self.num * self.S].reshape(self.num, self.S)

    def kraus_indices(self, i):
        lib = load()
        nch = C.c_uint32()
        _check(lib.qt_batch_kraus_indices(self.h, i, None, None, 0, C.byref(nch)))
        k = np.zeros(max(nch.value, 1), np.int32)
        st = np.zeros_like(k)
        _check(lib.qt_batch_kraus_indices(self.h, i, _ptr(k), _ptr(st), len(k), None))
        return k[:nch.value], st[:nch.value]

    def state(self, i):
        n = self.fused[i].circuit.num_qubits
        out = np.zeros(1 << n, dtype=np.complex64)
        _check(load().qt_batch_state(self.h, i, _ptr(out), out.nbytes))
        return out

    def stats(self):
        s = qt_batch_stats_t()
        _check(load().qt_batch_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in qt_batch_stats_t._fields_}

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.qt_batch_destroy(self.h)
            self.h = None


class qt_batch_tuning(C.Structure):
    _fields_ = [("k_shared", C.c_uint32), ("threads_shared", C.c_uint32),
                ("k_global", C.c_uint32), ("threads_global", C.c_uint32)]


SMEM_N_MAX = 14   # largest state (qubits) the batched kernel holds in shared memory


def autotune_batch(circuits, sample=256, kmin=2, kmax=4, stream=None):
    """qt_batch_autotune: returns ({"k_shared", "threads_shared", "k_global",
    "threads_global"}, {(class, k, threads): ms}) with class "shared" (n <= 14)
    or "global"."""
    lib = load()
    n = len(circuits)
    hs = (C.c_void_p * n)(*[c.h for c in circuits])
    best = qt_batch_tuning()
    nk = kmax - kmin + 1
    table = np.zeros(2 * nk * 3)
    _check(lib.qt_batch_autotune(n, C.cast(hs, C.c_void_p), sample, kmin, kmax, stream,
                                 C.byref(best), _ptr(table)))
    res = {}
    for ci, cls in enumerate(("shared", "global")):
        for k in range(kmin, kmax + 1):
            for ti, th in enumerate((128, 256, 512)):
                res[(cls, k, th)] = float(table[(ci * nk + k - kmin) * 3 + ti])
    return {f: getattr(best, f) for f, _ in qt_batch_tuning._fields_}, res


def fuse_by_class(circuits, tuning, threads=0):
    """Fuse each circuit at its class's width from autotune_batch (shared-memory
    states n <= 14: k_shared; larger: k_global); returns Fused handles in order."""
    out = [None] * len(circuits)
    for cls, k in (("shared", tuning["k_shared"]), ("global", tuning["k_global"])):
        idx = [i for i, c in enumerate(circuits) if (c.num_qubits > SMEM_N_MAX) == (cls == "global")]
        if idx:
            for i, f in zip(idx, fuse_many([circuits[i] for i in idx], k, threads)):
                out[i] = f
    return out


# ----------------------------------------------------------------------------
# serving form
# ----------------------------------------------------------------------------
class Server:
    """qt_server: continuous-batching request loop (plain-loop workers, one stream
    per slot, and a batch lane that merges small requests into shared launches)."""

    def __init__(self, budget_bytes, max_slots=8, small_n_max=16, dry_run=False, share_prefix=True):
        """small_n_max: the batch lane's limit (0: no lane); share_prefix=False: plain
        workers run each trajectory on its own (QT_SERVER_NO_SHARED_PREFIX)."""
        cfg = qt_server_config(int(budget_bytes), int(max_slots), int(small_n_max),
                               (QT_SERVER_DRY_RUN if dry_run else 0) |
                               (0 if share_prefix else QT_SERVER_NO_SHARED_PREFIX))
        self.h = C.c_void_p()
        _check(load().qt_server_create(C.byref(cfg), C.byref(self.h)))
        self._fused = {}

    def submit(self, fused, seed=0, first_traj=0, num_traj=1, samples_per_traj=0):
        r = qt_server_request(seed, first_traj, num_traj, samples_per_traj)
        i = C.c_uint64()
        _check(load().qt_server_submit(self.h, fused.h, C.byref(r), C.byref(i)))
        self._fused[i.value] = fused          # keep the circuit alive while the request lives
        return i.value

    def poll(self, rid):
        st = C.c_int32()
        _check(load().qt_server_poll(self.h, rid, C.byref(st)))
        return st.value

    def wait(self, rid, timeout_s=0.0):
        _check(load().qt_server_wait(self.h, rid, int(timeout_s * 1e9)))

    def cancel(self, rid):
        _check(load().qt_server_cancel(self.h, rid))

    def info(self, rid):
        inf = qt_server_req_info()
        _check(load().qt_server_result(self.h, rid, None, 0, C.byref(inf)))
        return {f: getattr(inf, f) for f, _ in qt_server_req_info._fields_}

    def result(self, rid):
        inf = self.info(rid)
        n = inf["num_traj"] * inf["samples_per_traj"]
        out = np.zeros(max(n, 1), dtype=np.uint64)
        _check(load().qt_server_result(self.h, rid, _ptr(out), len(out), None))
        return out[:n].reshape(inf["num_traj"], inf["samples_per_traj"]), inf

    def release(self, rid):
        _check(load().qt_server_release(self.h, rid))
        self._fused.pop(rid, None)

    def stats(self):
        s = qt_server_stats_t()
        _check(load().qt_server_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in qt_server_stats_t._fields_}

    def inject(self, fault, count=1):
        _check(load().qt_server_inject(self.h, fault, count))

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.qt_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
