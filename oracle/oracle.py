"""ctypes wrapper of oracle.c (test infrastructure; see oracle.h)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

DELAYED, EAGER, CUMULATIVE = 0, 1, 2


def lib_path() -> str:
    return _SO


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain C11 + OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared",
           "-fcx-limited-range", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Circ(C.Structure):
    _fields_ = [
        ("num_qubits", C.c_int32), ("num_ops", C.c_int32),
        ("kind", C.c_void_p), ("nq", C.c_void_p), ("qoff", C.c_void_p),
        ("qubits", C.c_void_p), ("nmat", C.c_void_p), ("moff", C.c_void_p),
        ("mats", C.c_void_p), ("poff", C.c_void_p), ("probs", C.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_SO)
            P = C.c_void_p
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_u01.restype = C.c_double
            lib.orc_u01.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32]
            lib.orc_apply.argtypes = [P, C.c_int, C.c_int, P, P]
            lib.orc_norm2.restype = C.c_double
            lib.orc_norm2.argtypes = [P, C.c_int]
            lib.orc_kraus_norms.argtypes = [P, C.c_int, C.c_int, P, C.c_int, P, P]
            lib.orc_lower_bound.restype = C.c_double
            lib.orc_lower_bound.argtypes = [C.c_int, P]
            lib.orc_run_trajectory.restype = C.c_int
            lib.orc_run_trajectory.argtypes = [P, C.c_int, C.c_uint64, C.c_uint64,
                                               C.c_int64, P, P, P, P]
            lib.orc_run_trajectories.argtypes = [P, C.c_int, C.c_uint64, C.c_uint64,
                                                 C.c_int, P, P, P, P, P]
            lib.orc_sample.argtypes = [P, C.c_int, C.c_uint64, C.c_uint64, C.c_int, P, P]
            lib.orc_expect_z.argtypes = [P, C.c_int, C.c_int, P, P]
            lib.orc_readout.argtypes = [P, C.c_int, C.c_int, P, C.c_uint64, C.c_uint64]
            lib.orc_density_evolve.argtypes = [P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class FlatCircuit:
    """A qtsynth Circuit flattened into the oracle's arrays."""

    def __init__(self, circ):
        ops = circ.ops
        self.circ = circ
        self.n = circ.num_qubits
        self.kind = np.array([o.kind for o in ops], dtype=np.int32)
        self.nq = np.array([len(o.qubits) for o in ops], dtype=np.int32)
        self.qoff = np.zeros(len(ops), dtype=np.int32)
        self.nmat = np.array([o.mats.shape[0] for o in ops], dtype=np.int32)
        self.moff = np.zeros(len(ops), dtype=np.int64)
        self.poff = np.zeros(len(ops), dtype=np.int64)
        qs, ms, ps = [], [], []
        qo = mo = po = 0
        for i, o in enumerate(ops):
            self.qoff[i] = qo
            self.moff[i] = mo
            self.poff[i] = po
            qs.extend(o.qubits)
            qo += len(o.qubits)
            ms.append(np.ascontiguousarray(o.mats, dtype=np.complex128).ravel())
            mo += o.mats.size
            if o.probs is not None:
                ps.extend(list(o.probs))
                po += len(o.probs)
        self.qubits = np.array(qs if qs else [0], dtype=np.int32)
        self.mats = np.concatenate(ms) if ms else np.zeros(1, np.complex128)
        self.probs = np.array(ps if ps else [0.0], dtype=np.float64)
        self.num_channels = int(np.sum(self.kind != 0))
        self.s = _Circ(self.n, len(ops), _ptr(self.kind), _ptr(self.nq), _ptr(self.qoff),
                       _ptr(self.qubits), _ptr(self.nmat), _ptr(self.moff), _ptr(self.mats),
                       _ptr(self.poff), _ptr(self.probs))

    @property
    def ref(self):
        return C.byref(self.s)


def _flat(circ):
    return circ if isinstance(circ, FlatCircuit) else FlatCircuit(circ)


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(seed, traj, stream, index):
    return _load().orc_u01(seed, traj, stream, index)


def apply(psi, qubits, U):
    """In place: Alg. 1 on a complex128 state."""
    lib = _load()
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    n = int(psi.size).bit_length() - 1
    q = np.asarray(qubits, dtype=np.int32)
    U = np.ascontiguousarray(U, dtype=np.complex128)
    lib.orc_apply(_ptr(psi), n, len(q), _ptr(q), _ptr(U))
    return psi


def norm2(psi):
    n = int(psi.size).bit_length() - 1
    return _load().orc_norm2(_ptr(psi), n)


def kraus_norms(psi, qubits, Ks):
    lib = _load()
    n = int(psi.size).bit_length() - 1
    q = np.asarray(qubits, dtype=np.int32)
    Ks = np.ascontiguousarray(Ks, dtype=np.complex128)
    P = np.zeros(Ks.shape[0])
    lib.orc_kraus_norms(_ptr(psi), n, len(q), _ptr(q), Ks.shape[0], _ptr(Ks), _ptr(P))
    return P


def lower_bound(K):
    K = np.ascontiguousarray(K, dtype=np.complex128)
    q = int(K.shape[0]).bit_length() - 1
    return _load().orc_lower_bound(q, _ptr(K))


def run_trajectory(circ, mode=DELAYED, seed=0, traj=0, max_ops=-1, psi=None):
    """One trajectory; returns dict(state, kraus_idx, stage, margin, flushes)."""
    lib = _load()
    fc = _flat(circ)
    if psi is None:
        psi = np.empty(1 << fc.n, dtype=np.complex128)
    nch = max(fc.num_channels, 1)
    ki = np.full(nch, -1, dtype=np.int32)
    st = np.zeros(nch, dtype=np.int32)
    mg = np.zeros(nch, dtype=np.float64)
    f = lib.orc_run_trajectory(fc.ref, mode, seed, traj, max_ops, _ptr(psi),
                               _ptr(ki), _ptr(st), _ptr(mg))
    k = fc.num_channels
    return dict(state=psi, kraus_idx=ki[:k], stage=st[:k], margin=mg[:k], flushes=f)


def run_trajectories(circ, T, mode=DELAYED, seed=0, traj0=0, keep_states=True):
    lib = _load()
    fc = _flat(circ)
    nch = max(fc.num_channels, 1)
    psis = np.empty((T, 1 << fc.n), dtype=np.complex128) if keep_states else None
    ki = np.full((T, nch), -1, dtype=np.int32)
    st = np.zeros((T, nch), dtype=np.int32)
    mg = np.zeros((T, nch), dtype=np.float64)
    fl = np.zeros(T, dtype=np.int32)
    lib.orc_run_trajectories(fc.ref, mode, seed, traj0, T, _ptr(psis), _ptr(ki), _ptr(st),
                             _ptr(mg), _ptr(fl))
    k = fc.num_channels
    return dict(states=psis, kraus_idx=ki[:, :k], stage=st[:, :k], margin=mg[:, :k],
                flushes=fl)


def sample(psi, seed, traj, S):
    lib = _load()
    n = int(psi.size).bit_length() - 1
    out = np.zeros(max(S, 1), dtype=np.uint64)
    mg = np.zeros(max(S, 1), dtype=np.float64)
    lib.orc_sample(_ptr(psi), n, seed, traj, S, _ptr(out), _ptr(mg))
    return out[:S], mg[:S]


def readout(bits, n, err, seed, traj):
    """Readout errors (Sec. V.A) applied to sampled bitstrings: err is [n, 2] with
    err[q] = (P(read 1 | 0), P(read 0 | 1)).  Returns a new array."""
    lib = _load()
    out = np.ascontiguousarray(np.array(bits, dtype=np.uint64, copy=True))
    e = np.ascontiguousarray(np.asarray(err, dtype=np.float64).reshape(n, 2))
    if out.size:
        lib.orc_readout(_ptr(out), int(out.size), n, _ptr(e), seed, traj)
    return out


def expect_z(psi, masks):
    lib = _load()
    n = int(psi.size).bit_length() - 1
    m = np.asarray(masks, dtype=np.uint64)
    out = np.zeros(max(len(m), 1))
    lib.orc_expect_z(_ptr(psi), n, len(m), _ptr(m), _ptr(out))
    return out[:len(m)]


def density_evolve(circ):
    lib = _load()
    fc = _flat(circ)
    assert fc.n <= 7
    rho = np.empty(1 << (2 * fc.n), dtype=np.complex128)
    lib.orc_density_evolve(fc.ref, _ptr(rho))
    # element (r, c) at r + c*2^n  ->  matrix [r, c]
    return rho.reshape(1 << fc.n, 1 << fc.n).T.copy()
