"""Array form of the layered random circuits, for workloads with thousands of circuits.

Builds exactly the op sequence of ``circuits._layered_circuit`` (same random
draws, same order, same moments) as flat arrays plus a small table of
distinct operators, without creating one Python object per op.  Like the
rest of qtsynth it only builds inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import circuits as C


@dataclass
class CompactCircuit:
    num_qubits: int
    kind: np.ndarray       # [ops] int32
    nq: np.ndarray         # [ops] int32 (1 or 2)
    qubits: np.ndarray     # [ops, 2] int32 (second entry unused for 1-qubit ops)
    moment: np.ndarray     # [ops] int32
    table_id: np.ndarray   # [ops] int32 into `table`
    table: List[tuple] = field(default_factory=list)   # (kind, mats, probs)
    name: str = ""

    @property
    def num_ops(self):
        return int(self.kind.size)

    @property
    def num_channels(self):
        return int(np.sum(self.kind != C.KIND_GATE))

    def to_circuit(self) -> C.Circuit:
        c = C.Circuit(self.num_qubits, name=self.name)
        for i in range(self.num_ops):
            kind, mats, probs = self.table[self.table_id[i]]
            qs = tuple(int(q) for q in self.qubits[i, :self.nq[i]])
            c.ops.append(C.Op(kind, qs, mats, probs, int(self.moment[i])))
        return c


class _Builder:
    def __init__(self):
        self.table = []
        self.index = {}
        self.kind, self.q0, self.q1, self.moment, self.tid_ = [], [], [], [], []

    def tid(self, key, make):
        t = self.index.get(key)
        if t is None:
            t = self.index[key] = len(self.table)
            self.table.append(make())
        return t

    def add1(self, kind, qubits, moment, tids):
        k = len(qubits)
        self.kind.extend([kind] * k)
        self.q0.extend(qubits)
        self.q1.extend([-1] * k)
        self.moment.extend([moment] * k)
        self.tid_.extend(tids if isinstance(tids, list) else [tids] * k)

    def add2(self, kind, pairs, moment, tid):
        k = len(pairs)
        self.kind.extend([kind] * k)
        self.q0.extend(p[0] for p in pairs)
        self.q1.extend(p[1] for p in pairs)
        self.moment.extend([moment] * k)
        self.tid_.extend([tid] * k)

    def build(self, n, name):
        q1 = np.asarray(self.q1, np.int32)
        qubits = np.stack([np.asarray(self.q0, np.int32), np.maximum(q1, 0)], axis=1)
        nq = np.where(q1 >= 0, 2, 1).astype(np.int32)
        return CompactCircuit(n, np.asarray(self.kind, np.int32), nq, qubits,
                              np.asarray(self.moment, np.int32), np.asarray(self.tid_, np.int32),
                              self.table, name)


def layered_compact(n, depth, rng, couplings, *, dep1=None, dep2=None, per_gate_ad=None,
                    layer_ad=None, layer_pd=None, name=""):
    """Same ops, order and random draws as circuits._layered_circuit."""
    b = _Builder()
    gate_tid = [b.tid(("g", g), lambda g=g: (C.KIND_GATE, C.GATE_SET[g][None].copy(), None))
                for g in range(3)]
    cz_tid = b.tid(("cz",), lambda: (C.KIND_GATE, C.CZ[None].copy(), None))

    def ch_tid(key, fn, p):
        return b.tid((key, p), lambda: fn(p))

    allq = list(range(n))
    prev = None
    m = 0
    for layer in range(depth):
        choice = C._one_qubit_layer(rng, n, prev)
        prev = choice
        b.add1(C.KIND_GATE, allq, m, [gate_tid[c] for c in choice.tolist()])
        m += 1
        if dep1 is not None or per_gate_ad is not None:
            if dep1 is not None:
                b.add1(C.KIND_MIXTURE, allq, m, ch_tid("dep", C.depolarizing, dep1))
                m += 1
            if per_gate_ad is not None:
                b.add1(C.KIND_KRAUS, allq, m, ch_tid("ad", C.amplitude_damping, per_gate_ad))
                m += 1
        pairs = couplings(layer)
        if pairs:
            b.add2(C.KIND_GATE, pairs, m, cz_tid)
        m += 1
        touched = sorted({q for p in pairs for q in p})
        if touched and (dep2 is not None or per_gate_ad is not None):
            if dep2 is not None:
                b.add1(C.KIND_MIXTURE, touched, m, ch_tid("dep", C.depolarizing, dep2))
                m += 1
            if per_gate_ad is not None:
                b.add1(C.KIND_KRAUS, touched, m, ch_tid("ad", C.amplitude_damping, per_gate_ad))
                m += 1
        if layer_ad is not None:
            b.add1(C.KIND_KRAUS, allq, m, ch_tid("ad", C.amplitude_damping, layer_ad))
            m += 1
        if layer_pd is not None:
            b.add1(C.KIND_KRAUS, allq, m, ch_tid("pd", C.phase_damping, layer_pd))
            m += 1
    return b.build(n, name)


def config2_compact(i, depth=40, nmin=8, nmax=18):
    """Array form of circuits.config2_circuit(i)."""
    rng = np.random.default_rng([0x53, i])
    n = int(rng.integers(nmin, nmax + 1))
    return layered_compact(n, depth, rng, lambda l: C._chain_couplings(n, l),
                           dep1=1e-3, dep2=1e-3, per_gate_ad=1e-3, name=f"batch{i}_n{n}")


def request_compact(req):
    """Array form of circuits.request_circuit(req)."""
    import math
    n, depth = req["n"], req["depth"]
    noise = dict(dep1=req["p_dep"], dep2=req["p_dep"], layer_ad=req["gamma"])
    if req["grid"]:
        cols = int(math.ceil(math.sqrt(n)))
        rows = int(math.ceil(n / cols))
        rng = np.random.default_rng([0x52, rows, cols, n, depth, req["seed"]])
        return layered_compact(n, depth, rng, lambda l: C._grid_couplings(rows, cols, n, l),
                               name=f"grid{rows}x{cols}x{depth}", **noise)
    rng = np.random.default_rng([0x51, n, depth, req["seed"]])
    return layered_compact(n, depth, rng, lambda l: C._chain_couplings(n, l),
                           name=f"chain{n}x{depth}", **noise)
