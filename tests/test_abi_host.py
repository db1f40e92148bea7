"""Host-side checks of libqt.so that need no GPU.

* the library builds for sm_103a, loads, and exports every function that
  include/qt.h declares;
* circuit validation (ranges, moments, unitarity, CPTP, mixture sums);
* the lower bounds pbar_i = sigma_min(K_i)^2 of Sec. III.E against numpy
  and closed forms;
* the fuser of Sec. III.B: widths, coverage, and the dense product of the
  fused gates equals the dense product of the unfused circuit.
"""
import os
import re

import numpy as np
import pytest

import qtsynth as qs
from test_oracle_apply import dense_operator

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qt():
    import paper_2111_02396_gb300 as pkg
    pkg.load()
    return pkg


def header_functions():
    src = open(os.path.join(ROOT, "include", "qt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qt_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(qt):
    lib = qt.load()
    names = header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), f"libqt.so does not export {name}"
    assert set(names) == set(qt.qt.EXPORTS)


def test_library_is_built_for_sm_103a(qt):
    # every translation unit is compiled with exactly one -gencode, for sm_103a
    # (the GPU tests also ask the runtime for the kernels' binary version)
    from paper_2111_02396_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def _circ(n, ops):
    c = qs.Circuit(n)
    c.ops = ops
    return c


def test_readout_errors_are_validated(qt):
    from paper_2111_02396_gb300.qt import QtError, QT_ERR_INVALID_ARG
    f = qt.Fused(qt.Circuit.from_synth(qs.config0_circuit()), 2)
    for bad in (np.full((10, 2), 1.5), np.full((10, 2), -0.1), np.full((10, 2), np.nan)):
        with pytest.raises(QtError) as ei:
            qt.Run(f, 1, samples_per_traj=4, readout_error=bad)
        assert ei.value.status == QT_ERR_INVALID_ARG


def test_validation_errors(qt):
    from paper_2111_02396_gb300.qt import QtError, QT_ERR_INVALID_ARG, QT_ERR_NOT_CPTP
    good = qs.Op(qs.KIND_GATE, (0,), qs.SQRT_X[None], None, 0)
    cases = [
        ([qs.Op(qs.KIND_GATE, (3,), qs.SQRT_X[None], None, 0)], QT_ERR_INVALID_ARG),   # qubit range
        ([good, qs.Op(qs.KIND_GATE, (0,), qs.H[None], None, 0)], QT_ERR_INVALID_ARG),    # moment overlap
        ([qs.Op(qs.KIND_GATE, (1,), (2 * qs.H)[None], None, 0)], QT_ERR_INVALID_ARG),   # not unitary
        ([qs.Op(qs.KIND_KRAUS, (1,), np.stack([qs.I2, qs.X]) * 0.9, None, 0)], QT_ERR_NOT_CPTP),
        ([qs.Op(qs.KIND_MIXTURE, (1,), np.stack([qs.I2, qs.X]), np.array([0.5, 0.6]), 0)],
         QT_ERR_INVALID_ARG),
        ([qs.Op(qs.KIND_GATE, (0, 0), qs.CZ[None], None, 0)], QT_ERR_INVALID_ARG),       # repeated qubit
        ([qs.Op(qs.KIND_GATE, (0,), qs.H[None], None, 2), good], QT_ERR_INVALID_ARG),    # moments decrease
    ]
    for ops, status in cases:
        with pytest.raises(QtError) as ei:
            qt.Circuit(3, ops)
        assert ei.value.status == status
    qt.Circuit(3, [good])   # accepted


@pytest.mark.parametrize("q", [1, 2, 3])
def test_lower_bounds_match_numpy(qt, q):
    rng = np.random.default_rng(q)
    for trial in range(4):
        Ks = qs.circuits.random_kraus(1 << q, 3, rng)
        c = qs.Circuit(q)
        c.kraus(Ks, tuple(range(q)), 0)
        got = qt.Circuit.from_synth(c).lower_bounds(0)
        want = [np.linalg.eigvalsh(K.conj().T @ K).min() for K in Ks]
        np.testing.assert_allclose(got, np.maximum(want, 0), atol=1e-12)


def test_lower_bounds_closed_forms(qt):
    c = qs.Circuit(2)
    c.channel(qs.amplitude_damping(0.3), (0,), 0)
    c.channel(qs.phase_damping(0.2), (1,), 0)
    c.channel(qs.depolarizing(0.01), (0,), 1)
    c.channel(qs.depolarizing(0.05, 2), (0, 1), 2)
    qc = qt.Circuit.from_synth(c)
    np.testing.assert_allclose(qc.lower_bounds(0), [0.7, 0.0], atol=1e-15)
    np.testing.assert_allclose(qc.lower_bounds(1), [0.8, 0.0], atol=1e-15)
    np.testing.assert_allclose(qc.lower_bounds(2), [0.99] + [0.01 / 3] * 3, atol=1e-15)
    lb = qc.lower_bounds(3)
    assert abs(lb.sum() - 1.0) < 1e-14          # mixtures: s = 1


def fused_dense(qt, fused, n):
    info = fused.info()
    D = 1 << n
    M = np.eye(D, dtype=np.complex128)
    seen = []
    for g in range(info["num_fused"]):
        fg = fused.gate(g)
        assert len(fg["targets"]) <= fused_kmax(fused)
        M = dense_operator(n, list(fg["targets"]), fg["matrix"]) @ M
        seen.extend(fg["members"].tolist())
    return M, seen


def fused_kmax(fused):
    return fused._kmax


def circuit_dense(circ, default_slots=True):
    n = circ.num_qubits
    M = np.eye(1 << n, dtype=np.complex128)
    for o in circ.ops:
        if o.kind == qs.KIND_GATE:
            U = o.mats[0]
        else:
            # default slot operator: the largest lower bound (mixtures: largest p)
            if o.kind == qs.KIND_MIXTURE:
                U = o.mats[int(np.argmax(o.probs))]
            else:
                lbs = [np.linalg.eigvalsh(K.conj().T @ K).min() for K in o.mats]
                U = o.mats[int(np.argmax(lbs))]
        M = dense_operator(n, list(o.qubits), U) @ M
    return M


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("seed", [0, 1])
def test_fused_product_equals_circuit(qt, k, seed):
    n = 7
    circ = qs.random_noisy_circuit(n, 60, seed, max_gate_qubits=min(k, 3), channel_prob=0.3,
                                   channel_kinds=("ad", "pd", "dep"))
    qc = qt.Circuit.from_synth(circ)
    f = qt.Fused(qc, k)
    f._kmax = k
    M, seen = fused_dense(qt, f, n)
    assert sorted(seen) == list(range(len(circ.ops)))        # every op exactly once
    want = circuit_dense(circ)
    np.testing.assert_allclose(M, want, atol=1e-11)
    if k >= 3:
        assert f.info()["num_fused"] < len(circ.ops) / 2       # fusion actually merges


def test_fusion_config1_shape(qt):
    circ = qs.config1_circuit(rows=3, cols=3, depth=6)
    qc = qt.Circuit.from_synth(circ)
    f = qt.Fused(qc, 4)
    f._kmax = 4
    M, seen = fused_dense(qt, f, 9)
    np.testing.assert_allclose(M, circuit_dense(circ), atol=1e-11)
    assert f.info()["max_width"] <= 4


def test_fused_members_respect_qubit_order(qt):
    """Within the fused sequence, ops sharing a qubit keep circuit order."""
    circ = qs.random_noisy_circuit(6, 80, 4, max_gate_qubits=2, channel_prob=0.3)
    qc = qt.Circuit.from_synth(circ)
    f = qt.Fused(qc, 4)
    order = []
    for g in range(f.info()["num_fused"]):
        order.extend(f.gate(g)["members"].tolist())
    last = {}
    for pos, i in enumerate(order):
        for q in circ.ops[i].qubits:
            if q in last:
                assert last[q] < i
            last[q] = i


@pytest.mark.parametrize("case", ["grid3x4_k4", "chain10_k3", "random11_k2"])
def test_first_touch_pieces_form_product_state(qt, orc, case):
    """The identity behind the product-state start: the fused gates that act
    first on each of their qubits (none of their qubits touched by an earlier
    gate) take |0...0> to the tensor product of their first columns, with |0>
    on every other qubit, and commute with every gate before them.  Folding
    them first and then applying the other gates in order gives the state of
    the plain sequence (FP64 oracle Alg. 1)."""
    circ, n, k = {
        "grid3x4_k4": (qs.config1_circuit(rows=3, cols=4, depth=8), 12, 4),
        "chain10_k3": (qs.config0_circuit(), 10, 3),
        "random11_k2": (qs.random_noisy_circuit(11, 120, 5, max_gate_qubits=2, channel_prob=0.3), 11, 2),
    }[case]
    f = qt.Fused(qt.Circuit.from_synth(circ), k)
    gates = [f.gate(g) for g in range(f.info()["num_fused"])]
    zero = np.zeros(1 << n, dtype=np.complex128)
    zero[0] = 1.0
    want = zero.copy()
    for d in gates:
        want = orc.apply(want, [int(q) for q in d["targets"]], d["matrix"])
    touched, first = 0, []
    for i, d in enumerate(gates):
        mask = sum(1 << int(q) for q in d["targets"])
        if not mask & touched:
            first.append(i)
        touched |= mask
    assert first
    x = np.arange(1 << n, dtype=np.int64)
    held = 0
    psi = np.ones(1 << n, dtype=np.complex128)
    for i in first:
        tg = [int(q) for q in gates[i]["targets"]]
        j = np.zeros_like(x)
        for b, q in enumerate(tg):
            j |= ((x >> q) & 1) << b
            held |= 1 << q
        psi *= gates[i]["matrix"][j, 0]
    psi[(x & ~held & ((1 << n) - 1)) != 0] = 0.0
    for i, d in enumerate(gates):
        if i not in first:
            psi = orc.apply(psi, [int(q) for q in d["targets"]], d["matrix"])
    np.testing.assert_allclose(psi, want, atol=1e-12)
