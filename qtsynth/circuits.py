"""Seeded noisy random circuits shaped like the paper's workloads.

Conventions (shared by every consumer of these inputs):

* An ``Op`` acts on ``qubits`` (q of them).  Its matrices are 2^q x 2^q,
  complex128, and bit ``b`` of a row/column index is the value of qubit
  ``qubits[b]`` (little-endian, the paper's "low qubit = low index" view of
  Sec. III.C).
* Amplitude index bit ``j`` of a state vector is qubit ``j``.
* ``KIND_GATE`` ops carry one unitary; ``KIND_KRAUS`` ops carry the Kraus
  operators K_i of a channel (sum K_i^dag K_i = I, Sec. III.E);
  ``KIND_MIXTURE`` ops carry unitaries U_i and probabilities p_i, i.e. the
  mixed-unitary channel with K_i = sqrt(p_i) U_i (Sec. II).
* ``moment`` groups ops that act during one time slice on disjoint qubits
  (Sec. II).

Gate set: sqrt(X), sqrt(Y), sqrt(W) are the det-1 rotations (I - iP)/sqrt(2)
for P = X, Y and W = (X+Y)/sqrt(2); the paper names them without matrices.
Noise channels: amplitude and phase damping are the T_phi -> inf and
T_1 -> inf cases of the decay/dephasing channel of Sec. V.B, depolarizing is
the Pauli mixture of Sec. V.B with D = 2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

KIND_GATE = 0
KIND_KRAUS = 1
KIND_MIXTURE = 2

_S2 = 1.0 / math.sqrt(2.0)
I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = _S2 * np.array([[1, 1], [1, -1]], dtype=np.complex128)
SQRT_X = _S2 * np.array([[1, -1j], [-1j, 1]], dtype=np.complex128)
SQRT_Y = _S2 * np.array([[1, -1], [1, 1]], dtype=np.complex128)
SQRT_W = _S2 * np.array([[1, np.exp(-0.75j * np.pi)],
                         [np.exp(-0.25j * np.pi), 1]], dtype=np.complex128)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
# control = qubits[0] (index bit 0), target = qubits[1] (index bit 1)
CNOT = np.zeros((4, 4), dtype=np.complex128)
CNOT[0, 0] = CNOT[3, 1] = CNOT[2, 2] = CNOT[1, 3] = 1.0
SWAP = np.zeros((4, 4), dtype=np.complex128)
SWAP[0, 0] = SWAP[2, 1] = SWAP[1, 2] = SWAP[3, 3] = 1.0

GATE_SET = (SQRT_X, SQRT_Y, SQRT_W)


@dataclass
class Op:
    kind: int
    qubits: tuple
    mats: np.ndarray                 # [num_ops, 2^q, 2^q] complex128
    probs: Optional[np.ndarray] = None   # [num_ops] for KIND_MIXTURE
    moment: int = 0

    @property
    def num_qubits(self) -> int:
        return len(self.qubits)

    @property
    def num_ops(self) -> int:
        return int(self.mats.shape[0])


@dataclass
class Circuit:
    num_qubits: int
    ops: List[Op] = field(default_factory=list)
    name: str = ""

    def gate(self, U, qubits, moment):
        U = np.asarray(U, dtype=np.complex128)
        self.ops.append(Op(KIND_GATE, tuple(int(q) for q in qubits), U[None].copy(),
                           None, int(moment)))

    def kraus(self, Ks, qubits, moment):
        Ks = np.asarray(Ks, dtype=np.complex128)
        self.ops.append(Op(KIND_KRAUS, tuple(int(q) for q in qubits), Ks.copy(),
                           None, int(moment)))

    def mixture(self, probs, Us, qubits, moment):
        Us = np.asarray(Us, dtype=np.complex128)
        self.ops.append(Op(KIND_MIXTURE, tuple(int(q) for q in qubits), Us.copy(),
                           np.asarray(probs, dtype=np.float64).copy(), int(moment)))

    def channel(self, ch, qubits, moment):
        kind, mats, probs = ch
        if kind == KIND_KRAUS:
            self.kraus(mats, qubits, moment)
        else:
            self.mixture(probs, mats, qubits, moment)

    @property
    def num_channels(self) -> int:
        return sum(1 for o in self.ops if o.kind != KIND_GATE)

    @property
    def num_gates(self) -> int:
        return sum(1 for o in self.ops if o.kind == KIND_GATE)


# --------------------------------------------------------------------------
# channels: (kind, mats, probs)
# --------------------------------------------------------------------------
def amplitude_damping(gamma: float):
    """Amplitude damping: decay channel of Sec. V.B with T_phi -> inf, gamma = 1 - exp(-t/T1)."""
    K0 = np.diag([1.0, math.sqrt(1.0 - gamma)]).astype(np.complex128)
    K1 = np.array([[0.0, math.sqrt(gamma)], [0.0, 0.0]], dtype=np.complex128)
    return (KIND_KRAUS, np.stack([K0, K1]), None)


def phase_damping(lam: float):
    """Phase damping: dephasing channel of Sec. V.B with T1 -> inf, lam = 1 - exp(-2t/T_phi)."""
    K0 = np.diag([1.0, math.sqrt(1.0 - lam)]).astype(np.complex128)
    K1 = np.diag([0.0, math.sqrt(lam)]).astype(np.complex128)
    return (KIND_KRAUS, np.stack([K0, K1]), None)


def depolarizing(p: float, num_qubits: int = 1):
    """Depolarizing channel of Sec. V.B as a Pauli mixture: (1-p) rho + p/(D^2-1) sum P rho P."""
    paulis1 = [I2, X, Y, Z]
    if num_qubits == 1:
        mats = paulis1
    elif num_qubits == 2:
        # index bit 0 <-> qubits[0]: kron(P_b, P_a) acts with P_a on bit 0
        mats = [np.kron(pb, pa) for pb in paulis1 for pa in paulis1]
    else:
        raise ValueError("depolarizing: 1 or 2 qubits")
    D2 = 4 ** num_qubits
    probs = [1.0 - p] + [p / (D2 - 1)] * (D2 - 1)
    return (KIND_MIXTURE, np.stack(mats), np.array(probs))


def decay_dephasing(t: float, T1: float, Tphi: float):
    """Three-operator decay + dephasing channel of Sec. V.B.

    1/T2 = 1/(2 T1) + 1/T_phi.  K0 = diag(1, e^{-t/T2}),
    K1 = [[0, sqrt(1 - e^{-t/T1})], [0, 0]],
    K2 = diag(0, sqrt(e^{-t/T1} - e^{-2t/T2})): the (0,0) entry of K2 as
    printed in the paper (1) breaks completeness; 0 restores it and
    reproduces the channel's closed form.
    """
    T2 = 1.0 / (1.0 / (2.0 * T1) + 1.0 / Tphi)
    a = math.exp(-t / T1)
    b = math.exp(-t / T2)
    K0 = np.diag([1.0, b]).astype(np.complex128)
    K1 = np.array([[0.0, math.sqrt(1.0 - a)], [0.0, 0.0]], dtype=np.complex128)
    K2 = np.diag([0.0, math.sqrt(max(a - b * b, 0.0))]).astype(np.complex128)
    return (KIND_KRAUS, np.stack([K0, K1, K2]), None)


def fsim(theta: float, phi: float):
    """fSim(theta, phi) of Sec. V.B; index bit 0 <-> qubits[0]."""
    U = np.zeros((4, 4), dtype=np.complex128)
    U[0, 0] = 1.0
    U[1, 1] = U[2, 2] = math.cos(theta)
    U[1, 2] = U[2, 1] = -1j * math.sin(theta)
    U[3, 3] = np.exp(-1j * phi)
    return U


def random_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    Q, R = np.linalg.qr(A)
    ph = np.diag(R) / np.abs(np.diag(R))
    return Q * ph[None, :]


def random_kraus(d: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """m random Kraus operators on dimension d (blocks of a random isometry)."""
    V = random_unitary(d * m, rng)[:, :d]
    return np.stack([V[i * d:(i + 1) * d, :] for i in range(m)])


# --------------------------------------------------------------------------
# random circuits shaped like the paper's workloads
# --------------------------------------------------------------------------
def _one_qubit_layer(rng, n, prev):
    """One gate per qubit from {sqrtX, sqrtY, sqrtW}, never the previous layer's gate:
    uniform over the three in the first layer, uniform over the other two after."""
    if prev is None:
        return rng.integers(3, size=n)
    return (prev + 1 + rng.integers(2, size=n)) % 3


def _grid_couplings(rows, cols, n, layer):
    """Cycle horizontal-even, vertical-even, horizontal-odd, vertical-odd couplings."""
    kind = layer % 4
    horizontal = kind in (0, 2)
    parity = 0 if kind in (0, 1) else 1
    pairs = []
    for r in range(rows):
        for c in range(cols):
            a = r * cols + c
            if a >= n:
                continue
            if horizontal and c % 2 == parity and c + 1 < cols:
                b = a + 1
            elif (not horizontal) and r % 2 == parity and r + 1 < rows:
                b = a + cols
            else:
                continue
            if b < n:
                pairs.append((a, b))
    return pairs


def _chain_couplings(n, layer):
    return [(i, i + 1) for i in range(layer % 2, n - 1, 2)]


def _layered_circuit(n, depth, rng, couplings, *, dep1=None, dep2=None,
                     per_gate_ad=None, layer_ad=None, layer_pd=None, name=""):
    """Random-circuit layers: 1q gates, CZ on the layer's couplings, noise.

    dep1 / dep2: depolarizing probability after 1q gates / on each qubit of a
    CZ.  per_gate_ad: amplitude damping after the depolarizing channel of each
    gate-qubit.  layer_ad / layer_pd: damping on every qubit at the end of a
    layer.
    """
    c = Circuit(n, name=name)
    prev = None
    m = 0
    for layer in range(depth):
        choice = _one_qubit_layer(rng, n, prev)
        prev = choice
        for q in range(n):
            c.gate(GATE_SET[choice[q]], (q,), m)
        m += 1
        if dep1 is not None or per_gate_ad is not None:
            if dep1 is not None:
                for q in range(n):
                    c.channel(depolarizing(dep1), (q,), m)
                m += 1
            if per_gate_ad is not None:
                for q in range(n):
                    c.channel(amplitude_damping(per_gate_ad), (q,), m)
                m += 1
        pairs = couplings(layer)
        for (a, b) in pairs:
            c.gate(CZ, (a, b), m)
        m += 1
        touched = sorted({q for p in pairs for q in p})
        if touched and (dep2 is not None or per_gate_ad is not None):
            if dep2 is not None:
                for q in touched:
                    c.channel(depolarizing(dep2), (q,), m)
                m += 1
            if per_gate_ad is not None:
                for q in touched:
                    c.channel(amplitude_damping(per_gate_ad), (q,), m)
                m += 1
        if layer_ad is not None:
            for q in range(n):
                c.channel(amplitude_damping(layer_ad), (q,), m)
            m += 1
        if layer_pd is not None:
            for q in range(n):
                c.channel(phase_damping(layer_pd), (q,), m)
            m += 1
    return c


def chain_circuit(n, depth, seed, **noise):
    rng = np.random.default_rng([0x51, n, depth, seed])
    return _layered_circuit(n, depth, rng, lambda l: _chain_couplings(n, l),
                            name=f"chain{n}x{depth}", **noise)


def grid_circuit(rows, cols, depth, seed, n=None, **noise):
    n = rows * cols if n is None else n
    rng = np.random.default_rng([0x52, rows, cols, n, depth, seed])
    return _layered_circuit(n, depth, rng, lambda l: _grid_couplings(rows, cols, n, l),
                            name=f"grid{rows}x{cols}x{depth}", **noise)


def config0_circuit(seed=0, n=10, depth=16):
    """10-qubit chain, depth 16; depolarizing 1e-3 after 1q gates, 1e-2 on
    each CZ qubit, amplitude damping 1e-3 on every qubit after each layer."""
    return chain_circuit(n, depth, seed, dep1=1e-3, dep2=1e-2, layer_ad=1e-3)


def config1_circuit(seed=0, rows=5, cols=6, depth=20, gamma=5e-4, lam=5e-4,
                    noiseless=False):
    """5x6 grid (30 qubits), depth 20, amplitude + phase damping per qubit per layer."""
    if noiseless:
        return grid_circuit(rows, cols, depth, seed)
    return grid_circuit(rows, cols, depth, seed, layer_ad=gamma, layer_pd=lam)


def config2_circuit(i, depth=40, nmin=8, nmax=18):
    """Circuit i of the batched workload: n_i ~ U{8..18}, chain, depth 40,
    depolarizing 1e-3 then amplitude damping 1e-3 on every gate-qubit."""
    rng = np.random.default_rng([0x53, i])
    n = int(rng.integers(nmin, nmax + 1))
    return _layered_circuit(n, depth, rng, lambda l: _chain_couplings(n, l),
                            dep1=1e-3, dep2=1e-3, per_gate_ad=1e-3,
                            name=f"batch{i}_n{n}")


def config3_circuit(seed=0, rows=4, cols=8, depth=24, p=1e-3):
    """4x8 grid (32 qubits) [2x13 for the error runs], depth 24, depolarizing p per gate-qubit."""
    return grid_circuit(rows, cols, depth, seed, dep1=p, dep2=p)


def serving_requests(num=2000, seed=0, rate=None, nmin=10, nmax=28,
                     dmin=10, dmax=30, tmax=512, samples=100):
    """Request stream: n ~ U{10..28}, depth ~ U{10..30}, chain or grid 50/50,
    p_dep and gamma ~ logU[1e-4, 1e-2], trajectories ~ floor(exp(U[0, ln 513)))
    clipped to 1..512, Poisson arrivals at ``rate`` per second (all at t=0
    when rate is None)."""
    rng = np.random.default_rng([0x54, seed])
    t = 0.0
    reqs = []
    for rid in range(num):
        n = int(rng.integers(nmin, nmax + 1))
        depth = int(rng.integers(dmin, dmax + 1))
        grid = bool(rng.integers(2))
        pdep = float(np.exp(rng.uniform(np.log(1e-4), np.log(1e-2))))
        gam = float(np.exp(rng.uniform(np.log(1e-4), np.log(1e-2))))
        ntraj = int(min(max(int(np.exp(rng.uniform(0.0, np.log(tmax + 1)))), 1), tmax))
        if rate is not None:
            t += float(rng.exponential(1.0 / rate))
        reqs.append(dict(id=rid, arrival=t, n=n, depth=depth, grid=grid,
                         p_dep=pdep, gamma=gam, num_traj=ntraj, samples=samples,
                         seed=rid))
    return reqs


def request_circuit(req):
    """Build the circuit of one serving request (config-0 structure)."""
    n, depth = req["n"], req["depth"]
    noise = dict(dep1=req["p_dep"], dep2=req["p_dep"], layer_ad=req["gamma"])
    if req["grid"]:
        cols = int(math.ceil(math.sqrt(n)))
        rows = int(math.ceil(n / cols))
        return grid_circuit(rows, cols, depth, req["seed"], n=n, **noise)
    return chain_circuit(n, depth, req["seed"], **noise)


# --------------------------------------------------------------------------
# small closed-form circuits and random test circuits
# --------------------------------------------------------------------------
def noise_model_circuit(rows, cols, depth, seed, *, t1q=25e-9, t2q=32e-9, T1=20e-6, Tphi=30e-6,
                        sigma_theta=0.01, sigma_phi=0.02, sigma_z=0.01, p1=1e-3, p2=5e-3,
                        p00=0.01, p11=0.04):
    """The approximate hardware noise model of Sec. V.B on a rows x cols grid,
    with synthetic parameters (no calibration data is used).

    Each layer: one gate per qubit from {sqrtX, sqrtY, sqrtW} (no repeat),
    followed on each qubit by the decay + dephasing channel for the gate
    duration t1q and by 1q depolarizing p1; then fSim(pi/2, pi/6) on the
    layer's grid couplings, each with Z phase errors exp(i a Z) before and
    after on both qubits, the coherent error fSim(dtheta, dphi) after it,
    the decay + dephasing channel for t2q on both qubits, and 2q
    depolarizing p2 (the D = 4 Pauli mixture).  The coherent error angles
    are drawn once per coupling (normal, sigma_theta / sigma_phi), the Z
    phases once per coupling and qubit (normal, sigma_z).

    Returns (circuit, readout) with readout [n, 2] = (p00 error, p11 error)
    per qubit, drawn around p00 and p11 (the p11 error is the larger, as
    the paper expects from decay during measurement)."""
    n = rows * cols
    rng = np.random.default_rng([0x57, rows, cols, depth, seed])
    c = Circuit(n, name=f"noise_model{rows}x{cols}x{depth}")
    coh = {}
    prev = None
    m = 0

    def rz(a):
        return np.diag([np.exp(1j * a), np.exp(-1j * a)]).astype(np.complex128)

    for layer in range(depth):
        choice = _one_qubit_layer(rng, n, prev)
        prev = choice
        for q in range(n):
            c.gate(GATE_SET[choice[q]], (q,), m)
        m += 1
        for q in range(n):
            c.channel(decay_dephasing(t1q, T1, Tphi), (q,), m)
        m += 1
        for q in range(n):
            c.channel(depolarizing(p1), (q,), m)
        m += 1
        pairs = _grid_couplings(rows, cols, n, layer)
        for (a, b) in pairs:
            if (a, b) not in coh:
                coh[(a, b)] = (rng.normal(0.0, sigma_theta), rng.normal(0.0, sigma_phi),
                               rng.normal(0.0, sigma_z, 4))
        for (a, b) in pairs:
            z = coh[(a, b)][2]
            c.gate(rz(z[0]), (a,), m)
            c.gate(rz(z[1]), (b,), m)
        m += 1
        for (a, b) in pairs:
            c.gate(fsim(np.pi / 2, np.pi / 6), (a, b), m)
        m += 1
        for (a, b) in pairs:
            dth, dph, _ = coh[(a, b)]
            c.gate(fsim(dth, dph), (a, b), m)
        m += 1
        for (a, b) in pairs:
            z = coh[(a, b)][2]
            c.gate(rz(z[2]), (a,), m)
            c.gate(rz(z[3]), (b,), m)
        m += 1
        touched = sorted({q for p in pairs for q in p})
        for q in touched:
            c.channel(decay_dephasing(t2q, T1, Tphi), (q,), m)
        m += 1
        for (a, b) in pairs:
            c.channel(depolarizing(p2, 2), (a, b), m)
        m += 1
    readout = np.stack([np.clip(rng.normal(p00, p00 / 4, n), 0.0, 1.0),
                        np.clip(rng.normal(p11, p11 / 4, n), 0.0, 1.0)], axis=1)
    return c, readout


def ghz_circuit(n):
    c = Circuit(n, name=f"ghz{n}")
    c.gate(H, (0,), 0)
    for q in range(n - 1):
        c.gate(CNOT, (q, q + 1), q + 1)
    return c


def qft_circuit(n, basis_state=0):
    """X gates preparing |basis_state>, then the QFT with output bit j on qubit j."""
    c = Circuit(n, name=f"qft{n}")
    m = 0
    for q in range(n):
        if (basis_state >> q) & 1:
            c.gate(X, (q,), m)
    m += 1
    for j in range(n - 1, -1, -1):
        c.gate(H, (j,), m)
        m += 1
        for mq in range(j - 1, -1, -1):
            theta = math.pi / (2 ** (j - mq))
            c.gate(np.diag([1, 1, 1, np.exp(1j * theta)]), (mq, j), m)
            m += 1
    for j in range(n // 2):
        c.gate(SWAP, (j, n - 1 - j), m)
    return c


def random_noisy_circuit(n, num_ops, seed, *, max_gate_qubits=3, noise=0.05,
                         channel_prob=0.4, channel_kinds=("ad", "pd", "dep", "dd", "rk", "dep2")):
    """Random gates on random qubit subsets interleaved with random channels."""
    rng = np.random.default_rng([0x55, n, num_ops, seed])
    c = Circuit(n, name=f"rand{n}_{num_ops}_{seed}")
    latest = [-1] * n

    def place(qs):
        m = max(latest[q] for q in qs) + 1
        for q in qs:
            latest[q] = m
        return m

    for _ in range(num_ops):
        if rng.random() < channel_prob:
            kind = channel_kinds[rng.integers(len(channel_kinds))]
            if kind == "dep2" and n >= 2:
                qs = tuple(int(x) for x in rng.choice(n, 2, replace=False))
                ch = depolarizing(noise * rng.random(), 2)
            else:
                qs = (int(rng.integers(n)),)
                g = noise * (0.2 + rng.random())
                if kind == "ad":
                    ch = amplitude_damping(g)
                elif kind == "pd":
                    ch = phase_damping(g)
                elif kind == "dep" or kind == "dep2":
                    ch = depolarizing(g)
                elif kind == "dd":
                    ch = decay_dephasing(1.0, 1.0 / g, 2.0 / g)
                else:
                    ch = (KIND_KRAUS, random_kraus(2, 2 + int(rng.integers(2)), rng), None)
            c.channel(ch, qs, place(qs))
        else:
            q = int(rng.integers(1, min(max_gate_qubits, n) + 1))
            qs = tuple(int(x) for x in rng.choice(n, q, replace=False))
            c.gate(random_unitary(2 ** q, rng), qs, place(qs))
    # a circuit is a sequence of moments: list ops moment by moment (stable,
    # so ops sharing a qubit keep their order)
    c.ops.sort(key=lambda o: o.moment)
    return c
