"""GPU checks at the full 30-qubit size, in the benchmark's launch configuration.

The FP64 oracle cannot run the whole 30-qubit workload in a test, so these
checks use outputs it can compute one by one, or properties that hold at
any size:
  * one fused 4-qubit gate on a seeded 2^30 state: sampled output
    amplitudes against the oracle applied to their 16-amplitude gather set;
  * a 30-qubit circuit made of six independent 5-qubit blocks (qubits
    interleaved across the index bits, fused to 4 qubits by the library):
    sampled amplitudes against the product of the six block states from
    the oracle, and the samples of that state against the oracle's exact
    per-block distributions (per-qubit marginals and a chi-square per block);
  * the 30-qubit 5x6 grid workload with damping: every stage-1 branch
    record equals the decision the oracle's own Philox draws and lower
    bounds give; flushes happen exactly where stage 1 cannot decide; as a
    consistency check of two different kernels, the sampled bitstrings'
    per-qubit frequencies agree with <Z_j> of the same final states;
  * opt-in (QT_FULL_ORACLE=1, about ten minutes of FP64 on the host cores):
    one whole trajectory of that workload, oracle against library.
"""
import os
import time

import numpy as np
import pytest

import qtsynth as qs
from gpu_util import KERNEL_L2, MARGIN, STATE_FID, STATE_L2, torch_cuda

pytestmark = pytest.mark.gpu
N = 30


@pytest.fixture(scope="module")
def qt():
    import paper_2111_02396_gb300 as pkg
    pkg.load()
    torch_cuda()
    return pkg


def test_single_gate_sampled_outputs(qt, orc):
    torch = torch_cuda()
    g = torch.Generator(device="cuda").manual_seed(1234)
    d = torch.randn(2 << N, device="cuda", generator=g, dtype=torch.float32).view(torch.complex64)
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 1 << N, 3000)
    for qubits in ([29, 3, 17, 8], [0, 1, 2, 3], [0, 29, 28, 14], [5, 6, 7, 8]):
        U = qs.random_unitary(16, rng)
        before = d.clone()
        qt.qt_state_apply(d.data_ptr(), N, qubits, U)
        mask = sum(1 << q for q in qubits)
        idx = []
        for x in xs:
            base = int(x) & ~mask
            idx.append([base | sum(((m >> b) & 1) << q for b, q in enumerate(qubits))
                        for m in range(16)])
        idx = torch.tensor(np.array(idx), device="cuda")
        vin = before[idx].cpu().numpy().astype(np.complex128)          # [S, 16] gather sets
        vout = d[idx].cpu().numpy().astype(np.complex128)
        want = np.stack([orc.apply(v.copy(), [0, 1, 2, 3], U) for v in vin])
        err = np.linalg.norm(vout - want) / np.linalg.norm(want)
        assert err < KERNEL_L2, (qubits, err)
        del before


def block_circuit(seed=0, blocks=6, width=5, depth=12):
    """Independent 5-qubit random circuits on qubits {b, b+6, b+12, ...}."""
    rng = np.random.default_rng([0x99, seed])
    n = blocks * width
    c = qs.Circuit(n)
    sub = []
    for b in range(blocks):
        qs_b = [b + blocks * j for j in range(width)]
        s = qs.Circuit(width)
        for layer in range(depth):
            for j in range(width):
                s.gate(qs.random_unitary(2, rng), (j,), 2 * layer)
            for j in range(layer % 2, width - 1, 2):
                s.gate(qs.CZ, (j, j + 1), 2 * layer + 1)
        sub.append((qs_b, s))
    m = 0
    for layer_ops in range(max(len(s.ops) for _, s in sub)):
        for qs_b, s in sub:
            if layer_ops < len(s.ops):
                o = s.ops[layer_ops]
                c.gate(o.mats[0], tuple(qs_b[j] for j in o.qubits), m)
        m += 1
    return c, sub


def test_block_product_circuit_sampled_amplitudes(qt, orc):
    circ, sub = block_circuit()
    qc = qt.Circuit.from_synth(circ)
    run = qt.Run(qt.Fused(qc, 4), 1, keep_states=True, samples_per_traj=2000)
    psi = run.state(0)
    states = [(qs_b, orc.run_trajectory(s)["state"]) for qs_b, s in sub]
    rng = np.random.default_rng(1)
    # uniform indices plus sampled ones (drawn from |psi|^2: the large amplitudes)
    xs = np.concatenate([rng.integers(0, 1 << N, 20000), run.samples()[0].astype(np.int64)])
    want = np.ones(len(xs), dtype=np.complex128)
    for qs_b, st in states:
        loc = np.zeros(len(xs), dtype=np.int64)
        for j, q in enumerate(qs_b):
            loc |= ((xs >> q) & 1) << j
        want *= st[loc]
    got = psi[xs].astype(np.complex128)
    # relative L2 over the sample, scaled by the state's norm density
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < STATE_L2, err
    # The sampled bitstrings against the oracle's exact distribution: the blocks
    # are independent, so the 5 bits of block b in a sample follow |st_b|^2,
    # and qubit q_j of block b is 1 with probability sum_{loc: bit j} |st_b[loc]|^2.
    smp = run.samples()[0].astype(np.int64)
    S = smp.size
    for qs_b, st in states:
        p = np.abs(st) ** 2
        p /= p.sum()
        loc = np.zeros(S, dtype=np.int64)
        for j, q in enumerate(qs_b):
            loc |= ((smp >> q) & 1) << j
            p1 = p[(np.arange(p.size) >> j) & 1 == 1].sum()
            freq = ((smp >> q) & 1).mean()
            se = np.sqrt(max(p1 * (1 - p1), 1e-4) / S)
            assert abs(freq - p1) < 5 * se, (q, freq, p1)
        # chi-square over the 32 outcomes of the block (outcomes expected fewer
        # than 5 times pooled into one bin)
        cnt = np.bincount(loc, minlength=p.size).astype(np.float64)
        exp = p * S
        big = exp >= 5
        obs_b = np.append(cnt[big], cnt[~big].sum())
        exp_b = np.append(exp[big], exp[~big].sum())
        keep = exp_b > 0
        chi2 = float(np.sum((obs_b[keep] - exp_b[keep]) ** 2 / exp_b[keep]))
        dof = int(keep.sum()) - 1
        # 1e-6 tail of chi-square by the Wilson-Hilferty normal approximation
        # (z = 4.75), so the 6 blocks fail together with probability < 1e-5
        crit = dof * (1 - 2 / (9 * dof) + 4.75 * np.sqrt(2 / (9 * dof))) ** 3
        assert chi2 < crit, (qs_b, chi2, crit)


def test_grid30_branch_records_and_marginals(qt, orc):
    circ = qs.config1_circuit()
    qc = qt.Circuit.from_synth(circ)
    f = qt.Fused(qc, 4)
    T, S = 2, 4000
    masks = [1 << j for j in range(N)]
    run = qt.Run(f, T, seed=0, samples_per_traj=S, z_masks=masks)
    kr, st = run.kraus_indices()
    # stage-1 decisions from the oracle's draws and lower bounds
    chans = [o for o in circ.ops if o.kind != qs.KIND_GATE]
    lbs = [[orc.lower_bound(K) for K in o.mats] for o in chans[:2]]   # AD and PD types
    lb_by_kind = {}
    for o in chans:
        key = (o.mats.shape[0], o.mats[1, 0, 1] != 0)   # AD has an off-diagonal K1
        if key not in lb_by_kind:
            lb_by_kind[key] = [orc.lower_bound(K) for K in o.mats]
    flushes = 0
    for t in range(T):
        for ch, o in enumerate(chans):
            lb = lb_by_kind[(o.mats.shape[0], o.mats[1, 0, 1] != 0)]
            r = orc.u01(0, t, 0, ch)
            if r < lb[0]:
                assert kr[t, ch] == 0 and st[t, ch] == 1
            else:
                assert st[t, ch] == 2
                flushes += 1
    assert run.stats()["flushes"] == flushes
    # sampled marginals vs <Z_j> of the same states
    smp = run.samples()
    z = run.expectation()
    for t in range(T):
        bits = ((smp[t][:, None] >> np.arange(N, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.float64)
        p1 = (1 - z[t]) / 2
        se = np.sqrt(np.maximum(p1 * (1 - p1), 1e-4) / S)
        assert np.all(np.abs(bits.mean(0) - p1) < 5 * se)
    assert lbs  # lower bounds were evaluated by the oracle


def _chunked_l2_fidelity(g, ref, chunk=1 << 26):
    """Relative L2 distance and fidelity of complex64 g against complex128 ref,
    a slice at a time (2^30 amplitudes do not fit comfortably in temporaries)."""
    diff = nref = ng = 0.0
    dot = 0j
    for i in range(0, ref.size, chunk):
        a = g[i:i + chunk].astype(np.complex128)
        b = ref[i:i + chunk]
        diff += float(np.sum(np.abs(a - b) ** 2))
        nref += float(np.sum(np.abs(b) ** 2))
        ng += float(np.sum(np.abs(a) ** 2))
        dot += np.vdot(b, a)
    return float(np.sqrt(diff / nref)), float(abs(dot) ** 2 / (ng * nref))


@pytest.mark.skipif(os.environ.get("QT_FULL_ORACLE") != "1",
                    reason="one whole 30-qubit FP64 oracle trajectory takes about ten minutes "
                           "(QT_FULL_ORACLE=1 runs it)")
def test_grid30_full_trajectory_against_oracle(qt, orc):
    """Trajectory 0 of the 30-qubit grid workload end to end: the FP64 oracle's
    whole unfused trajectory against the library's plain loop in the benchmark's
    configuration (fused k = 4, delayed inner products, 100 samples).  Every
    branch record where the oracle's margin exceeds 1e-6, the final state
    (relative L2, fidelity), the samples where the CDF margin exceeds 1e-6 and,
    for the others, the oracle's CDF neighbourhood of their targets.
    Prints the oracle's wall time for the whole trajectory, the figure that the
    benchmark's CPU baseline extrapolates from a prefix of the ops."""
    circ = qs.config1_circuit()
    f = qt.Fused(qt.Circuit.from_synth(circ), 4)
    S = 100
    run = qt.Run(f, 1, seed=0, first_traj=0, samples_per_traj=S, keep_states=True)
    kr, st = run.kraus_indices()
    smp = run.samples()[0]
    g = run.state(0)
    del run
    t0 = time.perf_counter()
    ref = orc.run_trajectory(circ, orc.DELAYED, seed=0, traj=0)
    t_traj = time.perf_counter() - t0
    t0 = time.perf_counter()
    want, margin = orc.sample(ref["state"], 0, 0, S)
    t_smp = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    print(f"\noracle, whole trajectory 0 of the 30-qubit grid workload ({len(circ.ops)} ops): "
          f"{t_traj:.1f} s + {S} samples {t_smp:.1f} s on {cores} cores = "
          f"{1.0 / (t_traj + t_smp):.6f} trajectories/s")
    # records up to the first tie (after a tie the two may take different branches)
    ties = np.flatnonzero(ref["margin"] <= MARGIN)
    first = int(ties[0]) if ties.size else ref["margin"].size
    assert np.array_equal(kr[0][:first], ref["kraus_idx"][:first])
    assert np.array_equal(st[0][:first], ref["stage"][:first])
    if ties.size:
        pytest.skip(f"branch tie at channel {first}: records compared up to it")
    l2, fid = _chunked_l2_fidelity(g, ref["state"])
    print(f"branch records compared: {first} (stage 2: {int((ref['stage'] == 2).sum())}); "
          f"state relative L2 {l2:.3e}, fidelity 1 - {1 - fid:.2e}; "
          f"samples compared: {int((margin > MARGIN).sum())} of {S}")
    assert l2 <= STATE_L2 and fid >= 1 - STATE_FID
    np.testing.assert_array_equal(smp[margin > MARGIN], want[margin > MARGIN])
    # At 2^30 amplitudes each probability is ~1e-9, so nearly every sample is a
    # tie by the 1e-6 margin.  Those must lie in the oracle's CDF neighbourhood
    # of their target u * C(2^n - 1): [C(x - 1) - delta, C(x) + delta].  delta
    # bounds |C_gpu - C_oracle|: the sampler's own rounding (FP32 squares, runs
    # of at most 1024 terms, FP64 across runs: 32 * 2^-24, as the sampler tests
    # check) plus the state difference, sum_y ||g_y|^2 - |r_y|^2| <= l2 (2 + l2).
    tie = margin <= MARGIN
    if tie.any():
        co = np.cumsum(np.abs(ref["state"]) ** 2)
        delta = 32 * 2.0 ** -24 * co[-1] + l2 * (2 + l2) * co[-1]
        u = np.array([orc.u01(0, 0, 1, j) for j in range(S)])
        t = u[tie] * co[-1]
        x = smp[tie].astype(np.int64)
        below = np.where(x > 0, co[np.maximum(x - 1, 0)], 0.0)
        print(f"ties checked against the oracle's CDF neighbourhood: {int(tie.sum())} (delta {delta:.2e}); "
              f"largest distance of a target outside its sample's CDF interval: "
              f"{float(max(np.max(below - t), np.max(t - co[x]), 0.0)):.2e}")
        assert np.all(t >= below - delta), np.min(t - below + delta)
        assert np.all(t <= co[x] + delta), np.min(co[x] + delta - t)
