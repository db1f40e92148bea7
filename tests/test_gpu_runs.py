"""GPU parity of whole trajectory runs (Alg. 2 and the conventional algorithm).

For the same circuits, seeds and Philox counters as the FP64 oracle:
  * Kraus branch records are equal wherever the draw's margin to the
    nearest partition boundary exceeds 1e-6 (a closer draw is a tie; the
    rest of that trajectory is then not compared);
  * final states agree within relative L2 2e-5 and fidelity 1 - 1e-5;
  * sampled bitstrings are equal where the CDF margin exceeds 1e-6;
  * expectations agree.
Covered: the 10-qubit chain workload (64 trajectories x 100 samples), random
circuits with every channel kind at fusion widths 2..5, delayed and eager
modes, and a 20-qubit grid with noise strong enough to force flushes.
"""
import numpy as np
import pytest

import qtsynth as qs
from gpu_util import MARGIN, STATE_FID, STATE_L2, fidelity, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qt():
    import paper_2111_02396_gb300 as pkg
    pkg.load()
    torch_cuda()
    return pkg


def compare_run(qt, orc, circ, T, *, k, mode, seed=0, S=0, masks=(), check_states=True,
                precision=0, grouping=False, share_prefix=False):
    qc = qt.Circuit.from_synth(circ)
    f = qt.Fused(qc, k)
    run = qt.Run(f, T, seed=seed, mode=mode, samples_per_traj=S, z_masks=masks,
                 keep_states=check_states, precision=precision, grouping=grouping,
                 share_prefix=share_prefix)
    kr, st = run.kraus_indices()
    omode = orc.DELAYED if mode == qt.QT_DELAYED else orc.EAGER
    ref = orc.run_trajectories(circ, T, mode=omode, seed=seed, keep_states=True)
    compared = ties = 0
    samples = run.samples() if S else None
    expv = run.expectation() if len(masks) else None
    for t in range(T):
        tie = False
        for ch in range(kr.shape[1]):
            if ref["margin"][t, ch] <= MARGIN:
                tie = True
                ties += 1
                break
            assert kr[t, ch] == ref["kraus_idx"][t, ch], (t, ch)
            assert st[t, ch] == ref["stage"][t, ch], (t, ch)
        if tie:
            continue
        compared += 1
        psi = ref["states"][t]
        if check_states:
            g = run.state(t)
            assert rel_l2(g, psi) <= STATE_L2, (t, rel_l2(g, psi))
            assert fidelity(g, psi) >= 1 - STATE_FID
        if S:
            want, margin = orc.sample(psi, seed, t, S)
            ok = margin > MARGIN
            np.testing.assert_array_equal(samples[t][ok], want[ok])
        if len(masks):
            np.testing.assert_allclose(expv[t], orc.expect_z(psi, masks), atol=2e-5)
    assert compared >= 0.75 * T, (compared, ties)
    return run, ref


def test_config0_chain10(qt, orc):
    circ = qs.config0_circuit()
    masks = [1 << j for j in range(10)] + [0b1111111111]
    run, ref = compare_run(qt, orc, circ, 64, k=2, mode=qt.QT_DELAYED, S=100, masks=masks)
    st = run.stats()
    assert st["num_traj"] == 64 and st["kernel_launches"] > 0


def test_config0_eager_same_branches(qt, orc):
    circ = qs.config0_circuit()
    compare_run(qt, orc, circ, 16, k=2, mode=qt.QT_EAGER, S=20)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
@pytest.mark.parametrize("mode", ["delayed", "eager"])
def test_random_channels(qt, orc, k, mode):
    m = qt.QT_DELAYED if mode == "delayed" else qt.QT_EAGER
    for seed in range(3):
        circ = qs.random_noisy_circuit(9, 70, 100 + seed, max_gate_qubits=3, noise=0.15,
                                       channel_prob=0.45)
        compare_run(qt, orc, circ, 12, k=k, mode=m, seed=seed, S=50, masks=[1, 6, 0x1ff])


def test_grid20_forced_flushes(qt, orc):
    circ = qs.config1_circuit(rows=4, cols=5, depth=12, gamma=1e-2, lam=1e-2)
    run, ref = compare_run(qt, orc, circ, 4, k=4, mode=qt.QT_DELAYED, S=200,
                           masks=[1 << j for j in range(20)])
    assert run.stats()["flushes"] > 0
    assert run.stats()["flushes"] == int(np.sum(ref["stage"] == 2))


def test_grid_depolarizing_k6_fp32(qt, orc):
    """The same circuit fused to k = 6 on the FP32 CUDA-core path."""
    circ = qs.config3_circuit(rows=2, cols=7, depth=12, p=0.02)
    compare_run(qt, orc, circ, 4, k=6, mode=qt.QT_DELAYED, S=100, precision=qt.QT_FP32)


@pytest.mark.parametrize("k", [5, 6])
def test_grid_depolarizing_tf32x3(qt, orc, k):
    """Depolarizing-only grid circuit (the precision workload's generator at
    n = 14) fused to k = 5, 6 and applied on tensor cores in split-TF32."""
    circ = qs.config3_circuit(rows=2, cols=7, depth=12, p=0.02)
    run, _ = compare_run(qt, orc, circ, 6, k=k, mode=qt.QT_DELAYED, S=100,
                         precision=qt.QT_TF32X3)
    assert run.stats()["flushes"] == 0


@pytest.mark.parametrize("k", [2, 3, 4])
def test_multi_gate_passes_match_oracle(qt, orc, k):
    """Multi-gate passes (several fused gates per pass over the state) against the
    FP64 oracle: branch records, states, samples and expectations, on a 20-qubit
    grid with flushes and on a 12-qubit random circuit with every channel kind."""
    circ = qs.config1_circuit(rows=4, cols=5, depth=12, gamma=1e-2, lam=1e-2)
    run, ref = compare_run(qt, orc, circ, 4, k=k, mode=qt.QT_DELAYED, seed=2, S=100,
                           masks=[1, 1 << 19, 0xfffff], grouping=True)
    st = run.stats()
    assert st["passes_by_width"][0] > 0          # multi-gate passes ran
    assert st["flushes"] == int(np.sum(ref["stage"] == 2)) and st["flushes"] > 0
    circ = qs.random_noisy_circuit(12, 90, 321 + k, max_gate_qubits=2, noise=0.1,
                                   channel_prob=0.4)
    run, _ = compare_run(qt, orc, circ, 8, k=k, mode=qt.QT_DELAYED, seed=k, S=50,
                         masks=[1, 0xfff], grouping=True)
    assert run.stats()["passes_by_width"][0] > 0


def test_multi_gate_passes_match_single_gate_passes(qt, orc):
    """Grouping fused gates into multi-gate passes changes only the pass count:
    same branch records, same states within float rounding, fewer passes."""
    circ = qs.config1_circuit(rows=4, cols=5, depth=12, gamma=1e-2, lam=1e-2)
    f = qt.Fused(qt.Circuit.from_synth(circ), 4)
    a = qt.Run(f, 4, seed=2, keep_states=True, grouping=True)
    b = qt.Run(f, 4, seed=2, keep_states=True, grouping=False)
    np.testing.assert_array_equal(a.kraus_indices()[0], b.kraus_indices()[0])
    for t in range(4):
        assert rel_l2(a.state(t), b.state(t)) < 2e-6
    sa, sb = a.stats(), b.stats()
    assert sa["fused_pieces"] == sb["fused_pieces"]
    assert sa["fused_passes"] < sb["fused_passes"]


@pytest.mark.parametrize("k", [3, 4])
def test_noise_model_with_readout_errors(qt, orc, k):
    """The approximate noise model of Sec. V.B (fSim with coherent errors and Z phases,
    three-operator decay + dephasing after every gate, 1q and 2q depolarizing) with
    short T1 / T_phi so that stage 2 flushes happen, plus readout errors on the samples:
    branch records, states, and samples after readout against the oracle."""
    circ, ro = qs.noise_model_circuit(3, 3, 8, 4, T1=1e-6, Tphi=1.5e-6)
    T, S = 12, 60
    run = qt.Run(qt.Fused(qt.Circuit.from_synth(circ), k), T, seed=6, samples_per_traj=S,
                 keep_states=True, readout_error=ro)
    kr, st = run.kraus_indices()
    ref = orc.run_trajectories(circ, T, seed=6, keep_states=True)
    smp = run.samples()
    compared = 0
    for t in range(T):
        if np.any(ref["margin"][t] <= MARGIN):
            continue
        compared += 1
        np.testing.assert_array_equal(kr[t], ref["kraus_idx"][t])
        np.testing.assert_array_equal(st[t], ref["stage"][t])
        g = run.state(t)
        assert rel_l2(g, ref["states"][t]) <= STATE_L2
        want, margin = orc.sample(ref["states"][t], 6, t, S)
        want = orc.readout(want, circ.num_qubits, ro, 6, t)
        ok = margin > MARGIN
        np.testing.assert_array_equal(smp[t][ok], want[ok])
    assert compared >= 0.75 * T
    assert run.stats()["flushes"] > 0
    assert np.any(ref["stage"] == 2) and np.any(ref["kraus_idx"] == 2)   # three-operator stage 2 reached


def test_product_state_start(qt, orc):
    # From 12 qubits on, the fused gates that act first on their own qubits
    # are folded into the initial product state (one write pass); branch
    # records, states, samples and expectations still match the oracle.
    circ = qs.config1_circuit(rows=3, cols=5)
    run, _ = compare_run(qt, orc, circ, 4, k=4, mode=qt.QT_DELAYED, S=100, masks=[1, 0x7fff])
    assert run.stats()["folded_pieces"] > 0
    small = qs.config1_circuit(rows=2, cols=5)
    r2, _ = compare_run(qt, orc, small, 2, k=4, mode=qt.QT_DELAYED, S=20)
    assert r2.stats()["folded_pieces"] == 0


@pytest.mark.parametrize("rows,cols", [(2, 11), (4, 6)])
def test_product_state_start_large_split(qt, orc, rows, cols):
    # At 22 and 24 qubits the split m of the product-state start must keep both
    # tables within 2^20 entries (m >= n - 20), unlike the 15-qubit case where any
    # split fits; one trajectory of each against the oracle.
    circ = qs.config1_circuit(rows=rows, cols=cols, depth=10)
    n = rows * cols
    run, _ = compare_run(qt, orc, circ, 1, k=4, mode=qt.QT_DELAYED, S=200, masks=[1, (1 << n) - 1])
    st = run.stats()
    assert st["folded_pieces"] > 0
    assert n - 20 <= st["fold_split"] <= 20


@pytest.mark.parametrize("keep", [True, False])
def test_shared_prefix_matches_oracle(qt, orc, keep):
    """QT_FLAG_SHARE_PREFIX: trajectories copy one shared state at their first
    non-default channel and run only their own suffix.  Branch records, states,
    samples and expectations against the FP64 oracle: on a 20-qubit grid with
    flushes (most trajectories diverge early), on a 15-qubit grid with weak
    damping (most never diverge and are measured on the shared final state),
    and on the 10-qubit chain workload."""
    strong = qs.config1_circuit(rows=4, cols=5, depth=12, gamma=1e-2, lam=1e-2)
    run, ref = compare_run(qt, orc, strong, 6, k=4, mode=qt.QT_DELAYED, seed=3, S=100,
                           masks=[1, 0xfffff], check_states=keep, share_prefix=True)
    st = run.stats()
    assert st["flushes"] == int(np.sum(ref["stage"] == 2)) and st["flushes"] > 0
    assert st["prefix_copies"] > 0
    weak = qs.config1_circuit(rows=3, cols=5, depth=16)
    run, ref = compare_run(qt, orc, weak, 12, k=4, mode=qt.QT_DELAYED, seed=1, S=100,
                           masks=[1, 0x7fff], check_states=keep, share_prefix=True)
    kr = run.kraus_indices()[0]
    never = int(np.sum(np.all(ref["stage"] == 1, axis=1) & np.all(kr == 0, axis=1)))
    assert never >= 3                              # measured on the shared final state
    st = run.stats()
    assert st["prefix_ops"] > 0
    if not keep:
        assert st["prefix_copies"] <= 12 - never
    compare_run(qt, orc, qs.config0_circuit(), 64, k=2, mode=qt.QT_DELAYED, S=100,
                masks=[1, 1023], check_states=keep, share_prefix=True)


def test_shared_prefix_equals_per_trajectory_loop(qt):
    """Sharing the prefix changes only where fused pieces are split: the same branch
    records, states within one kernel call's rounding, and fewer fused passes."""
    circ = qs.config1_circuit(rows=4, cols=5, depth=16, gamma=2e-3, lam=2e-3)
    f = qt.Fused(qt.Circuit.from_synth(circ), 4)
    a = qt.Run(f, 16, seed=9, keep_states=True, share_prefix=True)
    b = qt.Run(f, 16, seed=9, keep_states=True)
    np.testing.assert_array_equal(a.kraus_indices()[0], b.kraus_indices()[0])
    np.testing.assert_array_equal(a.kraus_indices()[1], b.kraus_indices()[1])
    for t in range(16):
        assert rel_l2(a.state(t), b.state(t)) < 2e-6
    assert a.stats()["fused_passes"] < b.stats()["fused_passes"]


@pytest.mark.parametrize("q,n,k,mode", [(4, 10, 4, "delayed"), (4, 12, 5, "delayed"), (5, 13, 5, "delayed"),
                                        (6, 13, 6, "delayed"), (4, 10, 4, "eager"), (5, 13, 6, "eager")])
def test_wide_kraus_channels_in_stage_two(qt, orc, q, n, k, mode):
    """Random Kraus channels on 4..6 qubits between random gates.  Their lower
    bounds are small, so most draws go to stage 2 and the probability pass runs on
    |K_i psi|^2 on the device: branch records (stage 2 included), states and
    samples against the oracle."""
    rng = np.random.default_rng([0x4b, q, n])
    c = qs.Circuit(n)
    m = 0
    for layer in range(4):
        for j in range(n):
            c.gate(qs.random_unitary(2, rng), (j,), m)
        m += 1
        for j in range(layer % 2, n - 1, 2):
            c.gate(qs.CZ, (j, j + 1), m)
        m += 1
        qubits = tuple(int(x) for x in rng.choice(n, q, replace=False))
        c.kraus(qs.circuits.random_kraus(1 << q, 3, rng), qubits, m)
        m += 1
    m = qt.QT_DELAYED if mode == "delayed" else qt.QT_EAGER
    run, ref = compare_run(qt, orc, c, 6, k=k, mode=m, seed=q, S=60, masks=[1, (1 << n) - 1])
    assert np.sum(ref["stage"] == 2) > 0
    assert run.stats()["flushes"] == int(np.sum(ref["stage"] == 2))
    if mode == "eager":                      # every channel evaluated
        assert run.stats()["prob_passes"] == 6 * 4


def test_mixture_only_circuit_never_flushes(qt, orc):
    circ = qs.config3_circuit(rows=2, cols=5, depth=10, p=0.05)
    run, _ = compare_run(qt, orc, circ, 8, k=4, mode=qt.QT_DELAYED, S=50)
    assert run.stats()["flushes"] == 0 and run.stats()["prob_passes"] == 0


def test_amplitude_damping_full_reset(qt, orc):
    c = qs.Circuit(5)
    for q in range(5):
        c.gate(qs.SQRT_X, (q,), 0)
    for q in range(5):
        c.channel(qs.amplitude_damping(1.0), (q,), 1)
    qc = qt.Circuit.from_synth(c)
    run = qt.Run(qt.Fused(qc, 3), 4, keep_states=True, samples_per_traj=10)
    for t in range(4):
        assert abs(abs(run.state(t)[0]) - 1) < 1e-6
    assert np.all(run.samples() == 0)


def test_trajectory_ranges_compose(qt):
    """Counter-based draws: trajectories [0,8) equal [0,4) + [4,8) (replica sharding)."""
    circ = qs.config1_circuit(rows=3, cols=4, depth=8, gamma=2e-2, lam=2e-2)
    qc = qt.Circuit.from_synth(circ)
    f = qt.Fused(qc, 4)
    a = qt.Run(f, 8, seed=5, samples_per_traj=30)
    b0 = qt.Run(f, 4, seed=5, first_traj=0, samples_per_traj=30)
    b1 = qt.Run(f, 4, seed=5, first_traj=4, samples_per_traj=30)
    np.testing.assert_array_equal(a.samples(), np.concatenate([b0.samples(), b1.samples()]))
    np.testing.assert_array_equal(a.kraus_indices()[0],
                                  np.concatenate([b0.kraus_indices()[0], b1.kraus_indices()[0]]))
