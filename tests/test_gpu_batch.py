"""GPU parity of the batched persistent form.

Every trajectory of a batch (each with its own circuit) is compared with
the FP64 oracle run of the same circuit, seed and trajectory id (branch
records where the margin exceeds 1e-6, final state within relative L2
2e-5 / fidelity 1 - 1e-5, samples where the CDF margin exceeds 1e-6), and
with the plain per-trajectory loop.  Covers states in shared memory
(n <= 14) and in global memory (n = 15..20), forced stage-2 flushes, the
product-state start, CUDA graph replay, and the autotuner.
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


def _workload_circuits(max_n=16, count=20):
    out, i = [], 0
    while len(out) < count:
        cc = qs.config2_compact(i)
        if cc.num_qubits <= max_n:
            out.append(cc)
        i += 1
    return out


def _noisy(n, depth, seed, gamma):
    rng = np.random.default_rng([0x61, n, seed])
    return qs.layered_compact(n, depth, rng, lambda l: qs.circuits._chain_couplings(n, l),
                              dep1=0.02, dep2=0.02, per_gate_ad=gamma)


def check_batch(qt, orc, ccs, k, *, seed=0, first=0, S=100, threads=0, threads_global=0):
    """k: one fusion width, or a tuning dict of per-class widths (fuse_by_class)."""
    qcs = [qt.Circuit.from_compact(c) for c in ccs]
    fs = qt.fuse_by_class(qcs, k) if isinstance(k, dict) else qt.fuse_many(qcs, k)
    b = qt.Batch(fs).run(seed=seed, first_traj=first, samples_per_traj=S, keep_states=True,
                         threads=threads, threads_global=threads_global)
    smp = b.samples()
    compared = 0
    for i, cc in enumerate(ccs):
        circ = cc.to_circuit()
        ref = orc.run_trajectory(circ, orc.DELAYED, seed=seed, traj=first + i)
        kr, st = b.kraus_indices(i)
        tie = False
        for ch in range(len(kr)):
            if ref["margin"][ch] <= MARGIN:
                tie = True
                break
            assert kr[ch] == ref["kraus_idx"][ch], (i, ch)
            assert st[ch] == ref["stage"][ch], (i, ch)
        if tie:
            continue
        compared += 1
        g = b.state(i)
        assert rel_l2(g, ref["state"]) <= STATE_L2, (i, rel_l2(g, ref["state"]))
        assert fidelity(g, ref["state"]) >= 1 - STATE_FID
        want, margin = orc.sample(ref["state"], seed, first + i, S)
        ok = margin > MARGIN
        np.testing.assert_array_equal(smp[i][ok], want[ok])
    assert compared >= 0.75 * len(ccs)
    return b, fs


def test_batch_workload_circuits_match_oracle(qt, orc):
    ccs = _workload_circuits()
    assert max(c.num_qubits for c in ccs) >= 15          # global-memory states are covered
    check_batch(qt, orc, ccs, 3)


@pytest.mark.parametrize("k", [2, 4, 5, 6])
def test_batch_forced_flushes(qt, orc, k):
    ccs = [_noisy(n, 10, s, 0.06) for s, n in enumerate([8, 9, 10, 11, 12, 15])]
    b, _ = check_batch(qt, orc, ccs, k, seed=3, first=100, S=64, threads=256)
    assert b.stats()["flushes"] > 0


@pytest.mark.parametrize("k,tg", [(1, 512), (2, 256), (3, 512), (4, 128), (5, 256), (6, 512)])
def test_batch_global_memory_states_match_oracle(qt, orc, k, tg):
    """States of 2^15..2^18 amplitudes (a CTA's slot of global memory, up to 32 loads in
    flight per thread, packed FMAs) next to shared-memory states in the second launch,
    with forced stage-2 flushes, at every fusion width and several CTA sizes."""
    ccs = [_noisy(n, 6, s, 0.08) for s, n in enumerate([15, 16, 17, 18, 9, 12])]
    b, _ = check_batch(qt, orc, ccs, k, seed=5, first=300, S=64, threads=512, threads_global=tg)
    assert b.stats()["flushes"] > 0


def test_batch_largest_states_match_oracle(qt, orc):
    """The largest states the batched form accepts (19 and 20 qubits: 4 and 8 MiB slots of
    global memory per CTA), with forced flushes, against the oracle."""
    ccs = [_noisy(n, 4, s, 0.08) for s, n in enumerate([19, 20, 20, 8])]
    b, _ = check_batch(qt, orc, ccs, 3, seed=11, first=900, S=64, threads=512)
    assert b.stats()["flushes"] > 0


def test_batch_per_class_widths_match_oracle(qt, orc):
    """Shared-memory states fused to k = 2 and global-memory states to k = 4 in one
    batch (the autotuner's per-class choice), against the oracle."""
    ccs = [_noisy(n, 8, s, 0.05) for s, n in enumerate([8, 11, 14, 15, 17, 18, 10, 16])]
    tune = {"k_shared": 2, "threads_shared": 256, "k_global": 4, "threads_global": 512}
    b, fs = check_batch(qt, orc, ccs, tune, seed=8, first=500, S=64, threads=256, threads_global=512)
    widths = [f.info()["max_width"] for f in fs]
    assert max(w for w, c in zip(widths, ccs) if c.num_qubits <= 14) <= 2
    assert max(w for w, c in zip(widths, ccs) if c.num_qubits > 14) == 4


def _first_on_qubits(fused, min_n):
    """Fused gates that are first on their qubits (none of their targets held by an
    earlier fused gate) in the circuits of at least min_n qubits: the pieces a
    noiseless circuit folds into its initial state."""
    count = 0
    for f in fused:
        if f.circuit.num_qubits < min_n:
            continue
        seen = 0
        for g in range(f.info()["num_fused"]):
            m = sum(1 << int(q) for q in f.gate(g)["targets"])
            count += not (m & seen)
            seen |= m
    return count


def test_batch_product_state_start(qt, orc):
    """Global-memory states (n > 14) start the first segment from a product state: a
    piece first on its qubits is folded into the initial state as its column U[:, 0]
    instead of making a pass.  Noiseless circuits (the whole circuit is one segment)
    fold exactly the fused gates first on their qubits; noisy ones also fold pieces
    composed from non-default stage-1 choices and pieces cut by the first flush
    point.  Shared-memory states in the same batch start from |0...0>.  All against
    the oracle."""
    chain = qs.circuits._chain_couplings
    clean = [qs.layered_compact(n, 5, np.random.default_rng([0x70, n]), lambda l, n=n: chain(n, l))
             for n in (5, 9, 13, 16, 18)]
    b, fs = check_batch(qt, orc, clean, 3, seed=2, S=32)
    st = b.stats()
    assert st["num_channels"] == 0 and st["flushes"] == 0
    assert st["folded_pieces"] == _first_on_qubits(fs, qt.SMEM_N_MAX + 1) > 0
    noisy = [qs.layered_compact(n, 6, np.random.default_rng([0x71, n]), lambda l, n=n: chain(n, l),
                                dep1=0.3, per_gate_ad=0.1) for n in (7, 10, 14, 15, 17)]
    b, fs = check_batch(qt, orc, noisy, 4, seed=4, first=60, S=32)
    st = b.stats()
    assert st["flushes"] > 0 and st["folded_pieces"] > 0


def test_batch_equals_plain_loop(qt):
    ccs = [_noisy(n, 8, s, 0.03) for s, n in enumerate([8, 10, 12, 13])]
    qcs = [qt.Circuit.from_compact(c) for c in ccs]
    fs = qt.fuse_many(qcs, 3)
    b = qt.Batch(fs).run(seed=9, first_traj=40, samples_per_traj=50)
    smp = b.samples()
    for i, f in enumerate(fs):
        r = qt.Run(f, 1, seed=9, first_traj=40 + i, samples_per_traj=50)
        kr_plain, _ = r.kraus_indices()
        kr_b, _ = b.kraus_indices(i)
        np.testing.assert_array_equal(kr_b, kr_plain[0])
        # same state up to float rounding: samples agree except near ties
        assert np.mean(smp[i] == r.samples()[0]) > 0.9


def test_batch_graph_replay(qt):
    torch = torch_cuda()
    ccs = _workload_circuits(max_n=13, count=12)
    fs = qt.fuse_many([qt.Circuit.from_compact(c) for c in ccs], 3)
    b = qt.Batch(fs)
    s = torch.cuda.Stream()
    a = b.run(seed=1, first_traj=7, samples_per_traj=32).samples().copy()
    g1 = b.run(seed=1, first_traj=7, samples_per_traj=32, use_graph=True, stream=s.cuda_stream).samples().copy()
    g2 = b.run(seed=1, first_traj=7, samples_per_traj=32, use_graph=True, stream=s.cuda_stream).samples().copy()
    np.testing.assert_array_equal(a, g1)
    np.testing.assert_array_equal(g1, g2)
    g3 = b.run(seed=2, first_traj=7, samples_per_traj=32, use_graph=True, stream=s.cuda_stream).samples()
    assert not np.array_equal(g3, g1)                    # new parameters reach the replayed graph


def test_batch_autotuner(qt):
    ccs = _workload_circuits(max_n=18, count=48)
    qcs = [qt.Circuit.from_compact(c) for c in ccs]
    tune, table = qt.autotune_batch(qcs, sample=24, kmin=2, kmax=6)
    assert len(table) == 30
    for cls in ("shared", "global"):
        k, threads = tune[f"k_{cls}"], tune[f"threads_{cls}"]
        assert k in (2, 3, 4, 5, 6) and threads in (128, 256, 512)
        mine = {key: v for key, v in table.items() if key[0] == cls}
        assert all(v > 0 for v in mine.values())
        assert table[(cls, k, threads)] == min(mine.values())
