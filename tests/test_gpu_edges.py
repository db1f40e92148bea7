"""GPU edge cases: empty and degenerate inputs, and the largest state.

  * no trajectories, no samples, a circuit without operations;
  * a one-qubit circuit, and a circuit made only of channels (no gates),
    against the FP64 oracle (branch records, states, samples);
  * batches of one circuit and of one fused circuit repeated;
  * the largest state the library accepts, 2^34 amplitudes (128 GiB): on
    the uniform superposition the read passes have closed forms
    (<Z_mask> = 0, every reduced-density entry 1/4, uniform samples), and
    a fused gate's output amplitude is c * sum_m U[j][m], with j the
    amplitude's index on the gate's qubits.
"""
import numpy as np
import pytest

import qtsynth as qs
from gpu_util import torch_cuda
from test_gpu_runs import compare_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qt():
    import paper_2111_02396_gb300 as pkg
    pkg.load()
    torch_cuda()
    return pkg


def test_kernels_are_sm_103a_code(qt):
    # the runtime reports the architecture of the loaded kernel image
    binary, ptx = qt.kernel_arch()
    assert binary == 103, (binary, ptx)


def test_zero_trajectories_and_zero_samples(qt):
    circ = qs.config0_circuit()
    f = qt.Fused(qt.Circuit.from_synth(circ), 3)
    r = qt.Run(f, 0, samples_per_traj=10, z_masks=[1, 2])
    assert r.samples().shape == (0, 10)
    assert r.expectation().shape == (0, 2)
    kr, st = r.kraus_indices()
    assert kr.shape == (0, circ.num_channels)
    s = r.stats()
    assert s["fused_passes"] == 0 and s["num_traj"] == 0
    r2 = qt.Run(f, 2, samples_per_traj=0)
    assert r2.samples().shape == (2, 0)


def test_circuit_without_operations(qt):
    qc = qt.Circuit(5, [])
    r = qt.Run(qt.Fused(qc, 2), 3, samples_per_traj=50, z_masks=[1, 3, 31], keep_states=True)
    assert np.all(r.samples() == 0)
    np.testing.assert_allclose(r.expectation(), 1.0, atol=1e-12)
    psi = r.state(1)
    assert psi[0] == 1 and np.count_nonzero(psi) == 1
    assert r.stats()["fused_passes"] == 0


def test_one_qubit_circuit(qt, orc):
    c = qs.Circuit(1)
    m = 0
    for g in (qs.SQRT_X, qs.SQRT_Y, qs.SQRT_W, qs.SQRT_X):
        c.gate(g, (0,), m)
        c.channel(qs.amplitude_damping(0.3), (0,), m + 1)
        c.channel(qs.phase_damping(0.2), (0,), m + 2)
        c.channel(qs.depolarizing(0.1), (0,), m + 3)
        m += 4
    compare_run(qt, orc, c, 24, k=1, mode=qt.QT_DELAYED, seed=11, S=40, masks=[1])


@pytest.mark.parametrize("mode", ["delayed", "eager"])
def test_channels_only_circuit(qt, orc, mode):
    c = qs.Circuit(3)
    rng = np.random.default_rng(7)
    m = 0
    for _ in range(4):
        for q in range(3):
            c.channel(qs.depolarizing(0.4), (q,), m)
        c.channel((qs.KIND_KRAUS, qs.circuits.random_kraus(4, 3, rng), None), (0, 2), m + 1)
        c.channel(qs.amplitude_damping(0.5), (1,), m + 1)
        m += 2
    md = qt.QT_DELAYED if mode == "delayed" else qt.QT_EAGER
    compare_run(qt, orc, c, 16, k=2, mode=md, seed=3, S=30, masks=[1, 5])


def test_batch_of_one_and_of_repeats(qt, orc):
    cc = qs.config2_compact(3)
    f = qt.fuse_many([qt.Circuit.from_compact(cc)], 3)
    one = qt.Batch(f).run(seed=4, first_traj=9, samples_per_traj=20)
    rep = qt.Batch([f[0]] * 5).run(seed=4, first_traj=9, samples_per_traj=20)
    s1, s5 = one.samples(), rep.samples()
    np.testing.assert_array_equal(s5[0], s1[0])          # same circuit, same trajectory id
    assert not all(np.array_equal(s5[0], s5[i]) for i in range(1, 5))   # ids 9..13 differ
    for i in range(5):
        want = qt.Batch(f).run(seed=4, first_traj=9 + i, samples_per_traj=20).samples()[0]
        np.testing.assert_array_equal(s5[i], want)


def test_largest_state(qt):
    torch = torch_cuda()
    n = 34
    c = 2.0 ** (-n / 2)
    d = torch.full((1 << n,), complex(c, 0.0), dtype=torch.complex64, device="cuda")
    try:
        np.testing.assert_allclose(qt.qt_state_expect_z(d.data_ptr(), n, [1, 1 << 33, (1 << n) - 1, 0b1011]),
                                   0.0, atol=1e-6)
        rho = qt.qt_state_reduced_density(d.data_ptr(), n, [0, 33])
        np.testing.assert_allclose(rho, np.full((4, 4), 0.25), atol=1e-6)
        smp = qt.qt_state_sample(d.data_ptr(), n, 5, 0, 4000)
        assert smp.max() < (1 << n)
        for q in (0, 17, 33):
            frac = np.mean((smp >> np.uint64(q)) & np.uint64(1))
            assert abs(frac - 0.5) < 0.04, (q, frac)
        rng = np.random.default_rng(17)
        for qubits in ([0, 13, 27, 33], [30, 31, 32, 33]):
            U = qs.random_unitary(16, rng)
            qt.qt_state_apply(d.data_ptr(), n, qubits, U)
            xs = rng.integers(0, 1 << n, 4096, dtype=np.int64)
            got = d[torch.tensor(xs, device="cuda")].cpu().numpy().astype(np.complex128)
            j = np.zeros(len(xs), dtype=np.int64)
            for b, q in enumerate(qubits):
                j |= ((xs >> q) & 1) << b
            want = c * U.sum(axis=1)[j]
            assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-6, qubits
            d.fill_(complex(c, 0.0))
    finally:
        del d
        torch.cuda.empty_cache()
