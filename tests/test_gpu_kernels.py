"""GPU parity of the hot kernels through the C ABI's state-level calls.

Each test puts a seeded complex64 state in device memory, calls the kernel
through libqt.so and compares with the FP64 oracle on the same input:
fused-gate application (Alg. 1) for every width 1..5 and target pattern
(all low qubits, all high, qubit 0 in or out, unsorted), the reduced
density block behind P_i = <psi|K_i^dag K_i|psi> (Alg. 2 step 14),
Z expectations and bitstring sampling.
"""
import numpy as np
import pytest

import qtsynth as qs
from gpu_util import (KERNEL_L2, MARGIN, STATE_L2, random_state, rel_l2, to_device,
                      torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qt():
    import paper_2111_02396_gb300 as pkg
    pkg.load()
    torch_cuda()
    return pkg


def patterns(n, k, rng):
    yield list(range(k))                                  # all low, includes qubit 0
    yield list(range(n - k, n))                           # all high
    yield [0] + list(range(n - k + 1, n))                 # qubit 0 + high
    yield list(range(1, k + 1))                           # low, qubit 0 free
    yield [int(x) for x in rng.choice(n, k, replace=False)]   # random, unsorted
    if n - 1 >= k:
        yield [int(x) for x in rng.choice(np.arange(1, n), k, replace=False)]


@pytest.mark.parametrize("n", [5, 11, 17])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_apply_every_pattern(qt, orc, n, k):
    if k > n:
        pytest.skip("k > n")
    rng = np.random.default_rng([n, k])
    for qubits in patterns(n, k, rng):
        if max(qubits) >= n:
            continue
        U = qs.random_unitary(1 << k, rng)
        psi = random_state(n, k)
        d = to_device(psi)
        qt.qt_state_apply(d.data_ptr(), n, qubits, U)
        got = d.cpu().numpy()
        want = orc.apply(psi.astype(np.complex128), qubits, U)
        assert rel_l2(got, want) < KERNEL_L2, (qubits, rel_l2(got, want))


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_apply_every_low_target_set(qt, orc, k):
    # The tile kernel picks its shared-memory swizzle from the targets below
    # bit 8 of the tile index: every k-subset of the 12 lowest qubits of a
    # 14-qubit state covers every such layout (C up to 11, high targets too).
    import itertools
    n = 14
    rng = np.random.default_rng([14, k])
    psi = random_state(n, k)
    want_norm = np.linalg.norm(psi)
    for qubits in itertools.combinations(range(12), k):
        qubits = list(qubits)
        U = qs.random_unitary(1 << k, rng)
        d = to_device(psi)
        qt.qt_state_apply(d.data_ptr(), n, qubits, U)
        got = d.cpu().numpy()
        want = orc.apply(psi.astype(np.complex128), qubits, U)
        assert rel_l2(got, want) < KERNEL_L2, (qubits, rel_l2(got, want))
        assert abs(np.linalg.norm(got) - want_norm) < 1e-5 * want_norm, qubits


# split-TF32 on tensor cores: three TF32 products per term, so each product
# carries ~3 * 2^-21 relative error and an output row sums 2^(k+1) of them;
# 1e-5 relative L2 bounds one call
TC_L2 = 1e-5


@pytest.mark.parametrize("n", [13, 16, 19])
@pytest.mark.parametrize("k", [4, 5, 6])
def test_apply_tf32x3_every_pattern(qt, orc, n, k):
    if n < k + 7:
        pytest.skip("tensor-core path needs n >= k + 7")
    rng = np.random.default_rng([n, k, 7])
    for qubits in patterns(n, k, rng):
        if max(qubits) >= n:
            continue
        U = qs.random_unitary(1 << k, rng)
        psi = random_state(n, k)
        d = to_device(psi)
        qt.qt_state_apply(d.data_ptr(), n, qubits, U, precision=qt.QT_TF32X3)
        want = orc.apply(psi.astype(np.complex128), qubits, U)
        assert rel_l2(d.cpu().numpy(), want) < TC_L2, (qubits, rel_l2(d.cpu().numpy(), want))


LOW_RUN_PATTERNS = [
    [0, 1, 2, 3, 4, 5], [0, 1, 6, 7, 8, 9], [1, 2, 3, 9, 10, 11], [3, 4, 5, 11, 12, 13],
    [0, 1, 8, 9, 16, 17], [1, 2, 3, 4, 10, 11], [1, 2, 9, 10, 17, 18], [0, 1, 2, 3, 8, 9],
    [0, 1, 2, 3], [0, 1, 8, 9], [1, 2, 9, 10], [0, 1, 2, 3, 4], [0, 1, 2, 8, 9], [1, 2, 3, 9, 10],
    [1, 2, 3, 9], [1, 2, 3, 5, 16], [1, 2, 3, 4, 5, 6], [2, 3, 9, 10, 17, 18],
]


def test_apply_tf32x3_low_target_runs(qt, orc):
    """Target patterns whose gather sets are aligned runs of low amplitudes (the
    6-qubit gates of the 32-qubit precision workload whose converter reads conflict
    in shared memory, and 4- and 5-qubit analogues), with and without high targets,
    against the oracle.  Covers the three ways the kernel moves amplitudes: member
    pairs (qubit 0 a target), set pairs exchanged by shuffles (qubits 1, 2 and 3
    targets, qubit 0 not) and single members."""
    n = 20
    rng = np.random.default_rng(77)
    for qubits in LOW_RUN_PATTERNS:
        k = len(qubits)
        U = qs.random_unitary(1 << k, rng)
        psi = random_state(n, k + 40)
        d = to_device(psi)
        qt.qt_state_apply(d.data_ptr(), n, qubits, U, precision=qt.QT_TF32X3)
        want = orc.apply(psi.astype(np.complex128), qubits, U)
        assert rel_l2(d.cpu().numpy(), want) < TC_L2, (qubits, rel_l2(d.cpu().numpy(), want))


@pytest.mark.parametrize("n", [13, 17])
def test_apply_k6_fp32_every_pattern(qt, orc, n):
    """6-qubit fused gates on CUDA cores (the FP32 comparator of the TF32x3 path)."""
    rng = np.random.default_rng([n, 6, 9])
    for qubits in patterns(n, 6, rng):
        if max(qubits) >= n:
            continue
        U = qs.random_unitary(64, rng)
        psi = random_state(n, 6)
        d = to_device(psi)
        qt.qt_state_apply(d.data_ptr(), n, qubits, U, precision=qt.QT_FP32)
        want = orc.apply(psi.astype(np.complex128), qubits, U)
        assert rel_l2(d.cpu().numpy(), want) < KERNEL_L2, (qubits, rel_l2(d.cpu().numpy(), want))


def test_apply_sequence_ragged_sizes(qt, orc):
    """Many gates in sequence on sizes that span several grid waves and a
    one-set edge case (n == k)."""
    for n in (4, 9, 20, 23):
        rng = np.random.default_rng(n)
        psi = random_state(n, 3)
        d = to_device(psi)
        ref = psi.astype(np.complex128)
        for _ in range(30):
            k = int(rng.integers(1, min(5, n) + 1))
            qubits = [int(x) for x in rng.choice(n, k, replace=False)]
            U = qs.random_unitary(1 << k, rng)
            qt.qt_state_apply(d.data_ptr(), n, qubits, U)
            orc.apply(ref, qubits, U)
        assert rel_l2(d.cpu().numpy(), ref) < STATE_L2


def test_apply_non_unitary_and_n_equals_k(qt, orc):
    rng = np.random.default_rng(9)
    for n in (1, 2, 3):
        psi = random_state(n, 1)
        d = to_device(psi)
        A = rng.normal(size=(1 << n, 1 << n)) + 1j * rng.normal(size=(1 << n, 1 << n))
        qt.qt_state_apply(d.data_ptr(), n, list(range(n))[::-1], A)
        want = orc.apply(psi.astype(np.complex128), list(range(n))[::-1], A)
        assert rel_l2(d.cpu().numpy(), want) < KERNEL_L2


@pytest.mark.parametrize("n,q", [(3, 1), (12, 1), (16, 2), (18, 3), (21, 2)])
def test_probabilities_from_reduced_density(qt, orc, n, q):
    rng = np.random.default_rng([n, q])
    psi = random_state(n, 5)
    d = to_device(psi)
    for _ in range(3):
        qubits = [int(x) for x in rng.choice(n, q, replace=False)]
        rho = qt.qt_state_reduced_density(d.data_ptr(), n, qubits)
        Ks = qs.circuits.random_kraus(1 << q, 3, rng)
        P_gpu = np.array([np.trace(K.conj().T @ K @ rho).real for K in Ks])
        P_orc = orc.kraus_norms(psi.astype(np.complex128), qubits, Ks)
        np.testing.assert_allclose(P_gpu, P_orc, rtol=1e-6, atol=1e-9)
        assert abs(np.trace(rho).real - orc.norm2(psi.astype(np.complex128))) < 1e-6


@pytest.mark.parametrize("n,q,nops", [(8, 4, 3), (9, 4, 17), (12, 5, 5), (13, 6, 2), (6, 6, 3), (20, 4, 4),
                                      (4, 2, 5)])
def test_kraus_probabilities(qt, orc, n, q, nops):
    """P_i = <psi|K_i^dag K_i|psi> of random Kraus channels on 2..6 qubits (17
    operators on 4 qubits take two passes of 16) against the FP64 oracle, N against
    <psi|psi>, and completeness sum_i P_i = N.  Tolerance: each |K_i v|^2 row is an
    FP32 sum of at most 64 products (rounding ~ 64 * 2^-24 ~ 4e-6 of the row), so
    rtol 2e-5 with an absolute floor of 1e-6 N."""
    psi = random_state(n, 21 + q) * np.float32(1.1)
    d = to_device(psi)
    rng = np.random.default_rng([n, q, nops])
    qubits = [int(x) for x in rng.choice(n, q, replace=False)]
    Ks = qs.circuits.random_kraus(1 << q, nops, rng)
    P, N = qt.qt_state_kraus_probabilities(d.data_ptr(), n, qubits, Ks)
    p64 = psi.astype(np.complex128)
    N_orc = orc.norm2(p64)
    np.testing.assert_allclose(P, orc.kraus_norms(p64, qubits, Ks), rtol=2e-5, atol=1e-6 * N_orc)
    assert abs(N - N_orc) <= 1e-6 * N_orc
    assert abs(P.sum() - N) <= 2e-5 * N


@pytest.mark.parametrize("n", [1, 6, 8, 9, 10, 15, 22])
def test_expect_z(qt, orc, n):
    psi = random_state(n, 7) * np.float32(1.3)
    d = to_device(psi)
    rng = np.random.default_rng(n)
    masks = [0, (1 << n) - 1] + [1 << j for j in range(n)] + [int(x) for x in rng.integers(0, 1 << n, 20)]
    got = qt.qt_state_expect_z(d.data_ptr(), n, masks)
    want = orc.expect_z(psi.astype(np.complex128), masks)
    np.testing.assert_allclose(got, want, atol=2e-6)


@pytest.mark.parametrize("n,S", [(1, 50), (4, 300), (11, 3000), (16, 3000), (20, 1000)])
def test_sample_parity(qt, orc, n, S):
    psi = random_state(n, 11)
    d = to_device(psi)
    got = qt.qt_state_sample(d.data_ptr(), n, 42, 3, S)
    want, margin = orc.sample(psi.astype(np.complex128), 42, 3, S)
    ok = margin > MARGIN
    assert np.all(got < (1 << n))
    np.testing.assert_array_equal(got[ok], want[ok])
    if n <= 11:
        assert ok.mean() > 0.9
    # Ties (the draw lies within 1e-6 of a CDF boundary; at n = 20 most draws
    # do): the GPU's index must lie in the oracle's CDF neighbourhood of the
    # target, u * C(2^n - 1) in [C(x - 1) - delta, C(x) + delta], where delta is
    # the measured largest difference between the sampler's own C (qt_state_cdf)
    # and C of the definition (sequential FP64 sum of |psi_y|^2 in index order,
    # as the oracle forms it), plus the difference of the totals.
    cg = qt.qt_state_cdf(d.data_ptr(), n)
    co = np.cumsum(np.abs(psi.astype(np.complex128)) ** 2)
    delta = float(np.max(np.abs(cg - co))) + abs(float(cg[-1] - co[-1]))
    # the sampler's arithmetic bounds delta: FP32 squares and runs of at most
    # 1024 terms (a 5-level warp scan plus 16 chunk sums, ~23 roundings of
    # 2^-24), carried in FP64 across runs
    assert delta <= 32 * 2.0 ** -24 * co[-1], delta
    if (~ok).any():
        u = np.array([orc.u01(42, 3, 1, j) for j in range(S)])
        t = u[~ok] * co[-1]
        x = got[~ok].astype(np.int64)
        below = np.where(x > 0, co[np.maximum(x - 1, 0)], 0.0)
        assert np.all(t >= below - delta), np.min(t - below + delta)
        assert np.all(t <= co[x] + delta), np.min(co[x] + delta - t)


@pytest.mark.parametrize("n,S", [(1, 200), (11, 3000), (33, 64)])
def test_sample_readout_errors(qt, orc, n, S):
    """Readout errors (Sec. V.A) on the device sampler: the same flips as the oracle's
    readout of the oracle's samples, wherever the sample itself is not a tie."""
    rng = np.random.default_rng(n + 5)
    ro = np.stack([rng.uniform(0, 0.3, n), rng.uniform(0, 0.5, n)], axis=1)
    if n <= 20:
        psi = random_state(n, 13)
        d = to_device(psi)
        want, margin = orc.sample(psi.astype(np.complex128), 8, 2, S)
    else:                                        # 2^33 amplitudes: the all-zero basis state
        torch = torch_cuda()
        d = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
        d[0] = 1.0
        want, margin = np.zeros(S, dtype=np.uint64), np.ones(S)
    got = qt.qt_state_sample(d.data_ptr(), n, 8, 2, S, readout_error=ro)
    want = orc.readout(want, n, ro, 8, 2)
    ok = margin > MARGIN
    np.testing.assert_array_equal(got[ok], want[ok])
    assert ok.mean() > 0.9
    del d


def test_sample_ghz_full_support(qt, orc):
    n = 12
    psi = np.zeros(1 << n, dtype=np.complex64)
    psi[0] = psi[-1] = np.float32(1 / np.sqrt(2))
    d = to_device(psi)
    got = qt.qt_state_sample(d.data_ptr(), n, 1, 0, 4000)
    assert set(np.unique(got).tolist()) <= {0, (1 << n) - 1}
    want, _ = orc.sample(psi.astype(np.complex128), 1, 0, 4000)
    np.testing.assert_array_equal(got, want)


def test_state_calls_reject_bad_arguments(qt):
    from paper_2111_02396_gb300.qt import QtError
    torch = torch_cuda()
    d = torch.zeros(64, dtype=torch.complex64, device="cuda")
    with pytest.raises(QtError):
        qt.qt_state_apply(d.data_ptr(), 6, [0, 0], np.eye(4))       # repeated qubit
    with pytest.raises(QtError):
        qt.qt_state_apply(d.data_ptr(), 6, [6], np.eye(2))          # out of range
    with pytest.raises(QtError):
        qt.qt_state_apply(d.data_ptr() + 8, 6, [1], np.eye(2))      # misaligned
    with pytest.raises(QtError):
        qt.qt_state_reduced_density(d.data_ptr(), 6, [0, 1, 2, 3])  # q > 3
