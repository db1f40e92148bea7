"""Pins of the oracle's readout errors (Sec. V.A, parallel readout errors).

A qubit whose true value is b is reported as 1 - b with the probability
measured for b: the p00 error (0 read as 1) or the p11 error (1 read as 0).
Pinned by the cases the definition fixes exactly (no error, certain error,
one-sided errors), by the flip rates of each qubit and each true value
against the binomial bounds, by the independence of qubits, and by the
draw convention (Philox stream 2, index (j << 6) | q), whose generator is
itself pinned by known-answer vectors.
"""
import numpy as np

N = 7


def _bits(rng, S, n=N):
    return rng.integers(0, 1 << n, S, dtype=np.uint64)


def test_no_error_is_identity(orc):
    rng = np.random.default_rng(1)
    b = _bits(rng, 500)
    np.testing.assert_array_equal(orc.readout(b, N, np.zeros((N, 2)), 3, 4), b)


def test_certain_errors(orc):
    rng = np.random.default_rng(2)
    b = _bits(rng, 400)
    full = np.uint64((1 << N) - 1)
    # every value flipped: the complement on the n qubits
    np.testing.assert_array_equal(orc.readout(b, N, np.ones((N, 2)), 5, 6), b ^ full)
    # only 0 -> 1 errors, certain: every qubit reads 1
    e = np.zeros((N, 2))
    e[:, 0] = 1.0
    np.testing.assert_array_equal(orc.readout(b, N, e, 5, 6), np.full_like(b, full))
    # only 1 -> 0 errors, certain: every qubit reads 0
    e = np.zeros((N, 2))
    e[:, 1] = 1.0
    np.testing.assert_array_equal(orc.readout(b, N, e, 5, 6), np.zeros_like(b))


def test_flip_rates_per_qubit_and_value(orc):
    rng = np.random.default_rng(3)
    S = 40000
    b = _bits(rng, S)
    e = np.stack([np.linspace(0.01, 0.2, N), np.linspace(0.3, 0.05, N)], axis=1)
    r = orc.readout(b, N, e, 11, 12)
    for q in range(N):
        true = (b >> np.uint64(q)) & np.uint64(1)
        read = (r >> np.uint64(q)) & np.uint64(1)
        for v in (0, 1):
            sel = true == v
            rate = np.mean(read[sel] != v)
            p = e[q, v]
            sigma = np.sqrt(p * (1 - p) / sel.sum())
            assert abs(rate - p) < 5 * sigma, (q, v, rate, p)


def test_qubits_flip_independently(orc):
    S = 40000
    b = np.zeros(S, dtype=np.uint64)
    e = np.full((N, 2), 0.5)
    r = orc.readout(b, N, e, 21, 22)
    f0 = ((r >> np.uint64(0)) & np.uint64(1)).astype(float)
    f1 = ((r >> np.uint64(1)) & np.uint64(1)).astype(float)
    assert abs(np.corrcoef(f0, f1)[0, 1]) < 5 / np.sqrt(S)


def test_draw_convention(orc):
    S = 64
    b = np.zeros(S, dtype=np.uint64)
    e = np.zeros((N, 2))
    e[3, 0] = 0.5
    r = orc.readout(b, N, e, 31, 32)
    want = np.array([orc.u01(31, 32, 2, (j << 6) | 3) < 0.5 for j in range(S)])
    np.testing.assert_array_equal(((r >> np.uint64(3)) & np.uint64(1)).astype(bool), want)
    assert np.all((r & ~np.uint64(1 << 3)) == 0)
