"""Pins for the oracle's Philox stream, sampling and Z expectations.

* Philox4x32-10 against the published known-answer vectors (golden file).
* Sampling against numpy's cumsum + searchsorted (the textbook inverse-CDF
  rule), a chi-square test against exact probabilities, and GHZ.
* Z-string expectations against the closed form of product states.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import qtsynth as qs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(orc.philox4x32_10(ctr, key)) == want


def test_u01_uniform(orc):
    u = np.array([orc.u01(7, t, 0, i) for t in range(40) for i in range(500)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # different streams / trajectories give different numbers
    assert orc.u01(0, 0, 0, 0) != orc.u01(0, 0, 1, 0)
    assert orc.u01(0, 0, 0, 0) != orc.u01(0, 1, 0, 0)
    assert orc.u01(0, 0, 0, 0) != orc.u01(1, 0, 0, 0)


def test_sample_matches_searchsorted(orc):
    rng = np.random.default_rng(1)
    n = 10
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    S = 500
    got, margin = orc.sample(psi, 9, 4, S)
    C = np.cumsum(np.abs(psi) ** 2)
    u = np.array([orc.u01(9, 4, 1, j) for j in range(S)])
    want = np.searchsorted(C, u * C[-1], side="right")
    ok = margin > 1e-12
    assert ok.mean() > 0.99
    np.testing.assert_array_equal(got[ok], want[ok])


def test_sample_chi_square(orc):
    rng = np.random.default_rng(2)
    n = 5
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    p = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    S = 40000
    got, _ = orc.sample(psi, 1, 0, S)
    counts = np.bincount(got.astype(np.int64), minlength=1 << n)
    assert stats.chisquare(counts, p * S).pvalue > 1e-4


def test_sample_ghz(orc):
    n = 9
    psi = orc.run_trajectory(qs.ghz_circuit(n))["state"]
    got, _ = orc.sample(psi, 0, 0, 2000)
    assert set(np.unique(got).tolist()) <= {0, (1 << n) - 1}
    assert 800 < np.sum(got == 0) < 1200


def test_expect_z_product_state(orc):
    rng = np.random.default_rng(3)
    n = 7
    th = rng.uniform(0, np.pi, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    psi = np.array([1.0 + 0j])
    for j in range(n):      # qubit j is bit j: kron puts later qubits in higher bits
        psi = np.kron(np.array([np.cos(th[j] / 2), np.exp(1j * ph[j]) * np.sin(th[j] / 2)]), psi)
    psi = psi * 1.7         # expectation is normalized by <psi|psi>
    masks = [1, 2, 5, 0b1111111, 0b1010010, 0]
    got = orc.expect_z(psi, masks)
    for g, m in zip(got, masks):
        want = np.prod([np.cos(th[j]) for j in range(n) if (m >> j) & 1])
        assert g == pytest.approx(want, abs=1e-13)
