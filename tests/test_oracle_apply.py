"""Pins for the oracle's Alg. 1 (Sec. III.A) gate application.

Checks against things other than the oracle itself: a dense 2^n x 2^n
operator assembled with numpy index arithmetic (brute force), the closed
forms of GHZ preparation and of the QFT of basis states, and norm
preservation of unitary circuits.
"""
import numpy as np
import pytest

import qtsynth as qs


def dense_operator(n, qubits, U):
    """Full 2^n x 2^n matrix of U acting on `qubits` (bit b of U's index = qubits[b])."""
    N = 1 << n
    x = np.arange(N)
    sub = np.zeros(N, dtype=np.int64)
    for b, q in enumerate(qubits):
        sub |= ((x >> q) & 1) << b
    mask = 0
    for q in qubits:
        mask |= 1 << q
    rest = x & ~mask
    same = rest[:, None] == rest[None, :]
    return np.where(same, U[sub[:, None], sub[None, :]], 0.0)


@pytest.mark.parametrize("n,q,seed", [(3, 1, 0), (4, 2, 1), (5, 3, 2), (6, 2, 3),
                                      (7, 4, 4), (8, 3, 5), (6, 6, 6), (7, 5, 7)])
def test_apply_matches_dense_operator(orc, n, q, seed):
    rng = np.random.default_rng(seed)
    qubits = [int(v) for v in rng.choice(n, q, replace=False)]   # unsorted on purpose
    U = rng.normal(size=(1 << q, 1 << q)) + 1j * rng.normal(size=(1 << q, 1 << q))
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    want = dense_operator(n, qubits, U) @ psi
    got = orc.apply(psi.copy(), qubits, U)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("n", [2, 5, 9])
def test_ghz_closed_form(orc, n):
    c = qs.ghz_circuit(n)
    res = orc.run_trajectory(c)
    want = np.zeros(1 << n, dtype=np.complex128)
    want[0] = want[-1] = 1 / np.sqrt(2)
    np.testing.assert_allclose(res["state"], want, atol=1e-14)


@pytest.mark.parametrize("n,x", [(3, 5), (5, 0), (5, 19), (7, 100)])
def test_qft_of_basis_state(orc, n, x):
    c = qs.qft_circuit(n, x)
    got = orc.run_trajectory(c)["state"]
    y = np.arange(1 << n)
    want = np.exp(2j * np.pi * x * y / (1 << n)) / np.sqrt(1 << n)
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_unitary_norm_preservation(orc):
    rng = np.random.default_rng(11)
    n = 12
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    for _ in range(40):
        q = int(rng.integers(1, 5))
        qubits = [int(v) for v in rng.choice(n, q, replace=False)]
        orc.apply(psi, qubits, qs.random_unitary(1 << q, rng))
    assert abs(orc.norm2(psi) - 1.0) < 1e-13


def test_norm2_matches_numpy(orc):
    rng = np.random.default_rng(3)
    psi = rng.normal(size=1 << 14) + 1j * rng.normal(size=1 << 14)
    assert orc.norm2(psi) == pytest.approx(np.vdot(psi, psi).real, rel=1e-13)
