"""Pins for the oracle's channel arithmetic (Sec. III.E, Sec. V.B).

* P_i = <psi|K_i^dag K_i|psi> against dense numpy operators (brute force).
* The lower bound pbar_i = sigma_min(K_i)^2 against numpy's eigvalsh and
  against closed forms (amplitude / phase damping, unitaries, Pauli mixtures).
* Kraus completeness of every generated channel.
* The exact density-matrix evolution against the closed form E(rho) of the
  decay/dephasing channel and against the two depolarizing formulas
  (Eq. depol_1 and the Pauli form of Sec. V.B).
"""
import math

import numpy as np
import pytest

import qtsynth as qs
from test_oracle_apply import dense_operator


def test_kraus_norms_match_dense(orc):
    rng = np.random.default_rng(5)
    for n, q in [(4, 1), (6, 2), (7, 3)]:
        qubits = [int(v) for v in rng.choice(n, q, replace=False)]
        Ks = qs.circuits.random_kraus(1 << q, 3, rng)
        psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        P = orc.kraus_norms(psi, qubits, Ks)
        for i, K in enumerate(Ks):
            w = dense_operator(n, qubits, K) @ psi
            assert P[i] == pytest.approx(np.vdot(w, w).real, rel=1e-12)
        # completeness: sum_i P_i = <psi|psi>
        assert P.sum() == pytest.approx(np.vdot(psi, psi).real, rel=1e-12)


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_lower_bound_matches_eigvalsh(orc, q):
    rng = np.random.default_rng(10 + q)
    for _ in range(5):
        K = rng.normal(size=(1 << q, 1 << q)) + 1j * rng.normal(size=(1 << q, 1 << q))
        want = np.linalg.eigvalsh(K.conj().T @ K).min()
        assert orc.lower_bound(K) == pytest.approx(want, rel=1e-9, abs=1e-12)


def test_lower_bound_closed_forms(orc):
    g = 0.137
    _, ad, _ = qs.amplitude_damping(g)
    assert orc.lower_bound(ad[0]) == pytest.approx(1 - g, rel=1e-13)
    assert orc.lower_bound(ad[1]) == pytest.approx(0.0, abs=1e-15)
    _, pd, _ = qs.phase_damping(g)
    assert orc.lower_bound(pd[0]) == pytest.approx(1 - g, rel=1e-13)
    assert orc.lower_bound(pd[1]) == pytest.approx(0.0, abs=1e-15)
    rng = np.random.default_rng(0)
    for q in (1, 2, 3):
        U = qs.random_unitary(1 << q, rng)
        assert orc.lower_bound(U) == pytest.approx(1.0, rel=1e-12)
        assert orc.lower_bound(math.sqrt(0.3) * U) == pytest.approx(0.3, rel=1e-12)
    _, dd, _ = qs.decay_dephasing(1.0, 10.0, 20.0)
    T2 = 1.0 / (1 / 20.0 + 1 / 20.0)
    assert orc.lower_bound(dd[0]) == pytest.approx(math.exp(-2 / T2), rel=1e-12)
    assert orc.lower_bound(dd[2]) == pytest.approx(0.0, abs=1e-15)


def test_lower_bound_below_probability(orc):
    """pbar_i <= p_i for every state (the bound Alg. 2 relies on)."""
    rng = np.random.default_rng(21)
    for _ in range(20):
        q = int(rng.integers(1, 3))
        n = 5
        Ks = qs.circuits.random_kraus(1 << q, 3, rng)
        qubits = [int(v) for v in rng.choice(n, q, replace=False)]
        psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        psi /= np.linalg.norm(psi)
        P = orc.kraus_norms(psi, qubits, Ks)
        for i, K in enumerate(Ks):
            assert orc.lower_bound(K) <= P[i] + 1e-14


@pytest.mark.parametrize("ch", [qs.amplitude_damping(0.3), qs.phase_damping(0.2),
                                qs.depolarizing(0.1), qs.depolarizing(0.2, 2),
                                qs.decay_dephasing(1.0, 5.0, 7.0)])
def test_kraus_completeness(ch):
    kind, mats, probs = ch
    if kind == qs.KIND_MIXTURE:
        Ks = [math.sqrt(p) * U for p, U in zip(probs, mats)]
        assert abs(sum(probs) - 1.0) < 1e-14
    else:
        Ks = list(mats)
    S = sum(K.conj().T @ K for K in Ks)
    np.testing.assert_allclose(S, np.eye(S.shape[0]), atol=1e-13)


def _one_qubit_rho(U):
    psi = U[:, 0]
    return np.outer(psi, psi.conj())


def test_density_decay_dephasing_closed_form(orc):
    rng = np.random.default_rng(2)
    U = qs.random_unitary(2, rng)
    t, T1, Tphi = 1.0, 4.0, 9.0
    c = qs.Circuit(1)
    c.gate(U, (0,), 0)
    c.channel(qs.decay_dephasing(t, T1, Tphi), (0,), 1)
    rho = orc.density_evolve(c)
    r0 = _one_qubit_rho(U)
    T2 = 1.0 / (1.0 / (2 * T1) + 1.0 / Tphi)
    e1, e2 = math.exp(-t / T1), math.exp(-t / T2)
    want = np.array([[1 - r0[1, 1] * e1, r0[0, 1] * e2],
                     [r0[1, 0] * e2, r0[1, 1] * e1]])
    np.testing.assert_allclose(rho, want, atol=1e-14)


def test_density_depolarizing_two_forms(orc):
    """Pauli form of Sec. V.B (D=2, 4) equals (1-eps) rho + eps I/D (Eq. depol_1)
    with p = eps (1 - 1/D^2)."""
    rng = np.random.default_rng(4)
    for nq in (1, 2):
        D = 2 ** nq
        eps = 0.23
        U = qs.random_unitary(D, rng)
        c = qs.Circuit(nq)
        c.gate(U, tuple(range(nq)), 0)
        c.channel(qs.depolarizing(eps * (1 - 1 / D ** 2), nq), tuple(range(nq)), 1)
        rho = orc.density_evolve(c)
        r0 = _one_qubit_rho(U)
        want = (1 - eps) * r0 + eps * np.eye(D) / D
        np.testing.assert_allclose(rho, want, atol=1e-14)


def test_density_unitary_matches_state(orc):
    """Noiseless: rho = |psi><psi| of the state-vector run (two code paths of Alg. 1)."""
    c = qs.random_noisy_circuit(4, 30, 1, channel_prob=0.0)
    rho = orc.density_evolve(c)
    psi = orc.run_trajectory(c)["state"]
    np.testing.assert_allclose(rho, np.outer(psi, psi.conj()), atol=1e-13)


def test_density_matches_dense_channel_sum(orc):
    """rho -> sum K rho K^dag assembled with dense numpy operators (brute force)."""
    rng = np.random.default_rng(8)
    n = 3
    c = qs.Circuit(n)
    U = qs.random_unitary(8, rng)
    c.gate(U, (2, 0, 1), 0)
    Ks = qs.circuits.random_kraus(4, 3, rng)
    c.kraus(Ks, (1, 2), 1)
    rho = orc.density_evolve(c)
    psi = dense_operator(n, (2, 0, 1), U)[:, 0]
    r = np.outer(psi, psi.conj())
    want = sum(dense_operator(n, (1, 2), K) @ r @ dense_operator(n, (1, 2), K).conj().T
               for K in Ks)
    np.testing.assert_allclose(rho, want, atol=1e-13)
