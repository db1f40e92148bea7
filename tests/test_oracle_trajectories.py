"""Pins for the oracle's trajectory sampling (Sec. III.E, Alg. 2).

* Trajectory averages of |psi><psi| agree with exact density-matrix
  evolution within 3 sigma (Bonferroni-adjusted), for the delayed, eager and
  cumulative samplers.
* Delayed and eager inner products pick identical Kraus branches for the
  same draws (both use the two-stage partition of [0,1) of Alg. 2).
* The two-stage partition differs from the cumulative one exactly where the
  paper's algorithm says it should.
* Special cases: gamma = 1 amplitude damping resets to |0>, zero noise gives
  the noiseless state, phase damping leaves Z populations unchanged.
* Stage-1 deferral happens with probability s = sum pbar_i.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import qtsynth as qs
from scipy import stats


def _traj_average(orc, c, T, mode, seed=0):
    res = orc.run_trajectories(c, T, mode=mode, seed=seed)
    S = res["states"]
    rho = np.einsum("ti,tj->ij", S, S.conj()) / T
    # per-element standard error of the mean of psi_i psi_j^* (real and imag)
    prod = S[:, :, None] * S.conj()[:, None, :]
    se_re = prod.real.std(axis=0, ddof=1) / math.sqrt(T)
    se_im = prod.imag.std(axis=0, ddof=1) / math.sqrt(T)
    return rho, se_re, se_im, res


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_trajectory_average_matches_density_matrix(orc, mode):
    n = 3
    c = qs.random_noisy_circuit(n, 40, 3, noise=0.25, channel_prob=0.5)
    exact = orc.density_evolve(c)
    T = 4000
    rho, se_re, se_im, _ = _traj_average(orc, c, T, mode)
    m = exact.size * 2
    z = stats.norm.isf(0.01 / (2 * m))          # family-wise 1% two-sided
    tol_re = z * np.maximum(se_re, 1e-3) + 1e-12
    tol_im = z * np.maximum(se_im, 1e-3) + 1e-12
    assert np.all(np.abs(rho.real - exact.real) <= tol_re)
    assert np.all(np.abs(rho.imag - exact.imag) <= tol_im)


def test_trajectory_observables_match_density_matrix_n6(orc):
    n = 6
    c = qs.random_noisy_circuit(n, 60, 9, noise=0.2, channel_prob=0.5, max_gate_qubits=2)
    exact = orc.density_evolve(c)
    T = 3000
    res = orc.run_trajectories(c, T, mode=0, seed=7)
    probs = np.abs(res["states"]) ** 2                     # [T, 2^n]
    masks = [1 << j for j in range(n)] + [3, 5, 0b111111, 0b101010]
    x = np.arange(1 << n)
    sign = np.array([[(-1) ** bin(int(v) & mk).count("1") for v in x] for mk in masks])
    per_traj = probs @ sign.T                               # [T, M]
    est = per_traj.mean(0)
    se = per_traj.std(0, ddof=1) / math.sqrt(T)
    want = sign @ np.real(np.diag(exact))
    z = stats.norm.isf(0.01 / (2 * len(masks)))
    assert np.all(np.abs(est - want) <= z * np.maximum(se, 1e-3))


def test_delayed_and_eager_pick_identical_branches(orc):
    c = qs.random_noisy_circuit(6, 80, 5, noise=0.3, channel_prob=0.6)
    T = 300
    d = orc.run_trajectories(c, T, mode=orc.DELAYED, seed=123)
    e = orc.run_trajectories(c, T, mode=orc.EAGER, seed=123)
    checked = 0
    for t in range(T):
        for ch in range(d["kraus_idx"].shape[1]):
            if min(d["margin"][t, ch], e["margin"][t, ch]) < 1e-9:
                break                                      # tie: stop this trajectory
            assert d["kraus_idx"][t, ch] == e["kraus_idx"][t, ch]
            checked += 1
        else:
            np.testing.assert_allclose(d["states"][t], e["states"][t], atol=1e-11)
    assert checked > 0.9 * T * d["kraus_idx"].shape[1]
    # the delayed run evaluates far fewer inner products
    assert d["flushes"].sum() < e["flushes"].sum()


def _two_stage_counterexample(qv=0.4, g=0.5):
    """K_a = sqrt(1-qv) A, K_b = sqrt(qv) A, K_c = sqrt(g)|0><1| with A = diag(1, sqrt(1-g))."""
    A = np.diag([1.0, math.sqrt(1 - g)])
    Ka = math.sqrt(1 - qv) * A
    Kb = math.sqrt(qv) * A
    Kc = np.array([[0.0, math.sqrt(g)], [0.0, 0.0]])
    return np.stack([Ka, Kb, Kc]).astype(np.complex128)


def test_two_stage_partition_differs_from_cumulative(orc):
    """On |+>, a draw r in [pbar_a, p_a) selects b under Alg. 2 (stage 1 covers
    [0, pbar_a + pbar_b), then stage 2 hands [s, s + p_a - pbar_a) to a) but a
    under the cumulative partition."""
    qv, g = 0.4, 0.5
    Ks = _two_stage_counterexample(qv, g)
    c = qs.Circuit(1)
    c.gate(qs.H, (0,), 0)
    c.kraus(Ks, (0,), 1)
    pbar_a = (1 - qv) * (1 - g)
    p_a = (1 - qv) * (1 - g / 2)
    pbar_b = qv * (1 - g)
    hits = 0
    for seed in range(4000):
        r = orc.u01(seed, 0, 0, 0)
        d = orc.run_trajectory(c, orc.DELAYED, seed=seed)["kraus_idx"][0]
        e = orc.run_trajectory(c, orc.EAGER, seed=seed)["kraus_idx"][0]
        cu = orc.run_trajectory(c, orc.CUMULATIVE, seed=seed)["kraus_idx"][0]
        assert d == e
        if pbar_a + 1e-9 < r < p_a - 1e-9:
            assert d == 1 and cu == 0
            hits += 1
        if r < pbar_a - 1e-9:
            assert d == 0 and cu == 0
        if pbar_a + 1e-9 < r < pbar_a + pbar_b - 1e-9:
            assert d == 1
    assert hits > 50


def test_stage1_deferral_rate(orc):
    g = 0.05
    c = qs.Circuit(2)
    for layer in range(20):
        c.gate(qs.SQRT_X, (0,), 2 * layer)
        c.gate(qs.SQRT_Y, (1,), 2 * layer)
        c.channel(qs.amplitude_damping(g), (0,), 2 * layer + 1)
        c.channel(qs.amplitude_damping(g), (1,), 2 * layer + 1)
    T = 2000
    res = orc.run_trajectories(c, T, mode=orc.DELAYED, seed=1)
    frac1 = np.mean(res["stage"] == 1)
    s = 1 - g
    se = math.sqrt(s * (1 - s) / res["stage"].size)
    assert abs(frac1 - s) < 5 * se


def test_full_amplitude_damping_resets(orc):
    c = qs.Circuit(3)
    for q in range(3):
        c.gate(qs.random_unitary(2, np.random.default_rng(q)), (q,), 0)
    c.gate(qs.CNOT, (0, 2), 1)
    for q in range(3):
        c.channel(qs.amplitude_damping(1.0), (q,), 2)
    for seed in range(20):
        psi = orc.run_trajectory(c, orc.DELAYED, seed=seed)["state"]
        assert abs(abs(psi[0]) - 1.0) < 1e-14


def test_zero_noise_equals_noiseless(orc):
    noisy = qs.chain_circuit(6, 8, 0, dep1=0.0, dep2=0.0, layer_ad=0.0)
    clean = qs.chain_circuit(6, 8, 0)
    a = orc.run_trajectory(noisy, orc.DELAYED, seed=3)["state"]
    b = orc.run_trajectory(clean)["state"]
    np.testing.assert_allclose(a, b, atol=1e-14)


def test_phase_damping_keeps_z_populations(orc):
    rng = np.random.default_rng(6)
    n = 4
    c = qs.Circuit(n)
    c.gate(qs.random_unitary(16, rng), (0, 1, 2, 3), 0)
    ref = orc.run_trajectory(c)["state"]
    for q in range(n):
        c.channel(qs.phase_damping(0.7), (q,), 1)
    exact = orc.density_evolve(c)
    np.testing.assert_allclose(np.real(np.diag(exact)), np.abs(ref) ** 2, atol=1e-14)


def test_reductions_independent_of_thread_count(orc, tmp_path):
    code = (
        "import sys, numpy as np; sys.path.insert(0, %r); import oracle as o;"
        "rng=np.random.default_rng(0); n=18;"
        "psi=rng.normal(size=1<<n)+1j*rng.normal(size=1<<n);"
        "K=np.stack([np.eye(2)*0.6, np.array([[0,0.8],[0,0]])]).astype(complex);"
        "P=o.kraus_norms(psi,[7],K); e=o.expect_z(psi,[5,1<<17]);"
        "print(repr(o.norm2(psi)), repr(list(P)), repr(list(e)))"
    ) % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for th in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=th)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, check=True,
                                   capture_output=True, text=True).stdout)
    assert outs[0] == outs[1]
