"""GPU checks of the serving loop (continuous batching).

Each request gives the same result served alone as in a mix of concurrent
requests (bitwise: its work depends only on its own circuit, seed and
trajectory ids), served small requests match the FP64 oracle (samples where
the CDF margin exceeds 1e-6), and the in-flight footprint never exceeds the
budget.
"""
import numpy as np
import pytest

import qtsynth as qs
from gpu_util import MARGIN, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qt():
    import paper_2111_02396_gb300 as pkg
    pkg.load()
    torch_cuda()
    return pkg


def _requests(qt, count=14, seed=5):
    reqs = qs.serving_requests(count, seed=seed, nmin=10, nmax=20, dmin=6, dmax=12, tmax=24, samples=20)
    out = []
    for r in reqs:
        f = qt.Fused(qt.Circuit.from_compact(qs.request_compact(r)), 4)
        out.append((r, f))
    return out


def test_alone_equals_in_mix(qt):
    reqs = _requests(qt)
    assert any(r["n"] <= 16 for r, _ in reqs) and any(r["n"] > 16 for r, _ in reqs)
    budget = 64 << 30
    mix = qt.Server(budget, max_slots=4, small_n_max=16)
    ids = [mix.submit(f, seed=r["seed"], first_traj=0, num_traj=r["num_traj"], samples_per_traj=r["samples"])
           for r, f in reqs]
    for i in ids:
        mix.wait(i, timeout_s=300)
    mixed = [mix.result(i)[0] for i in ids]
    st = mix.stats()
    assert st["done"] == len(reqs) and st["peak_inflight_bytes"] <= budget
    nb = sum(mix.info(i)["batched"] for i in ids)
    assert nb >= 2 and 1 <= st["lane_launches"] < nb           # small requests shared launches
    mix.close()
    alone_srv = qt.Server(budget, max_slots=1, small_n_max=16)
    for (r, f), m in zip(reqs, mixed):
        i = alone_srv.submit(f, seed=r["seed"], first_traj=0, num_traj=r["num_traj"],
                             samples_per_traj=r["samples"])
        alone_srv.wait(i, timeout_s=300)
        a, inf = alone_srv.result(i)
        np.testing.assert_array_equal(a, m)
    alone_srv.close()


def test_served_requests_match_oracle(qt, orc):
    reqs = [x for x in _requests(qt, count=10, seed=8) if x[0]["n"] <= 13][:3]
    srv = qt.Server(16 << 30, max_slots=2, small_n_max=16)
    for r, f in reqs:
        T = min(r["num_traj"], 6)
        i = srv.submit(f, seed=r["seed"], first_traj=0, num_traj=T, samples_per_traj=r["samples"])
        srv.wait(i, timeout_s=300)
        smp, inf = srv.result(i)
        assert inf["batched"] == 1
        circ = qs.request_compact(r).to_circuit()
        for t in range(T):
            ref = orc.run_trajectory(circ, orc.DELAYED, seed=r["seed"], traj=t)
            if np.any(ref["margin"] <= MARGIN):
                continue
            want, margin = orc.sample(ref["state"], r["seed"], t, r["samples"])
            ok = margin > MARGIN
            np.testing.assert_array_equal(smp[t][ok], want[ok])
    srv.close()


def test_served_plain_requests_match_oracle(qt, orc):
    """Requests on the plain workers (their trajectories share the default-choice
    prefix) against the oracle, and against the server's per-trajectory loop."""
    reqs = [x for x in _requests(qt, count=16, seed=11) if 15 <= x[0]["n"] <= 18][:2]
    assert reqs
    shared = qt.Server(16 << 30, max_slots=2, small_n_max=0)
    plain = qt.Server(16 << 30, max_slots=2, small_n_max=0, share_prefix=False)
    for r, f in reqs:
        T = min(r["num_traj"], 6)
        out = []
        for srv in (shared, plain):
            i = srv.submit(f, seed=r["seed"], first_traj=0, num_traj=T, samples_per_traj=r["samples"])
            srv.wait(i, timeout_s=300)
            smp, inf = srv.result(i)
            assert inf["batched"] == 0
            out.append(smp)
        circ = qs.request_compact(r).to_circuit()
        for t in range(T):
            ref = orc.run_trajectory(circ, orc.DELAYED, seed=r["seed"], traj=t)
            if np.any(ref["margin"] <= MARGIN):
                continue
            want, margin = orc.sample(ref["state"], r["seed"], t, r["samples"])
            ok = margin > MARGIN
            for smp in out:
                np.testing.assert_array_equal(smp[t][ok], want[ok])
    shared.close()
    plain.close()


def test_lane_merges_requests_with_their_own_seeds(qt, orc):
    """One merged launch over trajectories of several requests (different circuits,
    seeds and trajectory ranges): each request's samples equal the oracle's for its
    own seed and ids."""
    reqs = [x for x in _requests(qt, count=20, seed=13) if x[0]["n"] <= 12][:4]
    srv = qt.Server(16 << 30, max_slots=1, small_n_max=14)
    ids = []
    for k, (r, f) in enumerate(reqs):
        ids.append(srv.submit(f, seed=r["seed"], first_traj=10 * k, num_traj=3, samples_per_traj=r["samples"]))
    for i in ids:
        srv.wait(i, timeout_s=300)
    assert srv.stats()["lane_launches"] <= len(reqs)
    for k, ((r, f), i) in enumerate(zip(reqs, ids)):
        smp, inf = srv.result(i)
        assert inf["batched"] == 1
        circ = qs.request_compact(r).to_circuit()
        for t in range(3):
            ref = orc.run_trajectory(circ, orc.DELAYED, seed=r["seed"], traj=10 * k + t)
            if np.any(ref["margin"] <= MARGIN):
                continue
            want, margin = orc.sample(ref["state"], r["seed"], 10 * k + t, r["samples"])
            ok = margin > MARGIN
            np.testing.assert_array_equal(smp[t][ok], want[ok])
    srv.close()
