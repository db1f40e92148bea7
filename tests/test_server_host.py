"""Serving loop scheduling on the CPU (dry-run executor, no GPU work).

Plain workers: admission never lets the in-flight footprint exceed the
budget, every request finishes, a request larger than the budget is
refused at submit, injected worker deaths are requeued by id and the
workers replaced, injected allocation failures are deferred and retried,
and queued requests can be cancelled.  Batch lane: small requests that
arrive together share merged launches, its state slots are reserved
against the budget, a lane that dies holding a launch has every request
of it requeued and is replaced, and allocation failures defer the whole
launch.
"""
import time

import pytest

import qtsynth as qs


@pytest.fixture(scope="module")
def qt():
    import paper_2111_02396_gb300 as pkg
    pkg.load()
    return pkg


def _fused(qt, n, depth=4, seed=0):
    c = qt.Circuit.from_synth(qs.chain_circuit(n, depth, seed, dep1=1e-3, layer_ad=1e-3))
    return qt.Fused(c, 3)


def test_admission_respects_budget(qt):
    fs = [_fused(qt, n, seed=n) for n in (10, 14, 18, 20, 22, 24)]
    budget = 2 * (8 << 24) + (64 << 20)        # room for one 24-qubit request (two states) plus scratch
    srv = qt.Server(budget, max_slots=6, small_n_max=0, dry_run=True)
    ids = [srv.submit(fs[i % len(fs)], seed=i, num_traj=1 + i % 5, samples_per_traj=3) for i in range(60)]
    for i in ids:
        srv.wait(i, timeout_s=60)
    st = srv.stats()
    assert st["done"] == 60 and st["failed"] == 0
    assert 0 < st["peak_inflight_bytes"] <= budget
    assert st["inflight_bytes"] == 0
    for i in ids:
        smp, inf = srv.result(i)
        assert smp.shape == (inf["num_traj"], 3) and inf["latency_s"] >= 0
    srv.close()


def test_oversized_request_refused(qt):
    from paper_2111_02396_gb300.qt import QtError, QT_ERR_OUT_OF_MEMORY
    srv = qt.Server(1 << 20, max_slots=2, dry_run=True)
    with pytest.raises(QtError) as ei:
        srv.submit(_fused(qt, 20), num_traj=1)
    assert ei.value.status == QT_ERR_OUT_OF_MEMORY
    srv.close()


def test_worker_death_is_requeued(qt):
    from paper_2111_02396_gb300.qt import QT_FAULT_WORKER_EXIT
    f = _fused(qt, 12)
    srv = qt.Server(1 << 34, max_slots=3, small_n_max=0, dry_run=True)
    srv.inject(QT_FAULT_WORKER_EXIT, 2)
    ids = [srv.submit(f, seed=i, num_traj=2, samples_per_traj=4) for i in range(20)]
    for i in ids:
        srv.wait(i, timeout_s=60)
    st = srv.stats()
    assert st["done"] == 20 and st["requeued"] == 2
    deadline = time.time() + 10
    while srv.stats()["workers_alive"] < 3 and time.time() < deadline:
        time.sleep(0.01)
    assert srv.stats()["workers_alive"] == 3
    assert sum(srv.info(i)["attempts"] for i in ids) == 22
    srv.close()


def test_allocation_failure_is_deferred(qt):
    from paper_2111_02396_gb300.qt import QT_FAULT_ALLOC
    f = _fused(qt, 12)
    srv = qt.Server(1 << 34, max_slots=2, small_n_max=0, dry_run=True)
    srv.inject(QT_FAULT_ALLOC, 3)
    ids = [srv.submit(f, seed=i, num_traj=1, samples_per_traj=2) for i in range(8)]
    for i in ids:
        srv.wait(i, timeout_s=60)
    st = srv.stats()
    assert st["done"] == 8 and st["failed"] == 0 and st["deferred"] == 3
    srv.close()


def test_cancel_queued_request(qt):
    f_big = _fused(qt, 26)
    f = _fused(qt, 10)
    srv = qt.Server(1 << 34, max_slots=1, small_n_max=0, dry_run=True)
    first = srv.submit(f_big, num_traj=3)       # keeps the only slot busy for a while
    later = [srv.submit(f, seed=i) for i in range(4)]
    srv.cancel(later[2])
    for i in [first] + later:
        srv.wait(i, timeout_s=60)
    assert srv.poll(later[2]) == 4               # cancelled
    assert all(srv.poll(i) == 2 for i in [first, later[0], later[1], later[3]])
    srv.close()


def test_lane_merges_small_requests(qt):
    # small requests that arrive together share launches; the large ones run on
    # the plain workers; everything finishes with its own sample shape
    small = [_fused(qt, n, seed=n) for n in (8, 10, 12, 14)]
    big = _fused(qt, 22)
    srv = qt.Server(1 << 34, max_slots=2, small_n_max=16, dry_run=True)
    ids = [srv.submit(small[i % 4], seed=i, num_traj=1 + i % 7, samples_per_traj=5) for i in range(40)]
    ids += [srv.submit(big, seed=99, num_traj=2, samples_per_traj=5)]
    for i in ids:
        srv.wait(i, timeout_s=60)
    st = srv.stats()
    assert st["done"] == 41 and st["failed"] == 0
    assert 1 <= st["lane_launches"] < 40                       # merged launches
    assert st["lane_trajectories"] == sum(1 + i % 7 for i in range(40))
    for k, i in enumerate(ids):
        smp, inf = srv.result(i)
        assert inf["batched"] == (1 if k < 40 else 0)
        assert smp.shape == (inf["num_traj"], 5)
    srv.close()


def test_lane_reservation_counts_against_budget(qt):
    # 16-qubit lane states need one 2^16-amplitude slot per SM, reserved at start
    srv = qt.Server(1 << 34, max_slots=2, small_n_max=16, dry_run=True)
    st = srv.stats()
    assert st["lane_bytes"] == (8 << 16) * 152 and st["inflight_bytes"] == st["lane_bytes"]
    srv.close()
    # a budget too small for the slots keeps the lane to shared-memory states
    srv = qt.Server(100 << 20, max_slots=2, small_n_max=16, dry_run=True)
    assert srv.stats()["lane_bytes"] == 0
    f15 = _fused(qt, 15)
    i = srv.submit(f15, num_traj=100, samples_per_traj=2)    # 15 qubits: not for this lane
    srv.wait(i, timeout_s=60)
    assert srv.info(i)["batched"] == 0
    srv.close()


def test_lane_death_requeues_its_launch(qt):
    from paper_2111_02396_gb300.qt import QT_FAULT_WORKER_EXIT
    f = _fused(qt, 12)
    srv = qt.Server(1 << 34, max_slots=1, small_n_max=14, dry_run=True)
    srv.inject(QT_FAULT_WORKER_EXIT, 1)
    ids = [srv.submit(f, seed=i, num_traj=3, samples_per_traj=4) for i in range(12)]
    for i in ids:
        srv.wait(i, timeout_s=60)
    st = srv.stats()
    assert st["done"] == 12 and st["failed"] == 0 and st["requeued"] >= 1
    att = [srv.info(i)["attempts"] for i in ids]
    assert sum(att) == 12 + st["requeued"] and max(att) == 2
    deadline = time.time() + 10
    while srv.stats()["workers_alive"] < 2 and time.time() < deadline:
        time.sleep(0.01)
    assert srv.stats()["workers_alive"] == 2                 # worker + replacement lane
    srv.close()


def test_lane_allocation_failure_defers_the_launch(qt):
    from paper_2111_02396_gb300.qt import QT_FAULT_ALLOC
    f = _fused(qt, 11)
    srv = qt.Server(1 << 34, max_slots=1, small_n_max=14, dry_run=True)
    srv.inject(QT_FAULT_ALLOC, 2)
    ids = [srv.submit(f, seed=i, num_traj=2, samples_per_traj=3) for i in range(6)]
    for i in ids:
        srv.wait(i, timeout_s=60)
    st = srv.stats()
    assert st["done"] == 6 and st["failed"] == 0 and st["deferred"] >= 2
    srv.close()
