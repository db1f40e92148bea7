"""Multi-GPU replicas, tested on the CPU with two gloo ranks.

Trajectories are independent jobs (Sec. IV.C runs them as separate cluster
jobs), so the path shards by trajectory id with no data exchange: in step s,
rank w runs the ids bench.trajectory_ids(w, W, s, T) gives it, and only the
tiny results are gathered.  With counter-based Philox draws the union over
ranks must equal one process running all ids -- branch records, samples and
states.  Each rank runs the oracle here (no GPU) on the ids of bench.py's
own mapping, the one --gpus N uses.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import qtsynth as qs

T = 12
S = 40


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


STEPS = 2


def _bench():
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def _rank_main(rank, world, port, out_dir):
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = _bench()
    circ = qs.random_noisy_circuit(6, 50, 21, noise=0.2, channel_prob=0.5)
    mine = []
    for step in range(STEPS):
        lo, cnt = bench.trajectory_ids(rank, world, step, T // (world * STEPS))
        res = oracle.run_trajectories(circ, cnt, seed=77, traj0=lo)
        smp = np.stack([oracle.sample(res["states"][t], 77, lo + t, S)[0] for t in range(cnt)])
        mine.append((lo, res["kraus_idx"], smp, res["states"]))
    # gather the per-rank results (no other communication)
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    if rank == 0:
        parts = sorted((p for rp in parts for p in rp), key=lambda p: p[0])
        np.save(os.path.join(out_dir, "ids.npy"), np.concatenate([p[0] + np.arange(len(p[2])) for p in parts]))
        np.save(os.path.join(out_dir, "kraus.npy"), np.concatenate([p[1] for p in parts]))
        np.save(os.path.join(out_dir, "samples.npy"), np.concatenate([p[2] for p in parts]))
        np.save(os.path.join(out_dir, "states.npy"), np.concatenate([p[3] for p in parts]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_equal_single_process(orc, tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    circ = qs.random_noisy_circuit(6, 50, 21, noise=0.2, channel_prob=0.5)
    ref = orc.run_trajectories(circ, T, seed=77, traj0=0)
    ref_smp = np.stack([orc.sample(ref["states"][t], 77, t, S)[0] for t in range(T)])
    np.testing.assert_array_equal(np.load(tmp_path / "ids.npy"), np.arange(T))
    np.testing.assert_array_equal(np.load(tmp_path / "kraus.npy"), ref["kraus_idx"])
    np.testing.assert_array_equal(np.load(tmp_path / "samples.npy"), ref_smp)
    np.testing.assert_array_equal(np.load(tmp_path / "states.npy"), ref["states"])


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_bench_rank_trajectory_ranges_partition_the_ids(world):
    """bench.trajectory_ids over every rank and step covers the ids [0, steps * W * T)
    exactly once: no trajectory is run twice and none is skipped."""
    bench = _bench()
    per, steps = 16, 23
    ids = []
    for step in range(steps):
        for rank in range(world):
            lo, cnt = bench.trajectory_ids(rank, world, step, per)
            assert cnt == per
            ids.extend(range(lo, lo + cnt))
    assert sorted(ids) == list(range(steps * world * per))
    assert bench.dist_env() == (0, 1, 0) or "RANK" in os.environ
