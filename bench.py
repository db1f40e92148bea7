#!/usr/bin/env python
"""Trajectory throughput on one GB300 (or N replicas, one per GPU).

Workload (one step = one batch of trajectories per GPU): the 30-qubit 5x6
grid random circuit of depth 20 ({sqrt X, sqrt Y, sqrt W} layers, CZ on
alternating grid couplings), amplitude damping 5e-4 and phase damping 5e-4
on every qubit after every layer (1200 channels), fused to 4 qubits, 16
trajectories per GPU with the delayed inner-product algorithm (Alg. 2),
100 bitstrings sampled from every final state.  Complex64 state (8 GiB,
larger than L2, so no L2 flush is needed between steps).

Prints one JSON line (rank 0).  At N = 1 the line also carries the three
systems forms of the metric, each measured in its own timed region with its
own clock record: "batched" (8192 circuits of 8..18 qubits in one persistent
launch, against the plain loop on the same GPU), "served" (a Poisson request
stream with continuous batching, p50/p99 latency, against serving the same
stream request by request) and "precision" (32-qubit circuits fused to 6
qubits on tensor cores in split TF32, against FP32 CUDA-core comparators,
error against the FP64 oracle at 26 qubits).  --impl reference times the
FP64 CPU oracle on a bounded sample of the grid workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "trajectories/s & %HBM peak: served/batched vs plain, p50/p99 at L2 err≤2e-5"
UNIT = "trajectories/s"
N_QUBITS = 30
FUSE_K = 4
SAMPLES = 100
WORKLOAD = ("grid30: 5x6 grid, depth 20, sqrtX/sqrtY/sqrtW + CZ, amplitude damping 5e-4 + "
            "phase damping 5e-4 per qubit per layer, fused k=4, delayed inner products, "
            "100 samples per trajectory")

# DRAM bytes per launch of the fused-gate kernel from an ncu capture, keyed by
# the SHA-256 of the kernel code it was taken on, comments and blank lines left
# out (null once the code changes).
KNOWN_TRAFFIC = {
    # k_apply_tile<4, 4, 8>: 4.244 GB per launch at n = 28 (dram read + write), x4 for n = 30
    "5b97b48612739d2b": 4 * (2147519744 + 2096363776),
}


def kernel_source_hash() -> str:
    # code only: line comments and blank lines do not change the kernel
    with open(os.path.join(ROOT, "paper_2111_02396_gb300", "csrc", "k_apply.cu")) as f:
        lines = (re.sub(r"//.*$", "", line).rstrip() for line in f)
        code = "\n".join(x for x in lines if x)
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.uuid = device_uuid
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def trajectory_ids(rank, world, step, per_rank):
    """(first id, count) of the trajectories rank `rank` of `world` runs in step
    `step`: the step's world * per_rank ids form one contiguous range, split into
    contiguous per-rank parts, so the union over ranks of every step is the same
    set of ids one process would run (trajectories are independent jobs, and the
    counter-based draws depend only on the id)."""
    return (step * world + rank) * per_rank, per_rank


# ----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands on a bounded sample
# ----------------------------------------------------------------------------
def oracle_sample(target_s=15.0, psi=None):
    """Run the oracle on the first M ops of trajectory 0 of the workload, M
    doubled from 8 until one run takes at least a third of target_s (so the
    whole sampling stays within about target_s).  Returns trajectories/s
    scaled by (total ops / M) and a description."""
    import numpy as np

    import oracle
    import qtsynth as qs
    oracle.build()
    circ = qs.config1_circuit()
    fc = oracle.FlatCircuit(circ)
    total = len(circ.ops)
    if psi is None:
        psi = np.empty(1 << N_QUBITS, dtype=np.complex128)
    M = 8
    while True:
        t0 = time.perf_counter()
        oracle.run_trajectory(fc, oracle.DELAYED, seed=0, traj=0, max_ops=M, psi=psi)
        dt = time.perf_counter() - t0
        if dt >= target_s / 3 or M >= total:
            break
        M = min(total, 2 * M)
    value = (M / total) / dt
    cores = len(os.sched_getaffinity(0))
    desc = (f"first {M} of {total} ops of trajectory 0 of the 30-qubit workload (FP64 oracle, "
            f"unfused, {cores} OpenMP threads), {dt:.1f} s, scaled by {total}/{M}")
    return value, cores, desc, psi


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    psi = np.empty(1 << N_QUBITS, dtype=np.complex128)
    vals, step_ms = [], []
    desc = ""
    cores = len(os.sched_getaffinity(0))
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        v, cores, desc, psi = oracle_sample(target_s=args.ref_seconds, psi=psi)
        if step >= args.warmup:
            vals.append(v)
            step_ms.append((time.perf_counter() - t0) * 1e3)
    value = statistics.median(vals)
    # a step is one bounded sample of the workload (wall time, including the
    # doubling of the sample length); value is the throughput it measures
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "num_qubits": N_QUBITS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def delayed_vs_eager(pkg, fused, sh, traj0, T=2):
    """The same trajectories (seed 0, ids traj0..) with delayed and with eager inner products
    (Alg. 2 vs the conventional per-channel evaluation): device time per trajectory, and the
    number of branch records that differ (the two-stage partition makes both modes pick the
    same operator for the same draw; a difference can only come from a draw within rounding
    of a boundary)."""
    d = pkg.Run(fused, T, seed=0, first_traj=traj0, mode=pkg.QT_DELAYED, stream=sh)
    e = pkg.Run(fused, T, seed=0, first_traj=traj0, mode=pkg.QT_EAGER, stream=sh)
    kd, ke = d.kraus_indices()[0], e.kraus_indices()[0]
    sd, se = d.stats(), e.stats()
    return {"trajectories": T, "delayed_ms_per_traj": sd["device_ms"] / T,
            "eager_ms_per_traj": se["device_ms"] / T,
            "eager_over_delayed": se["device_ms"] / sd["device_ms"],
            "probability_passes_per_traj": {"delayed": sd["prob_passes"] / T, "eager": se["prob_passes"] / T},
            "branch_records": int(kd.size), "differing_branch_records": int((kd != ke).sum())}


def bandwidth_probe(pkg, qs, sh):
    """One noiseless trajectory of the 32-qubit 4x8 grid (32 GiB state), depth 20, fused to k = 4:
    the fused-gate passes' rate per gate width, timed with events around every pass."""
    circ = qs.grid_circuit(4, 8, 20, 0)
    f = pkg.Fused(pkg.Circuit.from_synth(circ), FUSE_K)
    r = pkg.Run(f, 1, seed=0, time_kernels=True, stream=sh)
    st = r.stats()
    by_w = {}
    for w in range(1, 8):
        if st["passes_by_width"][w]:
            by_w[str(w)] = {"passes": st["passes_by_width"][w],
                            "gbs": st["passes_by_width"][w] * (16 << 32) / (st["apply_ms_by_width"][w] / 1e3) / 1e9}
    return {"workload": "noiseless 4x8 grid (n = 32, 32 GiB complex64), depth 20, fused k = 4, one trajectory",
            "ms": st["device_ms"], "fused_passes": st["fused_passes"],
            "all_passes_gbs": st["apply_bytes"] / (st["apply_ms"] / 1e3) / 1e9, "by_width": by_w}


def run_ours(args):
    import torch

    import paper_2111_02396_gb300 as pkg
    import qtsynth as qs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.load()
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    circ = qs.config1_circuit()
    qc = pkg.Circuit.from_synth(circ)
    fused = pkg.Fused(qc, FUSE_K)
    T = args.traj

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def step(i, flags=False):
        first, cnt = trajectory_ids(rank, world, i, T)
        return pkg.Run(fused, cnt, seed=0, first_traj=first, samples_per_traj=SAMPLES,
                       time_kernels=flags, stream=sh)

    for i in range(args.warmup):
        step(i)
    # ---- device-timed loop (inputs resident: fused circuit built once) ----
    uuid = device_uuid(local)
    clocks = ClockSampler(uuid)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    apply_ms = apply_bytes = launches = passes = folded = flushes = gate_ops = 0
    ms_w = [0.0] * 8
    passes_w = [0] * 8
    for i in range(args.steps):
        r = step(args.warmup + i, flags=True)
        s = r.stats()
        gate_ops += s["gate_ops"]
        apply_ms += s["apply_ms"]
        apply_bytes += s["apply_bytes"]
        launches += s["kernel_launches"]
        passes += s["fused_passes"]
        folded += s["folded_pieces"]
        flushes += s["flushes"]
        for w in range(8):
            ms_w[w] += s["apply_ms_by_width"][w]
            passes_w[w] += s["passes_by_width"][w]
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * T * args.steps / (ms / 1e3)

    # ---- end-to-end loop through the public API with host buffers ----
    barrier()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for i in range(args.steps):
        qc2 = pkg.Circuit.from_synth(circ)             # host op arrays -> library
        f2 = pkg.Fused(qc2, FUSE_K)
        first, cnt = trajectory_ids(rank, world, args.warmup + i, T)
        r = pkg.Run(f2, cnt, seed=0, first_traj=first, samples_per_traj=SAMPLES, stream=sh)
        smp = r.samples()                              # result on the host
        s = r.stats()
        h2d += s["h2d_bytes"]
        d2h += s["d2h_bytes"]
        assert smp.shape == (T, SAMPLES)
    barrier()
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = world * T * args.steps / e2e_s

    peak, peak_kind = measured_peaks()
    # the dominant kernel: the gate width with the most fused-pass device time
    wdom = max(range(1, 8), key=lambda w: ms_w[w])
    pass_bytes = 16 << N_QUBITS
    achieved = passes_w[wdom] * pass_bytes / (ms_w[wdom] / 1e3) / 1e9 if ms_w[wdom] > 0 else 0.0
    achieved_all = (apply_bytes / (apply_ms / 1e3)) / 1e9 if apply_ms > 0 else 0.0
    traffic = KNOWN_TRAFFIC.get(kernel_source_hash()) if wdom == FUSE_K else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "num_qubits": N_QUBITS, "trajectories_per_step_per_gpu": T,
                   "fuse_k": FUSE_K, "mode": "delayed", "samples_per_traj": SAMPLES,
                   "fused_passes_per_traj": passes / (T * args.steps),
                   "folded_pieces_per_traj": folded / (T * args.steps),
                   "flushes_per_traj": flushes / (T * args.steps),
                   "l2": "no flush: every pass streams the 8 GiB state (> 129 MB L2)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": f"k_apply_tile<{wdom}> ({wdom}-qubit fused-gate apply)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "frac_of_8TBs_nominal": achieved / 8000.0,
                     "traffic": traffic,
                     "bytes_per_launch": pass_bytes,
                     "launches": passes_w[wdom],
                     "share_of_fused_pass_time": ms_w[wdom] / apply_ms if apply_ms > 0 else None,
                     "all_fused_passes_gbs": achieved_all},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                "d2h_bytes_per_step": d2h // args.steps},
        "gpu_launches": launches,
        "clocks": clk,
    }
    line["amplitude_updates_per_s"] = world * passes * float(1 << N_QUBITS) / (ms / 1e3)
    line["gate_equivalent_updates_per_s"] = world * gate_ops * float(1 << N_QUBITS) / (ms / 1e3)
    if rank == 0 and world == 1 and not args.no_extras:
        line["delayed_vs_eager"] = delayed_vs_eager(pkg, fused, sh, 9_000_000)
        line["bandwidth_probe_n32"] = bandwidth_probe(pkg, qs, sh)
    if rank == 0 and world == 1 and not args.no_forms:
        # the systems forms of the metric, each in its own timed region
        line["batched"] = batched_form(uuid=uuid)
        line["served"] = served_form(args.requests, args.slots, uuid)
        line["precision"] = precision_form(uuid=uuid)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc, _ = oracle_sample(target_s=args.ref_seconds)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------
# The three systems forms beside the plain loop.  Each form is a function that
# returns its result object; the default run adds all three to the grid30 line
# (each with the clocks sampled during its own GPU-timed region), and
# --workload batch / serve / precision prints one of them as a line of its own.
# ----------------------------------------------------------------------------
BATCH_WORKLOAD = ("batch8192: 8192 circuits, n ~ U{8..18}, 1D chain, depth 40, sqrtX/sqrtY/sqrtW + CZ, "
                  "depolarizing 1e-3 then amplitude damping 1e-3 on every gate-qubit, one trajectory each, "
                  "100 samples per trajectory")


def device_uuid(local=0):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:  # noqa: BLE001 -- sample all GPUs instead
        return None


def batched_form(steps=3, warmup=2, num=8192, plain_stride=32, uuid=None):
    """Config 2: 8192 circuits of uneven size, one trajectory each, in one persistent
    launch replayed as a CUDA graph, against the plain per-trajectory loop on the same
    GPU (every plain_stride-th circuit, scaled) and the FP64 oracle."""
    import concurrent.futures as cf

    import numpy as np
    import torch

    import oracle
    import paper_2111_02396_gb300 as pkg
    import qtsynth as qs

    pkg.load()
    oracle.build()
    t0 = time.perf_counter()
    ccs = [qs.config2_compact(i) for i in range(num)]
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        qcs = list(ex.map(pkg.Circuit.from_compact, ccs))
    t_create = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    t0 = time.perf_counter()
    tune, table = pkg.autotune_batch(qcs, sample=256, kmin=2, kmax=6, stream=sh)
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    fused = pkg.fuse_by_class(qcs, tune)
    t_fuse = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch = pkg.Batch(fused)
    t_pack = time.perf_counter() - t0
    launch = dict(use_graph=True, threads=tune["threads_shared"], threads_global=tune["threads_global"], stream=sh)
    for i in range(warmup):
        batch.run(seed=0, first_traj=i * num, samples_per_traj=SAMPLES, **launch)
    clk = ClockSampler(uuid)
    torch.cuda.synchronize()
    clk.start()
    ms = []
    for i in range(steps):
        batch.run(seed=0, first_traj=(warmup + i) * num, samples_per_traj=SAMPLES, **launch)
        ms.append(batch.stats()["device_ms"])
    clocks = clk.stop()
    batched = num / (statistics.median(ms) / 1e3)
    # plain per-trajectory loop on every stride-th circuit, scaled to the batch
    idx = list(range(0, num, plain_stride))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in idx:
        pkg.Run(fused[i], 1, seed=0, first_traj=i, samples_per_traj=SAMPLES, stream=sh)
    torch.cuda.synchronize()
    plain = num / ((time.perf_counter() - t0) * plain_stride)
    # accuracy against the FP64 oracle: trajectories of every size class
    pick = []
    for n in range(8, 19, 2):
        pick += [i for i in range(num) if ccs[i].num_qubits == n][:2]
    sub = pkg.Batch([fused[i] for i in pick]).run(seed=0, first_traj=0, samples_per_traj=0, keep_states=True,
                                                  stream=sh)
    errs = []
    for j, i in enumerate(pick):
        ref = oracle.run_trajectory(ccs[i].to_circuit(), oracle.DELAYED, seed=0, traj=j)
        if np.all(ref["margin"] > 1e-6):
            g = sub.state(j).astype(np.complex128)
            errs.append(float(np.linalg.norm(g - ref["state"]) / np.linalg.norm(ref["state"])))
    # the FP64 oracle on the host cores, on a spread sample of the batch
    stride_o = max(1, num // 32)
    sample_o = list(range(0, num, stride_o))
    t0 = time.perf_counter()
    for i in sample_o:
        ref = oracle.run_trajectory(ccs[i].to_circuit(), oracle.DELAYED, seed=0, traj=i)
        oracle.sample(ref["state"], 0, i, SAMPLES)
    t_orc = time.perf_counter() - t0
    st = batch.stats()
    amps = np.array([1 << c.num_qubits for c in ccs], dtype=np.float64)
    nf = np.array([f.info()["num_fused"] for f in fused], dtype=np.float64)
    med_s = statistics.median(ms) / 1e3
    eff_gbs = float(np.sum(nf * amps * 16)) / med_s / 1e9
    peak, peak_kind = measured_peaks()
    return {
        "workload": BATCH_WORKLOAD, "trajectories_per_run": num, "runs": steps, "warmup_runs": warmup,
        "traj_per_s": batched, "ms_per_run": statistics.median(ms),
        "autotuned": tune, "cuda_graph": True,
        "plain_loop": {"traj_per_s": plain,
                       "sample": f"every {plain_stride}th circuit ({len(idx)} trajectories), qt_run_trajectories "
                                 f"one trajectory at a time on the same GPU, scaled by {plain_stride}"},
        "speedup_vs_plain": batched / plain,
        "amplitude_updates_per_s": float(np.sum(nf * amps)) / med_s,
        "effective_bandwidth": {"achieved": eff_gbs, "peak": peak, "unit": "GB/s", "frac": eff_gbs / peak,
                                "peak_kind": peak_kind,
                                "note": "algorithmic bytes (16 B x 2^n per fused gate, those folded into the "
                                        "product-state start included) / kernel time; states of <= 2^14 "
                                        "amplitudes live in shared memory, so this is not an HBM figure"},
        "l2_err_max": max(errs) if errs else None,
        "l2_err_sample": f"{len(errs)} trajectories (2 of each n in 8, 10, .., 18) against the FP64 oracle",
        "autotune_ms": {f"{c}_k{k}_t{t}": v for (c, k, t), v in table.items()},
        "cpu_baseline": {"value": len(sample_o) / t_orc, "unit": UNIT, "cores": len(os.sched_getaffinity(0)),
                         "kind": "oracle",
                         "sample": f"every {stride_o}th circuit ({len(sample_o)} trajectories with {SAMPLES} "
                                   f"samples), FP64 oracle, {t_orc:.1f} s"},
        "host_s": {"generate": t_gen, "create": t_create, "autotune": t_tune, "fuse": t_fuse, "pack": t_pack},
        "flushes_per_traj": st["flushes"] / num,
        "fused_gates_per_traj": float(np.mean(nf)),
        "folded_pieces_per_traj": st["folded_pieces"] / num,
        "clocks": clocks,
    }


def run_batch(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    b = batched_form(args.steps, args.warmup, args.batch_size, args.plain_stride, device_uuid(local))
    line = {
        "metric": METRIC, "value": b["traj_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms_per_run"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "form": "batched",
        "config": {"workload": BATCH_WORKLOAD}, "batched": b,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


SERVE_WORKLOAD = ("serve: requests with n ~ U{10..28}, depth ~ U{10..30}, chain or grid, depolarizing and "
                  "amplitude damping ~ logU[1e-4, 1e-2], trajectories ~ logU[1, 512], 100 samples per "
                  "trajectory, Poisson arrivals at 0.9x the plain loop's service rate, 150 GB HBM budget")


def serve_stream(pkg, fused, reqs, arrivals, *, slots, small_n_max, budget, keep=(), share_prefix=True):
    """Serve the stream; keep: request indices whose samples are returned."""
    srv = pkg.Server(budget, max_slots=slots, small_n_max=small_n_max, share_prefix=share_prefix)
    ids = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for k, r in enumerate(reqs):
            dt = arrivals[k] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids[k] = srv.submit(fused[k], seed=r["seed"], first_traj=0, num_traj=r["num_traj"],
                                samples_per_traj=r["samples"])

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    for i in ids:
        srv.wait(i)
    lat = [srv.info(i)["latency_s"] for i in ids]
    done = time.perf_counter() - t0
    st = srv.stats()
    batched = sum(srv.info(i)["batched"] for i in ids)
    kept = {k: srv.result(ids[k])[0] for k in keep}
    srv.close()
    return lat, done, st, batched, kept


def served_form(requests=160, slots=8, uuid=None):
    """Config 4: the first `requests` requests of the seeded 2000-request stream, served
    with continuous batching under a 150 GB budget, against the plain loop serving the
    same stream request by request; Poisson arrivals at 0.9x the plain loop's service
    rate, and a burst (all at t = 0) for the capacity of each form."""
    import concurrent.futures as cf

    import numpy as np
    import torch

    import oracle
    import paper_2111_02396_gb300 as pkg
    import qtsynth as qs

    pkg.load()
    oracle.build()
    R = requests
    reqs = qs.serving_requests(R, seed=0)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        qcs = list(ex.map(lambda r: pkg.Circuit.from_compact(qs.request_compact(r)), reqs))
    fused = pkg.fuse_many(qcs, 4)
    budget = 150 * 10**9
    clk = ClockSampler(uuid)
    torch.cuda.synchronize()
    clk.start()
    # calibration = the plain loop's burst: the whole stream request by request,
    # every trajectory on its own
    plain = dict(slots=1, small_n_max=0, budget=budget, share_prefix=False)
    served = dict(slots=slots, small_n_max=20, budget=budget)
    lat_c, t_cal, _, _, _ = serve_stream(pkg, fused, reqs, [0.0] * R, **plain)
    rate = 0.9 * R / t_cal
    rng = np.random.default_rng(1234)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, R)).tolist()
    arrivals = [a - arrivals[0] for a in arrivals]
    total_traj = sum(r["num_traj"] for r in reqs)
    # oracle parity on a seeded subsample: every 25th request with n <= 20, its first trajectory
    sub = [k for k in range(0, R, 25) if reqs[k]["n"] <= 20]
    lat_s, t_s, st_s, nb, kept = serve_stream(pkg, fused, reqs, arrivals, keep=sub, **served)
    lat_p, t_p, _, _, _ = serve_stream(pkg, fused, reqs, arrivals, **plain)
    lat_b, t_b, st_b, _, _ = serve_stream(pkg, fused, reqs, [0.0] * R, **served)
    # the same served burst with the plain workers' trajectories run one by one
    # (merged launches and concurrency only, no shared prefixes)
    lat_n, t_n, _, _, _ = serve_stream(pkg, fused, reqs, [0.0] * R, share_prefix=False, **served)
    clocks = clk.stop()
    compared = mismatched = 0
    for k in sub:
        r = reqs[k]
        ref = oracle.run_trajectory(qs.request_compact(r).to_circuit(), oracle.DELAYED, seed=r["seed"], traj=0)
        want, margin = oracle.sample(ref["state"], r["seed"], 0, r["samples"])
        ok = margin > 1e-6
        compared += int(ok.sum())
        mismatched += int(np.sum(kept[k][0][ok] != want[ok]))
    pct = lambda v, q: float(np.percentile(np.asarray(v), q))
    return {
        "workload": SERVE_WORKLOAD, "requests": R, "of_stream": 2000, "trajectories": total_traj,
        "slots": slots, "arrival_rate_per_s": rate, "budget_bytes": budget,
        "batched_requests": "n <= 14, or n <= 20 with >= 64 trajectories",
        "poisson": {"served": {"traj_per_s": total_traj / t_s, "p50_s": pct(lat_s, 50), "p99_s": pct(lat_s, 99),
                               "makespan_s": t_s, "peak_inflight_bytes": st_s["peak_inflight_bytes"],
                               "requests_batched": nb, "lane_launches": st_s["lane_launches"]},
                    "plain_request_by_request": {"traj_per_s": total_traj / t_p, "p50_s": pct(lat_p, 50),
                                                 "p99_s": pct(lat_p, 99), "makespan_s": t_p}},
        "burst": {"served_traj_per_s": total_traj / t_b, "plain_traj_per_s": total_traj / t_cal,
                  "served_p50_s": pct(lat_b, 50), "served_p99_s": pct(lat_b, 99),
                  "plain_p50_s": pct(lat_c, 50), "plain_p99_s": pct(lat_c, 99),
                  "capacity_ratio": t_cal / t_b, "lane_launches": st_b["lane_launches"],
                  "served_without_shared_prefix": {"traj_per_s": total_traj / t_n, "p50_s": pct(lat_n, 50),
                                                   "p99_s": pct(lat_n, 99), "capacity_ratio": t_cal / t_n}},
        "forms": {"served": "batch lane (small requests merged into shared launches of the batched kernel) + "
                            f"{slots} plain workers whose requests share their trajectories' default-choice prefix",
                  "plain_request_by_request": "one worker, the plain per-trajectory loop, no lane, no sharing"},
        "parity": {"requests": sub, "samples_compared": compared, "sample_mismatches": mismatched,
                   "note": "first trajectory of every 25th request with n <= 20 against the FP64 oracle; "
                           "samples whose CDF margin is <= 1e-6 are ties and not compared"},
        "clocks": clocks,
    }


def run_serve(args):
    import torch

    torch.cuda.set_device(0)
    f = served_form(args.requests, args.slots, device_uuid(0))
    line = {
        "metric": METRIC, "value": f["poisson"]["served"]["traj_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": f["poisson"]["served"]["makespan_s"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "form": "served",
        "config": {"workload": SERVE_WORKLOAD, "requests": args.requests}, "served": f,
    }
    print(json.dumps(line), flush=True)
    return 0


PRECISION_WORKLOAD = ("precision: 4x8 grid (n=32) [2x13 grid (n=26) for the error], depth 24, "
                      "sqrtX/sqrtY/sqrtW + CZ, depolarizing 1e-3 on every gate-qubit")


def precision_form(traj=32, traj_fp32_k6=4, oracle_traj=2, uuid=None):
    """Config 3: 6-qubit fused gates on tensor cores in split TF32 against two FP32
    CUDA-core comparators: the same k = 6 plan (k_apply_tile6) and the same circuit
    fused to k = 4 (k_apply_tile<4>, the plain loop's kernel).  Throughput and norm
    drift at n = 32, error against the FP64 oracle at n = 26."""
    import numpy as np
    import torch

    import oracle
    import paper_2111_02396_gb300 as pkg
    import qtsynth as qs

    pkg.load()
    oracle.build()
    sh = torch.cuda.current_stream().cuda_stream
    forms = (("tf32x3_k6", pkg.QT_TF32X3, 6, traj), ("fp32_k6", pkg.QT_FP32, 6, traj_fp32_k6),
             ("fp32_k4", pkg.QT_FP32, 4, traj))
    # error against the FP64 oracle at n = 26
    c26 = qs.config3_circuit(rows=2, cols=13, depth=24)
    t0 = time.perf_counter()
    refs = [oracle.run_trajectory(c26, oracle.DELAYED, seed=0, traj=t)["state"] for t in range(oracle_traj)]
    t_orc = time.perf_counter() - t0
    errs = {}
    for name, prec, k, _ in forms:
        r = pkg.Run(pkg.Fused(pkg.Circuit.from_synth(c26), k), oracle_traj, seed=0, precision=prec,
                    keep_states=True, stream=sh)
        l2, fid = [], []
        for t in range(oracle_traj):
            g = r.state(t).astype(np.complex128)
            ref = refs[t]
            l2.append(float(np.linalg.norm(g - ref) / np.linalg.norm(ref)))
            fid.append(float(abs(np.vdot(ref, g)) ** 2 / (np.vdot(g, g).real * np.vdot(ref, ref).real)))
        errs[name] = {"trajectories": oracle_traj, "rel_l2_max": max(l2), "fidelity_min": min(fid)}
    # throughput and norm drift at n = 32
    c32 = qs.config3_circuit()
    res = {}
    clk = ClockSampler(uuid)
    for name, prec, k, T in forms:
        f = pkg.Fused(pkg.Circuit.from_synth(c32), k)
        pkg.Run(f, 1, seed=0, first_traj=10_000, precision=prec, stream=sh)     # warm-up
        if name == "tf32x3_k6":
            torch.cuda.synchronize()
            clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = pkg.Run(f, T, seed=0, precision=prec, samples_per_traj=SAMPLES, time_kernels=True, stream=sh)
        e1.record()
        torch.cuda.synchronize()
        st = r.stats()
        ms = e0.elapsed_time(e1)
        res[name] = {"trajectories": T, "traj_per_s": T / (ms / 1e3),
                     "amplitude_updates_per_s": st["fused_passes"] * float(1 << 32) / (ms / 1e3),
                     "apply_gbs": st["apply_bytes"] / (st["apply_ms"] / 1e3) / 1e9,
                     "fused_passes_per_traj": st["fused_passes"] / T,
                     "norm_drift_max": float(np.max(np.abs(r.norms() - 1.0))),
                     "error_n26": errs[name]}
    clocks = clk.stop()
    peak, kind = measured_peaks()
    tc = res["tf32x3_k6"]
    best_fp32 = max(("fp32_k6", "fp32_k4"), key=lambda nm: res[nm]["traj_per_s"])
    return {
        "workload": PRECISION_WORKLOAD, "n32": res, "traj_per_s": tc["traj_per_s"],
        "tf32x3_over_best_fp32": tc["traj_per_s"] / res[best_fp32]["traj_per_s"], "best_fp32": best_fp32,
        "roofline": {"bound": "hbm", "kernel": "k_apply_tc<6> (split-TF32 tcgen05)", "achieved": tc["apply_gbs"],
                     "peak": peak, "unit": "GB/s", "frac": tc["apply_gbs"] / peak, "peak_kind": kind},
        "cpu_baseline": {"value": oracle_traj / t_orc, "unit": "trajectories/s (n = 26)",
                         "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                         "sample": f"{oracle_traj} trajectories of the 26-qubit error workload (FP64, unfused), "
                                   f"{t_orc:.1f} s"},
        "clocks": clocks,
    }


def run_precision(args):
    import torch

    torch.cuda.set_device(0)
    f = precision_form(args.traj_precision, min(args.traj_precision, 4), 4, device_uuid(0))
    line = {"metric": METRIC, "value": f["traj_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * f["n32"]["tf32x3_k6"]["trajectories"] / f["traj_per_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "form": "precision", "config": {"workload": PRECISION_WORKLOAD},
            "precision": f, "roofline": f["roofline"]}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# runtime vs noise strength (the shape of the paper's Fig. 3): phase damping
# after every layer, delayed inner products vs the conventional algorithm
# ----------------------------------------------------------------------------
def run_noise_sweep(args):
    import numpy as np
    import torch

    import paper_2111_02396_gb300 as pkg
    import qtsynth as qs

    torch.cuda.set_device(0)
    pkg.load()
    sh = torch.cuda.current_stream().cuda_stream
    lams = [1e-4, 1e-3, 1e-2, 1e-1]
    table = {}
    for n, (rows, cols), T in ((20, (4, 5), 8), (27, (3, 9), 4)):
        rows_out = {}
        for lam in lams:
            circ = qs.grid_circuit(rows, cols, 20, 0, layer_pd=lam)
            f = pkg.Fused(pkg.Circuit.from_synth(circ), 4)
            entry = {}
            for name, mode in (("delayed", pkg.QT_DELAYED), ("eager", pkg.QT_EAGER)):
                pkg.Run(f, 1, seed=1, first_traj=999, mode=mode, stream=sh)        # warm-up
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0 = time.perf_counter()
                e0.record()
                r = pkg.Run(f, T, seed=1, mode=mode, samples_per_traj=SAMPLES, stream=sh)
                e1.record()
                torch.cuda.synchronize()
                wall = time.perf_counter() - t0
                st = r.stats()
                entry[name] = {"ms_per_traj": wall * 1e3 / T, "device_ms_per_traj": e0.elapsed_time(e1) / T,
                               "prob_passes_per_traj": st["prob_passes"] / T,
                               "fused_passes_per_traj": st["fused_passes"] / T}
            entry["eager_over_delayed"] = entry["eager"]["ms_per_traj"] / entry["delayed"]["ms_per_traj"]
            rows_out[str(lam)] = entry
        d = np.array([rows_out[str(l)]["delayed"]["ms_per_traj"] for l in lams])
        slope, icpt = np.polyfit(np.array(lams), d, 1)
        table[f"n{n}"] = {"lambda": rows_out, "delayed_linear_fit_ms": {"slope_per_unit_lambda": slope,
                                                                         "intercept": icpt}}
    line = {"metric": METRIC, "unit": UNIT, "form": "noise-sweep", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "grid random circuits depth 20, phase damping lambda per qubit per layer, "
                                   "fused k=4, 100 samples per trajectory (Fig. 3 shape)"},
            "sweep": table,
            "value": table["n27"]["lambda"]["0.0001"]["eager_over_delayed"],
            "value_meaning": "eager / delayed runtime at n=27, lambda=1e-4 (the paper reports ~10x)"}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# small workload: 10-qubit chain, 64 trajectories x 100 samples
# ----------------------------------------------------------------------------
def run_chain10(args):
    import numpy as np
    import torch

    import paper_2111_02396_gb300 as pkg
    import qtsynth as qs

    torch.cuda.set_device(0)
    pkg.load()
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    circ = qs.config0_circuit()
    f = pkg.Fused(pkg.Circuit.from_synth(circ), 2)
    T = 64
    res = {}
    for name in ("plain", "batched"):
        times = []
        b = pkg.Batch([f] * T) if name == "batched" else None
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            if b is None:
                r = pkg.Run(f, T, seed=0, first_traj=i * T, samples_per_traj=SAMPLES, stream=sh)
                smp = r.samples()
            else:
                smp = b.run(seed=0, first_traj=i * T, samples_per_traj=SAMPLES, use_graph=True,
                            stream=sh).samples()
            times.append(time.perf_counter() - t0)
            assert smp.shape == (T, SAMPLES)
        t = statistics.median(times[args.warmup:])
        res[name] = {"traj_per_s": T / t, "ms_per_64_traj": t * 1e3}
    # the FP64 oracle on the host cores: all 64 trajectories with their samples
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    ref = oracle.run_trajectories(circ, T, seed=0, traj0=0, keep_states=True)
    for t in range(T):
        oracle.sample(ref["states"][t], 0, t, SAMPLES)
    t_orc = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    # parity of the batched records against it (ties, margin <= 1e-6, are not compared)
    b = pkg.Batch([f] * T).run(seed=0, first_traj=0, samples_per_traj=SAMPLES, keep_states=True, stream=sh)
    smp = b.samples()
    errs, bad_rec, bad_smp, compared = [], 0, 0, 0
    for t in range(T):
        if np.any(ref["margin"][t] <= 1e-6):
            continue
        compared += 1
        kr, _ = b.kraus_indices(t)
        bad_rec += int(np.sum(kr != ref["kraus_idx"][t]))
        g = b.state(t).astype(np.complex128)
        w = ref["states"][t]
        errs.append(float(np.linalg.norm(g - w) / np.linalg.norm(w)))
        want, margin = oracle.sample(w, 0, t, SAMPLES)
        ok = margin > 1e-6
        bad_smp += int(np.sum(smp[t][ok] != want[ok]))
    line = {"metric": METRIC, "value": res["batched"]["traj_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "form": "chain10",
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": "chain10: 10-qubit chain, depth 16, depolarizing 1e-3 / 1e-2, amplitude "
                                   "damping 1e-3, 64 trajectories x 100 samples, fused k=2"},
            "plain": res["plain"], "batched": res["batched"],
            "speedup_vs_plain": res["batched"]["traj_per_s"] / res["plain"]["traj_per_s"],
            "cpu_baseline": {"value": T / t_orc, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"all {T} trajectories with {SAMPLES} samples each (FP64, unfused, "
                                       f"OpenMP over trajectories), {t_orc:.2f} s"},
            "parity": {"trajectories_compared": compared, "branch_record_mismatches": bad_rec,
                       "sample_mismatches": bad_smp, "state_rel_l2_max": max(errs) if errs else None}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--traj", type=int, default=16, help="trajectories per step per GPU")
    ap.add_argument("--ref-seconds", type=float, default=15.0, help="oracle sample length")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="grid30: skip the delayed-vs-eager comparison and the 32-qubit bandwidth probe")
    ap.add_argument("--workload", choices=["grid30", "chain10", "batch", "serve", "precision", "noise-sweep"],
                    default="grid30",
                    help="grid30: the plain loop at scale (default); batch: the batched form; "
                         "serve: the serving loop")
    ap.add_argument("--no-forms", action="store_true",
                    help="grid30: skip the batched, served and precision forms")
    ap.add_argument("--requests", type=int, default=160, help="serve: requests of the stream")
    ap.add_argument("--slots", type=int, default=8, help="serve: concurrent requests")
    ap.add_argument("--traj-precision", type=int, default=32, help="precision: trajectories at n=32")
    ap.add_argument("--batch-size", type=int, default=8192)
    ap.add_argument("--plain-stride", type=int, default=32)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "noise-sweep":
        return run_noise_sweep(args)
    if args.workload == "chain10":
        return run_chain10(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
