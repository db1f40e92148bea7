"""Kernel micro-benchmark, a companion of bench.py: the fused-gate kernel
(Alg. 1), the read passes, whole trajectories and the batched kernel, each
timed alone.

Times each kernel through the C ABI's state-level calls on a device state
of 2^n complex64 amplitudes, with CUDA events on the launching stream after
warm-up, and reports achieved bandwidth against the algorithmic bytes:
16 * 2^n per fused-gate pass (read + write), 8 * 2^n per read pass.

    python kernel_bench.py --n 30 --k 4
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

PATTERNS = {
    "high": lambda n, k: list(range(n - k, n)),
    "mid": lambda n, k: [n // 2 + 2 * j for j in range(k)],
    "low0": lambda n, k: list(range(k)),
    "low1": lambda n, k: list(range(1, k + 1)),
    "mixed": lambda n, k: [0] + list(range(n - k + 1, n)),
    "spread": lambda n, k: [int(round(j * (n - 1) / max(k - 1, 1))) for j in range(k)],
    "low123": lambda n, k: [1, 2, 3] + [n // 2 + j for j in range(k - 3)],
}


def main(argv=None):
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch

    import paper_2111_02396_gb300 as pkg

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=28)
    ap.add_argument("--k", type=int, nargs="+", default=[1, 2, 3, 4, 5])
    ap.add_argument("--patterns", nargs="+", default=list(PATTERNS))
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reads", action="store_true", help="also time the read passes")
    ap.add_argument("--tf32", action="store_true", help="split-TF32 tensor-core path (k = 4..6)")
    ap.add_argument("--grid", type=int, nargs=2, metavar=("ROWS", "COLS"),
                    help="instead: time whole trajectories of the damped grid workload on a ROWS x COLS grid")
    ap.add_argument("--fuse", type=int, default=4, help="--grid: fusion width")
    ap.add_argument("--grouping", action="store_true", help="--grid: multi-gate passes")
    ap.add_argument("--batch", type=int, metavar="COUNT",
                    help="time the batched persistent kernel on COUNT circuits of the mixed-width workload")
    ap.add_argument("--threads", type=int, default=512, help="--batch: threads per CTA")
    ap.add_argument("--min-n", type=int, default=0, help="--batch: keep circuits with n >= this")
    ap.add_argument("--max-n", type=int, default=64, help="--batch: keep circuits with n <= this")
    args = ap.parse_args(argv)
    if args.grid:
        return grid_runs(args)
    if args.batch:
        return batch_runs(args)
    pkg.load()
    n = args.n
    st = torch.cuda.current_stream()
    d = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    d[0] = 1
    rng = np.random.default_rng(0)
    rows = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timeit(fn, nbytes):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(args.reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
        return ms, nbytes / (ms / 1e3) / 1e9

    for k in args.k:
        q, _ = np.linalg.qr(rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k)))
        for pat in args.patterns:
            qubits = PATTERNS[pat](n, k)
            prec = pkg.QT_TF32X3 if args.tf32 else pkg.QT_FP32
            ms, gbs = timeit(lambda: pkg.qt_state_apply(d.data_ptr(), n, qubits, q, precision=prec,
                                                        stream=st.cuda_stream), 16 << n)
            rows.append(dict(kernel="apply_tf32x3" if args.tf32 else "apply", n=n, k=k, pattern=pat,
                             qubits=qubits, ms=ms, gbs=gbs))
            print(json.dumps(rows[-1]), flush=True)
    if args.reads:
        for q in (1, 2):
            ms, gbs = timeit(lambda: pkg.qt_state_reduced_density(d.data_ptr(), n, list(range(n - q, n)),
                                                                  stream=st.cuda_stream), 8 << n)
            print(json.dumps(dict(kernel="rdm", n=n, q=q, ms=ms, gbs=gbs)), flush=True)
        masks = [1 << j for j in range(min(n, 16))]
        ms, gbs = timeit(lambda: pkg.qt_state_expect_z(d.data_ptr(), n, masks, stream=st.cuda_stream), 8 << n)
        print(json.dumps(dict(kernel="expect16", n=n, ms=ms, gbs=gbs)), flush=True)
        ms, gbs = timeit(lambda: pkg.qt_state_sample(d.data_ptr(), n, 0, 0, 100, stream=st.cuda_stream), 8 << n)
        print(json.dumps(dict(kernel="sample100", n=n, ms=ms, gbs=gbs)), flush=True)


def batch_runs(args):
    """The batched persistent form on circuits of the 8192-circuit workload (n ~ U{8..18})."""
    import torch

    import paper_2111_02396_gb300 as pkg
    import qtsynth as qs
    pkg.load()
    ccs, i = [], 0
    while len(ccs) < args.batch:
        cc = qs.config2_compact(i)
        if args.min_n <= cc.num_qubits <= args.max_n:
            ccs.append(cc)
        i += 1
    fused = pkg.fuse_many([pkg.Circuit.from_compact(c) for c in ccs], args.fuse)
    b = pkg.Batch(fused)
    sh = torch.cuda.current_stream().cuda_stream
    for w in range(args.warmup):
        b.run(seed=0, first_traj=w * args.batch, samples_per_traj=100, threads=args.threads, stream=sh)
    ms = []
    for r in range(args.reps):
        b.run(seed=0, first_traj=(args.warmup + r) * args.batch, samples_per_traj=100, threads=args.threads,
              stream=sh)
        ms.append(b.stats()["device_ms"])
    amps = np.array([1 << c.num_qubits for c in ccs], dtype=np.float64)
    nf = np.array([f.info()["num_fused"] for f in fused], dtype=np.float64)
    med = float(np.median(ms))
    row = dict(kernel="batch", count=args.batch, fuse=args.fuse, threads=args.threads, min_n=args.min_n,
               max_n=args.max_n, ms=med, traj_per_s=args.batch / (med / 1e3),
               eff_gbs=float(np.sum(nf * amps * 16)) / (med / 1e3) / 1e9)
    print(json.dumps(row), flush=True)


def grid_runs(args):
    """Whole trajectories (all kernels of the plain loop) on a smaller grid."""
    import torch

    import paper_2111_02396_gb300 as pkg
    import qtsynth as qs
    pkg.load()
    rows, cols = args.grid
    n = rows * cols
    circ = qs.config1_circuit(rows=rows, cols=cols)
    f = pkg.Fused(pkg.Circuit.from_synth(circ), args.fuse)
    sh = torch.cuda.current_stream().cuda_stream
    for i in range(args.warmup):
        pkg.Run(f, 1, seed=0, first_traj=100 + i, grouping=args.grouping, stream=sh)
    torch.cuda.synchronize()
    r = pkg.Run(f, args.reps, seed=0, time_kernels=True, grouping=args.grouping, stream=sh)
    st = r.stats()
    row = dict(kernel="grid_run", n=n, fuse=args.fuse, grouping=args.grouping, traj=args.reps,
               ms_per_traj=st["device_ms"] / args.reps, passes_per_traj=st["fused_passes"] / args.reps,
               pieces_per_traj=st["fused_pieces"] / args.reps,
               pass_gbs=st["apply_bytes"] / (st["apply_ms"] / 1e3) / 1e9 if st["apply_ms"] else None,
               gate_equiv_gbs=(st["fused_pieces"] * 16 * (1 << n)) / (st["apply_ms"] / 1e3) / 1e9
               if st["apply_ms"] else None)
    print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
