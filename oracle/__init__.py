"""FP64 CPU oracle for the quantum-trajectory method of arXiv 2111.02396.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference arm of ``bench.py``.  The product path
(``paper_2111_02396_gb300``) never imports it, and it never imports the
product.  It shares nothing with the CUDA library except the seeded input
generators of ``qtsynth``.

Parity status of every function is pinned by ``tests/test_oracle_*.py``
(closed forms, brute force, exact density-matrix evolution, known-answer
vectors); no function is "parity unpinned".
"""
from .oracle import (  # noqa: F401
    build, lib_path, philox4x32_10, u01, apply, norm2, kraus_norms, lower_bound,
    run_trajectory, run_trajectories, sample, readout, expect_z, density_evolve,
    DELAYED, EAGER, CUMULATIVE, FlatCircuit,
)
