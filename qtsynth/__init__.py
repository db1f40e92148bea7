"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This package only builds inputs: noisy random circuits shaped like the
paper's workloads (random circuits of depth 16-40 on chains and grids,
Sec. III.F), the gate matrices they use and the Kraus / mixture lists of the
noise channels (Sec. II and Sec. V.B). It contains none of the simulation
arithmetic (no gate application, no lower bounds, no fusion, no sampling).
"""
from .circuits import (  # noqa: F401
    KIND_GATE, KIND_KRAUS, KIND_MIXTURE, Op, Circuit,
    SQRT_X, SQRT_Y, SQRT_W, CZ, H, CNOT, X, Y, Z, I2,
    amplitude_damping, phase_damping, depolarizing, decay_dephasing,
    fsim, random_unitary,
    chain_circuit, grid_circuit, config0_circuit, config1_circuit,
    config2_circuit, config3_circuit, serving_requests,
    ghz_circuit, qft_circuit, random_noisy_circuit, noise_model_circuit,
)
from .circuits import request_circuit  # noqa: F401,E402
from .compact import CompactCircuit, layered_compact, config2_compact, request_compact  # noqa: F401,E402
