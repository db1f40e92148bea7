"""GB300 (sm_103a) quantum-trajectory simulator for noisy circuits.

Implements the hot path of "Simulations of Quantum Circuits with
Approximate Noise using qsim and Cirq" (arXiv 2111.02396): fused k-qubit
gates (Sec. III.A-B, Alg. 1) and sampled Kraus operators applied to a
complex64 state vector, with branch probabilities from the delayed
inner-product algorithm (Sec. III.E, Alg. 2).  The compute runs in the
hand-written CUDA kernels of libqt.so (C ABI in include/qt.h); this package
is its Python binding.
"""
from . import qt  # noqa: F401
from .qt import (  # noqa: F401
    Circuit, Fused, Run, QtError, load, lib_path, use_torch_allocator,
    QT_DELAYED, QT_EAGER, QT_FP32, QT_TF32X3,
    qt_state_apply, qt_state_reduced_density, qt_state_sample, qt_state_expect_z, qt_state_cdf,
    qt_state_kraus_probabilities,
    kernel_arch,
    Batch, fuse_many, fuse_by_class, autotune_batch, Server, SMEM_N_MAX,
)
