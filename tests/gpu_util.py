"""Shared helpers of the GPU parity tests."""
import numpy as np


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.fail("GPU test selected but no CUDA device is visible")
    return torch


def random_state(n, seed, dtype=np.complex64):
    rng = np.random.default_rng([0x77, n, seed])
    v = rng.standard_normal(2 << n, dtype=np.float32).view(np.complex64)
    v /= np.float32(np.sqrt(np.vdot(v, v).real))
    return v.astype(dtype, copy=False)


def to_device(psi64):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(psi64)).cuda()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(abs(np.vdot(b, a)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


# Tolerances.  States after a whole circuit: relative L2 <= 2e-5 and
# fidelity >= 1 - 1e-5 against the FP64 oracle.  One kernel call on
# complex64 data: each output is a sum of at most 64 FP32 products, so its
# rounding error is below 64 * 2^-24 ~ 4e-6 of the row norm; 2e-6 in
# relative L2 is the bound used for a single fused gate (k <= 5).
STATE_L2 = 2e-5
STATE_FID = 1e-5
KERNEL_L2 = 2e-6
# Branch and sample parity: decisions must agree where the oracle's margin
# (distance of the draw to the nearest partition boundary, relative to the
# total) exceeds 1e-6; closer draws are ties.
MARGIN = 1e-6
