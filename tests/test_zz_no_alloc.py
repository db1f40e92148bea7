"""The allocation-free probability pass against the allocating one.

qt_state_reduced_density_noalloc serves callers that cannot let the library
allocate device memory (an application that owns all GPU memory through its
own pool, or a latency-critical loop that must not stall on cudaMalloc /
cudaFree): its scratch is a fixed array compiled into libqt.so.  This test
calls it through the C ABI twice in a row on different inputs (the array
keeps the previous call's contents, so the second call checks that nothing
stale leaks in) and compares each result with qt_state_reduced_density on
the same state.  It is collected last so that a run stopped at its first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_util import random_state, to_device, torch_cuda

pytestmark = pytest.mark.gpu


def _noalloc(lib, ptr, n, qubits):
    fn = lib.qt_state_reduced_density_noalloc
    fn.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    q = np.ascontiguousarray(qubits, dtype=np.uint32)
    D = 1 << len(q)
    out = np.zeros(D * D, dtype=np.complex128)
    st = fn(ptr, n, len(q), q.ctypes.data, out.ctypes.data, None)
    assert st == 0, lib.qt_last_error().decode()
    return out.reshape(D, D)


def test_noalloc_matches_allocating_entry_point():
    torch_cuda()
    import paper_2111_02396_gb300 as pkg
    lib = pkg.load()
    cases = [(20, [3, 17]), (16, [0, 5, 9]), (12, [11])]
    for call, (n, qubits) in enumerate(cases):
        psi = random_state(n, 30 + call)
        d = to_device(psi)
        got = _noalloc(lib, d.data_ptr(), n, qubits)
        want = pkg.qt_state_reduced_density(d.data_ptr(), n, qubits)
        np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-9)
        assert abs(np.trace(got).real - 1.0) < 1e-5


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch_cuda()
    import paper_2111_02396_gb300 as pkg
    lib = pkg.load()
    d = to_device(random_state(8, 1))
    fn = lib.qt_state_reduced_density_noalloc
    fn.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    q = np.arange(4, dtype=np.uint32)
    out = np.zeros(256, dtype=np.complex128)
    st = fn(d.data_ptr(), 8, 4, q.ctypes.data, out.ctypes.data, None)
    assert st == -6 and b"fixed scratch" in lib.qt_last_error()
