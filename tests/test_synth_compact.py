"""The array-form generator builds exactly the circuits of the object-form one."""
import numpy as np
import pytest

import qtsynth as qs


def _same(a, b):
    assert a.num_qubits == b.num_qubits and len(a.ops) == len(b.ops)
    for x, y in zip(a.ops, b.ops):
        assert x.kind == y.kind and x.qubits == y.qubits and x.moment == y.moment
        np.testing.assert_array_equal(x.mats, y.mats)
        if x.probs is None:
            assert y.probs is None
        else:
            np.testing.assert_array_equal(x.probs, y.probs)


@pytest.mark.parametrize("i", [0, 1, 7, 4095])
def test_config2_compact_matches(i):
    _same(qs.config2_compact(i).to_circuit(), qs.config2_circuit(i))


def test_request_compact_matches():
    for req in qs.serving_requests(6, seed=3, nmax=14, dmax=14):
        _same(qs.request_compact(req).to_circuit(), qs.request_circuit(req))
