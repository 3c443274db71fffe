"""The full-size tests' sigma gate (tests/golden_ref.py) on the CPU: the
stored oracle values pass against themselves, a planted error fails, and the
SHA-256 check refuses values stored for other bytes of G."""
import numpy as np
import pytest

import golden_ref
from paper_1008_1371_gb300 import workloads as W


def test_gate_on_stored_values():
    G, J = W.graded(1024, decades=6.0, seed=2)
    try:
        s, k = golden_ref.load("graded1024", G)
    except AssertionError as e:  # this host rounds G differently: nothing to compare
        pytest.skip(str(e))
    assert golden_ref.gate(J, s, s, k)[:2] == (0.0, 0.0)
    t = s.copy()
    j = int(np.argmax(2 * k <= 1e-12))  # a value held to 1e-12
    t[j] *= 1 + 2e-12
    assert golden_ref.gate(J, t, s, k)[1] > 1e-12
    with pytest.raises(AssertionError):
        golden_ref.assert_gate(J, t, s, k)
    t[j] = s[j] * (1 + 0.5e-12)
    golden_ref.assert_gate(J, t, s, k)
    loose = np.where(2 * k > 1e-12)[0]
    if loose.size:
        t = s.copy()
        t[loose[0]] *= 1 + 1.9 * k[loose[0]]
        golden_ref.assert_gate(J, t, s, k)
        t[loose[0]] = s[loose[0]] * (1 + 2.5 * k[loose[0]])
        with pytest.raises(AssertionError):
            golden_ref.assert_gate(J, t, s, k)


def test_load_refuses_other_bytes():
    G, J = W.graded(1024, decades=6.0, seed=2)
    G = G.copy()
    G[3, 4] = np.nextafter(G[3, 4], np.inf)
    with pytest.raises(AssertionError):
        golden_ref.load("graded1024", G)
