"""The parity rule (tests/parity.py) is itself checked on the CPU: it must
accept a correct implementation that rounds differently (the oracle compiled
with FMA contraction) and reject a planted error of 1e-4 in the rates."""
import platform

import numpy as np
import pytest

import oracle
from mc_inputs import network_13, synthetic_cells
from parity import classify, compare


@pytest.mark.skipif(platform.machine() not in ("x86_64", "AMD64"), reason="FMA twin needs x86-64 FMA")
def test_rule_accepts_rounding_twin_and_rejects_planted_error():
    net = network_13()
    cells = synthetic_cells(net, 2048, seed=3)
    on = oracle.OracleNetwork(net)
    (o, stable) = classify(on, cells, 1e10, oracle.burn)
    t = oracle.burn(on, cells, 1e10, rtol=1e-10, atol=1e-16)
    assert 0.7 < stable.mean() < 1.0
    twin = oracle.oracle.rounding_twin()
    b = twin.burn(twin.OracleNetwork(net), cells, 1e10)
    assert not np.array_equal(b[0], o[0])  # it really rounds differently
    rep = compare(b[0], b[1], b[2], o[0], o[1], o[2], o[3], stable=stable, tight=(t[0], t[1]))
    assert rep["pass"], rep
    bad = network_13()
    bad.A_r = bad.A_r * 1.0001
    m = oracle.burn(oracle.OracleNetwork(bad), cells, 1e10)
    rep = compare(m[0], m[1], m[2], o[0], o[1], o[2], o[3], stable=stable, tight=(t[0], t[1]))
    assert not rep["pass"], rep
