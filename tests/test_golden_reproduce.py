"""The stored steady states under tests/golden/ are the oracle's as it stands.

The JSON fixtures that the GPU steady-state tests compare against were written
by the committed scripts beside them, which call only the FP64 oracle.  Here
the cheapest case of each is run again through the same script functions, and
every stored number must come back (the step count exactly, the values within
1e-12 relative): a fixture edited by hand, written by anything else, or left
behind by a later change of the oracle's arithmetic fails.
"""
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


@pytest.fixture(scope="module")
def scripts():
    sys.path.insert(0, GOLDEN)
    try:
        import make_mass_flow_curve
        import make_pressure_steady
    finally:
        sys.path.remove(GOLDEN)
    return make_mass_flow_curve, make_pressure_steady


def same(got, want, keys):
    for k in keys:
        g, w = np.asarray(got[k], dtype=float), np.asarray(want[k], dtype=float)
        assert g.shape == w.shape, k
        assert np.all(np.abs(g - w) <= 1e-12 * np.maximum(np.abs(w), 1e-300)), (k, got[k], want[k])


def test_mass_flow_curve_case_reproduces(scripts):
    curve, _ = scripts
    doc = json.load(open(os.path.join(GOLDEN, "mass_flow_curve_801x8.json")))
    want = doc["cases"][0]
    assert want["kn_out"] == 0.02
    got = curve.run(want["kn_out"], 0)
    assert got["steps"] == want["steps"] and got["converged"]
    same(got, want, ("mass_flow", "S", "u_slip", "ux_max", "total_mass", "residual"))


def test_pressure_steady_case_reproduces(scripts):
    _, steady = scripts
    doc = json.load(open(os.path.join(GOLDEN, "pressure_1601x16_steady.json")))
    want = doc["cases"][0]
    assert want["kn_out"] == 0.0194
    got = steady.run(want["kn_out"], 0)
    assert got["steps"] == want["steps"] and got["converged"]
    assert got["cols"] == want["cols"]
    same(got, want, ("mass_flow", "q_norm", "u_slip", "ux_max", "total_mass", "residual", "ux_prof_outlet",
                     "dp_nonlin", "m_of_x"))
