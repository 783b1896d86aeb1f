"""The pressure-driven mass-flow study of Sec. 3.2 (Fig. 7): TMAC sigma =
0.93 (r_b from Eq. 21 with B1 = 1 - 0.1817 sigma), p_in/p_out = 1.8, the local
Knudsen number from the centreline pressure, L/H = 100 (ny = 8, nx = 801),
run to steady state for several outlet Knudsen numbers.  The experimental
and analytical curves the paper compares with are not available, so the
checks are the properties the method must show (a uniform mass flow along
the channel, and S = m/m_ns above 1 and growing with Kn_out) and, value by
value, the FP64 oracle's steady S at the same step count
(tests/golden/mass_flow_curve_801x8.json, written by the oracle alone).  The
paper's second abscissa is Kn_ave = (Kn_in + Kn_out)/2 with
Kn_in = Kn_out p_out/p_in."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KN_OUT = (0.02, 0.05, 0.1, 0.2, 0.4)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mass_flow_curve_801x8.json")


@pytest.fixture(scope="module")
def clb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1603_01955_gb300.clb as clb

    return clb


def steady(ch, chunk=20000, tol=1e-9, cap=2_000_000):
    o = ch.observables()
    done = 0
    while done < cap:
        ch.step(chunk)
        done += chunk
        o = ch.observables()
        if 0 <= o["residual"] < tol:
            break
    return o, done


def test_mass_flow_rate_curve(clb):
    S = []
    for kn in KN_OUT:
        ch = clb.Channel(801, 8, kn, sigma=0.93, drive="pressure", drive_value=1.8, storage="fp64", kn_mode=1)
        o, steps = steady(ch)
        assert o["residual"] < 1e-9, (kn, steps)
        m = o["m_of_x"][1:-1]
        assert np.abs(m - m.mean()).max() <= 1e-6 * m.mean()
        S.append(o["q_norm"])
        ch.close()
    S = np.array(S)
    assert (S > 1).all()
    assert (np.diff(S) > 0).all()
    # Kn_ave of the paper's second plot: the inlet Knudsen number is Kn_out p_out/p_in
    kn_ave = 0.5 * (np.array(KN_OUT) / 1.8 + np.array(KN_OUT))
    assert np.allclose(kn_ave, np.array(KN_OUT) * (1 + 1 / 1.8) / 2)


def test_steady_S_matches_oracle(clb):
    """S on the GPU after exactly the steps the FP64 oracle took to reach a
    change below 1e-11 per 1000 steps, against the oracle's S there."""
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    assert [c["kn_out"] for c in cases] == list(KN_OUT)
    for c in cases:
        assert c["converged"]
        ch = clb.Channel(801, 8, c["kn_out"], sigma=0.93, drive="pressure", drive_value=1.8, storage="fp64",
                         kn_mode=1)
        ch.step(c["steps"])
        o = ch.observables()
        ch.close()
        assert o["q_norm"] == pytest.approx(c["S"], rel=1e-10), c["kn_out"]
        assert o["mass_flow"] == pytest.approx(c["mass_flow"], rel=1e-10), c["kn_out"]
        assert o["u_slip"] == pytest.approx(c["u_slip"], rel=1e-9), c["kn_out"]
