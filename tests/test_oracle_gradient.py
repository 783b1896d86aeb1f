"""Pins of the oracle's complex-step gradient (the reference for the GPU
adjoint): derivatives of J = mean_x sum_y u_x with respect to the wall's
bounce-back fraction r_b (Eq. 20), the Bosanquet factor a (Eq. 16-18, 21) and
the body force G.

* the complex-step build reproduces the FP64 oracle in its real part;
* its derivatives equal central finite differences of the FP64 oracle;
* at steady state they equal the derivatives of the hand-derived closed-form
  slip-Poiseuille profile (see test_oracle_flow.closed_form_profile):
      J = N u_s + (3G/(2 tau)) sum_J (J-1/2)(N+1/2-J),
      u_s = (3G/2) [ (1-r) N / r + 2 tau_q - 1/(4 tau) ],
      tau = sqrt(6/pi) N Kn / (1 + a Kn),  tau_q = 3/(16 tau) + pi B2 tau / 4.
"""
import math
from dataclasses import replace

import numpy as np
import pytest


def J_real(oracle_mod, p, steps):
    s = oracle_mod.OracleSim(p)
    s.step(steps, 1)
    _, ux, _ = s.macro()
    return ux.sum() / p.nx


@pytest.mark.parametrize("kn,ny,G", [(0.3, 8, 1e-5), (1.0, 6, -3e-5)])
def test_complex_step_real_part_and_fd(oracle_mod, kn, ny, G):
    p = oracle_mod.OracleParams(nx=2, ny=ny, kn=kn, gx=G, r=0.7)
    steps = 400
    J, g = oracle_mod.gradient_cs(p, steps)
    J0 = J_real(oracle_mod, p, steps)
    assert J == pytest.approx(J0, rel=1e-14)
    for name, field, base in (("r", "r", p.r), ("a", "a", p.a), ("g", "gx", p.gx)):
        h = 1e-5 * abs(base)
        fd = (J_real(oracle_mod, replace(p, **{field: base + h}), steps)
              - J_real(oracle_mod, replace(p, **{field: base - h}), steps)) / (2 * h)
        assert g[name] == pytest.approx(fd, rel=1e-5), name


def closed_form_J_and_grad(ny, kn, a, r, G, b2=0.55):
    c6 = math.sqrt(6 / math.pi)
    tau = c6 * ny * kn / (1 + a * kn)
    tq = 3 / (16 * tau) + math.pi * b2 * tau / 4
    S2 = sum((j - 0.5) * (ny + 0.5 - j) for j in range(1, ny + 1))
    us = 1.5 * G * ((1 - r) * ny / r + 2 * tq - 1 / (4 * tau))
    J = ny * us + 1.5 * G / tau * S2
    dJ_dr = ny * 1.5 * G * ny * (-1 / r**2)
    dJ_dG = J / G
    dtau_da = -c6 * ny * kn * kn / (1 + a * kn) ** 2
    dtq_dtau = -3 / (16 * tau**2) + math.pi * b2 / 4
    dJ_dtau = ny * 1.5 * G * (2 * dtq_dtau + 1 / (4 * tau**2)) - 1.5 * G / tau**2 * S2
    return J, {"r": dJ_dr, "a": dJ_dtau * dtau_da, "g": dJ_dG}


@pytest.mark.parametrize("kn,ny,r", [(0.1, 16, 0.63), (0.5, 8, 0.9), (2.0, 12, 0.4)])
def test_steady_gradient_matches_closed_form(oracle_mod, kn, ny, r):
    G = 1e-7
    p = oracle_mod.OracleParams(nx=1, ny=ny, kn=kn, gx=G, r=r)
    sv, _ = oracle_mod.rates_kn(kn, ny)
    nu = (1 / sv - 0.5) / 3
    steps = int(40 * ny * ny / (math.pi**2 * nu)) + 3000
    J, g = oracle_mod.gradient_cs(p, steps)
    Jc, gc = closed_form_J_and_grad(ny, kn, 2.0, r, G)
    assert J == pytest.approx(Jc, rel=1e-6)
    for name in ("r", "a", "g"):
        assert g[name] == pytest.approx(gc[name], rel=1e-5), name
