"""Write ``mass_flow_curve_801x8.json``: the FP64 oracle's steady normalised
mass flow S = m/m_ns of the Sec. 3.2 mass-flow study (Fig. 7 workload).

Channel: nx = 801, ny = 8 (L/H = 100), p_in/p_out = 1.8 (rho_in = 1.8,
rho_out = 1), TMAC sigma = 0.93 (r_b from Eq. 21 with B1 = 1 - 0.1817 sigma),
Bosanquet a = 2, B2 = 0.55, s3 = 1.1, s8 = 1.2, local Knudsen number from the
centreline pressure of the previous step, initial state f^eq(rho_lin(x), 0).
For each Kn_out in {0.02, 0.05, 0.1, 0.2, 0.4}: step in chunks of 1000 and stop
at the first check where |m(t) - m(t - 1000)| / |m(t)| < 1e-11 (well past the
1e-9 of the paper-style runs, so that the stored values are the steady state
to about 1e-9; cap 3e6 steps).

Stored per case: the step count and the oracle's scalars (mass flow, S, slip,
u_x,max, total mass).  Only the oracle is called.  Run from the repository root:
    python tests/golden/make_mass_flow_curve.py [threads]
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

NX, NY, RATIO, SIGMA = 801, 8, 1.8, 0.93
KN_OUT = (0.02, 0.05, 0.1, 0.2, 0.4)
CHECK, TOL, CAP = 1000, 1e-11, 3_000_000
OUT = os.path.join(HERE, "mass_flow_curve_801x8.json")


def run(kn: float, threads: int) -> dict:
    p = oracle.OracleParams(nx=NX, ny=NY, pressure=True, kn=kn, sigma=SIGMA, rho_in=RATIO, rho_out=1.0,
                            kn_mode=1)
    s = oracle.OracleSim(p)
    t0 = time.perf_counter()
    prev = s.observables()["mass_flow"]
    steps, res = 0, float("inf")
    while steps < CAP:
        s.step(CHECK, threads)
        steps += CHECK
        m = s.observables()["mass_flow"]
        res = float(abs(m - prev) / abs(m))
        prev = m
        if res < TOL:
            break
    o = s.observables()
    s.close()
    return {"kn_out": kn, "steps": steps, "residual": float(res), "converged": bool(res < TOL),
            "oracle_seconds": round(time.perf_counter() - t0, 1), "mass_flow": float(o["mass_flow"]),
            "S": float(o["q_norm"]), "u_slip": float(o["u_slip"]), "ux_max": float(o["ux_max"]),
            "total_mass": float(o["total_mass"])}


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    cases = []
    for kn in KN_OUT:
        c = run(kn, threads)
        print(f"Kn_out {kn}: {c['steps']} steps, residual {c['residual']:.2e}, S = {c['S']:.8f} "
              f"({c['oracle_seconds']} s)", flush=True)
        cases.append(c)
    doc = {
        "what": "FP64 oracle steady S = m/m_ns of the Sec. 3.2 mass-flow study (Fig. 7 workload)",
        "channel": {"nx": NX, "ny": NY, "rho_in": RATIO, "rho_out": 1.0, "sigma": SIGMA, "a": 2.0, "b2": 0.55,
                    "s3": 1.1, "s8": 1.2, "kn_mode": 1},
        "steady_state": {"check_every": CHECK, "tol": TOL, "cap": CAP},
        "written_by": "tests/golden/make_mass_flow_curve.py (calls oracle/ only)",
        "cases": cases,
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
