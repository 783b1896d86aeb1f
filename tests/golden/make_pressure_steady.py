"""Write ``pressure_1601x16_steady.json``: the FP64 oracle's steady state of
the L/H = 100 pressure-driven channel of Sec. 3.2 (Fig. 3-5 workload).

Channel: nx = 1601, ny = 16, p_in/p_out = 2 (rho_in = 2, rho_out = 1), Bosanquet
a = 2, r_b from Eq. 21 with sigma = 1, B2 = 0.55, s3 = 1.1, s8 = 1.2, local
Knudsen number from the node's own pressure, initial state f^eq(rho_lin(x), 0)
with rho linear between the end densities.  For each outlet Knudsen number
Kn_out in {0.0194, 0.05, 0.1, 0.2}: step in chunks of K = 1000 and stop at the
first check where the relative change of the mean mass flow over the chunk,
|m(t) - m(t - K)| / |m(t)|, is below 1e-9 (cap 2e6 steps).

Stored per case: the step count, the scalars of the oracle's observables, the
outlet profile u_x(y), and the centreline non-linear pressure deviation and
column mass flow at every 16th column plus the last.

Only the oracle is called.  Run from the repository root:
    python tests/golden/make_pressure_steady.py [threads]
It takes tens of minutes on a few cores.
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

NX, NY, RATIO = 1601, 16, 2.0
KN_OUT = (0.0194, 0.05, 0.1, 0.2)
CHECK, TOL, CAP = 1000, 1e-9, 2_000_000
COLS = list(range(0, NX, 16)) + [NX - 1]
OUT = os.path.join(HERE, "pressure_1601x16_steady.json")


def run(kn: float, threads: int) -> dict:
    p = oracle.OracleParams(nx=NX, ny=NY, pressure=True, kn=kn, rho_in=RATIO, rho_out=1.0)
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
    return {
        "kn_out": kn,
        "steps": steps,
        "residual": float(res),
        "converged": bool(res < TOL),
        "oracle_seconds": round(time.perf_counter() - t0, 1),
        "mass_flow": float(o["mass_flow"]),
        "q_norm": float(o["q_norm"]),
        "u_slip": float(o["u_slip"]),
        "ux_max": float(o["ux_max"]),
        "total_mass": float(o["total_mass"]),
        "ux_prof_outlet": [float(v) for v in o["ux_prof"]],
        "cols": COLS,
        "dp_nonlin": [float(o["dp_nonlin"][x]) for x in COLS],
        "m_of_x": [float(o["m_of_x"][x]) for x in COLS],
    }


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    cases = []
    for kn in KN_OUT:
        c = run(kn, threads)
        print(f"Kn_out {kn}: {c['steps']} steps, residual {c['residual']:.2e}, "
              f"S = {c['q_norm']:.6f} ({c['oracle_seconds']} s)", flush=True)
        cases.append(c)
    doc = {
        "what": "FP64 oracle steady state of the Sec. 3.2 pressure-driven channel (Fig. 3-5 workload)",
        "channel": {"nx": NX, "ny": NY, "rho_in": RATIO, "rho_out": 1.0, "a": 2.0, "sigma": 1.0, "b2": 0.55,
                    "s3": 1.1, "s8": 1.2, "kn_mode": 0},
        "steady_state": {"check_every": CHECK, "tol": TOL, "cap": CAP},
        "written_by": "tests/golden/make_pressure_steady.py (calls oracle/ only)",
        "cases": cases,
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
