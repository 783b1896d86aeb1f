"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, a wrong sign, coefficient or index, a transposed operand, a swapped
rate, a wrong wall offset or partner, a wrong normalisation), builds it, and
runs the oracle's pin tests (test_oracle_algebra, test_oracle_flow,
test_oracle_gradient) against it in a child process.  The case passes when at
least one pin fails.  The copy lives in a temporary directory; the oracle's own
source is never touched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = [os.path.join(ROOT, "tests", f) for f in
        ("test_oracle_algebra.py", "test_oracle_flow.py", "test_oracle_gradient.py")]

# (name, text in clb_oracle.c, replacement): each text occurs exactly once.
MUTANTS = [
    # lattice, matrices, equilibrium (Eq. 1, 3, 6, 10, 11)
    ("diagonal_angles", "sin((2 * i - 9) * PI / 4.0)", "sin((2 * i - 7) * PI / 4.0)"),
    ("T_row_xyy", "T[7 * 9 + i] = x * y * y;", "T[7 * 9 + i] = x * y;"),
    ("K_column_6", "K[i * 9 + 6] = -3 * x * x * y + 2 * y;", "K[i * 9 + 6] = -3 * x * x * y + y;"),
    ("moment_indices_transposed", "ipow(EX[i], m) * ipow(EY[i], n)", "ipow(EX[i], n) * ipow(EY[i], m)"),
    ("Tinv_transposed", "s += TINV[i * 9 + j] * m[j];", "s += TINV[j * 9 + i] * m[j];"),
    ("K_transposed", "kg += KMAT[i * 9 + j] * g[j];", "kg += KMAT[j * 9 + i] * g[j];"),
    ("feq_fourth_moment", "m[8] = 1.0 / 9.0 * rho + 1.0 / 3.0 * rho", "m[8] = 1.0 / 9.0 * rho + 2.0 / 3.0 * rho"),
    # collision (Eq. 7, 9, 13)
    ("velocity_without_half_force", "const real_t ux = (kx + 0.5 * rho * Fx) / rho;",
     "const real_t ux = kx / rho;"),
    ("g3_coefficient", "g[3] = s[3] / 12.0 *", "g[3] = s[3] / 4.0 *"),
    ("g5_force_term_dropped", "(rho * ux * uy - kxy - 0.5 * rho * (Fx * uy + Fy * ux))",
     "(rho * ux * uy - kxy)"),
    ("g6_cascade_sign", "0.5 * uy * (3.0 * g[3] + g[4]) - 2.0 * ux * g[5];",
     "0.5 * uy * (3.0 * g[3] - g[4]) - 2.0 * ux * g[5];"),
    ("g8_drops_g6", "- 2.0 * uy * g[6] - 2.0 * ux * g[7];", "- 2.0 * ux * g[7];"),
    ("source_force_sign", "Sh[1] = rho * Fx;", "Sh[1] = -rho * Fx;"),
    ("source_xy_term", "Sh[5] = rho * (ux * Fy + uy * Fx);", "Sh[5] = rho * ux * Fy;"),
    # rates (Eq. 14, 18, 21)
    ("sv_sq_swapped", "s[4] = s[5] = sv; /* Eq. 14: s4 = s5 = s_v */\n    s[6] = s[7] = sq;",
     "s[4] = s[5] = sq;\n    s[6] = s[7] = sv;"),
    ("eq18_constant", "sqrt(6.0 / PI) * (double)ny * kn_local", "sqrt(PI / 6.0) * (double)ny * kn_local"),
    ("bosanquet_factor_as_one", "(double)ny * kn_local / (1.0 + a * kn_local)",
     "(double)ny * kn_local / (1.0 + kn_local)"),
    ("eq21_tau_power", "4.0 * PI * tq * tq * b2", "4.0 * PI * tq * b2"),
    ("eq21_B1_of_sigma", "1.0 - 0.1817 * sigma", "1.0 - 0.1817 / sigma"),
    ("local_kn_proportional_to_p", "p->kn * p->rho_out / rho", "p->kn * rho / p->rho_out"),
    # streaming and walls (Eq. 5, 20)
    ("push_x_reversed", "const int tx = xsrc(p, x + EX[i]);", "const int tx = xsrc(p, x - EX[i]);"),
    ("bsr_offsets_reversed",
     "const int xm = p->same_node_bsr ? x : xsrc(p, x - 1);\n    const int xp = p->same_node_bsr ? x : xsrc(p, x + 1);",
     "const int xm = p->same_node_bsr ? x : xsrc(p, x + 1);\n    const int xp = p->same_node_bsr ? x : xsrc(p, x - 1);"),
    ("bsr_r_and_1_minus_r_swapped",
     "return r * ft[IDX(7, 0, x, nx, ny)] + (1.0 - r) * ft[IDX(8, 0, xm, nx, ny)];",
     "return (1.0 - r) * ft[IDX(7, 0, x, nx, ny)] + r * ft[IDX(8, 0, xm, nx, ny)];"),
    ("top_specular_partner",
     "return r * ft[IDX(6, yt, x, nx, ny)] + (1.0 - r) * ft[IDX(5, yt, xm, nx, ny)];",
     "return r * ft[IDX(6, yt, x, nx, ny)] + (1.0 - r) * ft[IDX(6, yt, xm, nx, ny)];"),
    ("bottom_rest_partner", "if (i == 2) return ft[IDX(4, 0, x, nx, ny)];",
     "if (i == 2) return ft[IDX(2, 0, x, nx, ny)];"),
    # pressure columns (Sec. 3.2)
    ("pressure_velocity_not_extrapolated", "oracle_feq(rho_b, 2.0 * u1x - u2x, 2.0 * u1y - u2y, eb);",
     "oracle_feq(rho_b, u1x, u1y, eb);"),
    ("pressure_nonequilibrium_from_second_column", "out[i] = eb[i] + (f1[i] - e1[i]);",
     "out[i] = eb[i] + (f2[i] - e1[i]);"),
    ("pressure_columns_in_equilibrium", "out[i] = eb[i] + (f1[i] - e1[i]);", "out[i] = eb[i];"),
    ("inlet_gets_outlet_density", "pressure_rebuild(p, a1, a2, p->rho_in, in);",
     "pressure_rebuild(p, a1, a2, p->rho_out, in);"),
    # observables (Sec. 3.1, 3.2)
    ("macro_half_force_sign", "*ux = (raw_moment(f, 1, 0) - 0.5 * (*rho) * P_gx(p)) / (*rho);",
     "*ux = (raw_moment(f, 1, 0) + 0.5 * (*rho) * P_gx(p)) / (*rho);"),
    ("p_l_sign", "const real_t pl = p_in - (p_in - p_out) * (double)x / L;",
     "const real_t pl = p_in + (p_in - p_out) * (double)x / L;"),
    ("q_norm_sqrt_RT", "(3.0 * P_gx(p) * (double)ny * (double)ny * sqrt(1.0 / 6.0))",
     "(3.0 * P_gx(p) * (double)ny * (double)ny * sqrt(1.0 / 3.0))"),
    ("m_ns_constant", "(24.0 * mu * (1.0 / 3.0) * L)", "(12.0 * mu * (1.0 / 3.0) * L)"),
    ("m_ns_height_squared", "(double)ny * ny * ny * (p_in * p_in - p_out * p_out)",
     "(double)ny * ny * (p_in * p_in - p_out * p_out)"),
    ("mass_flow_mean_over_rows", "const real_t mbar = msum / (double)nx;", "const real_t mbar = msum / (double)ny;"),
    ("q_norm_mean_over_rows", "qnorm = (usum / (double)nx)", "qnorm = (usum / (double)ny)"),
    # observables along the channel (Sec. 3.2): centreline pressure, its non-linear deviation
    ("centreline_two_rows_summed", "if (ny % 2 == 0 && (y == ny / 2 - 1 || y == ny / 2)) rc += 0.5 * rho;",
     "if (ny % 2 == 0 && (y == ny / 2 - 1 || y == ny / 2)) rc += rho;"),
    ("dp_nonlin_over_p_in", "if (dp_nonlin) dp_nonlin[x] = (pc - pl) / p_out;",
     "if (dp_nonlin) dp_nonlin[x] = (pc - pl) / p_in;"),
    # slip velocity extrapolated to J = 0 instead of the wall at J = 1/2
    ("slip_extrapolated_to_J0_bottom", "const real_t sb = 1.5 * ucol_prof[0] - 0.5 * ucol_prof[1];",
     "const real_t sb = 2.0 * ucol_prof[0] - 1.0 * ucol_prof[1];"),
    ("slip_extrapolated_to_J0_top", "const real_t st = 1.5 * ucol_prof[3] - 0.5 * ucol_prof[2];",
     "const real_t st = 2.0 * ucol_prof[3] - 1.0 * ucol_prof[2];"),
    # centreline Knudsen number (Sec. 3.2, reading R8): the row, the time level, the mode itself
    ("centreline_wrong_row", "        const int y1 = (ny % 2) ? y0 : ny / 2;\n        for (int i = 0; i < NQ; ++i) {",
     "        const int y1 = (ny % 2) ? y0 : ny / 2 + 1;\n        for (int i = 0; i < NQ; ++i) {"),
    ("centreline_of_the_streamed_state",
     "        centreline_density(&s->p, s->ft, s->rc); /* of the state before the step */\n"
     "        stream_and_boundaries(&s->p, s->ft, s->fb, nthreads);",
     "        stream_and_boundaries(&s->p, s->ft, s->fb, nthreads);\n"
     "        centreline_density(&s->p, s->fb, s->rc);"),
    ("centreline_mode_ignored",
     "node_rates(p, (p->pressure && p->kn_mode == 1) ? rc[x] : raw_moment(f, 0, 0), s);",
     "node_rates(p, raw_moment(f, 0, 0), s);"),
    # complex-step derivative (the reference of the adjoint)
    ("complex_step_drops_r", "static real_t P_r(const oracle_params* p) { return p->r + I * p->r_im; }",
     "static real_t P_r(const oracle_params* p) { return p->r; }"),
]


def test_mutant_table_is_well_formed():
    src = open(os.path.join(ORACLE, "clb_oracle.c")).read()
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        assert old != new, name


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(os.path.join(ORACLE, "clb_oracle.c")).read()
    assert src.count(old) == 1
    (tmp_path / "clb_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE, "clb_oracle.h"), tmp_path / "clb_oracle.h")
    env = dict(os.environ, CLB_ORACLE_DIR=str(tmp_path), OMP_NUM_THREADS="4")
    # the planted mistake must still compile: a build failure is not a catch
    subprocess.run([sys.executable, "-c", "import oracle; oracle.build_oracle()"], cwd=ROOT, env=env,
                   check=True, capture_output=True, timeout=120)
    run = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert run.returncode == 1, f"mutant {name} survived the pins:\n{run.stdout[-2000:]}"
    assert " failed" in run.stdout, run.stdout[-2000:]
