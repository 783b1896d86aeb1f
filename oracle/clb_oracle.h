/*
 * FP64 CPU oracle of the cascaded lattice Boltzmann (CLB) method of Liu & He,
 * "Numerical modelling of microchannel gas flows in the transition flow regime
 * using the cascaded lattice Boltzmann method" (arXiv:1603.01955).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load it.  It shares no code,
 * header, table or constant with the CUDA library, and neither includes the
 * other.
 *
 * Canonical state: the post-collision populations f~_i (Eq. 4) after a whole
 * number of steps, laid out as [9][ny][nx] doubles, index
 * (i*ny + y)*nx + x, with x = 0..nx-1 along the channel and y = 0..ny-1 across
 * it (row y = 0 touches the bottom wall, which sits half a cell below it).
 *
 * Parity pins: every function here is pinned by a CPU test against something
 * other than itself (paper-printed matrices, central-moment relaxation,
 * equilibrium fixed point, conservation, symmetries, a closed-form steady
 * profile).  The pressure inlet/outlet reconstruction follows a reading of a
 * passage the paper leaves unspecified (Sec. 3.2: "consistent linear
 * extrapolation"); it is pinned only by invariants (imposed density, mass
 * balance), not by any value the paper prints.
 */
#ifndef CLB_ORACLE_H
#define CLB_ORACLE_H

#include <stdint.h>
#ifdef ORACLE_COMPLEX
#include <complex.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* The number type of states and of everything derived from r, a and F:
 * double, or double _Complex in the complex-step build (ORACLE_COMPLEX),
 * where arrays of real_t are arrays of (re, im) pairs. */
#ifdef ORACLE_COMPLEX
typedef double _Complex real_t;
#else
typedef double real_t;
#endif

typedef struct {
    int nx, ny;           /* lattice nodes along / across the channel */
    int pressure;         /* 0: periodic in x, body force; 1: pressure inlet/outlet */
    double kn;            /* Kn (periodic) or Kn_out (pressure), Sec. 2.2 / Sec. 3.2 */
    double a;             /* Bosanquet rarefaction factor, Eq. 16 */
    double r;             /* bounce-back fraction r_b of the CBBSR wall, Eq. 20 */
    double b2;            /* second-order slip coefficient B2, Eq. 19/21 */
    double s3, s8;        /* free relaxation rates (Sec. 3: 1.1 and 1.2) */
    double gx, gy;        /* body force per unit mass F (lattice units), Eq. 9/13 */
    double rho_in;        /* inlet density  (pressure mode), p = rho/3 */
    double rho_out;       /* outlet density (pressure mode) */
    double sv_override;   /* >0: use this s_v instead of Eq. 18 (tests) */
    double sq_override;   /* >0: use this s_q instead of Eq. 21 (tests) */
    int same_node_bsr;    /* test-only: Eq. 20 with no x offset on the specular part */
    double r_im, a_im, gx_im; /* complex-step build: imaginary parts of r, a, gx */
    int kn_mode;          /* pressure mode: 0 Kn from the node's own pressure; 1 from the
                             centreline pressure p(x) of the previous step (Sec. 3.2) */
} oracle_params;

/* Lattice and matrices built from their definitions (Eq. 1, 3, 10). */
void oracle_lattice(int ex[9], int ey[9]);
void oracle_tmat(double T[81]);     /* row-major, Eq. 10 */
void oracle_tinv(double Ti[81]);    /* Gauss-Jordan inverse of T */
void oracle_kmat(double K[81]);     /* row-major, Eq. 3 */

/* Eq. 11: equilibrium f^eq = T^-1 f^eq-hat. */
void oracle_feq(real_t rho, real_t ux, real_t uy, real_t out[9]);

/* Eq. 18 (s_v) and Eq. 21 (s_q) at a local Knudsen number. */
void oracle_rates_kn(real_t kn_local, int ny, real_t a, real_t b2,
                     real_t* sv, real_t* sq);
/* Eq. 21 first relation with B1 = 1 - 0.1817 sigma (Sec. 3). */
double oracle_r_from_sigma(double sigma);

/* One collision (Eq. 4 with Eq. 7-9, 12-13) of a single node.
 * fbar: pre-collision transformed populations; s[9]: relaxation rates (only
 * s[3..8] are used); out: post-collision populations; ghat (may be NULL): the
 * collision kernels g^_0..g^_8 of Eq. 7; S (may be NULL): the source of Eq. 9-10. */
void oracle_collide(const real_t fbar[9], real_t Fx, real_t Fy, const real_t s[9],
                    real_t out[9], real_t ghat[9], real_t S[9]);

/* Simulation. */
typedef struct oracle_sim oracle_sim;
oracle_sim* oracle_create(const oracle_params* p);
void oracle_destroy(oracle_sim* s);
void oracle_get_state(const oracle_sim* s, real_t* f);     /* [9][ny][nx] */
void oracle_set_state(oracle_sim* s, const real_t* f);
int64_t oracle_step(oracle_sim* s, int64_t nsteps, int nthreads);  /* returns steps done */
int oracle_threads_used(void);

/* Pre-collision populations after stream + walls + pressure columns of the
 * current state (what the next collision would see), [9][ny][nx]. */
void oracle_prestate(oracle_sim* s, real_t* fbar);

/* Next-step post-collision populations at a list of nodes, computed from a
 * full state f_prev ([9][ny][nx]) by a node-local pull.  out: [n][9]. */
void oracle_step_nodes(const oracle_params* p, const real_t* f_prev, int n,
                       const int* xs, const int* ys, real_t* out);

/* Observables of the current state (Sec. 3.1, 3.2).  Any output may be NULL.
 * scal[0] mean mass flow  m = mean_x sum_y rho u_x
 * scal[1] normalised flow: Q (periodic) or S = m/m_ns (pressure)
 * scal[2] slip velocity at the profile column (wall extrapolation)
 * scal[3] total mass sum rho
 * scal[4] u_x,max at the profile column */
void oracle_observables(const oracle_sim* s, int profile_col, real_t scal[5],
                        real_t* ux_prof, real_t* uy_prof, real_t* p_centre,
                        real_t* dp_nonlin, real_t* m_of_x);

/* Density and velocity fields of the current state, [ny][nx] each. */
void oracle_macro(const oracle_sim* s, real_t* rho, real_t* ux, real_t* uy);

#ifdef __cplusplus
}
#endif
#endif
