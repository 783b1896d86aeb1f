/*
 * FP64 CPU oracle of the cascaded lattice Boltzmann (CLB) method of Liu & He
 * (arXiv:1603.01955).  TEST INFRASTRUCTURE ONLY: the reference the CUDA path
 * is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.
 *
 * Written for reading, not speed: every step follows the paper's equations in
 * the paper's order and notation, with the matrices built from their
 * definitions (Eq. 1, 3, 10) and inverted numerically.  Compiled with
 * -ffp-contract=off so that no fused multiply-add changes its rounding.
 *
 * One time step on the canonical post-collision state f~ (see clb_oracle.h):
 *   1. push-stream f~_i(x) -> fbar_i(x + e_i)              (Eq. 5, Sec. 3.1 periodic x)
 *   2. CBBSR walls at the first and last rows              (Eq. 20, and its mirror)
 *   3. pressure inlet/outlet columns (pressure mode only)  (Sec. 3.2, reading below)
 *   4. collide every node                                  (Eq. 4, 7-9, 12-13, 18, 21)
 *
 * Readings of passages the paper leaves open (each one is also listed in the
 * design notes):
 *  - Eq. 20 gives no x offsets.  The bounce-back part comes from the same node,
 *    the specular part from the node the reflected particle left:
 *      bottom: fbar5(x) = r f~7(x) + (1-r) f~8(x-1),  fbar6(x) = r f~8(x) + (1-r) f~7(x+1)
 *      top:    fbar7(x) = r f~5(x) + (1-r) f~6(x+1),  fbar8(x) = r f~6(x) + (1-r) f~5(x-1)
 *    and fbar2 = f~4 (bottom), fbar4 = f~2 (top).  The top wall is the mirror
 *    image of the bottom one, which is the only wall the paper writes out.
 *  - Pressure columns ("consistent linear extrapolation", Sec. 3.2, details not
 *    given): after streaming, all nine populations of the inlet column are
 *      fbar_i(0,y) = f^eq_i(rho_in, u_b) + f^neq_i(1,y),
 *      u_b = 2 u(1,y) - u(2,y),  f^neq = fbar - f^eq(rho, u):
 *    the velocity is extrapolated linearly from the two interior neighbours,
 *    the non-equilibrium part is taken from the first one, and the density is
 *    imposed; the outlet mirrors it with rho_out and columns nx-2, nx-3.
 *    f^neq carries no mass, so rho(0,y) = rho_in exactly.  (Extrapolating
 *    f^neq linearly too, 2 f^neq(1) - f^neq(2), amplifies the shortest
 *    x-wavelength threefold and diverges at the outlet once tau ~ 30.)
 *  - Local Knudsen number (Sec. 3.2): Kn = Kn_out p_out / p, with p = rho/3
 *    taken per node (kn_mode 0), or, as the paper states it, from the
 *    centreline pressure of the column (kn_mode 1: the middle row, or the mean
 *    of the two middle rows, of the state before the step, i.e. one step
 *    behind; identical at steady state).
 *  - tau~_q in Eq. 21 is 1/s_v - 1/2, as the sentence after Eq. 21 defines it.
 *  - Initial state: f~ = f^eq(rho_init(x), 0), rho_init = rho_out (periodic)
 *    or linear from rho_in at x = 0 to rho_out at x = nx-1 (pressure).
 */
#include "clb_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 9

/* In the complex-step build (ORACLE_COMPLEX) every quantity that depends on
 * the state or on r, a or F carries an imaginary part: perturbing one of them
 * by i*h gives its exact derivative as Im(result)/h, with no cancellation.
 * The ordinary build has real_t = double and is unchanged arithmetic. */
#ifdef ORACLE_COMPLEX
#define RE(v) creal(v)
static real_t P_r(const oracle_params* p) { return p->r + I * p->r_im; }
static real_t P_a(const oracle_params* p) { return p->a + I * p->a_im; }
static real_t P_gx(const oracle_params* p) { return p->gx + I * p->gx_im; }
#else
#define RE(v) (v)
static real_t P_r(const oracle_params* p) { return p->r; }
static real_t P_a(const oracle_params* p) { return p->a; }
static real_t P_gx(const oracle_params* p) { return p->gx; }
#endif

static const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ lattice */

/* Eq. 1: e_i = (cos((i-1) pi/2), sin((i-1) pi/2)) for i = 1..4 and
 * sqrt(2) (cos((2i-9) pi/4), sin((2i-9) pi/4)) for i = 5..8, with c = 1. */
void oracle_lattice(int ex[9], int ey[9])
{
    ex[0] = 0;
    ey[0] = 0;
    for (int i = 1; i <= 4; ++i) {
        ex[i] = (int)lround(cos((i - 1) * PI / 2.0));
        ey[i] = (int)lround(sin((i - 1) * PI / 2.0));
    }
    for (int i = 5; i <= 8; ++i) {
        ex[i] = (int)lround(sqrt(2.0) * cos((2 * i - 9) * PI / 4.0));
        ey[i] = (int)lround(sqrt(2.0) * sin((2 * i - 9) * PI / 4.0));
    }
}

static int ipow(int b, int e)
{
    int v = 1;
    while (e-- > 0) v *= b;
    return v;
}

/* Eq. 10: rows |1>, |ex>, |ey>, |ex^2+ey^2>, |ex^2-ey^2>, |ex ey>, |ex^2 ey>,
 * |ex ey^2>, |ex^2 ey^2>. */
void oracle_tmat(double T[81])
{
    int ex[9], ey[9];
    oracle_lattice(ex, ey);
    for (int i = 0; i < NQ; ++i) {
        const int x = ex[i], y = ey[i];
        T[0 * 9 + i] = 1;
        T[1 * 9 + i] = x;
        T[2 * 9 + i] = y;
        T[3 * 9 + i] = x * x + y * y;
        T[4 * 9 + i] = x * x - y * y;
        T[5 * 9 + i] = x * y;
        T[6 * 9 + i] = x * x * y;
        T[7 * 9 + i] = x * y * y;
        T[8 * 9 + i] = x * x * y * y;
    }
}

/* Gauss-Jordan elimination with partial pivoting. */
static void invert9(const double A[81], double Ai[81])
{
    double M[9][18];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 18; ++c)
            M[r][c] = (c < 9) ? A[r * 9 + c] : (c - 9 == r ? 1.0 : 0.0);
    for (int c = 0; c < 9; ++c) {
        int piv = c;
        for (int r = c + 1; r < 9; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 18; ++k) {
                double t = M[c][k];
                M[c][k] = M[piv][k];
                M[piv][k] = t;
            }
        const double d = M[c][c];
        for (int k = 0; k < 18; ++k) M[c][k] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == c) continue;
            const double f = M[r][c];
            if (f == 0.0) continue;
            for (int k = 0; k < 18; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) Ai[r * 9 + c] = M[r][c + 9];
}

void oracle_tinv(double Ti[81])
{
    double T[81];
    oracle_tmat(T);
    invert9(T, Ti);
}

/* Eq. 3: columns |1>, |ex>, |ey>, 3|ex^2+ey^2> - 4|1>, |ex^2-ey^2>, |ex ey>,
 * -3|ex^2 ey> + 2|ey>, -3|ex ey^2> + 2|ex>, 9|ex^2 ey^2> - 6|ex^2+ey^2> + 4|1>. */
void oracle_kmat(double K[81])
{
    int ex[9], ey[9];
    oracle_lattice(ex, ey);
    for (int i = 0; i < NQ; ++i) {
        const int x = ex[i], y = ey[i];
        K[i * 9 + 0] = 1;
        K[i * 9 + 1] = x;
        K[i * 9 + 2] = y;
        K[i * 9 + 3] = 3 * (x * x + y * y) - 4;
        K[i * 9 + 4] = x * x - y * y;
        K[i * 9 + 5] = x * y;
        K[i * 9 + 6] = -3 * x * x * y + 2 * y;
        K[i * 9 + 7] = -3 * x * y * y + 2 * x;
        K[i * 9 + 8] = 9 * x * x * y * y - 6 * (x * x + y * y) + 4;
    }
}

/* Module-level tables, built once from the definitions above. */
static int g_ready = 0;
static int EX[NQ], EY[NQ];
static double TINV[81], KMAT[81];

static void ensure_tables(void)
{
    if (g_ready) return;
    oracle_lattice(EX, EY);
    oracle_tinv(TINV);
    oracle_kmat(KMAT);
    g_ready = 1;
}

/* Raw moment <ex^m ey^n | f> (the inner product defined under Eq. 7). */
static real_t raw_moment(const real_t f[9], int m, int n)
{
    real_t s = 0.0;
    for (int i = 0; i < NQ; ++i) s += (double)(ipow(EX[i], m) * ipow(EY[i], n)) * f[i];
    return s;
}

static void tinv_apply(const real_t m[9], real_t f[9])
{
    for (int i = 0; i < NQ; ++i) {
        real_t s = 0.0;
        for (int j = 0; j < NQ; ++j) s += TINV[i * 9 + j] * m[j];
        f[i] = s;
    }
}

/* Eq. 11 */
void oracle_feq(real_t rho, real_t ux, real_t uy, real_t out[9])
{
    ensure_tables();
    real_t m[9];
    m[0] = rho;
    m[1] = rho * ux;
    m[2] = rho * uy;
    m[3] = 2.0 / 3.0 * rho + rho * (ux * ux + uy * uy);
    m[4] = rho * (ux * ux - uy * uy);
    m[5] = rho * ux * uy;
    m[6] = 1.0 / 3.0 * rho * uy + rho * ux * ux * uy;
    m[7] = 1.0 / 3.0 * rho * ux + rho * ux * uy * uy;
    m[8] = 1.0 / 9.0 * rho + 1.0 / 3.0 * rho * (ux * ux + uy * uy) + rho * ux * ux * uy * uy;
    tinv_apply(m, out);
}

/* ------------------------------------------------------------------- rates */

/* Eq. 18: 1/s_v = 1/2 + sqrt(6/pi) N Kn / (1 + a Kn), N = H/dx = ny (walls half
 * a cell outside the first and last rows).
 * Eq. 21: 1/s_q = 1/2 + (3 + 4 pi tau_q^2 B2) / (16 tau_q), tau_q = 1/s_v - 1/2. */
void oracle_rates_kn(real_t kn_local, int ny, real_t a, real_t b2, real_t* sv, real_t* sq)
{
    const real_t inv_sv = 0.5 + sqrt(6.0 / PI) * (double)ny * kn_local / (1.0 + a * kn_local);
    const real_t tq = inv_sv - 0.5;
    const real_t inv_sq = 0.5 + (3.0 + 4.0 * PI * tq * tq * b2) / (16.0 * tq);
    *sv = 1.0 / inv_sv;
    *sq = 1.0 / inv_sq;
}

/* Eq. 21 with sigma_v = (2 - sigma)/sigma (Eq. 19) and B1 = 1 - 0.1817 sigma (Sec. 3). */
double oracle_r_from_sigma(double sigma)
{
    const double b1 = 1.0 - 0.1817 * sigma;
    const double sigv = (2.0 - sigma) / sigma;
    return 1.0 / (1.0 + b1 * sigv * sqrt(PI / 6.0));
}

/* --------------------------------------------------------------- collision */

void oracle_collide(const real_t fb[9], real_t Fx, real_t Fy, const real_t s[9],
                    real_t out[9], real_t ghat[9], real_t Sout[9])
{
    ensure_tables();
    /* Eq. 12 and the raw moments of Eq. 8 */
    const real_t rho = raw_moment(fb, 0, 0);
    const real_t kx = raw_moment(fb, 1, 0);
    const real_t ky = raw_moment(fb, 0, 1);
    const real_t kxx = raw_moment(fb, 2, 0);
    const real_t kyy = raw_moment(fb, 0, 2);
    const real_t kxy = raw_moment(fb, 1, 1);
    const real_t kxxy = raw_moment(fb, 2, 1);
    const real_t kxyy = raw_moment(fb, 1, 2);
    const real_t kxxyy = raw_moment(fb, 2, 2);
    /* Eq. 13 (delta_t = 1) */
    const real_t ux = (kx + 0.5 * rho * Fx) / rho;
    const real_t uy = (ky + 0.5 * rho * Fy) / rho;

    /* Eq. 7, in order: each kernel uses the lower ones */
    real_t g[9];
    g[0] = g[1] = g[2] = 0.0;
    g[3] = s[3] / 12.0 *
           (2.0 / 3.0 * rho + rho * (ux * ux + uy * uy) - (kxx + kyy) -
            0.5 * rho * (2.0 * Fx * ux + 2.0 * Fy * uy));
    g[4] = s[4] / 4.0 *
           (rho * (ux * ux - uy * uy) - (kxx - kyy) - 0.5 * rho * (2.0 * Fx * ux - 2.0 * Fy * uy));
    g[5] = s[5] / 4.0 * (rho * ux * uy - kxy - 0.5 * rho * (Fx * uy + Fy * ux));
    g[6] = s[6] / 4.0 *
               (2.0 * rho * ux * ux * uy + kxxy - 2.0 * ux * kxy - uy * kxx -
                0.5 * rho * (Fy * ux * ux + 2.0 * Fx * ux * uy)) -
           0.5 * uy * (3.0 * g[3] + g[4]) - 2.0 * ux * g[5];
    g[7] = s[7] / 4.0 *
               (2.0 * rho * ux * uy * uy + kxyy - 2.0 * uy * kxy - ux * kyy -
                0.5 * rho * (Fx * uy * uy + 2.0 * Fy * uy * ux)) -
           0.5 * ux * (3.0 * g[3] - g[4]) - 2.0 * uy * g[5];
    g[8] = s[8] / 4.0 *
               (1.0 / 9.0 * rho + 3.0 * rho * ux * ux * uy * uy -
                (kxxyy - 2.0 * ux * kxyy - 2.0 * uy * kxxy + ux * ux * kyy + uy * uy * kxx +
                 4.0 * ux * uy * kxy) -
                0.5 * rho * (2.0 * Fx * ux * uy * uy + 2.0 * Fy * uy * ux * ux)) -
           2.0 * g[3] - 0.5 * uy * uy * (3.0 * g[3] + g[4]) - 0.5 * ux * ux * (3.0 * g[3] - g[4]) -
           4.0 * ux * uy * g[5] - 2.0 * uy * g[6] - 2.0 * ux * g[7];

    /* Eq. 9 and S = T^-1 S^ (Eq. 10) */
    real_t Sh[9], S[9];
    Sh[0] = 0.0;
    Sh[1] = rho * Fx;
    Sh[2] = rho * Fy;
    Sh[3] = 2.0 * rho * (ux * Fx + uy * Fy);
    Sh[4] = 2.0 * rho * (ux * Fx - uy * Fy);
    Sh[5] = rho * (ux * Fy + uy * Fx);
    Sh[6] = rho * Fy * ux * ux + 2.0 * rho * Fx * ux * uy;
    Sh[7] = rho * Fx * uy * uy + 2.0 * rho * Fy * uy * ux;
    Sh[8] = 2.0 * rho * Fx * ux * uy * uy + 2.0 * rho * Fy * uy * ux * ux;
    tinv_apply(Sh, S);

    /* Eq. 4: f~ = fbar + K g^ + S  (delta_t = 1) */
    for (int i = 0; i < NQ; ++i) {
        real_t kg = 0.0;
        for (int j = 0; j < NQ; ++j) kg += KMAT[i * 9 + j] * g[j];
        out[i] = fb[i] + kg + S[i];
    }
    if (ghat)
        for (int j = 0; j < NQ; ++j) ghat[j] = g[j];
    if (Sout)
        for (int j = 0; j < NQ; ++j) Sout[j] = S[j];
}

/* -------------------------------------------------------------- simulation */

struct oracle_sim {
    oracle_params p;
    real_t* ft; /* post-collision state, [9][ny][nx] */
    real_t* fb; /* work: pre-collision populations */
    real_t* rc; /* work: centreline density per column (kn_mode 1) */
    real_t sv_const, sq_const;
};

static int g_threads_used = 1;

int oracle_threads_used(void) { return g_threads_used; }

#define IDX(i, y, x, nx, ny) ((((size_t)(i)) * (size_t)(ny) + (size_t)(y)) * (size_t)(nx) + (size_t)(x))

/* rho: the density that sets the local Knudsen number (the node's own, or
 * the column's centreline density in kn_mode 1). */
static void node_rates(const oracle_params* p, real_t rho, real_t s[9])
{
    real_t sv, sq;
    const real_t kn_local = p->pressure ? p->kn * p->rho_out / rho : p->kn;
    oracle_rates_kn(kn_local, p->ny, P_a(p), p->b2, &sv, &sq);
    if (p->sv_override > 0.0) sv = p->sv_override;
    if (p->sq_override > 0.0) sq = p->sq_override;
    s[0] = s[1] = s[2] = 0.0;
    s[3] = p->s3;
    s[4] = s[5] = sv; /* Eq. 14: s4 = s5 = s_v */
    s[6] = s[7] = sq; /* Eq. 21: s6 = s7 = s_q */
    s[8] = p->s8;
}

oracle_sim* oracle_create(const oracle_params* p)
{
    ensure_tables();
    if (p->nx < 1 || p->ny < 1) return NULL;
    if (p->pressure && p->nx < 4) return NULL;
    oracle_sim* s = (oracle_sim*)calloc(1, sizeof(oracle_sim));
    s->p = *p;
    const size_t n = (size_t)NQ * p->nx * p->ny;
    s->ft = (real_t*)malloc(n * sizeof(real_t));
    s->fb = (real_t*)malloc(n * sizeof(real_t));
    s->rc = (real_t*)malloc((size_t)p->nx * sizeof(real_t));
    for (int x = 0; x < p->nx; ++x) {
        real_t rho0 = p->rho_out;
        if (p->pressure)
            rho0 = p->rho_in + (p->rho_out - p->rho_in) * (double)x / (double)(p->nx - 1);
        real_t feq[9];
        oracle_feq(rho0, 0.0, 0.0, feq);
        for (int y = 0; y < p->ny; ++y)
            for (int i = 0; i < NQ; ++i) s->ft[IDX(i, y, x, p->nx, p->ny)] = feq[i];
    }
    return s;
}

void oracle_destroy(oracle_sim* s)
{
    if (!s) return;
    free(s->ft);
    free(s->fb);
    free(s->rc);
    free(s);
}

void oracle_get_state(const oracle_sim* s, real_t* f)
{
    memcpy(f, s->ft, (size_t)NQ * s->p.nx * s->p.ny * sizeof(real_t));
}

void oracle_set_state(oracle_sim* s, const real_t* f)
{
    memcpy(s->ft, f, (size_t)NQ * s->p.nx * s->p.ny * sizeof(real_t));
}

/* Wrap an x index in periodic mode; -1 if it leaves a pressure channel. */
static int xsrc(const oracle_params* p, int x)
{
    if (x >= 0 && x < p->nx) return x;
    if (!p->pressure) return ((x % p->nx) + p->nx) % p->nx;
    return -1;
}

/* Eq. 20 and its mirror: the populations entering row 0 from the bottom wall
 * and row ny-1 from the top wall, at column x, from the post-collision state. */
static real_t wall_value(const oracle_params* p, const real_t* ft, int i, int y, int x)
{
    const int nx = p->nx, ny = p->ny;
    const real_t r = P_r(p);
    const int xm = p->same_node_bsr ? x : xsrc(p, x - 1);
    const int xp = p->same_node_bsr ? x : xsrc(p, x + 1);
    if (y == 0 && (i == 2 || i == 5 || i == 6)) {
        if (i == 2) return ft[IDX(4, 0, x, nx, ny)];
        if (i == 5) {
            if (xm < 0) return NAN;
            return r * ft[IDX(7, 0, x, nx, ny)] + (1.0 - r) * ft[IDX(8, 0, xm, nx, ny)];
        }
        if (xp < 0) return NAN;
        return r * ft[IDX(8, 0, x, nx, ny)] + (1.0 - r) * ft[IDX(7, 0, xp, nx, ny)];
    }
    /* top wall, y == ny-1, i in {4, 7, 8} */
    const int yt = ny - 1;
    if (i == 4) return ft[IDX(2, yt, x, nx, ny)];
    if (i == 7) {
        if (xp < 0) return NAN;
        return r * ft[IDX(5, yt, x, nx, ny)] + (1.0 - r) * ft[IDX(6, yt, xp, nx, ny)];
    }
    if (xm < 0) return NAN;
    return r * ft[IDX(6, yt, x, nx, ny)] + (1.0 - r) * ft[IDX(5, yt, xm, nx, ny)];
}

static void macro_of(const real_t f[9], real_t Fx, real_t Fy, real_t* rho, real_t* ux, real_t* uy)
{
    /* Eq. 12-13 on pre-collision populations */
    *rho = raw_moment(f, 0, 0);
    *ux = (raw_moment(f, 1, 0) + 0.5 * (*rho) * Fx) / (*rho);
    *uy = (raw_moment(f, 0, 1) + 0.5 * (*rho) * Fy) / (*rho);
}

/* Pressure column rebuild (reading of Sec. 3.2, see file header).
 * f1, f2: pre-collision populations of the first and second interior
 * neighbours; rho_b: imposed density; out: the boundary populations. */
static void pressure_rebuild(const oracle_params* p, const real_t f1[9], const real_t f2[9],
                             real_t rho_b, real_t out[9])
{
    real_t r1, u1x, u1y, r2, u2x, u2y, e1[9], eb[9];
    macro_of(f1, P_gx(p), p->gy, &r1, &u1x, &u1y);
    macro_of(f2, P_gx(p), p->gy, &r2, &u2x, &u2y);
    oracle_feq(r1, u1x, u1y, e1);
    oracle_feq(rho_b, 2.0 * u1x - u2x, 2.0 * u1y - u2y, eb);
    for (int i = 0; i < NQ; ++i) out[i] = eb[i] + (f1[i] - e1[i]);
}

/* Steps 1-3 of a time step: streaming, walls, pressure columns. */
static void stream_and_boundaries(const oracle_params* p, const real_t* ft, real_t* fb, int nthreads)
{
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)NQ * nx * ny;
    for (size_t k = 0; k < n; ++k) fb[k] = NAN; /* anything left undefined shows up */

    /* 1. push streaming, Eq. 5 */
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int i = 0; i < NQ; ++i) {
                const int ty = y + EY[i];
                if (ty < 0 || ty >= ny) continue; /* leaves through a wall */
                const int tx = xsrc(p, x + EX[i]);
                if (tx < 0) continue; /* leaves through an open end */
                fb[IDX(i, ty, tx, nx, ny)] = ft[IDX(i, y, x, nx, ny)];
            }

    /* 2. walls, Eq. 20 (bottom) and its mirror (top) */
    for (int x = 0; x < nx; ++x) {
        fb[IDX(2, 0, x, nx, ny)] = wall_value(p, ft, 2, 0, x);
        fb[IDX(5, 0, x, nx, ny)] = wall_value(p, ft, 5, 0, x);
        fb[IDX(6, 0, x, nx, ny)] = wall_value(p, ft, 6, 0, x);
        fb[IDX(4, ny - 1, x, nx, ny)] = wall_value(p, ft, 4, ny - 1, x);
        fb[IDX(7, ny - 1, x, nx, ny)] = wall_value(p, ft, 7, ny - 1, x);
        fb[IDX(8, ny - 1, x, nx, ny)] = wall_value(p, ft, 8, ny - 1, x);
    }

    /* 3. pressure columns, from the streamed interior columns */
    if (p->pressure) {
        for (int y = 0; y < ny; ++y) {
            real_t a1[9], a2[9], b1[9], b2[9], in[9], outc[9];
            for (int i = 0; i < NQ; ++i) {
                a1[i] = fb[IDX(i, y, 1, nx, ny)];
                a2[i] = fb[IDX(i, y, 2, nx, ny)];
                b1[i] = fb[IDX(i, y, nx - 2, nx, ny)];
                b2[i] = fb[IDX(i, y, nx - 3, nx, ny)];
            }
            pressure_rebuild(p, a1, a2, p->rho_in, in);
            pressure_rebuild(p, b1, b2, p->rho_out, outc);
            for (int i = 0; i < NQ; ++i) {
                fb[IDX(i, y, 0, nx, ny)] = in[i];
                fb[IDX(i, y, nx - 1, nx, ny)] = outc[i];
            }
        }
    }
}

/* Centreline density of each column of a state: the middle row, or the mean
 * of the two middle rows. */
static void centreline_density(const oracle_params* p, const real_t* f, real_t* rc)
{
    const int nx = p->nx, ny = p->ny;
    for (int x = 0; x < nx; ++x) {
        real_t r0 = 0.0, r1 = 0.0;
        const int y0 = (ny % 2) ? (ny - 1) / 2 : ny / 2 - 1;
        const int y1 = (ny % 2) ? y0 : ny / 2;
        for (int i = 0; i < NQ; ++i) {
            r0 += f[IDX(i, y0, x, nx, ny)];
            r1 += f[IDX(i, y1, x, nx, ny)];
        }
        rc[x] = (ny % 2) ? r0 : 0.5 * (r0 + r1);
    }
}

static void collide_all(const oracle_params* p, const real_t* fb, real_t* ft, const real_t* rc, int nthreads)
{
    const int nx = p->nx, ny = p->ny;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < ny; ++y) {
#ifdef _OPENMP
        if (y == 0) g_threads_used = omp_get_num_threads();
#endif
        for (int x = 0; x < nx; ++x) {
            real_t f[9], o[9], s[9];
            for (int i = 0; i < NQ; ++i) f[i] = fb[IDX(i, y, x, nx, ny)];
            node_rates(p, (p->pressure && p->kn_mode == 1) ? rc[x] : raw_moment(f, 0, 0), s);
            oracle_collide(f, P_gx(p), p->gy, s, o, NULL, NULL);
            for (int i = 0; i < NQ; ++i) ft[IDX(i, y, x, nx, ny)] = o[i];
        }
    }
}

static int resolve_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    return nthreads;
}

int64_t oracle_step(oracle_sim* s, int64_t nsteps, int nthreads)
{
    nthreads = resolve_threads(nthreads);
    g_threads_used = 1;
    for (int64_t t = 0; t < nsteps; ++t) {
        centreline_density(&s->p, s->ft, s->rc); /* of the state before the step */
        stream_and_boundaries(&s->p, s->ft, s->fb, nthreads);
        collide_all(&s->p, s->fb, s->ft, s->rc, nthreads);
    }
    return nsteps;
}

void oracle_prestate(oracle_sim* s, real_t* fbar)
{
    stream_and_boundaries(&s->p, s->ft, fbar, 1);
}

/* ------------------------------------------------------ node-local stepping */

/* Pre-collision populations at (x, y): what streaming, the walls and the
 * pressure columns deliver there, gathered node by node. */
static void arrive(const oracle_params* p, const real_t* ft, int x, int y, real_t fb[9])
{
    const int nx = p->nx, ny = p->ny;
    if (p->pressure && (x == 0 || x == nx - 1)) {
        real_t f1[9], f2[9];
        const int d = (x == 0) ? 1 : -1;
        arrive(p, ft, x + d, y, f1);
        arrive(p, ft, x + 2 * d, y, f2);
        pressure_rebuild(p, f1, f2, x == 0 ? p->rho_in : p->rho_out, fb);
        return;
    }
    for (int i = 0; i < NQ; ++i) {
        const int sy = y - EY[i];
        if (sy < 0 || sy >= ny) {
            fb[i] = wall_value(p, ft, i, y, x);
            continue;
        }
        const int sx = xsrc(p, x - EX[i]);
        fb[i] = (sx < 0) ? NAN : ft[IDX(i, sy, sx, nx, ny)];
    }
}

void oracle_step_nodes(const oracle_params* p, const real_t* f_prev, int n, const int* xs,
                       const int* ys, real_t* out)
{
    ensure_tables();
    const int y0 = (p->ny % 2) ? (p->ny - 1) / 2 : p->ny / 2 - 1;
    const int y1 = (p->ny % 2) ? y0 : p->ny / 2;
    for (int k = 0; k < n; ++k) {
        real_t fb[9], s[9];
        arrive(p, f_prev, xs[k], ys[k], fb);
        real_t rho_kn = raw_moment(fb, 0, 0);
        if (p->pressure && p->kn_mode == 1) {
            real_t r0 = 0.0, r1 = 0.0;
            for (int i = 0; i < NQ; ++i) {
                r0 += f_prev[IDX(i, y0, xs[k], p->nx, p->ny)];
                r1 += f_prev[IDX(i, y1, xs[k], p->nx, p->ny)];
            }
            rho_kn = (p->ny % 2) ? r0 : 0.5 * (r0 + r1);
        }
        node_rates(p, rho_kn, s);
        oracle_collide(fb, P_gx(p), p->gy, s, out + 9 * (size_t)k, NULL, NULL);
    }
}

/* ------------------------------------------------------------- observables */

/* Density and velocity at a node from its post-collision populations: the
 * collision keeps rho and adds rho F to the first moment (Eq. 4, 9), so
 * rho u = sum e_i f~_i - rho F / 2 equals Eq. 13 at the same time level. */
static void node_macro(const oracle_sim* s, int x, int y, real_t* rho, real_t* ux, real_t* uy)
{
    const oracle_params* p = &s->p;
    real_t f[9];
    for (int i = 0; i < NQ; ++i) f[i] = s->ft[IDX(i, y, x, p->nx, p->ny)];
    *rho = raw_moment(f, 0, 0);
    *ux = (raw_moment(f, 1, 0) - 0.5 * (*rho) * P_gx(p)) / (*rho);
    *uy = (raw_moment(f, 0, 1) - 0.5 * (*rho) * p->gy) / (*rho);
}

void oracle_macro(const oracle_sim* s, real_t* rho, real_t* ux, real_t* uy)
{
    const int nx = s->p.nx, ny = s->p.ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            real_t r, a, b;
            node_macro(s, x, y, &r, &a, &b);
            if (rho) rho[(size_t)y * nx + x] = r;
            if (ux) ux[(size_t)y * nx + x] = a;
            if (uy) uy[(size_t)y * nx + x] = b;
        }
}

void oracle_observables(const oracle_sim* s, int profile_col, real_t scal[5], real_t* ux_prof,
                        real_t* uy_prof, real_t* p_centre, real_t* dp_nonlin, real_t* m_of_x)
{
    const oracle_params* p = &s->p;
    const int nx = p->nx, ny = p->ny;
    if (profile_col < 0 || profile_col >= nx) profile_col = p->pressure ? nx - 1 : 0;
    const real_t p_in = (p->pressure ? p->rho_in : p->rho_out) / 3.0;
    const real_t p_out = p->rho_out / 3.0;
    const real_t L = (nx > 1) ? (double)(nx - 1) : 1.0;

    real_t msum = 0.0, mass = 0.0, usum = 0.0;
    for (int x = 0; x < nx; ++x) {
        real_t mx = 0.0, ucol = 0.0, rc = 0.0;
        for (int y = 0; y < ny; ++y) {
            real_t rho, ux, uy;
            node_macro(s, x, y, &rho, &ux, &uy);
            mx += rho * ux;
            ucol += ux;
            mass += rho;
            /* centreline: the middle row, or the mean of the two middle rows */
            if (ny % 2 == 1 && y == (ny - 1) / 2) rc = rho;
            if (ny % 2 == 0 && (y == ny / 2 - 1 || y == ny / 2)) rc += 0.5 * rho;
        }
        msum += mx;
        usum += ucol;
        const real_t pc = rc / 3.0;
        /* Sec. 3.2: p_l decreases linearly from p_in to p_out over L */
        const real_t pl = p_in - (p_in - p_out) * (double)x / L;
        if (m_of_x) m_of_x[x] = mx;
        if (p_centre) p_centre[x] = pc;
        if (dp_nonlin) dp_nonlin[x] = (pc - pl) / p_out;
    }
    real_t umax = -INFINITY;
    real_t ucol_prof[4] = {0, 0, 0, 0};
    for (int y = 0; y < ny; ++y) {
        real_t rho, ux, uy;
        node_macro(s, profile_col, y, &rho, &ux, &uy);
        if (ux_prof) ux_prof[y] = ux;
        if (uy_prof) uy_prof[y] = uy;
        if (RE(ux) > RE(umax)) umax = ux;
        if (y < 2) ucol_prof[y] = ux;
        if (y >= ny - 2) ucol_prof[2 + (y - (ny - 2))] = ux;
    }
    real_t slip;
    if (ny >= 2) {
        /* linear extrapolation of the first two rows to the wall at half a cell */
        const real_t sb = 1.5 * ucol_prof[0] - 0.5 * ucol_prof[1];
        const real_t st = 1.5 * ucol_prof[3] - 0.5 * ucol_prof[2];
        slip = 0.5 * (sb + st);
    } else {
        slip = ucol_prof[0];
    }
    const real_t mbar = msum / (double)nx;
    real_t qnorm = 0.0;
    if (!p->pressure) {
        /* Sec. 3.1: Q = int u dy / (F H^2 sqrt(RT/2) / p), RT = 1/3, p = rho0 RT,
         * F = rho0 g, so Q = sum_y u / (3 g H^2 sqrt(1/6)). */
        if (p->gx != 0.0)
            qnorm = (usum / (double)nx) / (3.0 * P_gx(p) * (double)ny * (double)ny * sqrt(1.0 / 6.0));
    } else {
        /* Sec. 3.2: S = m / m_ns; m_ns is the isothermal no-slip flow with the
         * unreduced viscosity mu = rho_out sqrt(6/pi) Kn_out N / 3 (Eq. 17 with a = 0):
         * m_ns = H^3 (p_in^2 - p_out^2) / (24 mu RT L). */
        const real_t mu = p->rho_out * sqrt(6.0 / PI) * p->kn * (double)ny / 3.0;
        const real_t mns = (double)ny * ny * ny * (p_in * p_in - p_out * p_out) / (24.0 * mu * (1.0 / 3.0) * L);
        qnorm = mbar / mns;
    }
    if (scal) {
        scal[0] = mbar;
        scal[1] = qnorm;
        scal[2] = slip;
        scal[3] = mass;
        scal[4] = umax;
    }
}
