// Device-side arithmetic of the cascaded lattice Boltzmann (CLB) collision of
// Liu & He (arXiv:1603.01955), Sec. 2, written for GB300 (sm_103a).
//
// Every routine works on deviations d_i = f_i - w_i R from a reference density
// R (w_i the D2Q9 rest weights 4/9, 1/9, 1/36).  The moments' reference parts
// cancel analytically, so the braces of Eq. 7 only ever combine small numbers
// and FP32 keeps its precision; with R = 0 the same code is the plain form.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "clb_internal.h"

namespace clb {

// Storage element <-> compute value.  FP64 and FP32 store the deviation
// itself; the 16-bit formats store it times a power-of-two field scale
// (FP16: keeps the small deviations out of the subnormal range; BF16: 1) and
// are decoded to FP32 for the collision.
template <class T> struct Codec;
template <> struct Codec<double> {
    using R = double;
    static __device__ __forceinline__ double dec(double v, double) { return v; }
    static __device__ __forceinline__ double enc(double v, double) { return v; }
};
template <> struct Codec<float> {
    using R = float;
    static __device__ __forceinline__ float dec(float v, float) { return v; }
    static __device__ __forceinline__ float enc(float v, float) { return v; }
};
// unscale / prescale: the scaling of dec and enc alone, for callers that
// convert two values per instruction.
template <> struct Codec<__half> {
    using R = float;
    static __device__ __forceinline__ float unscale(float v, float isc) { return v * isc; }
    static __device__ __forceinline__ float prescale(float v, float sc) { return v * sc; }
    static __device__ __forceinline__ float dec(__half v, float isc) { return __half2float(v) * isc; }
    static __device__ __forceinline__ __half enc(float v, float sc) { return __float2half_rn(v * sc); }
};
// BF16 has FP32's exponent range, so its values are stored unscaled (scale 1).
template <> struct Codec<__nv_bfloat16> {
    using R = float;
    static __device__ __forceinline__ float unscale(float v, float) { return v; }
    static __device__ __forceinline__ float prescale(float v, float) { return v; }
    static __device__ __forceinline__ float dec(__nv_bfloat16 v, float) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 enc(float v, float) { return __float2bfloat16_rn(v); }
};

// D2Q9 rest weights: Eq. 11 at u = 0 through the closed-form inverse of Eq. 10.
template <typename R> struct Wt {
    static constexpr R w0 = R(4.0 / 9.0);
    static constexpr R wa = R(1.0 / 9.0);   // axis directions 1..4
    static constexpr R wd = R(1.0 / 36.0);  // diagonal directions 5..8
};

// FP32: the hardware reciprocal (PTX rcp.approx, within 1 ulp); its error is
// far below the FP32 storage rounding.  FP64: the IEEE quotient.
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// FP64 reciprocal by Newton-Raphson: the approximate hardware reciprocal
// (rcp.approx.ftz.f64) refined twice by r <- r + r (1 - x r), each step
// squaring the relative error, which ends within a few ulp of 1/x for the
// positive normal densities and rate denominators it is applied to.  GB300's
// FP64 rate is low, so this is cheaper than a correctly rounded division.
__device__ __forceinline__ double rcp(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// The launch constants of the compute type, read in place from the kernel
// parameters.
template <typename R> __device__ __forceinline__ const KC<R>& kc(const SweepArgs& a);
template <> __device__ __forceinline__ const KC<float>& kc<float>(const SweepArgs& a) { return a.kf; }
template <> __device__ __forceinline__ const KC<double>& kc<double>(const SweepArgs& a) { return a.kd; }

// Inverse of the moment matrix T of Eq. 10 in closed form: populations from the
// nine raw moments m0..m8 (1, x, y, xx+yy, xx-yy, xy, xxy, xyy, xxyy).
template <typename R>
__device__ __forceinline__ void tinv_apply(const R m[9], R f[9]) {
    const R q = R(0.25);
    f[0] = m[0] - m[3] + m[8];
    const R c = m[3] - R(2) * m[8];
    f[1] = q * (c + m[4] + R(2) * (m[1] - m[7]));
    f[3] = q * (c + m[4] - R(2) * (m[1] - m[7]));
    f[2] = q * (c - m[4] + R(2) * (m[2] - m[6]));
    f[4] = q * (c - m[4] - R(2) * (m[2] - m[6]));
    f[5] = q * (m[5] + m[6] + m[7] + m[8]);
    f[6] = q * (-m[5] + m[6] - m[7] + m[8]);
    f[7] = q * (m[5] - m[6] - m[7] + m[8]);
    f[8] = q * (-m[5] - m[6] + m[7] + m[8]);
}

// Equilibrium of Eq. 11 minus w_i R, for a node with density rho = R + drho
// and velocity (ux, uy).
template <typename R>
__device__ __forceinline__ void feq_dev(R drho, R rho, R ux, R uy, R f[9]) {
    const R ux2 = ux * ux, uy2 = uy * uy, u2 = ux2 + uy2;
    R m[9];
    m[0] = drho;
    m[1] = rho * ux;
    m[2] = rho * uy;
    m[3] = R(2.0 / 3.0) * drho + rho * u2;
    m[4] = rho * (ux2 - uy2);
    m[5] = rho * ux * uy;
    m[6] = rho * uy * (R(1.0 / 3.0) + ux2);
    m[7] = rho * ux * (R(1.0 / 3.0) + uy2);
    m[8] = R(1.0 / 9.0) * drho + rho * (R(1.0 / 3.0) * u2 + ux2 * uy2);
    tinv_apply(m, f);
}

// Density deviation and momentum sum e_i d_i of nine deviations.
template <typename R>
__device__ __forceinline__ void macro_dev(const R d[9], R& drho, R& jx, R& jy) {
    const R p57 = d[5] - d[7], p86 = d[8] - d[6];
    drho = d[0] + (d[1] + d[3]) + (d[2] + d[4]) + ((d[5] + d[7]) + (d[6] + d[8]));
    jx = (d[1] - d[3]) + (p57 + p86);
    jy = (d[2] - d[4]) + (p57 - p86);
}

// One cascaded collision (Eq. 4 with Eq. 6-9, 12-13), in place on the
// deviations d relative to R = ref.  MODE_PERIODIC: body force F, constant
// rates.  MODE_PRESSURE: no force, s_v and s_q from the local Knudsen number
// Kn = Kn_out rho_out / rho (Sec. 3.2) through Eq. 18 and Eq. 21.
// rho_kn (pressure channel, optional): the density that sets the local
// Knudsen number when it is not the node's own (the column's centreline).
template <typename R, int MODE>
__device__ __forceinline__ void collide(R (&d)[9], R ref, const KC<R>& c, const R* rho_kn = nullptr) {
    // raw moments of Eq. 8 (deviation parts)
    const R a57 = d[5] + d[7], a68 = d[6] + d[8];
    const R p57 = d[5] - d[7], p86 = d[8] - d[6];
    const R kxy = a57 - a68;
    const R kxxyy = a57 + a68;
    const R kxxy = p57 - p86;
    const R kxyy = p57 + p86;
    const R s13 = d[1] + d[3], s24 = d[2] + d[4];
    const R kxx = s13 + kxxyy;
    const R kyy = s24 + kxxyy;
    const R drho = d[0] + s13 + s24 + kxxyy;
    const R jx = (d[1] - d[3]) + kxyy;
    const R jy = (d[2] - d[4]) + kxxy;
    // Eq. 12-13
    const R rho = ref + drho;
    const R irho = rcp(rho);
    R ux = jx * irho, uy = jy * irho;
    if (MODE == MODE_PERIODIC) {
        ux += c.hfx;
        uy += c.hfy;
    }
    // relaxation rates
    R sv4, sq4;
    if (MODE == MODE_PRESSURE) {
        // tau = A/q, q = rho + B; 1/s_v = 1/2 + tau (Eq. 18);
        // 1/s_q = 1/2 + 3/(16 tau) + (pi B2/4) tau (Eq. 21)
        const R q = (rho_kn ? *rho_kn : rho) + c.B;
        sv4 = R(0.25) * q * rcp(R(0.5) * q + c.A);
        sq4 = R(0.25) * q * rcp(q * (R(0.5) + c.A316 * q) + c.CA);
    } else {
        sv4 = c.sv_4;
        sq4 = c.sq_4;
    }
    const R ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const R third = R(1.0 / 3.0) * ref;
    const R kxxf = third + kxx;  // full k'_xx
    const R kyyf = third + kyy;  // full k'_yy
    // Eq. 7, in cascade order
    R t3 = R(2.0 / 3.0) * drho - (kxx + kyy) + rho * (ux2 + uy2);
    R t4 = rho * (ux2 - uy2) - (kxx - kyy);
    R t5 = rho * uxy - kxy;
    R t6 = R(2) * rho * ux2 * uy + kxxy - R(2) * ux * kxy - uy * kxxf;
    R t7 = R(2) * rho * ux * uy2 + kxyy - R(2) * uy * kxy - ux * kyyf;
    R t8 = R(1.0 / 9.0) * drho + R(3) * rho * ux2 * uy2 -
           (kxxyy - R(2) * ux * kxyy - R(2) * uy * kxxy + ux2 * kyyf + uy2 * kxxf + R(4) * uxy * kxy);
    if (MODE == MODE_PERIODIC) {
        const R fx = c.fx, fy = c.fy;
        t3 -= rho * (fx * ux + fy * uy);
        t4 -= rho * (fx * ux - fy * uy);
        t5 -= R(0.5) * rho * (fx * uy + fy * ux);
        t6 -= R(0.5) * rho * (fy * ux2 + R(2) * fx * uxy);
        t7 -= R(0.5) * rho * (fx * uy2 + R(2) * fy * uxy);
        t8 -= rho * (fx * ux * uy2 + fy * uy * ux2);
    }
    const R g3 = c.s3_12 * t3;
    const R g4 = sv4 * t4;
    const R g5 = sv4 * t5;
    const R h34p = R(3) * g3 + g4, h34m = R(3) * g3 - g4;
    const R g6 = sq4 * t6 - R(0.5) * uy * h34p - R(2) * ux * g5;
    const R g7 = sq4 * t7 - R(0.5) * ux * h34m - R(2) * uy * g5;
    const R g8 = c.s8_4 * t8 - R(2) * g3 - R(0.5) * (uy2 * h34p + ux2 * h34m) - R(4) * uxy * g5 -
                 R(2) * (uy * g6 + ux * g7);
    // Eq. 6 (g0 = g1 = g2 = 0)
    const R ca = g4 - g3, cb = -g3 - g4, ce = R(2) * g3 + g8;
    d[0] += R(-4) * (g3 - g8);
    d[1] += ca + R(2) * (g7 - g8);
    d[3] += ca - R(2) * (g7 + g8);
    d[2] += cb + R(2) * (g6 - g8);
    d[4] += cb - R(2) * (g6 + g8);
    d[5] += ce + g5 - g6 - g7;
    d[6] += ce - g5 - g6 + g7;
    d[7] += ce + g5 + g6 + g7;
    d[8] += ce - g5 + g6 - g7;
    if (MODE == MODE_PERIODIC) {
        // source S = T^-1 S^ (Eq. 9-10)
        const R fx = c.fx, fy = c.fy;
        R m[9];
        m[0] = R(0);
        m[1] = rho * fx;
        m[2] = rho * fy;
        m[3] = R(2) * rho * (ux * fx + uy * fy);
        m[4] = R(2) * rho * (ux * fx - uy * fy);
        m[5] = rho * (ux * fy + uy * fx);
        m[6] = rho * (fy * ux2 + R(2) * fx * uxy);
        m[7] = rho * (fx * uy2 + R(2) * fy * uxy);
        m[8] = R(2) * rho * uxy * (fx * uy + fy * ux);
        R S[9];
        tinv_apply(m, S);
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] += S[i];
    }
}

// ------------------------------------------------- pressure boundary columns

// A stored population field: element (i, y, x) at
//   base + i * plane + (y & rmask) * pitch + xoff + x,
// rmask = -1 for a whole buffer, 2^k - 1 for a ring of 2^k rows.
template <class T> struct Field {
    const T* base;
    long long plane;
    int rmask;
};

// Read-only load (kCG = false: through the non-coherent path, for values
// written before this launch) or an L2-coherent load (kCG = true: for values
// other blocks wrote earlier in the same launch).
template <bool kCG, class T> __device__ __forceinline__ T ld_field(const T* p) {
    if constexpr (kCG)
        return __ldcg(p);
    else
        return __ldg(p);
}

// Pre-collision deviations at one interior node (x in 1..nx-2) of a pressure
// channel, gathered element by element; used only to rebuild the end columns.
template <class T, class R, bool kCG = false>
__device__ void gather_node(const SweepArgs& a, const KC<R>& c, const Field<T> f, int x, int y, R o[9]) {
    auto at = [&](int i, int dy, int xx) -> R {
        const T* p = f.base + i * f.plane + (long long)((y + dy) & f.rmask) * a.pitch + a.xoff + xx;
        return Codec<T>::dec(ld_field<kCG>(p), c.isc);
    };
    const int rt = row_kind(y, a.ny);
    const R sha = c.sha, shd = c.shd;  // source at x-1; the source at x+1 gets the negative
    o[0] = at(0, 0, x);
    o[1] = at(1, 0, x - 1) + sha;
    o[3] = at(3, 0, x + 1) - sha;
    if (rt & ROW_BOTTOM) {
        o[2] = at(4, 0, x);
        o[5] = c.r * at(7, 0, x) + c.rc * (at(8, 0, x - 1) + shd);
        o[6] = c.r * at(8, 0, x) + c.rc * (at(7, 0, x + 1) - shd);
    } else {
        o[2] = at(2, -1, x);
        o[5] = at(5, -1, x - 1) + shd;
        o[6] = at(6, -1, x + 1) - shd;
    }
    if (rt & ROW_TOP) {
        o[4] = at(2, 0, x);
        o[7] = c.r * at(5, 0, x) + c.rc * (at(6, 0, x + 1) - shd);
        o[8] = c.r * at(6, 0, x) + c.rc * (at(5, 0, x - 1) + shd);
    } else {
        o[4] = at(4, 1, x);
        o[7] = at(7, 1, x + 1) - shd;
        o[8] = at(8, 1, x - 1) + shd;
    }
}

// Pressure column rebuilt by linear extrapolation (reading of Sec. 3.2):
//   f_i(b) = f^eq_i(rho_b, u_b) + f^neq_i(b+d),  u_b = 2 u(b+d) - u(b+2d),
//   f^neq = f - f^eq(rho, u),
// with d = +1 at the inlet (rho_b = rho_in) and -1 at the outlet (rho_out):
// the velocity is extrapolated linearly, the non-equilibrium part comes from
// the first interior neighbour (a linear extrapolation of it as well would
// amplify the shortest x-wavelength threefold and diverge at tau ~ 30).
// Output: deviations relative to R(b).
template <class T, class R, bool kCG = false>
__device__ __forceinline__ void rebuild_column(const SweepArgs& a, const KC<R>& c, const Field<T> f, int x, int y,
                                            bool inlet, R* out) {
    const int dir = inlet ? 1 : -1;
    R n1[9], n2[9], e1[9], eb[9];
    gather_node<T, R, kCG>(a, c, f, x + dir, y, n1);
    gather_node<T, R, kCG>(a, c, f, x + 2 * dir, y, n2);
    R dr1, jx1, jy1, dr2, jx2, jy2;
    macro_dev(n1, dr1, jx1, jy1);
    macro_dev(n2, dr2, jx2, jy2);
    const R r1 = c.ref0 + c.slope * R(x + dir) + dr1;
    const R r2 = c.ref0 + c.slope * R(x + 2 * dir) + dr2;
    const R u1x = jx1 / r1, u1y = jy1 / r1, u2x = jx2 / r2, u2y = jy2 / r2;
    feq_dev(dr1, r1, u1x, u1y, e1);
    const R drb = inlet ? c.drho_in : c.drho_out;
    const R rb = c.ref0 + c.slope * R(x) + drb;
    feq_dev(drb, rb, R(2) * u1x - u2x, R(2) * u1y - u2y, eb);
    // the neighbour's deviations are relative to R(x+d); f^neq does not depend
    // on the reference, so only the equilibrium carries R(b)
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = eb[i] + (n1[i] - e1[i]);
}

}  // namespace clb
