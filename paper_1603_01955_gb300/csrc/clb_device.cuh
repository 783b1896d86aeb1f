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

#include <type_traits>

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
template <> struct Codec<__half> {
    using R = float;
    static __device__ __forceinline__ float dec(__half v, float isc) { return __fmul_rn(__half2float(v), isc); }
    static __device__ __forceinline__ __half enc(float v, float sc) { return __float2half_rn(__fmul_rn(v, sc)); }
};
// BF16 has FP32's exponent range, so its values are stored unscaled (scale 1).
template <> struct Codec<__nv_bfloat16> {
    using R = float;
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

// Lane arithmetic of the collision.  Every operation is written out with its
// rounding (no multiply-add is left for the compiler to contract), so a node
// gets the same bits whether it is collided alone (float, double) or together
// with its neighbour in packed FP32 (float2: the f32x2 instructions of
// sm_100-class GPUs add, multiply or fused-multiply-add both halves of a
// register pair at once, each half rounded as the scalar operation).  Other
// number types (the dual numbers of the adjoint) use their operators.
namespace ln {
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
// Packed FP32 in inline PTX: the .rn forms are never fused by the compiler.
#define CLB_F32X2_BINARY(NAME, OP)                                                  \
    __device__ __forceinline__ float2 NAME(float2 a, float2 b) {                    \
        float2 r;                                                                   \
        asm("{\n\t.reg .b64 pa, pb, pr;\n\t"                                       \
            "mov.b64 pa, {%2, %3};\n\t"                                             \
            "mov.b64 pb, {%4, %5};\n\t" OP                                           \
            " pr, pa, pb;\n\t"                                                       \
            "mov.b64 {%0, %1}, pr;\n\t}"                                             \
            : "=f"(r.x), "=f"(r.y)                                                    \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                \
        return r;                                                                   \
    }
CLB_F32X2_BINARY(add, "add.rn.f32x2")
CLB_F32X2_BINARY(sub, "sub.rn.f32x2")
CLB_F32X2_BINARY(mul, "mul.rn.f32x2")
#undef CLB_F32X2_BINARY
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pc, pr;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pc, {%6, %7};\n\t"
        "fma.rn.f32x2 pr, pa, pb, pc;\n\t"
        "mov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
// -a: free as an operand of a scalar fused multiply-add; one exact packed
// multiply for float2
__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ double neg(double a) { return -a; }
__device__ __forceinline__ float2 neg(float2 a) { return mul(a, make_float2(-1.0f, -1.0f)); }
template <class L> __device__ __forceinline__ L neg(L a) { return -a; }
template <class L> __device__ __forceinline__ L add(L a, L b) { return a + b; }
template <class L> __device__ __forceinline__ L sub(L a, L b) { return a - b; }
template <class L> __device__ __forceinline__ L mul(L a, L b) { return a * b; }
template <class L> __device__ __forceinline__ L fma(L a, L b, L c) { return a * b + c; }
// a scalar in every lane
template <class L, class S> __device__ __forceinline__ L bc(S s) {
    if constexpr (std::is_same<L, float2>::value)
        return make_float2(float(s), float(s));
    else
        return L(s);
}
}  // namespace ln

__device__ __forceinline__ float2 rcp(float2 a) { return make_float2(rcp(a.x), rcp(a.y)); }

// One cascaded collision (Eq. 4 with Eq. 6-9, 12-13), in place on the
// deviations d relative to R = ref.  MODE_PERIODIC: body force F, constant
// rates.  MODE_PRESSURE: no force, s_v and s_q from the local Knudsen number
// Kn = Kn_out rho_out / rho (Sec. 3.2) through Eq. 18 and Eq. 21.
// rho_kn (pressure channel, optional): the density that sets the local
// Knudsen number when it is not the node's own (the column's centreline).
// L: the lane type, R (one node) or float2 (two FP32 nodes, lane x the first).
//
// The order of operations is fixed: no product is ever an operand of an add
// or a subtract (a product that is summed is a fused multiply-add, ln::fma,
// or is formed with a zero addend, prod), so no compiler can fuse it
// differently for one lane type than for another, and each node gets the same
// bits alone or packed.  A few of Eq. 7's braces are regrouped for fewer
// operations; each regrouping is stated where it is made.
template <typename R, int MODE, class L = R>
__device__ __forceinline__ void collide(L (&d)[9], L ref, const KC<R>& c, const L* rho_kn = nullptr) {
    using namespace ln;
    auto k = [](double v) { return bc<L>(R(v)); };          // a literal in every lane
    auto prod = [&](L a, L b) { return fma(a, b, k(0.0)); };  // a product that is summed later
    // raw moments of Eq. 8 (deviation parts)
    const L a57 = add(d[5], d[7]), a68 = add(d[6], d[8]);
    const L p57 = sub(d[5], d[7]), p86 = sub(d[8], d[6]);
    const L nkxy = sub(a68, a57);  // -k'_xy
    const L kxxyy = add(a57, a68);
    const L kxxy = sub(p57, p86);
    const L kxyy = add(p57, p86);
    const L s13 = add(d[1], d[3]), s24 = add(d[2], d[4]);
    const L kxx = add(s13, kxxyy);
    const L kyy = add(s24, kxxyy);
    const L drho = add(add(add(d[0], s13), s24), kxxyy);
    const L jx = add(sub(d[1], d[3]), kxyy);
    const L jy = add(sub(d[2], d[4]), kxxy);
    // Eq. 12-13 and the relaxation rates: tau = A/q, q = rho + B;
    // s_v/4 = (q/4) / hv, hv = q/2 + A (Eq. 18);
    // s_q/4 = (q/4) / hq, hq = q (1/2 + 3q/(16A)) + (pi B2/4) A (Eq. 21)
    const L rho = add(ref, drho);
    L irho, sv4, sq4;
    if (MODE == MODE_PRESSURE) {
        const L q = add(rho_kn ? *rho_kn : rho, bc<L>(c.B));
        const L q4 = mul(q, k(0.25));
        const L hv = fma(q, k(0.5), bc<L>(c.A));
        const L hq = fma(q, fma(bc<L>(c.A316), q, k(0.5)), bc<L>(c.CA));
        if constexpr (std::is_same<L, double>::value) {
            // FP64 pipe bound: one reciprocal, 1 / (rho hv hq), for all three
            const L p = mul(hv, hq);
            const L inv = rcp(mul(rho, p));
            const L ri = mul(rho, inv);
            irho = mul(p, inv);
            sv4 = mul(mul(q4, hq), ri);
            sq4 = mul(mul(q4, hv), ri);
        } else {
            irho = rcp(rho);
            sv4 = mul(q4, rcp(hv));
            sq4 = mul(q4, rcp(hq));
        }
    } else {
        irho = rcp(rho);
        sv4 = bc<L>(c.sv_4);
        sq4 = bc<L>(c.sq_4);
    }
    L ux, uy;
    if (MODE == MODE_PERIODIC) {
        ux = fma(jx, irho, bc<L>(c.hfx));
        uy = fma(jy, irho, bc<L>(c.hfy));
    } else {
        ux = mul(jx, irho);
        uy = mul(jy, irho);
    }
    const L ux2 = mul(ux, ux), uy2 = mul(uy, uy), uxy = mul(ux, uy);
    const L nux = neg(ux), nuy = neg(uy);
    const L ux_2 = mul(k(2.0), ux), uy_2 = mul(k(2.0), uy);
    const L nux_2 = neg(ux_2), nuy_2 = neg(uy_2);
    const L kxxf = fma(k(1.0 / 3.0), ref, kxx);  // full k'_xx
    const L kyyf = fma(k(1.0 / 3.0), ref, kyy);  // full k'_yy
    // Eq. 7, in cascade order.  t5u = rho ux uy - k'_xy is the xy brace
    // without its force term; the xxy, xyy and xxyy braces are written through
    // it: 2 rho ux^2 uy - 2 ux k'_xy = 2 ux t5u, 2 rho ux uy^2 - 2 uy k'_xy =
    // 2 uy t5u, and 3 rho ux^2 uy^2 - 4 ux uy k'_xy = ux uy (3 t5u - k'_xy).
    const L t5u = fma(rho, uxy, nkxy);
    L t3 = sub(fma(rho, fma(ux, ux, uy2), mul(k(2.0 / 3.0), drho)), add(kxx, kyy));
    L t4 = fma(rho, fma(nuy, uy, ux2), sub(kyy, kxx));
    L t5 = t5u;
    L t6 = fma(ux_2, t5u, fma(nuy, kxxf, kxxy));
    L t7 = fma(uy_2, t5u, fma(nux, kyyf, kxyy));
    L t8 = sub(fma(uy_2, kxxy, fma(ux_2, kxyy, fma(uxy, fma(k(3.0), t5u, nkxy), mul(k(1.0 / 9.0), drho)))),
               fma(ux2, kyyf, fma(uy2, kxxf, kxxyy)));
    if (MODE == MODE_PERIODIC) {
        const L fx = bc<L>(c.fx), fy = bc<L>(c.fy);
        const L nrho = neg(rho), nrh = mul(k(0.5), nrho);
        t3 = fma(nrho, fma(fx, ux, mul(fy, uy)), t3);
        t4 = fma(nrho, fma(fx, ux, mul(fy, nuy)), t4);
        t5 = fma(nrh, fma(fx, uy, mul(fy, ux)), t5);
        t6 = fma(nrh, fma(fy, ux2, mul(mul(k(2.0), fx), uxy)), t6);
        t7 = fma(nrh, fma(fx, uy2, mul(mul(k(2.0), fy), uxy)), t7);
        t8 = fma(nrho, fma(fx, mul(ux, uy2), mul(fy, mul(uy, ux2))), t8);
    }
    // kernels g3..g8; hp, hm = (3 g3 +- g4) / 2
    const L g3 = prod(bc<L>(c.s3_12), t3);
    const L g4 = prod(sv4, t4);
    const L g5 = prod(sv4, t5);
    const L hp = fma(k(1.5), g3, mul(k(0.5), g4));
    const L hm = fma(k(1.5), g3, mul(k(-0.5), g4));
    const L g6 = fma(sq4, t6, fma(nuy, hp, mul(nux_2, g5)));
    const L g7 = fma(sq4, t7, fma(nux, hm, mul(nuy_2, g5)));
    // minus the bracket of g8: 2 g3 + uy^2 hp + ux^2 hm + 4 ux uy g5 + 2 uy g6 + 2 ux g7
    L nb8 = mul(k(-2.0), g3);
    nb8 = fma(neg(uy2), hp, nb8);
    nb8 = fma(neg(ux2), hm, nb8);
    nb8 = fma(mul(k(-4.0), uxy), g5, nb8);
    nb8 = fma(nuy_2, g6, nb8);
    nb8 = fma(nux_2, g7, nb8);
    const L g8 = fma(bc<L>(c.s8_4), t8, nb8);
    // Eq. 6 (g0 = g1 = g2 = 0)
    d[0] = fma(k(-4.0), sub(g3, g8), d[0]);
    const L ca = sub(g4, g3), s34 = add(g3, g4), ce = fma(k(2.0), g3, g8);
    d[1] = add(d[1], fma(k(2.0), sub(g7, g8), ca));
    d[3] = add(d[3], fma(k(-2.0), add(g7, g8), ca));
    d[2] = sub(d[2], fma(k(-2.0), sub(g6, g8), s34));
    d[4] = sub(d[4], fma(k(2.0), add(g6, g8), s34));
    const L e5 = add(ce, g5), e6 = sub(ce, g5), gp = add(g6, g7), gm = sub(g6, g7);
    d[5] = add(d[5], sub(e5, gp));
    d[7] = add(d[7], add(e5, gp));
    d[6] = add(d[6], sub(e6, gm));
    d[8] = add(d[8], add(e6, gm));
    if (MODE == MODE_PERIODIC) {
        // source S = T^-1 S^ (Eq. 9-10), T^-1 in closed form as tinv_apply
        const L fx = bc<L>(c.fx), fy = bc<L>(c.fy), two = k(2.0), qt = k(0.25);
        const L m1 = prod(rho, fx);
        const L m2 = prod(rho, fy);
        const L m3 = mul(two, prod(rho, fma(ux, fx, mul(uy, fy))));
        const L m4 = mul(two, prod(rho, fma(ux, fx, mul(nuy, fy))));
        const L m5 = prod(rho, fma(ux, fy, mul(uy, fx)));
        const L m6 = prod(rho, fma(fy, ux2, mul(mul(two, fx), uxy)));
        const L m7 = prod(rho, fma(fx, uy2, mul(mul(two, fy), uxy)));
        const L m8 = mul(two, prod(rho, mul(uxy, fma(fx, uy, mul(fy, ux)))));
        const L cm = fma(k(-2.0), m8, m3);
        const L b4 = add(cm, m4), e4 = sub(cm, m4);
        const L a17 = mul(two, sub(m1, m7)), a26 = mul(two, sub(m2, m6));
        const L p56 = add(m5, m6), n56 = sub(m6, m5);
        const L p78 = add(m7, m8), n78 = sub(m8, m7);
        d[0] = add(d[0], sub(m8, m3));  // S_0 = m0 - m3 + m8 with m0 = 0
        d[1] = add(d[1], mul(qt, add(b4, a17)));
        d[3] = add(d[3], mul(qt, sub(b4, a17)));
        d[2] = add(d[2], mul(qt, add(e4, a26)));
        d[4] = add(d[4], mul(qt, sub(e4, a26)));
        d[5] = add(d[5], mul(qt, add(p56, p78)));
        d[6] = add(d[6], mul(qt, add(n56, n78)));
        d[7] = add(d[7], mul(qt, sub(n78, n56)));
        d[8] = add(d[8], mul(qt, sub(p78, p56)));
    }
}

// ------------------------------------------------- pressure boundary columns

// A stored population field: element (i, y, x) at
//   base + i * plane + y * pitch + xoff + x.
template <class T> struct Field {
    const T* base;
    long long plane;
};

// Pre-collision deviations at one interior node (x in 1..nx-2) of a pressure
// channel, gathered element by element; used only to rebuild the end columns.
template <class T, class R>
__device__ void gather_node(const SweepArgs& a, const KC<R>& c, const Field<T> f, int x, int y, R o[9]) {
    auto at = [&](int i, int dy, int xx) -> R {
        const T* p = f.base + i * f.plane + (long long)(y + dy) * a.pitch + a.xoff + xx;
        return Codec<T>::dec(__ldg(p), c.isc);
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
template <class T, class R>
__device__ __forceinline__ void rebuild_column(const SweepArgs& a, const KC<R>& c, const Field<T> f, int x, int y,
                                            bool inlet, R* out) {
    const int dir = inlet ? 1 : -1;
    R n1[9], n2[9], e1[9], eb[9];
    gather_node<T, R>(a, c, f, x + dir, y, n1);
    gather_node<T, R>(a, c, f, x + 2 * dir, y, n2);
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
