// Pieces of the TMA-staged sweep (sweep_tma.cu): mbarrier and bulk-copy
// wrappers, the tile geometry, and one consumer thread's update of its nodes
// of a staged tile.
//
// A tile is a row segment of W = NC*V columns.  Its inputs are nine segments,
// one per direction i, taken from the row the population is pulled from
// (Eq. 5), each W + 2E elements wide (a 16-byte halo on both sides), so the
// x-shift of the moving populations is a shared-memory offset.  Wall rows need
// no extra data: for the bottom row the three segments that would come from
// row -1 are planes 4, 7, 8 of the row itself (Eq. 20), for the top row those
// from row ny are planes 2, 5, 6.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "clb_device.cuh"
#include "clb_internal.h"

namespace clb {
namespace tma {

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false if the deadline passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both ends 16-byte
// aligned), completing on `bar`.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <class T, int V> struct VecT;
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<float, 2> { using type = float2; };
template <> struct VecT<float, 1> { using type = float; };
template <> struct VecT<__half, 8> { using type = uint4; };
template <> struct VecT<__nv_bfloat16, 8> { using type = uint4; };
template <> struct VecT<__half, 1> { using type = __half; };
template <> struct VecT<__nv_bfloat16, 1> { using type = __nv_bfloat16; };
template <> struct VecT<__half, 4> { using type = uint2; };
template <> struct VecT<__half, 2> { using type = unsigned int; };
template <> struct VecT<__nv_bfloat16, 4> { using type = uint2; };
template <> struct VecT<__nv_bfloat16, 2> { using type = unsigned int; };

// A 16-bit value plus (kNeg: minus) an FP32 term s, rounded once to FP32: the
// mixed-precision add/sub of sm_100 and later (PTX ISA 8.6).  The widening of
// the 16-bit operand is exact, so this is bit for bit the conversion followed
// by an FP32 add.  The instruction counters show the same number of FP32 adds
// as the separate conversion and add (the compiler expands it); it is kept
// for the BF16 sweep, which measured 0.1-0.4 us per sweep faster with it.
template <bool kNeg> __device__ __forceinline__ float add_f16(__half h, float s) {
    float r;
    const unsigned short b = __half_as_ushort(h);
    if (kNeg)
        asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"(b), "f"(s));
    else
        asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(r) : "h"(b), "f"(s));
    return r;
}
template <bool kNeg> __device__ __forceinline__ float add_f16(__nv_bfloat16 h, float s) {
    float r;
    const unsigned short b = __bfloat16_as_ushort(h);
    if (kNeg)
        asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(r) : "h"(b), "f"(s));
    else
        asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(r) : "h"(b), "f"(s));
    return r;
}

// Pairs of 16-bit values converted by one instruction each way.
template <class T> struct Pair16 {
    static constexpr bool ok = false;
};
template <> struct Pair16<__half> {
    static constexpr bool ok = true;
    using P = __half2;
    static __device__ __forceinline__ float2 dec(P p) { return __half22float2(p); }
    static __device__ __forceinline__ P enc(float2 v) { return __floats2half2_rn(v.x, v.y); }
    template <bool kNeg> static __device__ __forceinline__ float2 dec_add(P p, float s) {
        return make_float2(add_f16<kNeg>(__low2half(p), s), add_f16<kNeg>(__high2half(p), s));
    }
};
template <> struct Pair16<__nv_bfloat16> {
    static constexpr bool ok = true;
    using P = __nv_bfloat162;
    static __device__ __forceinline__ float2 dec(P p) { return __bfloat1622float2(p); }
    static __device__ __forceinline__ P enc(float2 v) { return __floats2bfloat162_rn(v.x, v.y); }
    template <bool kNeg> static __device__ __forceinline__ float2 dec_add(P p, float s) {
        return make_float2(add_f16<kNeg>(__low2bfloat16(p), s), add_f16<kNeg>(__high2bfloat16(p), s));
    }
};

// A stored value as it is, in FP32 (no storage scale: the sweeps that use
// this collide in the units of the stored values, with SweepArgs::ks).
template <class T> struct Raw {
    static __device__ __forceinline__ float dec(T v) { return float(v); }
    static __device__ __forceinline__ T enc(float v) { return T(v); }
};
template <> struct Raw<float> {
    static __device__ __forceinline__ float dec(float v) { return v; }
    static __device__ __forceinline__ float enc(float v) { return v; }
};
template <> struct Raw<__half> {
    static __device__ __forceinline__ float dec(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half enc(float v) { return __float2half_rn(v); }
};
template <> struct Raw<__nv_bfloat16> {
    static __device__ __forceinline__ float dec(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 enc(float v) { return __float2bfloat16_rn(v); }
};

template <class T, int NC, int V, int S> struct Geometry {
    static constexpr int W = NC * V;                    // columns per tile
    static constexpr int E = 16 / (int)sizeof(T);       // halo elements per side
    static constexpr int SEG = W + 2 * E;                // elements per segment
    static constexpr int SEG_BYTES = SEG * (int)sizeof(T);
    static constexpr int STAGE_BYTES = 9 * SEG_BYTES;
    static constexpr int SMEM = S * STAGE_BYTES + 2 * S * 8;
};

// Plane held by the segment in slot i for a row of type rt.
__device__ __forceinline__ int seg_plane(int i, int rt) {
    if ((rt & ROW_BOTTOM) && (i == 2 || i == 5 || i == 6)) return i == 2 ? 4 : (i == 5 ? 7 : 8);
    if ((rt & ROW_TOP) && (i == 4 || i == 7 || i == 8)) return i == 4 ? 2 : (i == 7 ? 5 : 6);
    return i;
}
// Row offset of that segment's source row.
__device__ __forceinline__ int seg_dy(int i, int rt) {
    if ((rt & ROW_BOTTOM) && (i == 2 || i == 5 || i == 6)) return 0;
    if ((rt & ROW_TOP) && (i == 4 || i == 7 || i == 8)) return 0;
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return -ey[i];
}

// Issue the nine bulk copies of the tile starting at column x0 of row y from
// field f into `stage`, completing on `full` (one arrive with the byte count).
template <class T, int SEG>
__device__ __forceinline__ void load_tile(const SweepArgs& a, const Field<T> f, int y, int x0,
                                          unsigned char* stage, uint64_t* full) {
    constexpr int E = 16 / (int)sizeof(T);
    const int rt = row_kind(y, a.ny);
    // the segment starts E columns left of the tile; clip at the row end
    const long long first = (long long)a.xoff + x0 - E;
    const int n_el = (int)min((long long)SEG, (long long)a.pitch - first);
    const uint32_t bytes = (uint32_t)n_el * sizeof(T);
    mbar_arrive_expect_tx(full, 9 * bytes);
    for (int i = 0; i < 9; ++i) {
        const T* src = f.base + seg_plane(i, rt) * f.plane + (long long)(y + seg_dy(i, rt)) * a.pitch + first;
        bulk_copy(stage + i * SEG * (int)sizeof(T), src, bytes, full);
    }
}

// One consumer thread's share of a staged tile: nodes x0 .. x0+V-1 of row y
// (x0 = tile start + thread * V).  The row's wall bits and the columns' inlet,
// outlet and halo roles follow from the indices (x = 0 and x = nx - 1; y = 0
// and y = ny - 1), so no mask is loaded.  Pulls the populations out of the stage
// (slot i holds the plane direction i is pulled from, sv the thread's offset
// in it), applies the CBBSR walls (Eq. 20) and the shift of the deviation
// storage, releases the stage on `empty`, rebuilds pressure columns from the
// field `src` (Sec. 3.2), collides (Eq. 4-13, 18, 21) and stores to the
// field `dst` (periodic channels also write the halo columns -1 and nx).
// c: the constants in the units of the stored values (SweepArgs::ks), so
// 16-bit values are converted without a scale multiply.
// kPlain: the tile lies in an interior row and holds neither column 0 nor
// column nx - 1 (nor columns past nx - 1): the copy of this code for such
// tiles, most of them, has no wall, end-column or ragged-edge branches.
template <class T, int MODE, int V, int SEG, bool kPlain>
__device__ __forceinline__ void tile_update(const SweepArgs& a, const KC<typename Codec<T>::R>& c, const T* stage,
                                            int sv, int x0, int y, uint64_t* empty, const Field<T> src,
                                            T* dst) {
    using R = typename Codec<T>::R;
    const int rt = kPlain ? 0 : row_kind(y, a.ny);
    constexpr int E = 16 / (int)sizeof(T);
    constexpr bool kShift = (MODE == MODE_PRESSURE) && !std::is_same<T, double>::value;
    // The thread's window of slot i, columns x0 - 1 .. x0 + V (index k + 1):
    // the V middle values in one aligned vector load, an end value only for the
    // slots that pull from it (e_x = +1 from the left: 1, 5, 8; e_x = -1 from
    // the right: 3, 6, 7; a wall row's CBBSR also takes 6 and 7 from the left
    // and 5 and 8 from the right).
    using VT = typename VecT<T, V>::type;
    // Plain tiles of the 16-bit sweeps take the storage shift of the pulled
    // populations (+sha for 1, -sha for 3, +shd for 5 and 8, -shd for 6 and 7)
    // in the conversion of their slots: every value of those slots is pulled
    // across one column there.
    constexpr bool kFuse = kShift && kPlain && Pair16<T>::ok && V % 2 == 0;
    R w[9][V + 2];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const T* p = stage + i * SEG + E + sv;
        const VT v = *reinterpret_cast<const VT*>(p);
        const T* e = reinterpret_cast<const T*>(&v);
        const bool left = i == 1 || i == 5 || i == 8 || (!kPlain && (i == 6 || i == 7));
        const bool right = i == 3 || i == 6 || i == 7 || (!kPlain && (i == 5 || i == 8));
        if constexpr (kFuse) {
            if (i == 0 || i == 2 || i == 4) {
#pragma unroll
                for (int k = 0; k < V; k += 2) {
                    const float2 q = Pair16<T>::dec(reinterpret_cast<const typename Pair16<T>::P*>(e)[k / 2]);
                    w[i][k + 1] = q.x;
                    w[i][k + 2] = q.y;
                }
                w[i][0] = w[i][V + 1] = R(0);
            } else {
                const float s = (i == 1 || i == 3) ? c.sha : c.shd;
#pragma unroll
                for (int k = 0; k < V; k += 2) {
                    const typename Pair16<T>::P pk = reinterpret_cast<const typename Pair16<T>::P*>(e)[k / 2];
                    const float2 q = right ? Pair16<T>::template dec_add<true>(pk, s)
                                           : Pair16<T>::template dec_add<false>(pk, s);
                    w[i][k + 1] = q.x;
                    w[i][k + 2] = q.y;
                }
                w[i][0] = left ? add_f16<false>(p[-1], s) : R(0);
                w[i][V + 1] = right ? add_f16<true>(p[V], s) : R(0);
            }
            continue;
        }
        if constexpr (Pair16<T>::ok && V % 2 == 0) {
            // two 16-bit values per conversion (exact, as the scalar one)
#pragma unroll
            for (int k = 0; k < V; k += 2) {
                const float2 q = Pair16<T>::dec(reinterpret_cast<const typename Pair16<T>::P*>(e)[k / 2]);
                w[i][k + 1] = q.x;
                w[i][k + 2] = q.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) w[i][k + 1] = Raw<T>::dec(e[k]);
        }
        w[i][0] = left ? Raw<T>::dec(p[-1]) : R(0);
        w[i][V + 1] = right ? Raw<T>::dec(p[V]) : R(0);
    }
    // element of slot i at column x0 + k (k may be -1 .. V)
    auto at = [&](int i, int k) -> R { return w[i][k + 1]; };
    R f[9][V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
        f[0][k] = at(0, k);
        f[1][k] = at(1, k - 1);
        f[3][k] = at(3, k + 1);
        if (rt & ROW_BOTTOM) {
            f[2][k] = at(2, k);
            f[5][k] = ln::fma(c.r, at(5, k), ln::mul(c.rc, at(6, k - 1) + (kShift ? c.shd : R(0))));
            f[6][k] = ln::fma(c.r, at(6, k), ln::mul(c.rc, at(5, k + 1) - (kShift ? c.shd : R(0))));
        } else {
            f[2][k] = at(2, k);
            f[5][k] = at(5, k - 1);
            f[6][k] = at(6, k + 1);
            if (kShift && !kFuse) {
                f[5][k] += c.shd;
                f[6][k] -= c.shd;
            }
        }
        if (rt & ROW_TOP) {
            f[4][k] = at(4, k);
            f[7][k] = ln::fma(c.r, at(7, k), ln::mul(c.rc, at(8, k + 1) - (kShift ? c.shd : R(0))));
            f[8][k] = ln::fma(c.r, at(8, k), ln::mul(c.rc, at(7, k - 1) + (kShift ? c.shd : R(0))));
        } else {
            f[4][k] = at(4, k);
            f[7][k] = at(7, k + 1);
            f[8][k] = at(8, k - 1);
            if (kShift && !kFuse) {
                f[7][k] -= c.shd;
                f[8][k] += c.shd;
            }
        }
        if (kShift && !kFuse) {
            f[1][k] += c.sha;
            f[3][k] -= c.sha;
        }
    }
    mbar_arrive(empty);  // the stage's data is in registers now
    if (!kPlain && x0 >= a.nx) return;

    // the thread's node in the first and in the last column, if any (x0 < nx)
    const int kfirst = !kPlain && x0 == 0 ? 0 : -1;
    const int klast = !kPlain && a.nx - 1 - x0 < V ? a.nx - 1 - x0 : -1;
    if (MODE == MODE_PRESSURE && !kPlain) {
        const int kin = kfirst, kout = klast;  // inlet x = 0, outlet x = nx - 1
        if (kin >= 0) {
            R t[9];
            rebuild_column<T, R>(a, c, src, x0 + kin, y, true, t);
#pragma unroll
            for (int k = 0; k < V; ++k)
                if (k == kin)
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i][k] = t[i];
        }
        if (kout >= 0) {
            R t[9];
            rebuild_column<T, R>(a, c, src, x0 + kout, y, false, t);
#pragma unroll
            for (int k = 0; k < V; ++k)
                if (k == kout)
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i][k] = t[i];
        }
    }
    // The 16-bit sweeps are bound by instruction issue as much as by HBM, so
    // they collide nodes k and k + 1 together in packed FP32 (bit for bit the
    // scalar collision, with about a third fewer instructions per node).  The
    // FP32 sweep is bound by HBM alone: there the packed form finished its
    // arithmetic sooner but moved the bytes less evenly, and back-to-back
    // steps got slower, so it collides one node per lane.
    if constexpr (Pair16<T>::ok && V % 2 == 0) {
#pragma unroll
        for (int k = 0; k < V; k += 2) {
            float2 d[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) d[i] = make_float2(f[i][k], f[i][k + 1]);
            const float2 ref = (MODE == MODE_PRESSURE)
                                   ? ln::fma(ln::bc<float2>(c.slope), make_float2(float(x0 + k), float(x0 + k + 1)),
                                             ln::bc<float2>(c.ref0))
                                   : ln::bc<float2>(c.ref0);
            collide<R, MODE, float2>(d, ref, c);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i][k] = d[i].x;
                f[i][k + 1] = d[i].y;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            R d[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) d[i] = f[i][k];
            const R ref = (MODE == MODE_PRESSURE) ? ln::fma(c.slope, R(x0 + k), c.ref0) : c.ref0;
            collide<R, MODE>(d, ref, c);
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i][k] = d[i];
        }
    }
    const long long P = a.plane;
    T* orow = dst + (long long)y * a.pitch + a.xoff;
    if (kPlain || x0 + V <= a.nx) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            VT v;
            T* e = reinterpret_cast<T*>(&v);
            if constexpr (Pair16<T>::ok && V % 2 == 0) {
                // two values per conversion, each rounded as by the scalar one
#pragma unroll
                for (int k = 0; k < V; k += 2)
                    reinterpret_cast<typename Pair16<T>::P*>(e)[k / 2] =
                        Pair16<T>::enc(make_float2(f[i][k], f[i][k + 1]));
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) e[k] = Raw<T>::enc(f[i][k]);
            }
            *reinterpret_cast<VT*>(orow + i * P + x0) = v;
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (x0 + k < a.nx)
#pragma unroll
                for (int i = 0; i < 9; ++i) orow[i * P + x0 + k] = Raw<T>::enc(f[i][k]);
    }
    if (MODE == MODE_PERIODIC && !kPlain) {
        // column 0 is mirrored into the halo column nx, column nx - 1 into -1
#pragma unroll
        for (int k = 0; k < V; ++k) {
            if (k == kfirst) {
                orow[3 * P + a.nx] = Raw<T>::enc(f[3][k]);
                orow[6 * P + a.nx] = Raw<T>::enc(f[6][k]);
                orow[7 * P + a.nx] = Raw<T>::enc(f[7][k]);
            }
            if (k == klast) {
                orow[1 * P - 1] = Raw<T>::enc(f[1][k]);
                orow[5 * P - 1] = Raw<T>::enc(f[5][k]);
                orow[8 * P - 1] = Raw<T>::enc(f[8][k]);
            }
        }
    }
}

}  // namespace tma
}  // namespace clb
