// Fused D2Q9 stream-and-collide sweep of the cascaded lattice Boltzmann (CLB)
// channel solver (Liu & He, arXiv:1603.01955), hand-written for GB300 (sm_103a).
//
// One launch = one time step for every node: pull-streaming of the
// post-collision populations of the last step (Eq. 5), CBBSR walls in the
// first and last rows (Eq. 20 and its mirror), pressure inlet/outlet columns
// (Sec. 3.2) or periodic x (Sec. 3.1), then the cascaded collision (Eq. 4,
// 6-13) with per-node relaxation rates (Eq. 18, 21), stored into the other
// buffer.
//
// Layout: structure of arrays, plane i (direction e_i of Eq. 1) of ny rows,
// each row `pitch` elements with column x at element xoff + x (xoff = 128
// bytes), so that every row and every vector of V columns is aligned.  Column
// -1 and column nx are halo columns that the previous sweep filled with the
// periodic images, so no wrap-around appears in the loads.
//
// Launch: one row per blockIdx.y, V consecutive nodes per thread along x.  A
// thread loads each plane as one 8/16-byte vector; the populations that move
// along x arrive from the neighbouring lane by a warp shuffle, and only lanes 0
// and 31 load the one element across the warp edge.  The wall rows are whole
// blocks, so the wall branch never diverges inside a warp.  The inlet and
// outlet columns of a pressure channel are recognised from their indices
// (x = 0 and x = nx - 1) and rebuilt before their collision.  No value is read twice from DRAM: every population of the
// last step is pulled by exactly one node.
#include <cstdint>
#include <type_traits>

#include "clb_device.cuh"
#include "clb_internal.h"

// Build-time knobs (defaults: the measured best on GB300).
// CLB_SWEEP_MIN_BLOCKS: resident 256-thread blocks per SM asked of the
// compiler for the FP32/16-bit sweeps, which caps their registers: 4 -> 64
// registers, 8 blocks of 128 threads per SM.  These kernels are bound by DRAM
// latency, and the occupancy this buys outweighs a 36-byte spill.
// CLB_SWEEP_MIN_BLOCKS_FP64: the same for the FP64 sweep (FP64-pipe bound).
// CLB_SWEEP_STREAMING: 1 = evict-first (.cs) hints on the population loads
// and stores, which are touched exactly once per step (measured slower).
#ifndef CLB_SWEEP_MIN_BLOCKS
#define CLB_SWEEP_MIN_BLOCKS 4
#endif
#ifndef CLB_SWEEP_MIN_BLOCKS_FP64
#define CLB_SWEEP_MIN_BLOCKS_FP64 2
#endif
#ifndef CLB_SWEEP_STREAMING
#define CLB_SWEEP_STREAMING 0
#endif

namespace clb {

template <class T> struct MinBlocks { static constexpr int value = CLB_SWEEP_MIN_BLOCKS; };
template <> struct MinBlocks<double> { static constexpr int value = CLB_SWEEP_MIN_BLOCKS_FP64; };

template <class T> __device__ __forceinline__ T ld_stream(const T* p) {
#if CLB_SWEEP_STREAMING
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}
template <class T> __device__ __forceinline__ void st_stream(T* p, const T& v) {
#if CLB_SWEEP_STREAMING
    __stcs(p, v);
#else
    *p = v;
#endif
}

template <class T, int V> struct Vec;
template <> struct Vec<__half, 4> { using type = uint2; };
template <> struct Vec<__half, 8> { using type = uint4; };
template <> struct Vec<__nv_bfloat16, 4> { using type = uint2; };
template <> struct Vec<__nv_bfloat16, 8> { using type = uint4; };
template <> struct Vec<float, 1> { using type = float; };
template <> struct Vec<float, 2> { using type = float2; };
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<double, 1> { using type = double; };
template <> struct Vec<double, 2> { using type = double2; };

template <class T, int V>
__device__ __forceinline__ void vload(const T* p, T (&v)[V]) {
    using VT = typename Vec<T, V>::type;
    const VT w = ld_stream(reinterpret_cast<const VT*>(p));
    const T* e = reinterpret_cast<const T*>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = e[k];
}

template <class T, int V>
__device__ __forceinline__ void vstore(T* p, const T (&v)[V]) {
    using VT = typename Vec<T, V>::type;
    VT w;
    T* e = reinterpret_cast<T*>(&w);
#pragma unroll
    for (int k = 0; k < V; ++k) e[k] = v[k];
    st_stream(reinterpret_cast<VT*>(p), w);
}

// V columns x0..x0+V-1 of one row, decoded (zeros for threads past the halo
// column).
template <class T, class R, int V>
__device__ __forceinline__ void row_vec(const T* row, int x0, bool live, R isc, R (&o)[V]) {
    if (live) {
        T v[V];
        vload<T, V>(row + x0, v);
#pragma unroll
        for (int k = 0; k < V; ++k) o[k] = Codec<T>::dec(v[k], isc);
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) o[k] = R(0);
    }
}

// Columns x0-1..x0+V-2 from the vector of columns x0..x0+V-1 (a population
// moving in +x): the first element comes from the previous lane.
template <class T, class R, int V>
__device__ __forceinline__ void from_left(const R (&v)[V], const T* row, int x0, int lane, R isc, R (&o)[V]) {
    R prev = __shfl_up_sync(0xffffffffu, v[V - 1], 1);
    if (lane == 0) prev = Codec<T>::dec(__ldg(row + x0 - 1), isc);
    o[0] = prev;
#pragma unroll
    for (int k = 1; k < V; ++k) o[k] = v[k - 1];
}

// Columns x0+1..x0+V (a population moving in -x): the last element comes from
// the next lane.
template <class T, class R, int V>
__device__ __forceinline__ void from_right(const R (&v)[V], const T* row, int x0, int lane, bool live, R isc,
                                           R (&o)[V]) {
    R next = __shfl_down_sync(0xffffffffu, v[0], 1);
    if (lane == 31 && live) next = Codec<T>::dec(__ldg(row + x0 + V), isc);
#pragma unroll
    for (int k = 0; k < V - 1; ++k) o[k] = v[k + 1];
    o[V - 1] = next;
}

template <class R, int V>
__device__ __forceinline__ void add_shift(R (&o)[V], R s) {
#pragma unroll
    for (int k = 0; k < V; ++k) o[k] += s;
}

template <class T, int MODE, int V>
__global__ void __launch_bounds__(256, MinBlocks<T>::value) sweep_kernel(const SweepArgs a) {
    using R = typename Codec<T>::R;
    constexpr bool kShift = (MODE == MODE_PRESSURE) && !std::is_same<T, double>::value;  // R(x) != 0
    const T* __restrict__ fin = static_cast<const T*>(a.fin);
    T* __restrict__ fout = static_cast<T*>(a.fout);

    const int lane = threadIdx.x & 31;
    const int y = blockIdx.y;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (x0 - lane * V > a.nx) return;  // the whole warp lies past the halo column
    const bool live = x0 <= a.nx;      // this thread's vector can feed a real node

    const KC<R>& c = kc<R>(a);
    const long long P = a.plane;
    const T* row = fin + (long long)y * a.pitch + a.xoff;  // plane 0, row y, column 0
    const int rt = row_kind(y, a.ny);

    R f[9][V];
    // rest population and the two that move along x only (Eq. 5)
    row_vec<T, R, V>(row, x0, live, c.isc, f[0]);
    {
        R v[V];
        row_vec<T, R, V>(row + 1 * P, x0, live, c.isc, v);
        from_left<T, R, V>(v, row + 1 * P, x0, lane, c.isc, f[1]);
        row_vec<T, R, V>(row + 3 * P, x0, live, c.isc, v);
        from_right<T, R, V>(v, row + 3 * P, x0, lane, live, c.isc, f[3]);
        if (kShift) {
            add_shift<R, V>(f[1], c.sha);
            add_shift<R, V>(f[3], -c.sha);
        }
    }
    // populations entering from the row below: 2, 5, 6
    if (rt & ROW_BOTTOM) {
        // Eq. 20: fbar2 = f~4, fbar5 = r f~7 + (1-r) f~8(x-1), fbar6 = r f~8 + (1-r) f~7(x+1)
        R v4[V], v7[V], v8[V], s8[V], s7[V];
        row_vec<T, R, V>(row + 4 * P, x0, live, c.isc, v4);
        row_vec<T, R, V>(row + 7 * P, x0, live, c.isc, v7);
        row_vec<T, R, V>(row + 8 * P, x0, live, c.isc, v8);
        from_left<T, R, V>(v8, row + 8 * P, x0, lane, c.isc, s8);
        from_right<T, R, V>(v7, row + 7 * P, x0, lane, live, c.isc, s7);
        if (kShift) {
            add_shift<R, V>(s8, c.shd);
            add_shift<R, V>(s7, -c.shd);
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
            f[2][k] = v4[k];
            f[5][k] = ln::fma(c.r, v7[k], ln::mul(c.rc, s8[k]));
            f[6][k] = ln::fma(c.r, v8[k], ln::mul(c.rc, s7[k]));
        }
    } else {
        const T* rd = row - a.pitch;
        R v[V];
        row_vec<T, R, V>(rd + 2 * P, x0, live, c.isc, f[2]);
        row_vec<T, R, V>(rd + 5 * P, x0, live, c.isc, v);
        from_left<T, R, V>(v, rd + 5 * P, x0, lane, c.isc, f[5]);
        row_vec<T, R, V>(rd + 6 * P, x0, live, c.isc, v);
        from_right<T, R, V>(v, rd + 6 * P, x0, lane, live, c.isc, f[6]);
        if (kShift) {
            add_shift<R, V>(f[5], c.shd);
            add_shift<R, V>(f[6], -c.shd);
        }
    }
    // populations entering from the row above: 4, 7, 8
    if (rt & ROW_TOP) {
        // mirror of Eq. 20: fbar4 = f~2, fbar7 = r f~5 + (1-r) f~6(x+1), fbar8 = r f~6 + (1-r) f~5(x-1)
        R v2[V], v5[V], v6[V], s6[V], s5[V];
        row_vec<T, R, V>(row + 2 * P, x0, live, c.isc, v2);
        row_vec<T, R, V>(row + 5 * P, x0, live, c.isc, v5);
        row_vec<T, R, V>(row + 6 * P, x0, live, c.isc, v6);
        from_right<T, R, V>(v6, row + 6 * P, x0, lane, live, c.isc, s6);
        from_left<T, R, V>(v5, row + 5 * P, x0, lane, c.isc, s5);
        if (kShift) {
            add_shift<R, V>(s6, -c.shd);
            add_shift<R, V>(s5, c.shd);
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
            f[4][k] = v2[k];
            f[7][k] = ln::fma(c.r, v5[k], ln::mul(c.rc, s6[k]));
            f[8][k] = ln::fma(c.r, v6[k], ln::mul(c.rc, s5[k]));
        }
    } else {
        const T* ru = row + a.pitch;
        R v[V];
        row_vec<T, R, V>(ru + 4 * P, x0, live, c.isc, f[4]);
        row_vec<T, R, V>(ru + 7 * P, x0, live, c.isc, v);
        from_right<T, R, V>(v, ru + 7 * P, x0, lane, live, c.isc, f[7]);
        row_vec<T, R, V>(ru + 8 * P, x0, live, c.isc, v);
        from_left<T, R, V>(v, ru + 8 * P, x0, lane, c.isc, f[8]);
        if (kShift) {
            add_shift<R, V>(f[7], -c.shd);
            add_shift<R, V>(f[8], c.shd);
        }
    }
    if (!live || x0 >= a.nx) return;  // nothing of this thread's own to store

    // the thread's node in the first and in the last column, if any: the
    // pressure inlet and outlet, rebuilt here (Sec. 3.2) before the collision
    // loop, or the columns mirrored into the periodic halo
    const int kfirst = x0 == 0 ? 0 : -1;
    const int klast = a.nx - 1 - x0 < V ? a.nx - 1 - x0 : -1;
    if (MODE == MODE_PRESSURE) {
        const int kin = kfirst, kout = klast;
        if (kin >= 0) {
            R t[9];
            rebuild_column<T, R>(a, c, Field<T>{fin, a.plane}, x0 + kin, y, true, t);
#pragma unroll
            for (int k = 0; k < V; ++k)
                if (k == kin)
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i][k] = t[i];
        }
        if (kout >= 0) {
            R t[9];
            rebuild_column<T, R>(a, c, Field<T>{fin, a.plane}, x0 + kout, y, false, t);
#pragma unroll
            for (int k = 0; k < V; ++k)
                if (k == kout)
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i][k] = t[i];
        }
    }

    // centreline Knudsen number: the column's centre density of the last step
    R rk[V];
    const bool centre_kn = MODE == MODE_PRESSURE && a.kn_mode == 1;
    if (centre_kn) {
        const R* rc0 = static_cast<const R*>(a.rc_in);
        const R* rc1 = rc0 + a.rc_stride;
#pragma unroll
        for (int k = 0; k < V; ++k)
            rk[k] = a.yc0 == a.yc1 ? rc0[x0 + k] : R(0.5) * (rc0[x0 + k] + rc1[x0 + k]);
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
        R d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = f[i][k];
        const R ref = (MODE == MODE_PRESSURE) ? ln::fma(c.slope, R(x0 + k), c.ref0) : c.ref0;
        if (centre_kn && (y == a.yc0 || y == a.yc1) && x0 + k < a.nx) {
            R dr = d[0];
#pragma unroll
            for (int i = 1; i < 9; ++i) dr += d[i];
            R* out = static_cast<R*>(a.rc_out) + (y == a.yc0 ? 0 : a.rc_stride);
            out[x0 + k] = ref + dr;
        }
        collide<R, MODE>(d, ref, c, centre_kn ? &rk[k] : nullptr);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i][k] = d[i];
    }

    T* orow = fout + (long long)y * a.pitch + a.xoff;
    if (x0 + V <= a.nx) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            T v[V];
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = Codec<T>::enc(f[i][k], c.sc);
            vstore<T, V>(orow + i * P + x0, v);
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (x0 + k < a.nx)
#pragma unroll
                for (int i = 0; i < 9; ++i) orow[i * P + x0 + k] = Codec<T>::enc(f[i][k], c.sc);
    }
    if (MODE == MODE_PERIODIC) {
        // periodic images for the next sweep: column 0 -> halo column nx
        // (populations moving in -x), column nx-1 -> halo column -1 (moving in +x)
#pragma unroll
        for (int k = 0; k < V; ++k) {
            if (k == kfirst) {
                orow[3 * P + a.nx] = Codec<T>::enc(f[3][k], c.sc);
                orow[6 * P + a.nx] = Codec<T>::enc(f[6][k], c.sc);
                orow[7 * P + a.nx] = Codec<T>::enc(f[7][k], c.sc);
            }
            if (k == klast) {
                orow[1 * P - 1] = Codec<T>::enc(f[1][k], c.sc);
                orow[5 * P - 1] = Codec<T>::enc(f[5][k], c.sc);
                orow[8 * P - 1] = Codec<T>::enc(f[8][k], c.sc);
            }
        }
    }
}

template <class T, int MODE, int V>
static cudaError_t launch_one(int block_x, const SweepArgs& a, cudaStream_t s) {
    const int groups = (a.nx + V) / V;  // vectors covering columns 0..nx (halo included)
    dim3 block(block_x, 1, 1);
    dim3 grid((groups + block_x - 1) / block_x, a.ny, 1);
    sweep_kernel<T, MODE, V><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <class T, int V>
static cudaError_t launch_mode(int mode, int block_x, const SweepArgs& a, cudaStream_t s) {
    if (mode == MODE_PRESSURE) return launch_one<T, MODE_PRESSURE, V>(block_x, a, s);
    return launch_one<T, MODE_PERIODIC, V>(block_x, a, s);
}

template <typename R> static void fill(KC<R>& c, const SweepArgs& a) {
    c.s3_12 = R(a.s3 / 12.0);
    c.s8_4 = R(a.s8 / 4.0);
    c.sv_4 = R(a.sv / 4.0);
    c.sq_4 = R(a.sq / 4.0);
    c.A = R(a.rate_A);
    c.B = R(a.rate_B);
    c.A316 = a.rate_A > 0 ? R(3.0 / (16.0 * a.rate_A)) : R(0);
    c.CA = R(a.rate_C * a.rate_A);
    c.hfx = R(0.5 * a.gx);
    c.hfy = R(0.5 * a.gy);
    c.fx = R(a.gx);
    c.fy = R(a.gy);
    c.r = R(a.r);
    c.rc = R(1.0 - a.r);
    c.ref0 = R(a.ref0);
    c.slope = R(a.ref_slope);
    c.sha = R(-a.ref_slope / 9.0);
    c.shd = R(-a.ref_slope / 36.0);
    c.drho_in = R(a.drho_in);
    c.drho_out = R(a.drho_out);
    c.sc = R(a.store_scale);
    c.isc = R(1.0 / a.store_scale);
}

void derive_constants(SweepArgs& a) {
    fill(a.kf, a);
    fill(a.kd, a);
    // densities scale, 1/densities scale inversely, rates and velocities do not
    KC<float>& k = a.ks;
    k = a.kf;
    const float s = a.kf.sc;
    k.A *= s;
    k.B *= s;
    k.CA *= s;
    k.A316 /= s;
    k.ref0 *= s;
    k.slope *= s;
    k.sha *= s;
    k.shd *= s;
    k.drho_in *= s;
    k.drho_out *= s;
    k.sc = k.isc = 1.0f;
}

bool sweep_supported(int storage, int vec) {
    if (storage == 0) return vec == 1 || vec == 2;
    if (storage == 1) return vec == 1 || vec == 2 || vec == 4;
    if (storage == 2 || storage == 3) return vec == 4 || vec == 8;
    return false;
}

cudaError_t launch_sweep(int storage, int mode, int vec, int block_x, const SweepArgs& a, cudaStream_t s) {
    if (storage == 0) {
        if (vec == 1) return launch_mode<double, 1>(mode, block_x, a, s);
        if (vec == 2) return launch_mode<double, 2>(mode, block_x, a, s);
    } else if (storage == 1) {
        if (vec == 1) return launch_mode<float, 1>(mode, block_x, a, s);
        if (vec == 2) return launch_mode<float, 2>(mode, block_x, a, s);
        if (vec == 4) return launch_mode<float, 4>(mode, block_x, a, s);
    } else if (storage == 2) {
        if (vec == 4) return launch_mode<__half, 4>(mode, block_x, a, s);
        if (vec == 8) return launch_mode<__half, 8>(mode, block_x, a, s);
    } else if (storage == 3) {
        if (vec == 4) return launch_mode<__nv_bfloat16, 4>(mode, block_x, a, s);
        if (vec == 8) return launch_mode<__nv_bfloat16, 8>(mode, block_x, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace clb
