// Fused D2Q9 stream-and-collide sweep with TMA-staged inputs (GB300, sm_103a).
//
// Same arithmetic as sweep.cu (Eq. 4-13, 18, 20, 21 of Liu & He,
// arXiv:1603.01955, node for node), organised so that the bytes in flight do
// not depend on registers: a persistent grid walks row segments ("tiles") of
// W = NC*V columns; a producer warp streams each tile's nine plane segments
// (one per direction, from the row the population is pulled from) into a ring
// of S shared-memory stages with bulk asynchronous copies (cp.async.bulk, the
// Tensor Memory Accelerator), completing on an mbarrier; NC consumer threads
// collide V nodes each from shared memory and store 16-byte vectors straight
// to global memory, then release the stage.  The x-shift of the moving
// populations is a shared-memory offset (a 16-byte halo on both sides of each
// segment), so no shuffles are needed.
//
// Wall rows need no extra data: for the bottom row the three segments that
// would come from row -1 are replaced by planes 4, 7, 8 of the row itself
// (Eq. 20), for the top row those from row ny by planes 2, 5, 6 of the row.
//
// Every mbarrier wait is bounded (about a second of clock cycles); on expiry
// the kernel records an error bit in *status, the producer waits (bounded) for
// the copies it issued, and all threads return.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "clb_device.cuh"
#include "clb_internal.h"

namespace clb {
namespace {

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

template <class T, int NC, int V, int S> struct Geometry {
    static constexpr int W = NC * V;                    // columns per tile
    static constexpr int E = 16 / (int)sizeof(T);       // halo elements per side
    static constexpr int SEG = W + 2 * E;                // elements per segment
    static constexpr int SEG_BYTES = SEG * (int)sizeof(T);
    static constexpr int STAGE_BYTES = 9 * SEG_BYTES;
    static constexpr int SMEM = S * STAGE_BYTES + 2 * S * 8;
};

// Source row offset of the segment in slot i for a row of type rt.
__device__ __forceinline__ int seg_plane(int i, int rt) {
    if ((rt & ROW_BOTTOM) && (i == 2 || i == 5 || i == 6)) return i == 2 ? 4 : (i == 5 ? 7 : 8);
    if ((rt & ROW_TOP) && (i == 4 || i == 7 || i == 8)) return i == 4 ? 2 : (i == 7 ? 5 : 6);
    return i;
}
__device__ __forceinline__ int seg_dy(int i, int rt) {
    if ((rt & ROW_BOTTOM) && (i == 2 || i == 5 || i == 6)) return 0;
    if ((rt & ROW_TOP) && (i == 4 || i == 7 || i == 8)) return 0;
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return -ey[i];
}

template <class T, int MODE, int NC, int V, int S, int MB>
__global__ void __launch_bounds__(NC + 32, MB) sweep_tma_kernel(const SweepArgs a, int ntiles, int tiles_per_row,
                                                            unsigned* status) {
    using G = Geometry<T, NC, V, S>;
    using R = typename Codec<T>::R;
    constexpr bool kShift = (MODE == MODE_PRESSURE) && !std::is_same<T, double>::value;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * G::STAGE_BYTES);
    uint64_t* empty = full + S;
    __shared__ int abort_flag;
    const T* __restrict__ fin = static_cast<const T*>(a.fin);
    T* __restrict__ fout = static_cast<T*>(a.fout);
    const KC<R>& c = kc<R>(a);
    const long long P = a.plane;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, NC);
        }
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();

    const int my_tiles = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (threadIdx.x >= NC) {
        // ---------------------------------------------------------- producer
        if (threadIdx.x != NC) return;
        int issued = 0;
        for (int it = 0; it < my_tiles; ++it) {
            const int s = it % S;
            if (it >= S && !mbar_wait(empty + s, ((it / S) - 1) & 1)) {
                atomicOr(status, 1u);
                abort_flag = 1;
                break;
            }
            if (*(volatile int*)&abort_flag) break;
            const int tile = (int)blockIdx.x + it * (int)gridDim.x;
            if (tile == a.withhold_tile) continue;  // testing: the consumers' waits must expire
            const int y = tile / tiles_per_row;
            const int x0 = (tile % tiles_per_row) * G::W;
            const int rt = a.row_type[y];
            // the segment starts E columns left of the tile; clip at the row end
            const long long first = (long long)a.xoff + x0 - G::E;
            const int n_el = (int)min((long long)G::SEG, (long long)a.pitch - first);
            const uint32_t bytes = (uint32_t)n_el * sizeof(T);
            unsigned char* stage = smem + s * G::STAGE_BYTES;
            mbar_arrive_expect_tx(full + s, 9 * bytes);
            for (int i = 0; i < 9; ++i) {
                const T* src = fin + seg_plane(i, rt) * P + (long long)(y + seg_dy(i, rt)) * a.pitch + first;
                bulk_copy(stage + i * G::SEG_BYTES, src, bytes, full + s);
            }
            issued = it + 1;
        }
        // copies still in flight for stages nobody will consume: wait (bounded)
        if (*(volatile int*)&abort_flag)
            for (int it = max(0, issued - S); it < issued; ++it) mbar_wait(full + it % S, (it / S) & 1);
        return;
    }

    // -------------------------------------------------------------- consumers
    const int tcx = threadIdx.x;
    for (int it = 0; it < my_tiles; ++it) {
        const int s = it % S;
        if (!mbar_wait(full + s, (it / S) & 1)) {
            atomicOr(status, 2u);
            abort_flag = 1;
            return;
        }
        const int tile = (int)blockIdx.x + it * (int)gridDim.x;
        const int y = tile / tiles_per_row;
        const int x0 = (tile % tiles_per_row) * G::W + tcx * V;
        const int rt = a.row_type[y];
        const T* stage = reinterpret_cast<const T*>(smem + s * G::STAGE_BYTES);
        // element of slot i at column x0 + k (k may be -1 .. V)
        auto at = [&](int i, int k) -> R {
            return Codec<T>::dec(stage[i * G::SEG + G::E + tcx * V + k], c.isc);
        };
        R f[9][V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            f[0][k] = at(0, k);
            f[1][k] = at(1, k - 1);
            f[3][k] = at(3, k + 1);
            if (rt & ROW_BOTTOM) {
                f[2][k] = at(2, k);
                f[5][k] = c.r * at(5, k) + c.rc * (at(6, k - 1) + (kShift ? c.shd : R(0)));
                f[6][k] = c.r * at(6, k) + c.rc * (at(5, k + 1) - (kShift ? c.shd : R(0)));
            } else {
                f[2][k] = at(2, k);
                f[5][k] = at(5, k - 1);
                f[6][k] = at(6, k + 1);
                if (kShift) {
                    f[5][k] += c.shd;
                    f[6][k] -= c.shd;
                }
            }
            if (rt & ROW_TOP) {
                f[4][k] = at(4, k);
                f[7][k] = c.r * at(7, k) + c.rc * (at(8, k + 1) - (kShift ? c.shd : R(0)));
                f[8][k] = c.r * at(8, k) + c.rc * (at(7, k - 1) + (kShift ? c.shd : R(0)));
            } else {
                f[4][k] = at(4, k);
                f[7][k] = at(7, k + 1);
                f[8][k] = at(8, k - 1);
                if (kShift) {
                    f[7][k] -= c.shd;
                    f[8][k] += c.shd;
                }
            }
            if (kShift) {
                f[1][k] += c.sha;
                f[3][k] -= c.sha;
            }
        }
        mbar_arrive(empty + s);  // the stage's data is in registers now
        if (x0 >= a.nx) continue;

        uint8_t ct[V];
        int kin = -1, kout = -1;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            ct[k] = a.col_type[x0 + k];
            if (MODE == MODE_PRESSURE) {
                if (ct[k] & COL_INLET) kin = k;
                if (ct[k] & COL_OUTLET) kout = k;
            }
        }
        if (MODE == MODE_PRESSURE) {
            if (kin >= 0) {
                R t[9];
                rebuild_column<T, R>(a, c, fin, x0 + kin, y, true, t);
#pragma unroll
                for (int k = 0; k < V; ++k)
                    if (k == kin)
#pragma unroll
                        for (int i = 0; i < 9; ++i) f[i][k] = t[i];
            }
            if (kout >= 0) {
                R t[9];
                rebuild_column<T, R>(a, c, fin, x0 + kout, y, false, t);
#pragma unroll
                for (int k = 0; k < V; ++k)
                    if (k == kout)
#pragma unroll
                        for (int i = 0; i < 9; ++i) f[i][k] = t[i];
            }
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
            R d[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) d[i] = f[i][k];
            const R ref = (MODE == MODE_PRESSURE) ? c.ref0 + c.slope * R(x0 + k) : c.ref0;
            collide<R, MODE>(d, ref, c);
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i][k] = d[i];
        }
        T* orow = fout + (long long)y * a.pitch + a.xoff;
        if (x0 + V <= a.nx) {
            using VT = typename VecT<T, V>::type;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                VT w;
                T* e = reinterpret_cast<T*>(&w);
#pragma unroll
                for (int k = 0; k < V; ++k) e[k] = Codec<T>::enc(f[i][k], c.sc);
                *reinterpret_cast<VT*>(orow + i * P + x0) = w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k)
                if (x0 + k < a.nx)
#pragma unroll
                    for (int i = 0; i < 9; ++i) orow[i * P + x0 + k] = Codec<T>::enc(f[i][k], c.sc);
        }
        if (MODE == MODE_PERIODIC) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                if (ct[k] & COL_HALO_RIGHT) {
                    orow[3 * P + a.nx] = Codec<T>::enc(f[3][k], c.sc);
                    orow[6 * P + a.nx] = Codec<T>::enc(f[6][k], c.sc);
                    orow[7 * P + a.nx] = Codec<T>::enc(f[7][k], c.sc);
                }
                if (ct[k] & COL_HALO_LEFT) {
                    orow[1 * P - 1] = Codec<T>::enc(f[1][k], c.sc);
                    orow[5 * P - 1] = Codec<T>::enc(f[5][k], c.sc);
                    orow[8 * P - 1] = Codec<T>::enc(f[8][k], c.sc);
                }
            }
        }
    }
}

template <class T, int MODE, int NC, int V, int S, int MB>
cudaError_t launch_tma_one(const SweepArgs& a, cudaStream_t st, unsigned* status) {
    using G = Geometry<T, NC, V, S>;
    auto kern = sweep_tma_kernel<T, MODE, NC, V, S, MB>;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NC + 32, G::SMEM);
    if (e != cudaSuccess) return e;
    const int tiles_per_row = (a.nx + G::W - 1) / G::W;
    const int ntiles = tiles_per_row * a.ny;
    const int grid = min(ntiles, max(1, per_sm) * sms);
    kern<<<grid, NC + 32, G::SMEM, st>>>(a, ntiles, tiles_per_row, status);
    return cudaGetLastError();
}

}  // namespace

// TMA-staged sweep; variant picks (consumer threads, nodes per thread,
// stages, blocks per SM the registers are sized for) from this table.
#define CLB_TMA_VARIANTS(X)                                                                             \
    X(0, 128, 4, 4, 3) X(1, 256, 4, 3, 2) X(2, 256, 2, 4, 2) X(3, 256, 2, 6, 2) X(4, 256, 1, 8, 2)      \
    X(5, 256, 4, 4, 2) X(6, 512, 1, 4, 1) X(7, 128, 2, 8, 3) X(8, 512, 1, 6, 1) X(9, 512, 1, 4, 2)      \
    X(10, 384, 1, 4, 2) X(11, 384, 1, 6, 2) X(12, 512, 2, 3, 1)

int tma_variant_count() { return 13; }

template <class T>
static cudaError_t dispatch_tma(int mode, int variant, const SweepArgs& a, cudaStream_t st, unsigned* status) {
#define CLB_TMA_CASE(id, nc, v, s, mb)                                                               \
    case id:                                                                                        \
        return mode == MODE_PRESSURE ? launch_tma_one<T, MODE_PRESSURE, nc, v, s, mb>(a, st, status) \
                                     : launch_tma_one<T, MODE_PERIODIC, nc, v, s, mb>(a, st, status);
    switch (variant) { CLB_TMA_VARIANTS(CLB_TMA_CASE) }
#undef CLB_TMA_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_tma(int storage, int mode, int variant, const SweepArgs& a, cudaStream_t st,
                             unsigned* status) {
    if (storage == 1) return dispatch_tma<float>(mode, variant, a, st, status);
    if (storage == 2) return dispatch_tma<__half>(mode, variant, a, st, status);
    if (storage == 3) return dispatch_tma<__nv_bfloat16>(mode, variant, a, st, status);
    return cudaErrorInvalidValue;
}

}  // namespace clb
