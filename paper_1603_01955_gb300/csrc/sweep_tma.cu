// Fused D2Q9 stream-and-collide sweep with TMA-staged inputs (GB300, sm_103a).
//
// Same arithmetic as sweep.cu (Eq. 4-13, 18, 20, 21 of Liu & He,
// arXiv:1603.01955, node for node), organised so that the bytes in flight do
// not depend on registers: the blocks of a persistent grid claim row segments
// ("tiles") of W = NC*V columns from a counter; a producer warp streams each
// tile's nine plane segments (one per direction, from the row the population
// is pulled from) into a ring of S shared-memory stages with bulk asynchronous
// copies (cp.async.bulk, the Tensor Memory Accelerator), completing on an
// mbarrier; NC consumer threads take their V nodes of each plane out of the
// stage, release it, collide, and store vectors of V values straight to global
// memory.  The tile geometry and the consumer's update are in tma_common.cuh.
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
#include "tma_common.cuh"

namespace clb {
namespace {

using namespace tma;

// Tiles are handed out in claim order from a counter in global memory
// (sched[0]), so that blocks finishing early take more of them: most rows end
// in a short tile, and a fixed round-robin would give some blocks a whole tile
// more work than others in every step.  The producer thread claims a tile one
// tile ahead, passes its row and column to the consumers in shared memory, and
// after its last claim counts itself in sched[1]; the last block to do so
// puts both counters back to zero for the next launch.
template <class T, int MODE, int NC, int V, int S, int MB>
__global__ void __launch_bounds__(NC + 32, MB) sweep_tma_kernel(const SweepArgs a, int ntiles, int tiles_per_row,
                                                            unsigned* sched, unsigned* status) {
    using G = Geometry<T, NC, V, S>;
    using R = typename Codec<T>::R;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * G::STAGE_BYTES);
    uint64_t* empty = full + S;
    __shared__ int abort_flag;
    __shared__ int2 stage_tile[S];  // (row, column tile) of each stage; row -1: no more tiles
    const T* __restrict__ fin = static_cast<const T*>(a.fin);
    T* __restrict__ fout = static_cast<T*>(a.fout);
    const KC<R>& c = a.ks;  // constants in the units of the stored values
    const Field<T> src{fin, a.plane};

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, NC);
        }
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    // Programmatic dependent launch: the next sweep may begin launching now
    // (its blocks start as this one's leave their SMs); no global memory is
    // touched before the previous sweep has completed and its writes are
    // visible, so reading its output, overwriting its input and claiming from
    // the counters it reset are safe.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (threadIdx.x >= NC) {
        // ---------------------------------------------------------- producer
        if (threadIdx.x != NC) return;
        // claim k is tile k, or ntiles-1-k when a.tile_order is 1 (every other
        // step: the rows the last sweep wrote last are read first, while many
        // of them are still in L2)
        const bool rev = a.tile_order != 0;
        int issued = 0;
        unsigned next = atomicAdd(sched, 1u);
        for (int q = 0;; ++q) {
            const int s = q % S;
            if (q >= S && !mbar_wait(empty + s, ((q / S) - 1) & 1)) {
                atomicOr(status, 1u);
                abort_flag = 1;
                break;
            }
            if (*(volatile int*)&abort_flag) break;
            const unsigned k = next;
            if (k >= (unsigned)ntiles) {
                stage_tile[s] = make_int2(-1, 0);
                mbar_arrive(full + s);  // completes the stage's phase with no bytes
                break;
            }
            next = atomicAdd(sched, 1u);
            const int t = rev ? ntiles - 1 - (int)k : (int)k;
            const int y = t / tiles_per_row, xt = t - y * tiles_per_row;
            stage_tile[s] = make_int2(y, xt);
            if ((int)k == a.withhold_tile) continue;  // testing: the consumers' waits must expire
            load_tile<T, G::SEG>(a, src, y, xt * G::W, smem + s * G::STAGE_BYTES, full + s);
            issued = q + 1;
        }
        if (atomicAdd(sched + 1, 1u) == gridDim.x - 1) {  // every block has made its last claim
            atomicExch(sched, 0u);
            atomicExch(sched + 1, 0u);
        }
        // copies still in flight for stages nobody will consume: wait (bounded)
        if (*(volatile int*)&abort_flag)
            for (int it = max(0, issued - S); it < issued; ++it) mbar_wait(full + it % S, (it / S) & 1);
        return;
    }

    // -------------------------------------------------------------- consumers
    const int tcx = threadIdx.x;
    for (int q = 0;; ++q) {
        const int s = q % S;
        if (!mbar_wait(full + s, (q / S) & 1)) {
            atomicOr(status, 2u);
            abort_flag = 1;
            return;
        }
        const int2 yt = stage_tile[s];  // written before the stage's arrive (the wait's asm is a memory barrier)
        const int y = yt.x, xt = yt.y;
        if (y < 0) return;
        const T* stage = reinterpret_cast<const T*>(smem + s * G::STAGE_BYTES);
        // most tiles are plain: an interior row, neither end column (the
        // first and the last tile of a row hold those)
        if (row_kind(y, a.ny) == 0 && xt != 0 && xt != tiles_per_row - 1)
            tile_update<T, MODE, V, G::SEG, true>(a, c, stage, tcx * V, xt * G::W + tcx * V, y, empty + s, src, fout);
        else
            tile_update<T, MODE, V, G::SEG, false>(a, c, stage, tcx * V, xt * G::W + tcx * V, y, empty + s, src, fout);
    }
}

template <class T, int MODE, int NC, int V, int S, int MB>
cudaError_t launch_tma_one(const SweepArgs& a, cudaStream_t st, unsigned* sched, unsigned* status) {
    using G = Geometry<T, NC, V, S>;
    auto kern = sweep_tma_kernel<T, MODE, NC, V, S, MB>;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    // resident blocks (SMs x blocks per SM), worked out once per device: the
    // occupancy query would otherwise add host time to every launch
    constexpr int kMaxDevices = 64;
    static int resident[kMaxDevices] = {};  // per instantiation
    int dev = 0;
    cudaGetDevice(&dev);
    int slots = (dev >= 0 && dev < kMaxDevices) ? resident[dev] : 0;
    if (slots == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NC + 32, G::SMEM);
        if (e != cudaSuccess) return e;
        slots = max(1, per_sm) * sms;
        if (dev >= 0 && dev < kMaxDevices) resident[dev] = slots;
    }
    const int tiles_per_row = (a.nx + G::W - 1) / G::W;
    const int ntiles = tiles_per_row * a.ny;
    const int grid = min(ntiles, slots);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NC + 32);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, ntiles, tiles_per_row, sched, status);
}

}  // namespace

// TMA-staged sweep; variant picks (consumer threads, nodes per thread,
// stages, blocks per SM the registers are sized for) from this table.
// Variant 0 is the default for FP32 storage, 1 for FP16 and BF16: the fastest
// of the shapes measured on the 25601 x 256 pressure channel; 2 (the 16-bit
// default before tiles were claimed dynamically) is the one alternative.
#define CLB_TMA_VARIANTS(X) X(0, 512, 2, 3, 1) X(1, 128, 4, 2, 4) X(2, 256, 4, 3, 2)

int tma_variant_count() { return 3; }

template <class T>
static cudaError_t dispatch_tma(int mode, int variant, const SweepArgs& a, cudaStream_t st, unsigned* sched,
                                unsigned* status) {
#define CLB_TMA_CASE(id, nc, v, s, mb)                                                               \
    case id:                                                                                        \
        return mode == MODE_PRESSURE ? launch_tma_one<T, MODE_PRESSURE, nc, v, s, mb>(a, st, sched, status) \
                                     : launch_tma_one<T, MODE_PERIODIC, nc, v, s, mb>(a, st, sched, status);
    switch (variant) { CLB_TMA_VARIANTS(CLB_TMA_CASE) }
#undef CLB_TMA_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_tma(int storage, int mode, int variant, const SweepArgs& a, cudaStream_t st,
                             unsigned* sched, unsigned* status) {
    if (storage == 1) return dispatch_tma<float>(mode, variant, a, st, sched, status);
    if (storage == 2) return dispatch_tma<__half>(mode, variant, a, st, sched, status);
    if (storage == 3) return dispatch_tma<__nv_bfloat16>(mode, variant, a, st, sched, status);
    return cudaErrorInvalidValue;
}

}  // namespace clb
