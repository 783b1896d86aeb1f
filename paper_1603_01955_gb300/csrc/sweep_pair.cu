// Two time steps per launch, the intermediate state kept in L2 (GB300, sm_103a).
//
// Each node update is exactly the one of sweep.cu / sweep_tma.cu (Eq. 4-13,
// 18, 20, 21 of Liu & He, arXiv:1603.01955), so two steps here equal two
// single-step launches bit for bit.  What changes is where the state of the
// middle time level lives: the first step of a row writes it into a ring of
// RR rows (all nine planes, same pitch as the buffers) instead of a full
// buffer, and the second step pulls it from there while it is still in L2.
// Per two steps the HBM sees one read of buffer A and one write of buffer B:
// 36 B per node update in FP32 instead of 72.
//
// Work items are row tiles of W = NC*V columns at level 0 (first step, A ->
// ring) or level 1 (second step, ring -> B), numbered in a fixed order: phase
// k holds the level-0 tiles of row k followed by the level-1 tiles of row
// k - L.  Block b takes items b, b + G, b + 2G, ... (G blocks) in that order.
// Dependencies, always on items with smaller numbers:
//   level 1, row j : level 0 of rows j-1, j, j+1 complete (its pull stencil);
//   level 0, row k : level 1 of rows k-RR-1 .. k-RR+1 complete (the readers
//                    of the ring slot row k overwrites), so RR > L + 1.
// The lag L (16 phases) puts most items in flight (grid x stages) between a
// row's two levels: a level-1 producer then mostly finds its dependencies
// already met instead of stalling its pipeline.  The launch is cooperative,
// so all blocks are resident; the block holding the smallest unfinished item
// has all of that item's dependencies complete, so the schedule cannot
// deadlock.  Completion is counted per row and level: the consumers arrive on
// an mbarrier once their stores are issued, a publisher thread waits on it
// and does one release-add per tile.  The producer polls the counters of an
// item's dependencies with relaxed loads (all rows of a stencil at once),
// acquires with a fence, and orders its bulk copies of the ring after that
// with a proxy fence.
//
// Counters never need clearing between launches: launch e (the host's epoch)
// expects the row counters at e * tiles.  Every wait is bounded (about a
// second); on expiry a status bit is set, the epoch arithmetic no longer
// holds, later launches return at once, and the host clears the counters when
// it reads the status.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "clb_device.cuh"
#include "clb_internal.h"
#include "tma_common.cuh"

// Build-time knob: CLB_PAIR_LAG > 0 sets the lag (phases between a row's two
// levels) instead of the default 16.
#ifndef CLB_PAIR_LAG
#define CLB_PAIR_LAG 0
#endif

namespace clb {
namespace {

using namespace tma;

// Item idx (0 <= idx < 2 ny T) -> (level, row, tile); T tiles per row, lag
// L phases between a row's two levels.
__device__ __forceinline__ void pair_item(int idx, int T, int ny, int L, int& level, int& y, int& tile) {
    const int cA = min(L, ny) * T;            // phases 0 .. L-1: level 0 only
    const int nB = max(0, ny - L);            // phases L .. ny-1: both levels
    const int cB = nB * 2 * T;
    if (idx < cA) {
        level = 0;
        y = idx / T;
        tile = idx % T;
    } else if (idx < cA + cB) {
        const int j = idx - cA, w = j % (2 * T);
        level = w / T;
        tile = w % T;
        y = L + j / (2 * T) - level * L;
    } else {                                   // phases ny .. ny+L-1: level 1 only
        const int j = idx - cA - cB;
        level = 1;
        y = nB + j / T;
        tile = j % T;
    }
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until done[r] has reached target for the rows r0 .. r0+2 that lie in
// 0 .. ny-1: the three counters are polled together with relaxed loads, and
// one fence then makes the wait an acquire of every release it observed.
__device__ bool wait_rows(const unsigned* done, int r0, int ny, unsigned target) {
    const int a = max(r0, 0), b = min(r0 + 2, ny - 1);
    if (a > b) return true;
    long long t0 = -1;
    for (;;) {
        bool ok = true;
        // all loads issued before any is compared
        unsigned v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = (a + k <= b) ? ld_relaxed(done + a + k) : target;
#pragma unroll
        for (int k = 0; k < 3; ++k) ok = ok && (int)(v[k] - target) >= 0;
        if (ok) break;
        if (t0 < 0) t0 = clock64();
        else if (clock64() - t0 > kWaitCycles) return false;
        __nanosleep(64);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return true;
}

// Wait until the publisher has counted n tiles (bounded).
__device__ bool wait_published(const int* published, int n) {
    if (*(volatile const int*)published >= n) return true;
    const long long t0 = clock64();
    while (*(volatile const int*)published < n) {
        if (clock64() - t0 > kWaitCycles) return false;
        __nanosleep(32);
    }
    return true;
}

// Shared memory of the two-step sweep: the staged tiles, the full and empty
// mbarriers of each stage, then the Q stored mbarriers of the publication
// queue.
template <class T, int NC, int V, int S> struct PairSmem {
    using G = Geometry<T, NC, V, S>;
    static constexpr int Q = 2 * S;  // tiles the publisher may lag behind the producer
    static constexpr int BYTES = S * G::STAGE_BYTES + (2 * S + Q) * 8;
};

// Block: NC consumer threads, then a producer warp (lane 0 works) and a
// publisher warp (lane 0 works).  Per stage: `full` completes when the
// producer's copies have landed, `empty` when the consumers hold the values
// in registers.  Per tile of the publication queue (Q slots): `stored`
// completes when every consumer has issued its stores, and the publisher then
// counts the tile in its row counter with a release-add.  Consumers never
// wait for each other or for the publication: its latency overlaps the next
// tiles.  The producer issues tile i only after the publisher has counted
// tile i - Q, so no queue slot is reused before it was read.
template <class T, int MODE, int NC, int V, int S, int MB>
__global__ void __launch_bounds__(NC + 64, MB) sweep_pair_kernel(const SweepArgs a, const PairArgs p, unsigned* status) {
    using G = Geometry<T, NC, V, S>;
    using R = typename Codec<T>::R;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int Q = PairSmem<T, NC, V, S>::Q;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * G::STAGE_BYTES);
    uint64_t* empty = full + S;
    uint64_t* stored = empty + S;
    __shared__ int item[S];      // work item of each stage (-1: stop)
    __shared__ int pub_item[Q];  // work item of each publication slot
    __shared__ int published;    // tiles counted by the publisher
    __shared__ int abort_flag;
    const KC<R>& c = a.ks;  // constants in the units of the stored values
    T* ring = static_cast<T*>(p.ring);
    // The source field of a work item is built from scalar selects: with
    // whole-struct selects or copies of two such fields (`level ? fR : fA`)
    // the generated code took the pointer of the wrong one.
    auto source = [&](int level) {
        return Field<T>{level ? static_cast<const T*>(ring) : static_cast<const T*>(a.fin),
                        level ? p.ring_plane : a.plane, level ? p.ring_rows - 1 : -1};
    };
    const int Tn = p.tiles_per_row;
    const int total = 2 * a.ny * Tn;
    unsigned* done0 = p.done;
    unsigned* done1 = p.done + a.ny;
    const unsigned target = (unsigned)(p.epoch + 1) * (unsigned)Tn;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, NC);
        }
        for (int q = 0; q < Q; ++q) mbar_init(stored + q, NC);
        published = 0;
        // an earlier launch gave up: the counters are stale until the host clears them
        abort_flag = *(volatile unsigned*)status != 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (abort_flag) return;

    if (threadIdx.x >= NC + 32) {
        // --------------------------------------------------------- publisher
        if (threadIdx.x != NC + 32) return;
        for (int it = 0;; ++it) {
            const int q = it % Q;
            if (!mbar_wait(stored + q, (it / Q) & 1)) {
                atomicOr(status, 8u);
                abort_flag = 1;
                return;
            }
            const int idx = pub_item[q];
            if (idx < 0) return;
            int level, y, tile;
            pair_item(idx, Tn, a.ny, p.lag, level, y, tile);
            // the consumers' stores (ordered before `stored`) become visible
            // to every block that acquires the row counter
            red_release_add((level ? done1 : done0) + y, 1u);
            *(volatile int*)&published = it + 1;
        }
    }

    if (threadIdx.x >= NC) {
        // ---------------------------------------------------------- producer
        if (threadIdx.x != NC) return;
        int issued = 0;
        for (int it = 0;; ++it) {
            const int s = it % S;
            // wait for the item's dependencies before its stage is free, so that
            // this latency overlaps the consumers' work on the occupied stages
            const int idx = (int)blockIdx.x + it * (int)gridDim.x;
            const bool last = idx >= total;
            int level = 0, y = 0, tile = 0;
            bool ok = true;
            if (!last) {
                pair_item(idx, Tn, a.ny, p.lag, level, y, tile);
                ok = level == 1 ? wait_rows(done0, y - 1, a.ny, target)
                                : wait_rows(done1, y - p.ring_rows - 1, a.ny, target);
            }
            if (!ok) {
                atomicOr(status, 4u);
                abort_flag = 1;
                break;
            }
            if (it >= S && !mbar_wait(empty + s, ((it / S) - 1) & 1)) {
                atomicOr(status, 1u);
                abort_flag = 1;
                break;
            }
            if (it >= Q && !wait_published(&published, it - Q + 1)) {
                atomicOr(status, 16u);
                abort_flag = 1;
                break;
            }
            if (*(volatile int*)&abort_flag) break;
            if (last) {
                item[s] = -1;
                pub_item[it % Q] = -1;
                mbar_arrive(full + s);  // tells the consumers, and through them the publisher, to stop
                break;
            }
            if (level == 1) fence_proxy_async_global();  // ring rows written by other blocks are read by bulk copies
            item[s] = idx;
            pub_item[it % Q] = idx;
            if (idx == a.withhold_tile) continue;  // testing: the consumers' waits must expire
            load_tile<T, G::SEG>(a, source(level), y, tile * G::W, smem + s * G::STAGE_BYTES,
                                 full + s);
            issued = it + 1;
        }
        // copies still in flight for stages nobody will consume: wait (bounded)
        if (*(volatile int*)&abort_flag)
            for (int it = max(0, issued - S); it < issued; ++it) mbar_wait(full + it % S, (it / S) & 1);
        return;
    }

    // -------------------------------------------------------------- consumers
    const int tcx = threadIdx.x;
    for (int it = 0;; ++it) {
        const int s = it % S;
        if (!mbar_wait(full + s, (it / S) & 1)) {
            atomicOr(status, 2u);
            abort_flag = 1;
            return;
        }
        const int idx = item[s];
        if (idx < 0) {
            mbar_arrive(stored + it % Q);
            return;
        }
        int level, y, tile;
        pair_item(idx, Tn, a.ny, p.lag, level, y, tile);
        const T* stage = reinterpret_cast<const T*>(smem + s * G::STAGE_BYTES);
        T* dst = level ? static_cast<T*>(a.fout) : ring;
        tile_update<T, MODE, V, G::SEG, true, true>(a, c, stage, tcx * V, tile * G::W + tcx * V, y,
                                              empty + s, source(level), dst, level ? a.plane : p.ring_plane,
                                              level ? -1 : p.ring_rows - 1);
        mbar_arrive(stored + it % Q);
    }
}

template <class T, int MODE, int NC, int V, int S, int MB>
cudaError_t launch_pair_one(const SweepArgs& a, const PairArgs& p, cudaStream_t st, unsigned* status) {
    using G = Geometry<T, NC, V, S>;
    using PS = PairSmem<T, NC, V, S>;
    auto kern = sweep_pair_kernel<T, MODE, NC, V, S, MB>;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, PS::BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (p.tiles_per_row != (a.nx + G::W - 1) / G::W || p.grid <= 0 || p.lag < 1 || p.ring_rows <= p.lag + 1)
        return cudaErrorInvalidValue;
    // cooperative: every block resident at once (the schedule relies on it)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.grid);
    cfg.blockDim = dim3(NC + 64);
    cfg.dynamicSmemBytes = PS::BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, p, status);
}

template <class T, int MODE, int NC, int V, int S, int MB>
cudaError_t plan_pair_one(int nx, int* tiles_per_row, int* grid, int* lag) {
    using G = Geometry<T, NC, V, S>;
    using PS = PairSmem<T, NC, V, S>;
    auto kern = sweep_pair_kernel<T, MODE, NC, V, S, MB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, PS::BYTES);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NC + 64, PS::BYTES);
    if (e != cudaSuccess) return e;
    *tiles_per_row = (nx + G::W - 1) / G::W;
    *grid = max(1, per_sm) * sms;
    // 16 phases: the best of 8 .. 24 measured on GB300 for every tile shape at
    // 25601 x 256 (the items in flight span 9 to 18 phases there)
    *lag = min(kPairRingRows - 2, CLB_PAIR_LAG > 0 ? CLB_PAIR_LAG : 16);
    return cudaSuccess;
}

}  // namespace

// Tile shapes of the two-step sweep: (id, consumer threads, nodes per thread,
// stages, blocks per SM the registers are sized for, single-step TMA variant
// of the same shape for an odd last step).
#define CLB_PAIR_VARIANTS(X) \
    X(0, 512, 2, 3, 1, 12) X(1, 256, 4, 3, 2, 1) X(2, 512, 1, 4, 2, 9) X(3, 256, 2, 4, 2, 2) X(4, 128, 4, 4, 3, 0)

int pair_variant_count() { return 5; }

int pair_single_variant(int variant) {
#define CLB_PAIR_SINGLE(id, nc, v, s, mb, single) \
    case id:                                      \
        return single;
    switch (variant) { CLB_PAIR_VARIANTS(CLB_PAIR_SINGLE) }
#undef CLB_PAIR_SINGLE
    return -1;
}

template <class T>
static cudaError_t dispatch_pair(int mode, int variant, const SweepArgs* a, const PairArgs* p, cudaStream_t st,
                                 unsigned* status, int nx, int* tiles_per_row, int* grid, int* lag) {
#define CLB_PAIR_CASE(id, nc, v, s, mb, single)                                                        \
    case id:                                                                                          \
        if (!a)                                                                                       \
            return mode == MODE_PRESSURE ? plan_pair_one<T, MODE_PRESSURE, nc, v, s, mb>(nx, tiles_per_row, grid, lag) \
                                         : plan_pair_one<T, MODE_PERIODIC, nc, v, s, mb>(nx, tiles_per_row, grid, lag); \
        return mode == MODE_PRESSURE ? launch_pair_one<T, MODE_PRESSURE, nc, v, s, mb>(*a, *p, st, status)  \
                                     : launch_pair_one<T, MODE_PERIODIC, nc, v, s, mb>(*a, *p, st, status);
    switch (variant) { CLB_PAIR_VARIANTS(CLB_PAIR_CASE) }
#undef CLB_PAIR_CASE
    return cudaErrorInvalidValue;
}

static cudaError_t pair_any(int storage, int mode, int variant, const SweepArgs* a, const PairArgs* p,
                            cudaStream_t st, unsigned* status, int nx, int* tiles_per_row, int* grid, int* lag) {
    if (storage == 1) return dispatch_pair<float>(mode, variant, a, p, st, status, nx, tiles_per_row, grid, lag);
    if (storage == 2) return dispatch_pair<__half>(mode, variant, a, p, st, status, nx, tiles_per_row, grid, lag);
    if (storage == 3) return dispatch_pair<__nv_bfloat16>(mode, variant, a, p, st, status, nx, tiles_per_row, grid, lag);
    return cudaErrorInvalidValue;
}

cudaError_t plan_sweep_pair(int storage, int mode, int variant, int nx, int* tiles_per_row, int* grid, int* lag) {
    return pair_any(storage, mode, variant, nullptr, nullptr, nullptr, nullptr, nx, tiles_per_row, grid, lag);
}

cudaError_t launch_sweep_pair(int storage, int mode, int variant, const SweepArgs& a, const PairArgs& p,
                              cudaStream_t st, unsigned* status) {
    return pair_any(storage, mode, variant, &a, &p, st, status, 0, nullptr, nullptr, nullptr);
}

}  // namespace clb
