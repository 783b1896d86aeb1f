// Batched Knudsen sweep: many small periodic channels (Sec. 3.1, Fig. 2 of
// Liu & He, arXiv:1603.01955) advanced together by one persistent launch.
//
// Each channel (at most a few hundred nodes: Nx = 4 columns, Ny <= ~256 rows)
// lives for the whole launch in the shared memory of one thread block, which
// runs many time steps with only block barriers between them: gather the
// pulled populations into registers (Eq. 5, CBBSR walls Eq. 20, periodic x),
// barrier, collide (Eq. 4, 6-13 with the channel's own s_v, s_q from Eq. 18,
// 21) and write back in place, barrier.  Global memory is touched once at
// the start and once at the end of a launch.  The host replays a CUDA graph
// holding one such launch of a fixed number of steps.
//
// Schedule: each channel is updated by a warp-aligned range of a block's
// threads, each thread taking `npt` nodes (1, 2, 4 or 8).  Unpacked, every
// channel has a block of its own; packed, small channels share a block (each
// on its own thread range and shared-memory region, all behind the same block
// barriers), which cuts the blocks of a sweep with many small channels.  An
// autotuner times every feasible (npt, packed) pair on a copy of the state
// and keeps the fastest.  Every schedule computes the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/clb.h"
#include "clb_device.cuh"
#include "clb_internal.h"

using namespace clb;

namespace {

struct BatchChannel {
    int nx, ny;
    long long offset;  // element offset of the channel's [9][ny][nx] block
};

// Where a channel runs under a schedule: threads [t0, t0 + threads) of its
// block, its copy (copies) in the block's shared memory from element smem_off.
struct BatchSlot {
    int t0, threads, smem_off, block;
};

struct BatchArgs {
    void* state;
    const BatchChannel* ch;
    const KC<float>* kf;   // per-channel constants
    const KC<double>* kd;
};

// A schedule's device tables: per block, the first entry and the count of its
// channels in `order`; per channel, its slot.
struct SchedArgs {
    const int2* groups;
    const int* order;
    const BatchSlot* slots;
};

template <typename R> __device__ __forceinline__ const KC<R>* kcs(const BatchArgs& a);
template <> __device__ __forceinline__ const KC<float>* kcs<float>(const BatchArgs& a) { return a.kf; }
template <> __device__ __forceinline__ const KC<double>* kcs<double>(const BatchArgs& a) { return a.kd; }

// Pre-collision populations of node (x, y) of a channel held in shared memory
// as s[i][y][x], nx columns periodic, walls below row 0 and above row ny-1.
template <class R>
__device__ __forceinline__ void gather(const R* s, int nx, int ny, int x, int y, R r, R rc, R (&f)[9]) {
    const int nn = nx * ny;
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;
    auto at = [&](int i, int yy, int xx) -> R { return s[i * nn + yy * nx + xx]; };
    f[0] = at(0, y, x);
    f[1] = at(1, y, xm);
    f[3] = at(3, y, xp);
    if (y == 0) {  // Eq. 20
        f[2] = at(4, 0, x);
        f[5] = ln::fma(r, at(7, 0, x), ln::mul(rc, at(8, 0, xm)));
        f[6] = ln::fma(r, at(8, 0, x), ln::mul(rc, at(7, 0, xp)));
    } else {
        f[2] = at(2, y - 1, x);
        f[5] = at(5, y - 1, xm);
        f[6] = at(6, y - 1, xp);
    }
    if (y == ny - 1) {  // mirror of Eq. 20
        f[4] = at(2, y, x);
        f[7] = ln::fma(r, at(5, y, x), ln::mul(rc, at(6, y, xp)));
        f[8] = ln::fma(r, at(6, y, x), ln::mul(rc, at(5, y, xm)));
    } else {
        f[4] = at(4, y + 1, x);
        f[7] = at(7, y + 1, xp);
        f[8] = at(8, y + 1, xm);
    }
}

// two_buffers: the block holds two copies of its channel and alternates
// between them, one barrier per step; otherwise it updates one copy in place,
// with a barrier between the gather and the writes.
// Where node (x, y) pulls its populations from (as gather above), as offsets
// into the channel's [9][ny][nx] block, worked out once per launch: o[i] for
// population i; at the walls f5, f6 (bottom) and f7, f8 (top) also take a
// partner, wb / wt, with weight 1 - r.
struct Pull {
    int o[9];
    int wb[2], wt[2];
    bool bottom, top;
};

__device__ __forceinline__ Pull pull_of(int nx, int ny, int x, int y) {
    Pull p;
    const int nn = nx * ny;
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;
    auto at = [&](int i, int yy, int xx) { return i * nn + yy * nx + xx; };
    p.bottom = y == 0;
    p.top = y == ny - 1;
    p.o[0] = at(0, y, x);
    p.o[1] = at(1, y, xm);
    p.o[3] = at(3, y, xp);
    p.wb[0] = p.wb[1] = p.wt[0] = p.wt[1] = 0;
    if (p.bottom) {
        p.o[2] = at(4, 0, x);
        p.o[5] = at(7, 0, x);
        p.wb[0] = at(8, 0, xm);
        p.o[6] = at(8, 0, x);
        p.wb[1] = at(7, 0, xp);
    } else {
        p.o[2] = at(2, y - 1, x);
        p.o[5] = at(5, y - 1, xm);
        p.o[6] = at(6, y - 1, xp);
    }
    if (p.top) {
        p.o[4] = at(2, y, x);
        p.o[7] = at(5, y, x);
        p.wt[0] = at(6, y, xp);
        p.o[8] = at(6, y, x);
        p.wt[1] = at(5, y, xm);
    } else {
        p.o[4] = at(4, y + 1, x);
        p.o[7] = at(7, y + 1, xp);
        p.o[8] = at(8, y + 1, xm);
    }
    return p;
}

// gather() through precomputed offsets (the same loads and arithmetic).
template <class R>
__device__ __forceinline__ void gather_at(const R* s, const Pull& p, R r, R rc, R (&f)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = s[p.o[i]];
    if (p.bottom) {  // Eq. 20
        f[5] = ln::fma(r, f[5], ln::mul(rc, s[p.wb[0]]));
        f[6] = ln::fma(r, f[6], ln::mul(rc, s[p.wb[1]]));
    }
    if (p.top) {  // mirror of Eq. 20
        f[7] = ln::fma(r, f[7], ln::mul(rc, s[p.wt[0]]));
        f[8] = ln::fma(r, f[8], ln::mul(rc, s[p.wt[1]]));
    }
}

template <class T, int NPT>
__global__ void __launch_bounds__(512) batch_kernel(const BatchArgs a, const SchedArgs sc, int nsteps, int two_buffers) {
    using R = T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // this thread's channel: the block's channel whose thread range holds it
    // (none for the padding threads, which only take part in the barriers)
    const int2 gr = sc.groups[blockIdx.x];
    int k = -1;
    BatchSlot sl{0, 1, 0, 0};
    for (int j = 0; j < gr.y; ++j) {
        const int kk = sc.order[gr.x + j];
        const BatchSlot q = sc.slots[kk];
        if ((int)threadIdx.x >= q.t0 && (int)threadIdx.x < q.t0 + q.threads) {
            k = kk;
            sl = q;
        }
    }
    const bool mine = k >= 0;
    const BatchChannel ch = mine ? a.ch[k] : BatchChannel{1, 1, 0};
    KC<R> c{};
    if (mine) c = kcs<R>(a)[k];
    const int nx = ch.nx, ny = ch.ny, nn = nx * ny;
    const int lt = (int)threadIdx.x - sl.t0, nth = sl.threads;  // thread within the channel's range
    R* s = reinterpret_cast<R*>(smem_raw) + sl.smem_off;
    T* g = static_cast<T*>(a.state) + ch.offset;
    if (mine)
        for (int e = lt; e < 9 * nn; e += nth) s[e] = g[e];
    const R r = c.r, rc = c.rc, ref = c.ref0;
    __syncthreads();
    R* out = two_buffers ? s + 9 * nn : s;
    // with few nodes per thread, the pull offsets are worked out once
    constexpr bool kPre = NPT <= 2;
    Pull pl[kPre ? NPT : 1];
    if constexpr (kPre) {
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            const int node = lt + q * nth;
            pl[q] = pull_of(nx, ny, node % nx, node / nx);
        }
    }
    for (int t = 0; t < nsteps; ++t) {
        R f[NPT][9];
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            const int node = lt + q * nth;
            if (mine && node < nn) {
                if constexpr (kPre)
                    gather_at(s, pl[q], r, rc, f[q]);
                else
                    gather(s, nx, ny, node % nx, node / nx, r, rc, f[q]);
            }
        }
        if (!two_buffers) __syncthreads();
        if (mine) {
            if constexpr (std::is_same<R, float>::value && NPT % 2 == 0) {
                // two nodes per packed FP32 instruction (bit for bit the one-node collision)
#pragma unroll
                for (int q = 0; q < NPT; q += 2) {
                    const int n0 = lt + q * nth, n1 = n0 + nth;
                    if (n1 < nn) {
                        float2 d[9];
#pragma unroll
                        for (int i = 0; i < 9; ++i) d[i] = make_float2(f[q][i], f[q + 1][i]);
                        collide<R, MODE_PERIODIC, float2>(d, ln::bc<float2>(ref), c);
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            out[i * nn + n0] = d[i].x;
                            out[i * nn + n1] = d[i].y;
                        }
                    } else if (n0 < nn) {
                        collide<R, MODE_PERIODIC>(f[q], ref, c);
#pragma unroll
                        for (int i = 0; i < 9; ++i) out[i * nn + n0] = f[q][i];
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < NPT; ++q) {
                    const int node = lt + q * nth;
                    if (node < nn) {
                        collide<R, MODE_PERIODIC>(f[q], ref, c);
#pragma unroll
                        for (int i = 0; i < 9; ++i) out[i * nn + node] = f[q][i];
                    }
                }
            }
        }
        __syncthreads();
        if (two_buffers) {
            R* t2 = s;
            s = out;
            out = t2;
        }
    }
    if (mine)
        for (int e = lt; e < 9 * nn; e += nth) g[e] = s[e];
}

// Per channel: mass flow (mean over x of sum_y rho u_x), sum of u_x (for Q),
// total mass, a non-finite count, and u_x in the first two and last two rows
// of column 0 (slip).  One block of kObsThreads per channel; FP64 sums in a
// fixed order.
constexpr int kObsThreads = 256;

template <class T>
__global__ void __launch_bounds__(kObsThreads) batch_obs_kernel(const BatchArgs a, double ref0, double gx, double* out) {
    __shared__ double sh[4][kObsThreads];
    const BatchChannel ch = a.ch[blockIdx.x];
    const int nx = ch.nx, ny = ch.ny, nn = nx * ny;
    const T* g = static_cast<const T*>(a.state) + ch.offset;
    double v[4] = {0, 0, 0, 0};
    double* o = out + 9 * blockIdx.x;
    for (int node = threadIdx.x; node < nn; node += kObsThreads) {
        double drho = 0, jx = 0;
        for (int i = 0; i < 9; ++i) {
            const double f = (double)g[i * nn + node];
            drho += f;
            jx += (i == 1 || i == 5 || i == 8) ? f : (i == 3 || i == 6 || i == 7) ? -f : 0.0;
        }
        const double rho = ref0 + drho;
        const double ux = (jx - 0.5 * rho * gx) / rho;  // Eq. 13 from the post-collision state
        if (!isfinite(rho) || !isfinite(ux)) v[3] += 1;
        v[0] += rho * ux;
        v[1] += ux;
        v[2] += rho;
        const int x = node % nx, y = node / nx;
        if (x == 0) {
            if (y == 0) o[4] = ux;
            if (y == 1) o[5] = ux;
            if (y == ny - 2) o[6] = ux;
            if (y == ny - 1) o[7] = ux;
        }
    }
    for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int w = kObsThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) o[k] = sh[k][0];
}

template <class T>
__global__ void batch_canon_kernel(void* state, long long offset, long long n, double* buf, double ref0,
                                   int to_canonical, int nn) {
    // w_i by direction i = idx / nn
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    T* g = static_cast<T*>(state) + offset;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const double wr = w[idx / nn] * ref0;
        if (to_canonical)
            buf[idx] = wr + (double)g[idx];
        else
            g[idx] = T(buf[idx] - wr);
    }
}

}  // namespace

// A schedule (see the file comment) with its device tables.
struct BatchSched {
    int npt = 0, packed = 0;
    int block = 0;        // threads per block
    int nblocks = 0;
    int two_buffers = 0;  // every channel keeps two copies in shared memory
    size_t smem = 0;      // bytes of shared memory per block (the largest group)
    void* mem = nullptr;  // one device allocation: groups, order, slots
    SchedArgs args{};
};

struct clb_batch {
    int n = 0, storage = 0, block_x = 0;
    bool tuned = false;
    size_t elem = 0;
    long long total = 0;  // elements of the state
    int max_nodes = 0;
    BatchSched sched;     // the schedule in use
    std::vector<BatchChannel> hch;
    std::vector<double> kn;
    std::vector<int> nx, ny;
    void* state = nullptr;
    BatchChannel* dch = nullptr;
    KC<float>* dkf = nullptr;
    KC<double>* dkd = nullptr;
    double* dobs = nullptr;
    double g = 0, ref0 = 0, rho0 = 1, r = 0;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    void* (*alloc)(size_t, void*) = nullptr;
    void (*dealloc)(void*, void*) = nullptr;
    void* alloc_ctx = nullptr;

    void* dalloc(size_t bytes) {
        if (alloc) return alloc(bytes ? bytes : 256, alloc_ctx);
        void* p = nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 256) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void dfree(void* p) {
        if (!p) return;
        if (dealloc)
            dealloc(p, alloc_ctx);
        else
            cudaFree(p);
    }
};

namespace {

constexpr int kGraphSteps = 500;  // time steps per persistent launch in the replayed graph
constexpr size_t kSmemCap = 200 * 1024;  // shared memory a block may take
constexpr int kPackedBlock = 256;        // threads per block of a packed schedule

void free_sched(clb_batch* b, BatchSched& sc) {
    b->dfree(sc.mem);
    sc = BatchSched{};
}

// Build schedule (npt, packed): per channel ceil(nodes / npt) threads rounded
// up to whole warps; unpacked, one channel per block, blocks as wide as the
// widest channel; packed, blocks of kPackedBlock threads (or the widest
// channel, if wider), filled first-fit with the channels by decreasing width,
// each block within kSmemCap bytes.  Two copies per
// channel when every block's channels still fit.  Returns false (no device
// work) if the schedule is not feasible.
bool plan_sched(const clb_batch* b, int npt, int packed, int block_min, BatchSched& sc, std::vector<int2>& groups,
                std::vector<int>& order, std::vector<BatchSlot>& slots) {
    const int n = b->n;
    std::vector<int> width(n);
    int block = block_min, total = 0;
    for (int k = 0; k < n; ++k) {
        const int nodes = b->nx[k] * b->ny[k];
        width[k] = ((nodes + npt - 1) / npt + 31) / 32 * 32;
        block = std::max(block, width[k]);
        total += width[k];
    }
    if (block > 512) return false;
    if (packed) block = std::max(block, std::min(kPackedBlock, total));
    const size_t one = 9 * b->elem;  // bytes per node and copy
    int two = 2 * one * b->max_nodes <= kSmemCap;
    std::vector<int> idx(n);
    for (int k = 0; k < n; ++k) idx[k] = k;
    if (packed) std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return width[x] > width[y]; });
    for (;;) {
        groups.clear();
        order.clear();
        slots.assign(n, BatchSlot{0, 0, 0, 0});
        std::vector<int> used_t, used_m;  // per block: threads and shared-memory elements taken
        std::vector<std::vector<int>> members;
        for (int k : idx) {
            const int elems = ((two ? 2 : 1) * 9 * b->nx[k] * b->ny[k] + 3) / 4 * 4;  // 16-byte aligned regions
            int blk = -1;
            if (packed)
                for (size_t j = 0; j < used_t.size() && blk < 0; ++j)
                    if (used_t[j] + width[k] <= block && (used_m[j] + elems) * b->elem <= kSmemCap) blk = (int)j;
            if (blk < 0) {
                blk = (int)used_t.size();
                used_t.push_back(0);
                used_m.push_back(0);
                members.emplace_back();
            }
            slots[k] = BatchSlot{used_t[blk], width[k], used_m[blk], blk};
            used_t[blk] += width[k];
            used_m[blk] += elems;
            members[blk].push_back(k);
        }
        size_t smem = 0;
        for (size_t j = 0; j < members.size(); ++j) {
            groups.push_back(make_int2((int)order.size(), (int)members[j].size()));
            for (int k : members[j]) order.push_back(k);
            smem = std::max(smem, used_m[j] * b->elem);
        }
        if (smem > kSmemCap) {
            if (!two) return false;
            two = 0;  // retry with one copy per channel
            continue;
        }
        sc.npt = npt;
        sc.packed = packed;
        sc.block = block;
        sc.nblocks = (int)groups.size();
        sc.two_buffers = two;
        sc.smem = std::max<size_t>(smem, 16);
        return true;
    }
}

template <class T> cudaError_t set_smem_limit(size_t bytes) {
    cudaError_t e = cudaSuccess;
    const void* ks[] = {(const void*)batch_kernel<T, 1>, (const void*)batch_kernel<T, 2>,
                        (const void*)batch_kernel<T, 4>, (const void*)batch_kernel<T, 8>};
    for (const void* k : ks) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) break;
    }
    return e;
}

// Plan and upload schedule (npt, packed); CLB_EINVAL if it is not feasible.
clb_status make_sched(clb_batch* b, int npt, int packed, int block_min, BatchSched& sc) {
    std::vector<int2> groups;
    std::vector<int> order;
    std::vector<BatchSlot> slots;
    BatchSched t;
    if (!plan_sched(b, npt, packed, block_min, t, groups, order, slots))
        return (clb_status)set_error(CLB_EINVAL, "clb_batch: schedule (%d nodes per thread, packed %d) does not fit",
                                     npt, packed);
    const size_t bg = groups.size() * sizeof(int2), bo = order.size() * sizeof(int), bs = slots.size() * sizeof(BatchSlot);
    const size_t og = 0, oo = (bg + 15) / 16 * 16, os = oo + (bo + 15) / 16 * 16;
    t.mem = b->dalloc(os + bs);
    if (!t.mem) return (clb_status)set_error(CLB_ENOMEM, "clb_batch: device allocation of a schedule failed");
    char* m = static_cast<char*>(t.mem);
    cudaError_t e = cudaMemcpyAsync(m + og, groups.data(), bg, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m + oo, order.data(), bo, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m + os, slots.data(), bs, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = b->storage == CLB_FP64 ? set_smem_limit<double>(t.smem) : set_smem_limit<float>(t.smem);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // the host vectors go out of scope
    if (e != cudaSuccess) {
        b->dfree(t.mem);
        return (clb_status)set_error(CLB_ECUDA, "clb_batch: schedule upload: %s", cudaGetErrorString(e));
    }
    t.args = SchedArgs{reinterpret_cast<const int2*>(m + og), reinterpret_cast<const int*>(m + oo),
                       reinterpret_cast<const BatchSlot*>(m + os)};
    sc = t;
    return CLB_OK;
}

template <class T>
cudaError_t launch_batch(clb_batch* b, const BatchSched& sc, void* state, int nsteps, cudaStream_t st) {
    BatchArgs a{state, b->dch, b->dkf, b->dkd};
    dim3 grid(sc.nblocks), blk(sc.block);
    switch (sc.npt) {
        case 1: batch_kernel<T, 1><<<grid, blk, sc.smem, st>>>(a, sc.args, nsteps, sc.two_buffers); break;
        case 2: batch_kernel<T, 2><<<grid, blk, sc.smem, st>>>(a, sc.args, nsteps, sc.two_buffers); break;
        case 4: batch_kernel<T, 4><<<grid, blk, sc.smem, st>>>(a, sc.args, nsteps, sc.two_buffers); break;
        case 8: batch_kernel<T, 8><<<grid, blk, sc.smem, st>>>(a, sc.args, nsteps, sc.two_buffers); break;
        default: return cudaErrorInvalidConfiguration;
    }
    return cudaGetLastError();
}

cudaError_t launch(clb_batch* b, const BatchSched& sc, void* state, int nsteps, cudaStream_t st) {
    return b->storage == CLB_FP64 ? launch_batch<double>(b, sc, state, nsteps, st)
                                  : launch_batch<float>(b, sc, state, nsteps, st);
}

void drop_graph(clb_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

clb_status build_graph(clb_batch* b) {
    drop_graph(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = launch(b, b->sched, b->state, kGraphSteps, b->stream);
        e = cudaStreamEndCapture(b->stream, &g);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return (clb_status)set_error(CLB_ECUDA, "clb_batch: graph capture: %s", cudaGetErrorString(e));
    }
    b->graph_steps = kGraphSteps;
    return CLB_OK;
}

// Make `sc` the schedule in use (the old one is released, the graph rebuilt on demand).
void adopt_sched(clb_batch* b, BatchSched& sc) {
    drop_graph(b);
    free_sched(b, b->sched);
    b->sched = sc;
    sc = BatchSched{};
    b->block_x = b->sched.block;
}

}  // namespace

extern "C" {

clb_status clb_batch_destroy(clb_batch* b) {
    if (!b) return CLB_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    free_sched(b, b->sched);
    b->dfree(b->state);
    b->dfree(b->dch);
    b->dfree(b->dkf);
    b->dfree(b->dkd);
    b->dfree(b->dobs);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return CLB_OK;
}

clb_status clb_batch_create(int n, const int* nx, const int* ny, const double* kn, double a, double r, double g,
                            const clb_opts* opts, clb_batch** out) {
    if (!out) return (clb_status)set_error(CLB_EINVAL, "clb_batch_create: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 65535 || !nx || !ny || !kn)
        return (clb_status)set_error(CLB_EINVAL, "clb_batch_create: need 1..65535 channels and their sizes");
    clb_opts o;
    clb_opts_default(&o);
    if (opts) o = *opts;
    if (o.storage != CLB_FP64 && o.storage != CLB_FP32_SHIFTED)
        return (clb_status)set_error(CLB_EINVAL, "clb_batch_create: storage must be FP64 or FP32-shifted");
    if (!(a >= 0) || !std::isfinite(g) || !std::isfinite(r) || r > 1 || !(o.rho_out > 0))
        return (clb_status)set_error(CLB_EINVAL, "clb_batch_create: a, r, g or rho_out out of range");
    if ((o.alloc == nullptr) != (o.free == nullptr))
        return (clb_status)set_error(CLB_EINVAL, "clb_batch_create: alloc and free hooks must be given together");
    const size_t elem = o.storage == CLB_FP64 ? 8 : 4;
    int max_nodes = 0;
    for (int k = 0; k < n; ++k) {
        // a block holds a whole channel (at most 8 x 512 nodes), so larger
        // sides are rejected here, before their product can overflow
        if (nx[k] < 1 || ny[k] < 1 || nx[k] > 8 * 512 || ny[k] > 8 * 512 || !(kn[k] > 0) || !std::isfinite(kn[k]))
            return (clb_status)set_error(CLB_EINVAL, "clb_batch_create: channel %d: bad nx, ny or Kn", k);
        max_nodes = std::max(max_nodes, nx[k] * ny[k]);
    }
    const size_t smem = (size_t)9 * max_nodes * elem;
    if (smem > 200 * 1024 || max_nodes > 8 * 512)
        return (clb_status)set_error(CLB_EINVAL,
                                     "clb_batch_create: the largest channel (%d nodes) does not fit one block's "
                                     "shared memory",
                                     max_nodes);
    if (o.block_x && (o.block_x < 32 || o.block_x > 512 || o.block_x % 32))
        return (clb_status)set_error(CLB_EINVAL, "clb_batch_create: block_x must be a multiple of 32 in 32..512");

    clb_batch* b = new (std::nothrow) clb_batch;
    if (!b) return (clb_status)set_error(CLB_ENOMEM, "clb_batch_create: host allocation failed");
    b->n = n;
    b->storage = o.storage;
    b->elem = elem;
    b->max_nodes = max_nodes;
    b->alloc = o.alloc;
    b->dealloc = o.free;
    b->alloc_ctx = o.alloc_ctx;
    b->g = g;
    b->rho0 = o.rho_out;
    b->ref0 = o.storage == CLB_FP64 ? 0.0 : o.rho_out;
    b->r = r >= 0 ? r : r_from_sigma(o.sigma);
    b->tuned = o.block_x != 0;
    long long off = 0;
    std::vector<KC<float>> kf(n);
    std::vector<KC<double>> kd(n);
    for (int k = 0; k < n; ++k) {
        b->nx.push_back(nx[k]);
        b->ny.push_back(ny[k]);
        b->kn.push_back(kn[k]);
        BatchChannel c{nx[k], ny[k], off};
        b->hch.push_back(c);
        off += ((9LL * nx[k] * ny[k] + 3) / 4) * 4;  // 16-byte aligned blocks
        SweepArgs sa{};
        sa.s3 = o.s3;
        sa.s8 = o.s8;
        rates_at(kn[k], ny[k], a, o.b2, &sa.sv, &sa.sq);
        sa.rate_A = 1.0;  // unused in the body-force collision
        sa.r = b->r;
        sa.gx = g;
        sa.ref0 = b->ref0;
        sa.store_scale = 1.0;
        derive_constants(sa);
        kf[k] = sa.kf;
        kd[k] = sa.kd;
    }
    b->total = off;
    if (o.stream) {
        b->stream = static_cast<cudaStream_t>(o.stream);
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
        b->own_stream = true;
    } else {
        cudaError_t e = cudaGetLastError();
        delete b;
        return (clb_status)set_error(CLB_ECUDA, "clb_batch_create: stream: %s", cudaGetErrorString(e));
    }
    b->state = b->dalloc(b->total * elem);
    b->dch = static_cast<BatchChannel*>(b->dalloc(n * sizeof(BatchChannel)));
    b->dkf = static_cast<KC<float>*>(b->dalloc(n * sizeof(KC<float>)));
    b->dkd = static_cast<KC<double>*>(b->dalloc(n * sizeof(KC<double>)));
    b->dobs = static_cast<double*>(b->dalloc(9 * (size_t)n * sizeof(double)));
    if (!b->state || !b->dch || !b->dkf || !b->dkd || !b->dobs) {
        clb_batch_destroy(b);
        return (clb_status)set_error(CLB_ENOMEM, "clb_batch_create: device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(b->dch, b->hch.data(), n * sizeof(BatchChannel), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->dkf, kf.data(), n * sizeof(KC<float>), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->dkd, kd.data(), n * sizeof(KC<double>), cudaMemcpyHostToDevice, b->stream);
    // initial state f^eq(rho_out, 0) = w_i rho_out: zero deviations (FP32) or w_i rho_out (FP64)
    if (e == cudaSuccess) e = cudaMemsetAsync(b->state, 0, b->total * elem, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        clb_batch_destroy(b);
        return (clb_status)set_error(CLB_ECUDA, "clb_batch_create: %s", cudaGetErrorString(e));
    }
    {
        // first schedule: opts.block_x threads per block, one channel per
        // block (fixed); or one node per thread where that fits (tuned on
        // first use)
        const int want = o.block_x ? o.block_x : 512;
        int npt = 1;
        while (npt < 8 && (max_nodes + npt - 1) / npt > want) npt *= 2;
        BatchSched sc;
        clb_status st = make_sched(b, npt, 0, o.block_x, sc);
        if (st != CLB_OK) {
            clb_batch_destroy(b);
            return st;
        }
        adopt_sched(b, sc);
    }
    if (b->storage == CLB_FP64) {
        const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
        for (int k = 0; k < n; ++k) {
            const int nn = nx[k] * ny[k];
            std::vector<double> f((size_t)9 * nn);
            for (int i = 0; i < 9; ++i)
                for (int j = 0; j < nn; ++j) f[(size_t)i * nn + j] = w[i] * o.rho_out;
            e = cudaMemcpy(static_cast<double*>(b->state) + b->hch[k].offset, f.data(), f.size() * sizeof(double),
                           cudaMemcpyHostToDevice);
            if (e != cudaSuccess) break;
        }
        if (e != cudaSuccess) {
            clb_batch_destroy(b);
            return (clb_status)set_error(CLB_ECUDA, "clb_batch_create: init: %s", cudaGetErrorString(e));
        }
    }
    *out = b;
    return CLB_OK;
}

clb_status clb_batch_tune(clb_batch* b, int* block_out) {
    if (!b) return (clb_status)set_error(CLB_EINVAL, "clb_batch_tune: batch is NULL");
    // time every feasible schedule on a scratch copy of the state (results do
    // not depend on the schedule, only the speed does)
    void* scratch = b->dalloc(b->total * b->elem);
    if (!scratch) return (clb_status)set_error(CLB_ENOMEM, "clb_batch_tune: device allocation failed");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    BatchSched best_sc;
    cudaError_t err = cudaSuccess;
    clb_status st = CLB_OK;
    const int trial_steps = 200;
    int unpacked_blocks = 0;
    for (int npt = 1; npt <= 8 && err == cudaSuccess && st == CLB_OK; npt *= 2) {
        for (int packed = 0; packed <= 1 && err == cudaSuccess; ++packed) {
            BatchSched sc;
            if (make_sched(b, npt, packed, 0, sc) != CLB_OK) {
                set_error(CLB_OK, "%s", "");  // an infeasible schedule is not an error of the tuner
                if (!packed) unpacked_blocks = -1;
                continue;
            }
            if (!packed) unpacked_blocks = sc.nblocks;
            if (packed && sc.nblocks == unpacked_blocks) {  // nothing was packed: the same schedule
                free_sched(b, sc);
                continue;
            }
            err = cudaMemcpyAsync(scratch, b->state, b->total * b->elem, cudaMemcpyDeviceToDevice, b->stream);
            if (err == cudaSuccess) err = launch(b, sc, scratch, 20, b->stream);  // warm-up
            if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
            if (err == cudaSuccess) err = launch(b, sc, scratch, trial_steps, b->stream);
            if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && ms < best) {
                best = ms;
                free_sched(b, best_sc);
                best_sc = sc;
            } else {
                free_sched(b, sc);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(b->stream);
    b->dfree(scratch);
    if (err != cudaSuccess || !best_sc.mem) {
        free_sched(b, best_sc);
        return (clb_status)set_error(CLB_ECUDA, "clb_batch_tune: %s",
                                     err != cudaSuccess ? cudaGetErrorString(err) : "no schedule fits");
    }
    adopt_sched(b, best_sc);
    b->tuned = true;
    if (block_out) *block_out = b->block_x;
    return CLB_OK;
}

clb_status clb_batch_set_schedule(clb_batch* b, int nodes_per_thread, int packed) {
    if (!b) return (clb_status)set_error(CLB_EINVAL, "clb_batch_set_schedule: batch is NULL");
    if (nodes_per_thread != 1 && nodes_per_thread != 2 && nodes_per_thread != 4 && nodes_per_thread != 8)
        return (clb_status)set_error(CLB_EINVAL, "clb_batch_set_schedule: nodes per thread must be 1, 2, 4 or 8");
    cudaStreamSynchronize(b->stream);  // the old tables may be in use by queued launches
    BatchSched sc;
    clb_status st = make_sched(b, nodes_per_thread, packed ? 1 : 0, 0, sc);
    if (st != CLB_OK) return st;
    adopt_sched(b, sc);
    b->tuned = true;
    return CLB_OK;
}

clb_status clb_batch_schedule(const clb_batch* b, int* threads_per_block, int* nodes_per_thread, int* blocks,
                              int* packed) {
    if (!b) return (clb_status)set_error(CLB_EINVAL, "clb_batch_schedule: batch is NULL");
    if (threads_per_block) *threads_per_block = b->sched.block;
    if (nodes_per_thread) *nodes_per_thread = b->sched.npt;
    if (blocks) *blocks = b->sched.nblocks;
    if (packed) *packed = b->sched.packed;
    return CLB_OK;
}

clb_status clb_batch_step(clb_batch* b, int64_t n) {
    clb::TraceRange trace_("clb_batch_step");
    if (!b || n < 0) return (clb_status)set_error(CLB_EINVAL, "clb_batch_step: bad arguments");
    if (!b->tuned) {
        clb_status st = clb_batch_tune(b, nullptr);
        if (st != CLB_OK) return st;
    }
    if (n >= kGraphSteps && !b->graph) {
        clb_status st = build_graph(b);
        if (st != CLB_OK) return st;
    }
    int64_t left = n;
    while (left >= kGraphSteps) {
        cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
        if (e != cudaSuccess) return (clb_status)set_error(CLB_ECUDA, "clb_batch_step: graph: %s", cudaGetErrorString(e));
        left -= kGraphSteps;
    }
    if (left > 0) {
        cudaError_t e = launch(b, b->sched, b->state, (int)left, b->stream);
        if (e != cudaSuccess) return (clb_status)set_error(CLB_ECUDA, "clb_batch_step: %s", cudaGetErrorString(e));
    }
    b->step += n;
    return CLB_OK;
}

clb_status clb_batch_observables(clb_batch* b, clb_scalars* s) {
    if (!b || !s) return (clb_status)set_error(CLB_EINVAL, "clb_batch_observables: NULL argument");
    BatchArgs a{b->state, b->dch, b->dkf, b->dkd};
    if (b->storage == CLB_FP64)
        batch_obs_kernel<double><<<b->n, kObsThreads, 0, b->stream>>>(a, b->ref0, b->g, b->dobs);
    else
        batch_obs_kernel<float><<<b->n, kObsThreads, 0, b->stream>>>(a, b->ref0, b->g, b->dobs);
    std::vector<double> h(9 * (size_t)b->n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), b->dobs, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return (clb_status)set_error(CLB_ECUDA, "clb_batch_observables: %s", cudaGetErrorString(e));
    int bad = 0;
    for (int k = 0; k < b->n; ++k) {
        const double* o = h.data() + 9 * k;
        const int ny = b->ny[k], nx = b->nx[k];
        clb_scalars& sc = s[k];
        sc.mass_flow = o[0] / nx;
        // Q of Sec. 3.1: sum_y u_x / (3 G ny^2 sqrt(1/6)), averaged over the columns
        sc.q_norm = b->g != 0 ? (o[1] / nx) / (3.0 * b->g * (double)ny * ny * std::sqrt(1.0 / 6.0)) : 0.0;
        sc.u_slip = ny >= 2 ? 0.5 * ((1.5 * o[4] - 0.5 * o[5]) + (1.5 * o[7] - 0.5 * o[6])) : o[4];
        sc.residual = -1.0;
        sc.total_mass = o[2];
        sc.ux_max = 0.0;
        sc.step = b->step;
        bad += o[3] > 0;
    }
    if (bad) return (clb_status)set_error(CLB_ENUMERIC, "clb_batch_observables: %d channels hold NaN/Inf", bad);
    return CLB_OK;
}

static clb_status batch_copy(clb_batch* b, int k, double* host, int to_host) {
    if (!b || !host || k < 0 || k >= b->n) return (clb_status)set_error(CLB_EINVAL, "clb_batch state: bad arguments");
    const int nn = b->nx[k] * b->ny[k];
    const long long n = 9LL * nn;
    double* tmp = static_cast<double*>(b->dalloc(n * sizeof(double)));
    if (!tmp) return (clb_status)set_error(CLB_ENOMEM, "clb_batch state: device allocation failed");
    cudaError_t e = cudaSuccess;
    if (!to_host) e = cudaMemcpyAsync(tmp, host, n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
        if (b->storage == CLB_FP64)
            batch_canon_kernel<double><<<64, 256, 0, b->stream>>>(b->state, b->hch[k].offset, n, tmp, b->ref0, to_host,
                                                                 nn);
        else
            batch_canon_kernel<float><<<64, 256, 0, b->stream>>>(b->state, b->hch[k].offset, n, tmp, b->ref0, to_host,
                                                                nn);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && to_host) e = cudaMemcpyAsync(host, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    b->dfree(tmp);
    if (e != cudaSuccess) return (clb_status)set_error(CLB_ECUDA, "clb_batch state: %s", cudaGetErrorString(e));
    return CLB_OK;
}

clb_status clb_batch_get_state(clb_batch* b, int k, double* host_f) { return batch_copy(b, k, host_f, 1); }

clb_status clb_batch_set_state(clb_batch* b, int k, const double* host_f) {
    return batch_copy(b, k, const_cast<double*>(host_f), 0);
}

clb_status clb_batch_info(const clb_batch* b, int* block_x, int64_t* step, void** stream) {
    if (!b) return (clb_status)set_error(CLB_EINVAL, "clb_batch_info: batch is NULL");
    if (block_x) *block_x = b->block_x;
    if (step) *step = b->step;
    if (stream) *stream = b->stream;
    return CLB_OK;
}

}  // extern "C"
