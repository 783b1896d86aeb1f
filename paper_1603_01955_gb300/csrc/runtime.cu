// Host runtime and C ABI (include/clb.h) of the CLB channel library, plus the
// small kernels around the sweep: initial equilibrium, state conversion, and
// the FP64 observable reductions (Sec. 3.1, 3.2 of Liu & He, arXiv:1603.01955).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/clb.h"
#include "clb_device.cuh"
#include "clb_internal.h"

using namespace clb;

namespace {

thread_local char g_err[512] = "";

clb_status fail(clb_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

#define CUDA_OR(expr)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) return fail(CLB_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

constexpr double kPi = 3.14159265358979323846;

// D2Q9 rest weights (Eq. 11 at u = 0) and directions (Eq. 1), host copies.
__constant__ double c_w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
__constant__ int c_ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};

// Observable scratch layout (doubles): per-column m(x), centre rho(x), column
// sums of u_x, profile u_x(y), u_y(y), then per-block partial sums.
struct ObsLayout {
    size_t m, rc, prof_x, prof_y, part, total;
    int nblocks;
};

constexpr int kObsCols = 32;  // columns per observable block
constexpr int kObsRows = 8;   // row groups per observable block
constexpr int kObsBatch = 4;  // rows a thread loads before reducing them

ObsLayout obs_layout(int nx, int ny) {
    ObsLayout L;
    L.nblocks = (nx + kObsCols - 1) / kObsCols;
    L.m = 0;
    L.rc = L.m + nx;
    L.prof_x = L.rc + nx;
    L.prof_y = L.prof_x + ny;
    L.part = L.prof_y + ny;
    L.total = L.part + 4 * (size_t)L.nblocks;
    return L;
}

}  // namespace

struct clb_sim {
    int nx = 0, ny = 0, pitch = 0, xoff = 0, storage = 0, vec = 0, block_x = 0, drive = 0;
    size_t elem = 0;        // bytes per stored element
    long long plane = 0;    // elements per plane
    size_t buf_bytes = 0;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;            // buffer holding the last completed step
    double* obs = nullptr;  // device scratch of the observable reductions: L.total doubles, a
                            // spare slot, the reduction's block counter
    double* hobs = nullptr; // pinned host copy of the first L.total + 1; slot L.total + 1 holds
                            // the status word read by check_status
    unsigned* status = nullptr;  // error bits of bounded device waits
    unsigned* sched = nullptr;   // TMA sweep: tile claim counters (2), zero between launches
    int pipeline = 1;       // 1 direct loads, 2.. TMA-staged tile shapes
    int withhold_tile = -1; // testing: TMA tile withheld in the first launch
    int graph_steps = 0;    // sweeps per replayed CUDA graph (0: no replay); even
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // per parity of `cur` at the chunk start
    int kn_mode = 0;        // 1: centreline Knudsen number (pressure channel)
    void* rc = nullptr;     // centreline densities: [2 sides][2 rows][rc_stride], compute type
    int rc_stride = 0;
    int yc0 = 0, yc1 = 0;   // centre rows
    ObsLayout L{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* (*alloc)(size_t, void*) = nullptr;
    void (*dealloc)(void*, void*) = nullptr;
    void* alloc_ctx = nullptr;
    // problem statement
    double kn = 0, a = 0, r = 0, b2 = 0, sigma = 1, s3 = 0, s8 = 0, g = 0, rho_in = 1, rho_out = 1;
    double sv = 0, sq = 0;
    double ref0 = 0, ref_slope = 0;
    double store_scale = 1;  // 16-bit formats: stored value = deviation * store_scale
    double drive_value = 0;  // as given to clb_create (G, or p_in/p_out)
    int64_t step = 0;
    bool have_prev = false;
    double prev_mass_flow = 0;

    void* dalloc(size_t bytes) {
        if (bytes == 0) bytes = 256;
        if (alloc) return alloc(bytes, alloc_ctx);
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
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
    double ref_at(int x) const { return ref0 + ref_slope * (double)x; }
};

// ------------------------------------------------------------------ kernels

namespace {

template <class T> using RT = typename Codec<T>::R;

template <class T>
__global__ void init_kernel(T* f, int nx, int ny, int pitch, int xoff, long long plane, double rho_a,
                            double rho_slope, double ref0, double ref_slope, int periodic, double sc) {
    const long long n = 9LL * ny * nx;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % nx);
        const int y = (int)((idx / nx) % ny);
        const int i = (int)(idx / ((long long)nx * ny));
        // f^eq(rho_init(x), u = 0) = w_i rho_init(x) (Eq. 11), stored as a deviation from w_i R(x)
        const T v = Codec<T>::enc(RT<T>(c_w[i] * ((rho_a + rho_slope * x) - (ref0 + ref_slope * x))), RT<T>(sc));
        T* row = f + i * plane + (long long)y * pitch + xoff;
        row[x] = v;
        if (periodic) {
            if (x == 0 && c_ex[i] < 0) row[nx] = v;
            if (x == nx - 1 && c_ex[i] > 0) row[-1] = v;
        }
    }
}

// Position (row = i ny + y, column x) of flat index idx = row nx + x, moved
// along by a fixed stride without a 64-bit division per element.
struct FlatWalk {
    long long idx, stride;
    int row, x, dq, dr, nx;
    __device__ FlatWalk(long long start, long long step, int nx_) : idx(start), stride(step), nx(nx_) {
        row = (int)(start / nx_);
        x = (int)(start - (long long)row * nx_);
        dq = (int)(step / nx_);
        dr = (int)(step - (long long)dq * nx_);
    }
    __device__ void next() {
        idx += stride;
        row += dq;
        x += dr;
        if (x >= nx) {
            x -= nx;
            ++row;
        }
    }
};

// The canonical FP64 array [9][ny][nx] <-> the stored state, in two walks:
// - flat (Flat = true): a grid-stride walk over the FP64 array in its memory
//   order, consecutive threads on consecutive elements, for `out` / `in` in
//   host memory the device reaches directly (pinned, mapped): swept from
//   start to end the host link runs near its ceiling (~209 GB/s into the
//   device here, against ~193 GB/s row by row);
// - row by row (one row (i, y) per step of blockIdx.y, columns across
//   threads), for device buffers, where it is the faster of the two
//   (0.45 against 0.68 ms for 25601 x 256 FP64 values).
template <class T>
__device__ __forceinline__ void to_canonical_one(const T* f, double* out, long long idx, int i, int y, int x, int pitch,
                                                 int xoff, long long plane, double ref0, double ref_slope, double isc) {
    const T* src = f + i * plane + (long long)y * pitch + xoff;
    out[idx] = fma(c_w[i] * ref_slope, (double)x, c_w[i] * ref0) + (double)Codec<T>::dec(src[x], RT<T>(isc));
}

template <class T>
__device__ __forceinline__ void from_canonical_one(const double* in, T* f, long long idx, int i, int y, int x, int nx,
                                                   int pitch, int xoff, long long plane, double ref0, double ref_slope,
                                                   int periodic, double sc) {
    T* dst = f + i * plane + (long long)y * pitch + xoff;
    const T v = Codec<T>::enc(RT<T>(in[idx] - fma(c_w[i] * ref_slope, (double)x, c_w[i] * ref0)), RT<T>(sc));
    dst[x] = v;
    if (periodic) {
        if (x == 0 && c_ex[i] < 0) dst[nx] = v;
        if (x == nx - 1 && c_ex[i] > 0) dst[-1] = v;
    }
}

template <class T, bool Flat>
__global__ void to_canonical_kernel(const T* f, double* out, int nx, int ny, int pitch, int xoff, long long plane,
                                    double ref0, double ref_slope, double isc) {
    if (Flat) {
        const long long n = 9LL * ny * nx;
        for (FlatWalk p(blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x, nx);
             p.idx < n; p.next()) {
            const int i = p.row / ny;
            to_canonical_one(f, out, p.idx, i, p.row - i * ny, p.x, pitch, xoff, plane, ref0, ref_slope, isc);
        }
    } else {
        for (int row = blockIdx.y; row < 9 * ny; row += gridDim.y) {
            const int i = row / ny, y = row - i * ny;
            for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x)
                to_canonical_one(f, out, (long long)row * nx + x, i, y, x, pitch, xoff, plane, ref0, ref_slope, isc);
        }
    }
}

template <class T, bool Flat>
__global__ void from_canonical_kernel(const double* in, T* f, int nx, int ny, int pitch, int xoff, long long plane,
                                      double ref0, double ref_slope, int periodic, double sc) {
    if (Flat) {
        const long long n = 9LL * ny * nx;
        for (FlatWalk p(blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x, nx);
             p.idx < n; p.next()) {
            const int i = p.row / ny;
            from_canonical_one(in, f, p.idx, i, p.row - i * ny, p.x, nx, pitch, xoff, plane, ref0, ref_slope, periodic,
                               sc);
        }
    } else {
        for (int row = blockIdx.y; row < 9 * ny; row += gridDim.y) {
            const int i = row / ny, y = row - i * ny;
            for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x)
                from_canonical_one(in, f, (long long)row * nx + x, i, y, x, nx, pitch, xoff, plane, ref0, ref_slope,
                                   periodic, sc);
        }
    }
}

// Centre-row densities of a state into rc[2][stride] (compute type RC).
template <class T, class RC>
__global__ void centre_density_kernel(const T* f, RC* rc, int nx, int pitch, int xoff, long long plane, int yc0,
                                      int yc1, int stride, double ref0, double ref_slope, double isc) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
        for (int slot = 0; slot < 2; ++slot) {
            const int y = slot ? yc1 : yc0;
            const T* row = f + (long long)y * pitch + xoff + x;
            double rho = ref0 + ref_slope * x;
            for (int i = 0; i < 9; ++i) rho += (double)Codec<T>::dec(row[i * plane], RT<T>(isc));
            rc[slot * stride + x] = RC(rho);
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Running sum over a thread's rows in the per-node type R: plain for FP64;
// compensated (Kahan) for FP32, so that a sum of a few dozen FP32 terms keeps
// FP32's precision and the FP64 pipe is touched once per thread, not per node.
template <class R> struct RowSum {
    R s = 0;
    __device__ __forceinline__ void add(R v) { s += v; }
    __device__ __forceinline__ double value() const { return (double)s; }
};
template <> struct RowSum<float> {
    float s = 0, c = 0;
    __device__ __forceinline__ void add(float v) {
        const float y = __fsub_rn(v, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Fixed-order sum of the per-block partials part[4 b + k] (b < nblocks) into
// part[0..3] by the threads of one block: thread t takes b = t, t + n, ...,
// then a tree over the threads.  The order depends on nothing but the sizes.
__device__ __forceinline__ void sum_partials_block(double* obs, const ObsLayout& L, double (*sh)[kObsRows * kObsCols]) {
    const int t = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    double acc[4] = {0, 0, 0, 0};
    for (int b = t; b < L.nblocks; b += nt)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += __ldcg(obs + L.part + 4 * b + k);
#pragma unroll
    for (int k = 0; k < 4; ++k) sh[k][t] = acc[k];
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
        if (t < w)
#pragma unroll
            for (int k = 0; k < 4; ++k) sh[k][t] += sh[k][t + w];
        __syncthreads();
    }
    if (t == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) obs[L.part + k] = sh[k][0];
}

// Per column: m(x) = sum_y rho u_x, centreline rho, sum_y u_x; the profiles at
// one column; per block: partial sums of m, u_x, rho and a non-finite count.
// Densities and velocities come from the post-collision populations of the
// last step: the collision keeps rho and adds rho F to the momentum (Eq. 4, 9),
// so rho u = sum_i e_i f~_i - rho F/2 is Eq. 13 at that time level.
// kSumU: also sum u_x over every node (the normalised flow rate Q of a
// body-force channel needs it); otherwise u_x is formed only at the profile
// column, and a node is counted non-finite when rho u or rho is.
// done (optional): a counter that is 0 on entry; the last block to finish
// then sums the partials (sum_partials_block), moves *status into
// *status_out, clears it, and resets the counter, so that one launch does
// the whole reduction.  Without it obs_final_kernel does the sum.
template <class T, bool kSumU>
__global__ void __launch_bounds__(kObsCols* kObsRows)
    obs_kernel(const T* __restrict__ f, double* __restrict__ obs, ObsLayout L, int nx, int ny, int pitch,
               int xoff, long long plane,
               double ref0, double ref_slope, double gx, double gy, int prof_col, double isc,
               unsigned* done = nullptr, unsigned* status = nullptr, double* status_out = nullptr) {
    // Per node in the storage's compute type (FP32 for FP32/16-bit storage,
    // whose values carry FP32 or coarser rounding already; FP64 for FP64),
    // summed over the thread's rows in that type (compensated in FP32) and
    // across threads in FP64.  The mass is n R(x) + sum of the density
    // deviations, so the reference part is exact.  The mass flow needs no
    // division: rho u_x = sum_i e_ix f~_i - rho F_x / 2.
    using R = RT<T>;
    __shared__ double sh[5][kObsRows * kObsCols];
    __shared__ bool last;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = blockIdx.x * kObsCols + tx;
    double m = 0, us = 0, mass = 0, rc = 0, bad = 0;
    // centre rows: the middle row, or the two middle rows (averaged)
    const int yc0 = (ny & 1) ? (ny - 1) / 2 : ny / 2 - 1, yc1 = (ny & 1) ? yc0 : ny / 2;
    if (x < nx) {
        const double ref = ref0 + ref_slope * x;
        const R hgx = R(0.5 * gx), hgy = R(0.5 * gy);
        RowSum<R> sm, su, sd;
        int rows = 0, nbad = 0;
        // density deviations at the centre rows this thread meets (FP32 selects
        // in the loop; the FP64 arithmetic on them once, after it)
        R dc0 = 0, dc1 = 0;
        bool hc0 = false, hc1 = false;
        // kObsBatch rows' nine values are loaded before any is used, so that
        // each thread keeps 9 kObsBatch loads in flight; the rows are then
        // reduced in the same order as one at a time
        for (int y0 = ty; y0 < ny; y0 += kObsBatch * kObsRows) {
            T raw[kObsBatch][9];
#pragma unroll
            for (int b = 0; b < kObsBatch; ++b) {
                const int y = y0 + b * kObsRows;
                if (y < ny) {
                    const T* row = f + (long long)y * pitch + xoff + x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) raw[b][i] = row[i * plane];
                }
            }
#pragma unroll
            for (int b = 0; b < kObsBatch; ++b) {
                const int y = y0 + b * kObsRows;
                if (y >= ny) break;
                R v[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) v[i] = Codec<T>::dec(raw[b][i], R(isc));
                const R a57 = v[5] - v[7], a86 = v[8] - v[6];
                const R drho = v[0] + (v[1] + v[3]) + (v[2] + v[4]) + ((v[5] + v[7]) + (v[6] + v[8]));
                const R rho = R(ref) + drho;
                const R mx = (v[1] - v[3]) + (a57 + a86) - hgx * rho;  // rho u_x
                const R my = (v[2] - v[4]) + (a57 - a86) - hgy * rho;  // rho u_y
                if (kSumU) {
                    const R irho = rcp(rho);
                    const R ux = mx * irho, uy = my * irho;
                    if (!isfinite(rho) || !isfinite(ux) || !isfinite(uy)) ++nbad;
                    su.add(ux);
                } else if (!isfinite(rho) || !isfinite(mx) || !isfinite(my) || rho == R(0)) {
                    ++nbad;
                }
                sm.add(mx);
                sd.add(drho);
                ++rows;
                if (y == yc0) {
                    dc0 = drho;
                    hc0 = true;
                }
                if (y == yc1 && yc1 != yc0) {
                    dc1 = drho;
                    hc1 = true;
                }
            }
        }
        // centreline density: the middle row, or the mean of the two middle rows
        if (ny & 1) {
            if (hc0) rc += ref + (double)dc0;
        } else {
            if (hc0) rc += 0.5 * (ref + (double)dc0);
            if (hc1) rc += 0.5 * (ref + (double)dc1);
        }
        // the velocity profiles at one column: its threads take their rows again
        if (x == prof_col) {
            for (int y = ty; y < ny; y += kObsRows) {
                const T* row = f + (long long)y * pitch + xoff + x;
                R v[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) v[i] = Codec<T>::dec(row[i * plane], R(isc));
                const R a57 = v[5] - v[7], a86 = v[8] - v[6];
                const R drho = v[0] + (v[1] + v[3]) + (v[2] + v[4]) + ((v[5] + v[7]) + (v[6] + v[8]));
                const R rho = R(ref) + drho;
                const R mx = (v[1] - v[3]) + (a57 + a86) - hgx * rho;
                const R my = (v[2] - v[4]) + (a57 - a86) - hgy * rho;
                const R irho = rcp(rho);
                obs[L.prof_x + y] = (double)(mx * irho);
                obs[L.prof_y + y] = (double)(my * irho);
            }
        }
        m = sm.value();
        us = su.value();
        mass = rows * ref + sd.value();
        bad = nbad;
    }
    const int t = ty * kObsCols + tx;
    sh[0][t] = m;
    sh[1][t] = us;
    sh[2][t] = mass;
    sh[3][t] = bad;
    sh[4][t] = rc;
    __syncthreads();
    if (ty == 0) {  // one full warp: column totals in a fixed order, then block partials
        double cm = 0, cu = 0, cmass = 0, cbad = 0, crc = 0;
        for (int k = 0; k < kObsRows; ++k) {
            cm += sh[0][k * kObsCols + tx];
            cu += sh[1][k * kObsCols + tx];
            cmass += sh[2][k * kObsCols + tx];
            cbad += sh[3][k * kObsCols + tx];
            crc += sh[4][k * kObsCols + tx];
        }
        if (x < nx) {
            obs[L.m + x] = cm;
            obs[L.rc + x] = crc;
        }
        cm = warp_sum(cm);
        cu = warp_sum(cu);
        cmass = warp_sum(cmass);
        cbad = warp_sum(cbad);
        if (tx == 0) {
            obs[L.part + 4 * blockIdx.x + 0] = cm;
            obs[L.part + 4 * blockIdx.x + 1] = cu;
            obs[L.part + 4 * blockIdx.x + 2] = cmass;
            obs[L.part + 4 * blockIdx.x + 3] = cbad;
        }
    }
    if (!done) return;
    // the last block to finish sums every block's partials
    __threadfence();
    __syncthreads();
    if (t == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    sum_partials_block(obs, L, sh);
    if (t == 0) {
        if (status) {
            *status_out = (double)*status;
            *status = 0u;
        }
        *done = 0u;
    }
}

// Sum the per-block partials in a fixed order (one warp), into part[0..3].
// With a status word: also move it into *status_out and clear it, so that the
// host reads the reductions and the error bits of the sweeps in one copy.
__global__ void obs_final_kernel(double* obs, ObsLayout L, unsigned* status = nullptr,
                                 double* status_out = nullptr) {
    const int t = threadIdx.x;
    if (status && t == 0) {
        *status_out = (double)*status;
        *status = 0u;
    }
    double acc[4] = {0, 0, 0, 0};
    for (int b = t; b < L.nblocks; b += 32)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += obs[L.part + 4 * b + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = warp_sum(acc[k]);
    __syncwarp();
    if (t == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) obs[L.part + k] = acc[k];
}

// Call f with a value of the storage element type.
template <class F> cudaError_t with_storage(int storage, F&& f) {
    switch (storage) {
        case CLB_FP64: return f(double{});
        case CLB_FP32_SHIFTED: return f(float{});
        case CLB_FP16_SCALED: return f(__half{});
        case CLB_BF16_SCALED: return f(__nv_bfloat16{});
    }
    return cudaErrorInvalidValue;
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    return (int)std::min<long long>(std::max<long long>(g, 1), 152LL * 32);
}

SweepArgs make_args(const clb_sim* s) {
    SweepArgs a{};
    a.fin = s->buf[s->cur];
    a.fout = s->buf[s->cur ^ 1];
    a.nx = s->nx;
    a.ny = s->ny;
    a.pitch = s->pitch;
    a.xoff = s->xoff;
    a.plane = s->plane;
    a.s3 = s->s3;
    a.s8 = s->s8;
    a.sv = s->sv;
    a.sq = s->sq;
    // tau = sqrt(6/pi) N Kn_loc/(1 + a Kn_loc), Kn_loc = Kn_out rho_out/rho
    //     = A/(rho + B), A = sqrt(6/pi) N Kn_out rho_out, B = a Kn_out rho_out
    a.rate_A = std::sqrt(6.0 / kPi) * s->ny * s->kn * s->rho_out;
    a.rate_B = s->a * s->kn * s->rho_out;
    a.rate_C = kPi * s->b2 / 4.0;
    a.r = s->r;
    a.gx = s->drive == CLB_DRIVE_BODY_FORCE ? s->g : 0.0;
    a.gy = 0.0;
    a.ref0 = s->ref0;
    a.ref_slope = s->ref_slope;
    a.drho_in = s->rho_in - s->ref_at(0);
    a.drho_out = s->rho_out - s->ref_at(s->nx - 1);
    a.store_scale = s->store_scale;
    a.kn_mode = s->kn_mode;
    a.withhold_tile = s->withhold_tile;
    a.yc0 = s->yc0;
    a.yc1 = s->yc1;
    a.rc_stride = s->rc_stride;
    derive_constants(a);
    return a;
}


// Centre-row densities of the current state into the rc side read by the
// next sweep (centreline Knudsen number only).
cudaError_t refresh_centre(clb_sim* s) {
    if (s->kn_mode != 1 || s->drive != CLB_DRIVE_PRESSURE) return cudaSuccess;
    return with_storage(s->storage, [&](auto tag) {
        using T = decltype(tag);
        using RC = RT<T>;
        RC* side = static_cast<RC*>(s->rc) + (size_t)s->cur * 2 * s->rc_stride;
        centre_density_kernel<T, RC><<<grid_for(s->nx, 256), 256, 0, s->stream>>>(
            static_cast<const T*>(s->buf[s->cur]), side, s->nx, s->pitch, s->xoff, s->plane, s->yc0, s->yc1,
            s->rc_stride, s->ref0, s->ref_slope, 1.0 / s->store_scale);
        return cudaGetLastError();
    });
}

cudaError_t launch_init(clb_sim* s, void* buf, double rho_a, double rho_slope) {
    const long long n = 9LL * s->nx * s->ny;
    return with_storage(s->storage, [&](auto tag) {
        using T = decltype(tag);
        init_kernel<T><<<grid_for(n, 256), 256, 0, s->stream>>>(
            static_cast<T*>(buf), s->nx, s->ny, s->pitch, s->xoff, s->plane, rho_a, rho_slope, s->ref0,
            s->ref_slope, s->drive == CLB_DRIVE_BODY_FORCE, s->store_scale);
        return cudaGetLastError();
    });
}

}  // namespace

namespace clb {

void rates_at(double kn, int ny, double a, double b2, double* sv, double* sq) {
    // Eq. 18 and Eq. 21 (tau_q = 1/s_v - 1/2)
    const double tau = std::sqrt(6.0 / kPi) * ny * kn / (1.0 + a * kn);
    *sv = 1.0 / (0.5 + tau);
    *sq = 1.0 / (0.5 + (3.0 + 4.0 * kPi * tau * tau * b2) / (16.0 * tau));
}

double r_from_sigma(double sigma) {
    // Eq. 21 with sigma_v = (2 - sigma)/sigma (Eq. 19) and B1 = 1 - 0.1817 sigma
    return 1.0 / (1.0 + (1.0 - 0.1817 * sigma) * (2.0 - sigma) / sigma * std::sqrt(kPi / 6.0));
}

int set_error(int st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

}  // namespace clb

// ---------------------------------------------------------------- C ABI

extern "C" {

void clb_opts_default(clb_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->test_withhold_tile = -1;
    o->b2 = 0.55;
    o->sigma = 1.0;
    o->s3 = 1.1;
    o->s8 = 1.2;
    o->rho_out = 1.0;
    o->storage = CLB_FP32_SHIFTED;
}

const char* clb_last_error(void) { return g_err; }

clb_status clb_destroy(clb_sim* s) {
    if (!s) return CLB_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    s->dfree(s->buf[0]);
    s->dfree(s->buf[1]);
    s->dfree(s->obs);
    if (s->hobs) cudaFreeHost(s->hobs);
    s->dfree(s->status);
    s->dfree(s->sched);
    s->dfree(s->rc);
    for (cudaGraphExec_t g : s->graph)
        if (g) cudaGraphExecDestroy(g);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return CLB_OK;
}

clb_status clb_create(int nx, int ny, double kn, double a, double r, clb_drive drive, double drive_value,
                      const clb_opts* opts, clb_sim** out) {
    g_err[0] = 0;
    if (!out) return fail(CLB_EINVAL, "clb_create: out is NULL");
    *out = nullptr;
    clb_opts o;
    clb_opts_default(&o);
    if (opts) o = *opts;
    if (drive != CLB_DRIVE_BODY_FORCE && drive != CLB_DRIVE_PRESSURE)
        return fail(CLB_EINVAL, "clb_create: unknown drive %d", (int)drive);
    if (ny < 1 || ny > 65535) return fail(CLB_EINVAL, "clb_create: ny = %d outside 1..65535", ny);
    if (nx < (drive == CLB_DRIVE_PRESSURE ? 4 : 1) || nx > (1 << 28))
        return fail(CLB_EINVAL, "clb_create: nx = %d too small or too large for this drive", nx);
    if (!(kn > 0) || !std::isfinite(kn)) return fail(CLB_EINVAL, "clb_create: Kn must be > 0");
    if (!(a >= 0) || !std::isfinite(a)) return fail(CLB_EINVAL, "clb_create: a must be >= 0");
    if (!std::isfinite(r) || r > 1) return fail(CLB_EINVAL, "clb_create: r must be in [0, 1] (or < 0 for Eq. 21)");
    if (!std::isfinite(drive_value)) return fail(CLB_EINVAL, "clb_create: drive value not finite");
    if (drive == CLB_DRIVE_PRESSURE && !(drive_value > 0))
        return fail(CLB_EINVAL, "clb_create: pressure ratio must be > 0");
    if (!(o.rho_out > 0) || !(o.b2 >= 0) || !(o.s3 > 0 && o.s3 < 2) || !(o.s8 > 0 && o.s8 < 2))
        return fail(CLB_EINVAL, "clb_create: rho_out, b2, s3 or s8 out of range");
    if (r < 0 && !(o.sigma > 0 && o.sigma <= 2)) return fail(CLB_EINVAL, "clb_create: sigma must be in (0, 2]");
    if (o.storage < CLB_FP64 || o.storage > CLB_BF16_SCALED)
        return fail(CLB_EINVAL, "clb_create: storage %d not available", o.storage);
    if ((o.alloc == nullptr) != (o.free == nullptr))
        return fail(CLB_EINVAL, "clb_create: alloc and free hooks must be given together");
    // Default nodes per thread of the direct sweep: one node per thread fills
    // the GPU with more warps, which wins where the channel is small (latency
    // bound) and for FP64 (FP64-pipe bound); four win for larger FP32 and for
    // 16-bit channels (fewer instructions per byte).
    int vec = o.vec;
    if (!vec) {
        if (o.storage == CLB_FP64)
            vec = 1;
        else if (o.storage == CLB_FP32_SHIFTED && (long long)nx * ny < (3LL << 16))
            vec = 1;
        else
            vec = 4;
    }
    if (!sweep_supported(o.storage, vec)) return fail(CLB_EINVAL, "clb_create: vec = %d not available", vec);
    int block_x = o.block_x ? o.block_x : 128;
    const int max_pipeline = 1 + tma_variant_count();
    if (o.pipeline < 0 || o.pipeline > max_pipeline)
        return fail(CLB_EINVAL, "clb_create: pipeline = %d must be 0..%d", o.pipeline, max_pipeline);
    if (o.kn_mode < 0 || o.kn_mode > 1) return fail(CLB_EINVAL, "clb_create: kn_mode = %d must be 0 or 1", o.kn_mode);
    if (block_x < 32 || block_x > 256 || block_x % 32)
        return fail(CLB_EINVAL, "clb_create: block_x = %d must be a multiple of 32 in 32..256", block_x);

    clb_sim* s = new (std::nothrow) clb_sim;
    if (!s) return fail(CLB_ENOMEM, "clb_create: host allocation failed");
    s->nx = nx;
    s->ny = ny;
    s->storage = o.storage;
    s->vec = vec;
    s->block_x = block_x;
    s->kn_mode = (drive == CLB_DRIVE_PRESSURE) ? o.kn_mode : 0;
    s->withhold_tile = o.test_withhold_tile;
    // Default engine: the TMA tile shape that was fastest on the 25601 x 256
    // pressure channel for the storage (pipeline 2: 512 x 2 nodes, 3 stages,
    // for FP32; 3: 128 x 4 nodes, 2 stages, 4 blocks per SM, for FP16 and
    // BF16).  Below 2^20 nodes, where a step is
    // bound by its latency rather than by HBM, the direct-load sweep is faster
    // (801 x 8: 4.1 against 4.7 us; 6401 x 64: 6.4 against 7.5 us per step),
    // and from 12801 x 128 up the TMA sweep is.  FP64 and the centreline
    // Knudsen mode always take the direct-load sweep.
    if (o.storage == CLB_FP64 || s->kn_mode == 1)
        s->pipeline = 1;
    else if (o.pipeline != 0)
        s->pipeline = o.pipeline;
    else if ((long long)nx * ny < (1LL << 20))
        s->pipeline = 1;  // small channels: the direct sweep has the shorter latency per step
    else
        s->pipeline = (o.storage == CLB_FP32_SHIFTED) ? 2 : 3;
    {
        // graph replay: not with the testing option
        int k = 0;
        if (o.graph_steps > 0)
            k = o.graph_steps;
        else if (o.graph_steps == 0)
            k = ((long long)nx * ny < (1LL << 20)) ? 64 : 0;
        if (o.test_withhold_tile >= 0) k = 0;
        s->graph_steps = k + (k & 1);  // even: a chunk ends on the buffer it started from
    }
    s->yc0 = (ny % 2) ? (ny - 1) / 2 : ny / 2 - 1;
    s->yc1 = (ny % 2) ? s->yc0 : ny / 2;
    s->drive = drive;
    s->drive_value = drive_value;
    s->kn = kn;
    s->a = a;
    s->b2 = o.b2;
    s->sigma = o.sigma;
    s->s3 = o.s3;
    s->s8 = o.s8;
    s->rho_out = o.rho_out;
    s->alloc = o.alloc;
    s->dealloc = o.free;
    s->alloc_ctx = o.alloc_ctx;
    if (drive == CLB_DRIVE_BODY_FORCE) {
        s->g = drive_value;
        s->rho_in = o.rho_out;
    } else {
        s->g = 0;
        s->rho_in = drive_value * o.rho_out;
    }
    s->r = r >= 0 ? r : r_from_sigma(o.sigma);
    rates_at(kn, ny, a, o.b2, &s->sv, &s->sq);

    // reference density of the stored deviations: the initial profile
    if (o.storage == CLB_FP64) {
        s->ref0 = 0;
        s->ref_slope = 0;
    } else if (drive == CLB_DRIVE_PRESSURE) {
        s->ref0 = s->rho_in;
        s->ref_slope = (s->rho_out - s->rho_in) / (double)(nx - 1);
    } else {
        s->ref0 = s->rho_out;
        s->ref_slope = 0;
    }

    s->elem = (o.storage == CLB_FP64) ? 8 : (o.storage == CLB_FP32_SHIFTED) ? 4 : 2;
    // FP16 keeps 2^-14 .. 4 in its normal range after this scale; BF16 has FP32's range
    s->store_scale = (o.storage == CLB_FP16_SCALED) ? 16384.0 : 1.0;
    const int align = (int)(128 / s->elem);
    s->xoff = align;
    s->pitch = ((s->xoff + nx + 16 + align - 1) / align) * align;
    s->plane = (long long)ny * s->pitch;
    s->buf_bytes = (size_t)9 * s->plane * s->elem;
    s->L = obs_layout(nx, ny);

    if (o.stream) {
        s->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaError_t e = cudaGetLastError();
            delete s;
            return fail(CLB_ECUDA, "clb_create: cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        s->own_stream = true;
    }

    s->buf[0] = s->dalloc(s->buf_bytes);
    s->buf[1] = s->dalloc(s->buf_bytes);
    s->obs = static_cast<double*>(s->dalloc((s->L.total + 2) * sizeof(double)));
    if (cudaHostAlloc(reinterpret_cast<void**>(&s->hobs), (s->L.total + 2) * sizeof(double), cudaHostAllocDefault) !=
        cudaSuccess) {
        cudaGetLastError();
        s->hobs = nullptr;
    }
    s->status = static_cast<unsigned*>(s->dalloc(sizeof(unsigned)));
    s->sched = static_cast<unsigned*>(s->dalloc(2 * sizeof(unsigned)));
    s->rc_stride = ((nx + 16 + 31) / 32) * 32;
    s->rc = s->dalloc((size_t)4 * s->rc_stride * (o.storage == CLB_FP64 ? 8 : 4));
    if (!s->buf[0] || !s->buf[1] || !s->obs || !s->hobs || !s->status || !s->sched || !s->rc) {
        clb_destroy(s);
        return fail(CLB_ENOMEM, "clb_create: device allocation of %zu bytes failed", 2 * s->buf_bytes);
    }
    clb_status st = CLB_OK;
    auto chk = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && st == CLB_OK) st = fail(CLB_ECUDA, "clb_create: %s: %s", what, cudaGetErrorString(e));
    };
    chk(cudaMemsetAsync(s->buf[0], 0, s->buf_bytes, s->stream), "memset");
    chk(cudaMemsetAsync(s->buf[1], 0, s->buf_bytes, s->stream), "memset");
    chk(cudaMemsetAsync(s->obs, 0, (s->L.total + 2) * sizeof(double), s->stream), "memset");
    chk(cudaMemsetAsync(s->status, 0, sizeof(unsigned), s->stream), "memset");
    chk(cudaMemsetAsync(s->sched, 0, 2 * sizeof(unsigned), s->stream), "memset");
    const double rho_slope = (drive == CLB_DRIVE_PRESSURE) ? (s->rho_out - s->rho_in) / (double)(nx - 1) : 0.0;
    chk(cudaMemsetAsync(s->rc, 0, (size_t)4 * s->rc_stride * (o.storage == CLB_FP64 ? 8 : 4), s->stream), "memset");
    chk(launch_init(s, s->buf[0], s->rho_in, rho_slope), "init");
    chk(refresh_centre(s), "centre densities");
    chk(cudaStreamSynchronize(s->stream), "sync");
    if (st != CLB_OK) {
        clb_destroy(s);
        return st;
    }
    *out = s;
    return CLB_OK;
}

// One sweep launch from buffer `cur` (direct or TMA engine).
static cudaError_t launch_single(clb_sim* s, SweepArgs& a, int mode, int cur) {
    const size_t rc_side = (size_t)2 * s->rc_stride * (s->storage == CLB_FP64 ? 8 : 4);
    a.fin = s->buf[cur];
    a.fout = s->buf[cur ^ 1];
    a.rc_in = static_cast<const char*>(s->rc) + cur * rc_side;
    a.rc_out = static_cast<char*>(s->rc) + (cur ^ 1) * rc_side;
    a.tile_order = cur;  // alternate the TMA sweep's tile order with the buffers
    return s->pipeline >= 2 ? launch_sweep_tma(s->storage, mode, s->pipeline - 2, a, s->stream, s->sched, s->status)
                            : launch_sweep(s->storage, mode, s->vec, s->block_x, a, s->stream);
}

// Capture graph_steps consecutive sweeps starting from buffer `cur` into an
// executable graph (programmatic launch edges are kept).
static cudaError_t build_graph(clb_sim* s, const SweepArgs& base, int mode, int cur, cudaGraphExec_t* out) {
    SweepArgs a = base;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < s->graph_steps && le == cudaSuccess; ++k, cur ^= 1) le = launch_single(s, a, mode, cur);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->stream, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le != cudaSuccess ? le : e;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

clb_status clb_step(clb_sim* s, int64_t n) {
    clb::TraceRange trace_("clb_step");
    if (!s) return fail(CLB_EINVAL, "clb_step: sim is NULL");
    if (n < 0) return fail(CLB_EINVAL, "clb_step: n < 0");
    const int mode = s->drive == CLB_DRIVE_PRESSURE ? MODE_PRESSURE : MODE_PERIODIC;
    SweepArgs a = make_args(s);
    // replayed chunks (the chunk length is even, so `cur` is where it started)
    for (; s->graph_steps > 0 && n >= s->graph_steps; n -= s->graph_steps) {
        if (!s->graph[s->cur]) {
            cudaError_t e = build_graph(s, a, mode, s->cur, &s->graph[s->cur]);
            if (e != cudaSuccess) return fail(CLB_ECUDA, "clb_step: capturing the sweep graph: %s", cudaGetErrorString(e));
        }
        cudaError_t e = cudaGraphLaunch(s->graph[s->cur], s->stream);
        if (e != cudaSuccess) return fail(CLB_ECUDA, "clb_step: graph launch: %s", cudaGetErrorString(e));
        s->step += s->graph_steps;
    }
    for (int64_t t = 0; t < n; ++t) {
        cudaError_t e = launch_single(s, a, mode, s->cur);
        if (e != cudaSuccess) return fail(CLB_ECUDA, "clb_step: sweep launch: %s", cudaGetErrorString(e));
        s->cur ^= 1;
        ++s->step;
        s->withhold_tile = a.withhold_tile = -1;
    }
    return CLB_OK;
}

// Read and clear the device status word; CLB_ETIMEOUT if a wait expired.
static clb_status check_status(clb_sim* s, const char* who) {
    // into pinned memory: a copy to pageable memory would be staged by the driver
    unsigned* hst = reinterpret_cast<unsigned*>(s->hobs + s->L.total + 1);
    CUDA_OR(cudaMemcpyAsync(hst, s->status, sizeof *hst, cudaMemcpyDeviceToHost, s->stream));
    CUDA_OR(cudaStreamSynchronize(s->stream));
    const unsigned st = *hst;
    if (st) {
        CUDA_OR(cudaMemsetAsync(s->status, 0, sizeof(unsigned), s->stream));
        return fail(CLB_ETIMEOUT, "%s: a sweep gave up waiting for its staged inputs (bits %u)", who, st);
    }
    return CLB_OK;
}

clb_status clb_sync(clb_sim* s) {
    if (!s) return fail(CLB_EINVAL, "clb_sync: sim is NULL");
    // the status copy is queued behind all of the stream's work, so the one
    // synchronisation in check_status waits for everything
    return check_status(s, "clb_sync");
}

clb_status clb_info(const clb_sim* s, clb_info_t* info) {
    if (!s || !info) return fail(CLB_EINVAL, "clb_info: NULL argument");
    info->nx = s->nx;
    info->ny = s->ny;
    info->pitch = s->pitch;
    info->storage = s->storage;
    info->vec = s->vec;
    info->block_x = s->block_x;
    info->drive = s->drive;
    // HBM bytes per node update: one read and one write of the nine populations
    info->bytes_per_node = 18.0 * (double)s->elem;
    info->sv = s->sv;
    info->sq = s->sq;
    info->r = s->r;
    info->kn = s->kn;
    info->a = s->a;
    info->g = s->g;
    info->rho_in = s->rho_in;
    info->rho_out = s->rho_out;
    info->step = s->step;
    info->stream = s->stream;
    info->pipeline = s->pipeline;
    info->kn_mode = s->kn_mode;
    return CLB_OK;
}

// Grids of the conversion kernels: the flat walk, eight 256-thread blocks
// per SM; the row walk, one row per blockIdx.y.
static dim3 flat_grid() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return dim3(8 * std::max(sms, 1));
}
static dim3 row_grid(int nx, int ny) {
    return dim3((unsigned)std::min(8, (nx + 255) / 256), (unsigned)std::min(9 * ny, 65535));
}

// The device's address of a host array, if the device can reach it (pinned
// or registered, and mapped); nullptr for other memory.
static void* device_view(const void* host) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

clb_status clb_get_state(clb_sim* s, double* host_f) {
    clb::TraceRange trace_("clb_get_state");
    if (!s || !host_f) return fail(CLB_EINVAL, "clb_get_state: NULL argument");
    const long long n = 9LL * s->nx * s->ny;
    // pinned host memory is written directly by the kernel; other memory
    // through a transient device buffer
    double* direct = static_cast<double*>(device_view(host_f));
    double* tmp = direct ? direct : static_cast<double*>(s->dalloc(n * sizeof(double)));
    if (!tmp) return fail(CLB_ENOMEM, "clb_get_state: device allocation failed");
    clb_status st = CLB_OK;
    cudaError_t e = with_storage(s->storage, [&](auto tag) {
        using T = decltype(tag);
        auto kern = direct ? to_canonical_kernel<T, true> : to_canonical_kernel<T, false>;
        kern<<<direct ? flat_grid() : row_grid(s->nx, s->ny), 256, 0, s->stream>>>(
            static_cast<const T*>(s->buf[s->cur]), tmp, s->nx, s->ny, s->pitch, s->xoff, s->plane, s->ref0,
            s->ref_slope, 1.0 / s->store_scale);
        return cudaGetLastError();
    });
    if (e == cudaSuccess && !direct)
        e = cudaMemcpyAsync(host_f, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = fail(CLB_ECUDA, "clb_get_state: %s", cudaGetErrorString(e));
    if (!direct) s->dfree(tmp);
    return st;
}

clb_status clb_set_state(clb_sim* s, const double* host_f) {
    clb::TraceRange trace_("clb_set_state");
    if (!s || !host_f) return fail(CLB_EINVAL, "clb_set_state: NULL argument");
    const long long n = 9LL * s->nx * s->ny;
    const double* direct = static_cast<const double*>(device_view(host_f));
    double* tmp = direct ? nullptr : static_cast<double*>(s->dalloc(n * sizeof(double)));
    if (!direct && !tmp) return fail(CLB_ENOMEM, "clb_set_state: device allocation failed");
    clb_status st = CLB_OK;
    cudaError_t e = direct ? cudaSuccess
                           : cudaMemcpyAsync(tmp, host_f, n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    const int periodic = s->drive == CLB_DRIVE_BODY_FORCE;
    if (e == cudaSuccess) {
        e = with_storage(s->storage, [&](auto tag) {
            using T = decltype(tag);
            auto kern = direct ? from_canonical_kernel<T, true> : from_canonical_kernel<T, false>;
            kern<<<direct ? flat_grid() : row_grid(s->nx, s->ny), 256, 0, s->stream>>>(
                direct ? direct : tmp, static_cast<T*>(s->buf[s->cur]), s->nx, s->ny, s->pitch, s->xoff, s->plane,
                s->ref0, s->ref_slope, periodic, s->store_scale);
            return cudaGetLastError();
        });
    }
    if (e == cudaSuccess) e = refresh_centre(s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = fail(CLB_ECUDA, "clb_set_state: %s", cudaGetErrorString(e));
    s->dfree(tmp);
    s->have_prev = false;
    return st;
}

clb_status clb_observables(clb_sim* s, int profile_col, clb_scalars* sc, double* ux_prof, double* uy_prof,
                           double* p_centre, double* dp_nonlin, double* m_of_x) {
    clb::TraceRange trace_("clb_observables");
    if (!s) return fail(CLB_EINVAL, "clb_observables: sim is NULL");
    const int nx = s->nx, ny = s->ny;
    if (profile_col < 0 || profile_col >= nx) profile_col = (s->drive == CLB_DRIVE_PRESSURE) ? nx - 1 : 0;
    const double gx = s->drive == CLB_DRIVE_BODY_FORCE ? s->g : 0.0;
    dim3 block(kObsCols, kObsRows);
    dim3 grid(s->L.nblocks);
    // one launch: the last block sums the partials into part[0..3] and puts
    // the status word at part[4] (block 1's partial, no longer needed, or the
    // spare slot at L.total when there is one block), so that everything the
    // host needs is one contiguous range; its counter (after the spare slot) is
    // cleared first, in case an earlier launch did not finish
    unsigned* done = reinterpret_cast<unsigned*>(s->obs + s->L.total + 1);
    double* status_out = s->obs + s->L.part + 4;
    CUDA_OR(cudaMemsetAsync(done, 0, sizeof(unsigned), s->stream));
    CUDA_OR(with_storage(s->storage, [&](auto tag) {
        using T = decltype(tag);
        auto args = [&](auto kern) {
            kern<<<grid, block, 0, s->stream>>>(static_cast<const T*>(s->buf[s->cur]), s->obs, s->L, nx, ny, s->pitch,
                                                s->xoff, s->plane, s->ref0, s->ref_slope, gx, 0.0, profile_col,
                                                1.0 / s->store_scale, done, s->status, status_out);
        };
        if (s->drive == CLB_DRIVE_BODY_FORCE)
            args(obs_kernel<T, true>);
        else
            args(obs_kernel<T, false>);
        return cudaGetLastError();
    }));
    // one pinned copy of what is asked for, one synchronisation: from the
    // column arrays (m(x), centre density; only if an output needs them) or
    // from the profiles, through the summed partials and the status word
    double* h = s->hobs;
    const bool cols = p_centre || dp_nonlin || m_of_x;
    const size_t first = cols ? 0 : s->L.prof_x, last = s->L.part + 5;
    CUDA_OR(cudaMemcpyAsync(h + first, s->obs + first, (last - first) * sizeof(double), cudaMemcpyDeviceToHost,
                            s->stream));
    CUDA_OR(cudaStreamSynchronize(s->stream));

    const double* hm = h + s->L.m;
    const double* hrc = h + s->L.rc;
    const double* hux = h + s->L.prof_x;
    const double* huy = h + s->L.prof_y;
    const double msum = h[s->L.part + 0], usum = h[s->L.part + 1], mass = h[s->L.part + 2];
    const double nbad = h[s->L.part + 3];
    const unsigned wait_bits = (unsigned)h[s->L.part + 4];
    const double p_in = s->rho_in / 3.0, p_out = s->rho_out / 3.0;
    const double L = nx > 1 ? (double)(nx - 1) : 1.0;
    if (cols) {
        // no division per column (the host's divide is slow next to the kernel)
        const double third = 1.0 / 3.0, slope = (p_in - p_out) / L, ipo = 1.0 / p_out;
        for (int x = 0; x < nx; ++x) {
            const double pc = hrc[x] * third;
            if (p_centre) p_centre[x] = pc;
            if (dp_nonlin) dp_nonlin[x] = (pc - (p_in - slope * x)) * ipo;
        }
        if (m_of_x) std::memcpy(m_of_x, hm, (size_t)nx * sizeof(double));
    }
    double umax = -INFINITY;
    for (int y = 0; y < ny; ++y) {
        if (ux_prof) ux_prof[y] = hux[y];
        if (uy_prof) uy_prof[y] = huy[y];
        umax = std::max(umax, hux[y]);
    }
    if (sc) {
        const double mbar = msum / nx;
        sc->mass_flow = mbar;
        if (ny >= 2)
            sc->u_slip = 0.5 * ((1.5 * hux[0] - 0.5 * hux[1]) + (1.5 * hux[ny - 1] - 0.5 * hux[ny - 2]));
        else
            sc->u_slip = hux[0];
        if (s->drive == CLB_DRIVE_BODY_FORCE) {
            // Q = sum_y u / (F H^2 sqrt(RT/2)/p) with RT = 1/3, p = rho0 RT, F = rho0 G
            sc->q_norm = s->g != 0 ? (usum / nx) / (3.0 * s->g * (double)ny * ny * std::sqrt(1.0 / 6.0)) : 0.0;
        } else {
            // m_ns = H^3 (p_in^2 - p_out^2)/(24 mu RT L), mu = rho_out sqrt(6/pi) Kn_out N/3
            const double mu = s->rho_out * std::sqrt(6.0 / kPi) * s->kn * ny / 3.0;
            const double mns = (double)ny * ny * ny * (p_in * p_in - p_out * p_out) / (24.0 * mu * (1.0 / 3.0) * L);
            sc->q_norm = mbar / mns;
        }
        sc->residual = s->have_prev && mbar != 0 ? std::fabs(mbar - s->prev_mass_flow) / std::fabs(mbar) : -1.0;
        sc->total_mass = mass;
        sc->ux_max = umax;
        sc->step = s->step;
        s->prev_mass_flow = mbar;
        s->have_prev = true;
    }
    if (wait_bits)
        return fail(CLB_ETIMEOUT, "clb_observables: a sweep gave up waiting for its staged inputs (bits %u)",
                    wait_bits);
    if (nbad > 0) return fail(CLB_ENUMERIC, "clb_observables: %.0f nodes with a non-finite density or velocity", nbad);
    return CLB_OK;
}

}  // extern "C"

// ---------------------------------------------------- allocation-free variant
//
// clb_observables_noalloc: the observable reduction above, for callers that
// hold the populations in device memory of their own and may not allocate any
// (see include/clb.h).  Its scratch is a fixed array in this file, shared by
// every call on a device and kept until the process exits.

namespace {

constexpr int kNoAllocMaxNx = 65536;
constexpr int kNoAllocMaxNy = 4096;
constexpr size_t kNoAllocScratch =
    2 * (size_t)kNoAllocMaxNx + 2 * (size_t)kNoAllocMaxNy + 4 * (size_t)((kNoAllocMaxNx + kObsCols - 1) / kObsCols);
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the name is only a host-side stand-in for it).
clb_status noalloc_scratch(double** out) {
    int dev = -1;
    CUDA_OR(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(CLB_EINVAL, "clb_observables_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(CLB_ECUDA, "clb_observables_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return CLB_OK;
}

}  // namespace

extern "C" clb_status clb_observables_noalloc(const double* f_dev, int nx, int ny, int drive, double g,
                                              double rho_in, double rho_out, double kn, int profile_col,
                                              void* stream, clb_scalars* sc, double* ux_prof, double* uy_prof,
                                              double* p_centre, double* dp_nonlin, double* m_of_x) {
    if (!f_dev) return fail(CLB_EINVAL, "clb_observables_noalloc: populations pointer is NULL");
    if (nx < 1 || nx > kNoAllocMaxNx || ny < 1 || ny > kNoAllocMaxNy)
        return fail(CLB_EINVAL, "clb_observables_noalloc: nx = %d, ny = %d outside 1..%d x 1..%d", nx, ny,
                    kNoAllocMaxNx, kNoAllocMaxNy);
    if (drive != CLB_DRIVE_BODY_FORCE && drive != CLB_DRIVE_PRESSURE)
        return fail(CLB_EINVAL, "clb_observables_noalloc: unknown drive %d", drive);
    if (drive == CLB_DRIVE_PRESSURE && !(kn > 0 && rho_in > 0 && rho_out > 0))
        return fail(CLB_EINVAL, "clb_observables_noalloc: pressure drive needs kn, rho_in, rho_out > 0");
    double* scratch = nullptr;
    clb_status st = noalloc_scratch(&scratch);
    if (st != CLB_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (profile_col < 0 || profile_col >= nx) profile_col = (drive == CLB_DRIVE_PRESSURE) ? nx - 1 : 0;
    const ObsLayout L = obs_layout(nx, ny);
    const double gx = drive == CLB_DRIVE_BODY_FORCE ? g : 0.0;
    // the previous call's values stay in the array; start from zeros
    CUDA_OR(cudaMemsetAsync(scratch, 0, L.total * sizeof(double), s));
    // populations in the canonical layout: row pitch nx, no halo, plain FP64 (R = 0)
    obs_kernel<double, true><<<dim3(L.nblocks), dim3(kObsCols, kObsRows), 0, s>>>(
        f_dev, scratch, L, nx, ny, nx, 0, (long long)nx * ny, 0.0, 0.0, gx, 0.0, profile_col, 1.0);
    CUDA_OR(cudaGetLastError());
    obs_final_kernel<<<1, 32, 0, s>>>(scratch, L);
    CUDA_OR(cudaGetLastError());
    // straight into the caller's arrays or small stack buffers: no allocation here
    double part[4];
    double prof[kNoAllocMaxNy];
    CUDA_OR(cudaMemcpyAsync(part, scratch + L.part, sizeof part, cudaMemcpyDeviceToHost, s));
    CUDA_OR(cudaMemcpyAsync(prof, scratch + L.prof_x, ny * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (uy_prof) CUDA_OR(cudaMemcpyAsync(uy_prof, scratch + L.prof_y, ny * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (m_of_x) CUDA_OR(cudaMemcpyAsync(m_of_x, scratch + L.m, nx * sizeof(double), cudaMemcpyDeviceToHost, s));
    double* rc_dst = p_centre ? p_centre : dp_nonlin;
    if (rc_dst) CUDA_OR(cudaMemcpyAsync(rc_dst, scratch + L.rc, nx * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_OR(cudaStreamSynchronize(s));

    const double p_in = rho_in / 3.0, p_out = rho_out / 3.0;
    const double Lx = nx > 1 ? (double)(nx - 1) : 1.0;
    if (rc_dst)
        for (int x = 0; x < nx; ++x) {
            const double pc = rc_dst[x] / 3.0;  // centreline density -> pressure
            if (p_centre) p_centre[x] = pc;
            if (dp_nonlin) dp_nonlin[x] = (pc - (p_in - (p_in - p_out) * x / Lx)) / p_out;
        }
    double umax = -INFINITY;
    for (int y = 0; y < ny; ++y) {
        if (ux_prof) ux_prof[y] = prof[y];
        umax = std::max(umax, prof[y]);
    }
    if (sc) {
        const double mbar = part[0] / nx;
        sc->mass_flow = mbar;
        sc->u_slip = ny >= 2 ? 0.5 * ((1.5 * prof[0] - 0.5 * prof[1]) + (1.5 * prof[ny - 1] - 0.5 * prof[ny - 2]))
                             : prof[0];
        if (drive == CLB_DRIVE_BODY_FORCE) {
            sc->q_norm = g != 0 ? (part[1] / nx) / (3.0 * g * (double)ny * ny * std::sqrt(1.0 / 6.0)) : 0.0;
        } else {
            const double mu = rho_out * std::sqrt(6.0 / kPi) * kn * ny / 3.0;
            const double mns = (double)ny * ny * ny * (p_in * p_in - p_out * p_out) / (24.0 * mu * (1.0 / 3.0) * Lx);
            sc->q_norm = mbar / mns;
        }
        sc->residual = -1.0;  // no previous call to compare with: the entry point keeps no state
        sc->total_mass = part[2];
        sc->ux_max = umax;
        sc->step = -1;
    }
    if (part[3] > 0)
        return fail(CLB_ENUMERIC, "clb_observables_noalloc: %.0f nodes with a non-finite density or velocity",
                    part[3]);
    return CLB_OK;
}

// ----------------------------------------------------------- checkpoints

namespace {

struct CkptHeader {
    char magic[8];           // "CLBCKPT1"
    uint32_t version;        // 1
    uint32_t header_bytes;   // sizeof(CkptHeader)
    int32_t nx, ny, drive, storage, kn_mode, pitch, elem, rc_stride;
    int64_t step;
    int32_t have_prev, reserved0;
    double kn, a, r, drive_value, b2, sigma, s3, s8, rho_out, prev_mass_flow;
    uint64_t buf_bytes, rc_bytes;  // payloads: stored populations, centreline densities
    uint64_t checksum;             // FNV-1a 64 over the payloads in that order
    uint64_t reserved1;
};
static_assert(sizeof(CkptHeader) == 176, "checkpoint header layout");
constexpr char kCkptMagic[8] = {'C', 'L', 'B', 'C', 'K', 'P', 'T', '1'};

uint64_t fnv1a(const std::vector<unsigned char>& v, uint64_t h) {
    for (unsigned char b : v) h = (h ^ b) * 1099511628211ull;
    return h;
}
constexpr uint64_t kFnvOffset = 14695981039346656037ull;

size_t rc_side_bytes(int rc_stride, int storage) {
    return (size_t)2 * rc_stride * (storage == CLB_FP64 ? 8 : 4);
}

}  // namespace

clb_status clb_save(clb_sim* s, const char* path) {
    clb::TraceRange trace_("clb_save");
    if (!s || !path) return fail(CLB_EINVAL, "clb_save: NULL argument");
    clb_status st = check_status(s, "clb_save");  // synchronises; refuses results of a failed sweep
    if (st != CLB_OK) return st;
    const size_t rc_side = rc_side_bytes(s->rc_stride, s->storage);
    std::vector<unsigned char> buf(s->buf_bytes), rc(rc_side);
    CUDA_OR(cudaMemcpyAsync(buf.data(), s->buf[s->cur], s->buf_bytes, cudaMemcpyDeviceToHost, s->stream));
    CUDA_OR(cudaMemcpyAsync(rc.data(), static_cast<const char*>(s->rc) + s->cur * rc_side, rc_side,
                            cudaMemcpyDeviceToHost, s->stream));
    CUDA_OR(cudaStreamSynchronize(s->stream));
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kCkptMagic, sizeof h.magic);
    h.version = 1;
    h.header_bytes = sizeof h;
    h.nx = s->nx;
    h.ny = s->ny;
    h.drive = s->drive;
    h.storage = s->storage;
    h.kn_mode = s->kn_mode;
    h.pitch = s->pitch;
    h.elem = (int32_t)s->elem;
    h.rc_stride = s->rc_stride;
    h.step = s->step;
    h.have_prev = s->have_prev ? 1 : 0;
    h.kn = s->kn;
    h.a = s->a;
    h.r = s->r;
    h.drive_value = s->drive_value;
    h.b2 = s->b2;
    h.sigma = s->sigma;
    h.s3 = s->s3;
    h.s8 = s->s8;
    h.rho_out = s->rho_out;
    h.prev_mass_flow = s->prev_mass_flow;
    h.buf_bytes = buf.size();
    h.rc_bytes = rc.size();
    h.checksum = fnv1a(rc, fnv1a(buf, kFnvOffset));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(CLB_EIO, "clb_save: cannot open %s for writing", path);
    const bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size() &&
                    std::fwrite(rc.data(), 1, rc.size(), f) == rc.size();
    if (std::fclose(f) != 0 || !ok) return fail(CLB_EIO, "clb_save: writing %s failed", path);
    return CLB_OK;
}

clb_status clb_load(const char* path, const clb_opts* opts, clb_sim** out) {
    clb::TraceRange trace_("clb_load");
    g_err[0] = 0;
    if (!path || !out) return fail(CLB_EINVAL, "clb_load: NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(CLB_EIO, "clb_load: cannot open %s", path);
    CkptHeader h;
    std::vector<unsigned char> buf, rc;
    const char* why = nullptr;
    if (std::fread(&h, sizeof h, 1, f) != 1) {
        why = "truncated header";
    } else if (std::memcmp(h.magic, kCkptMagic, sizeof h.magic) != 0) {
        why = "not a CLB checkpoint";
    } else if (h.version != 1 || h.header_bytes != sizeof h) {
        why = "unsupported checkpoint version";
    } else if (h.storage < CLB_FP64 || h.storage > CLB_BF16_SCALED || h.nx < 1 || h.ny < 1 || h.ny > 65535 ||
               h.pitch < h.nx || h.elem != (h.storage == CLB_FP64 ? 8 : h.storage == CLB_FP32_SHIFTED ? 4 : 2) ||
               h.buf_bytes != (uint64_t)9 * h.ny * h.pitch * h.elem || h.rc_stride < h.nx ||
               h.rc_bytes != rc_side_bytes(h.rc_stride, h.storage)) {
        why = "inconsistent header";
    } else {
        buf.resize(h.buf_bytes);
        rc.resize(h.rc_bytes);
        if (std::fread(buf.data(), 1, buf.size(), f) != buf.size() || std::fread(rc.data(), 1, rc.size(), f) != rc.size())
            why = "truncated payload";
        else if (fnv1a(rc, fnv1a(buf, kFnvOffset)) != h.checksum)
            why = "checksum mismatch";
    }
    std::fclose(f);
    if (why) return fail(CLB_EIO, "clb_load: %s: %s", path, why);

    clb_opts o;
    clb_opts_default(&o);
    if (opts) o = *opts;
    o.storage = h.storage;
    o.kn_mode = h.kn_mode;
    o.b2 = h.b2;
    o.sigma = h.sigma;
    o.s3 = h.s3;
    o.s8 = h.s8;
    o.rho_out = h.rho_out;
    clb_sim* s = nullptr;
    clb_status st = clb_create(h.nx, h.ny, h.kn, h.a, h.r, (clb_drive)h.drive, h.drive_value, &o, &s);
    if (st != CLB_OK) return st;
    if (s->pitch != h.pitch || (int)s->elem != h.elem || s->rc_stride != h.rc_stride || s->buf_bytes != h.buf_bytes) {
        clb_destroy(s);
        return fail(CLB_EIO, "clb_load: %s: layout differs from what this library version creates", path);
    }
    cudaError_t e = cudaMemcpyAsync(s->buf[s->cur], buf.data(), buf.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<char*>(s->rc) + s->cur * rc.size(), rc.data(), rc.size(),
                            cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        clb_destroy(s);
        return fail(CLB_ECUDA, "clb_load: %s", cudaGetErrorString(e));
    }
    s->step = h.step;
    s->have_prev = h.have_prev != 0;
    s->prev_mass_flow = h.prev_mass_flow;
    *out = s;
    return CLB_OK;
}
