// Discrete adjoint of the body-force channel (Sec. 3.1 of Liu & He,
// arXiv:1603.01955): gradient of the flow sum J = mean_x sum_y u_x after N
// steps with respect to the CBBSR bounce-back fraction r_b (Eq. 20), the
// Bosanquet factor a (Eq. 16-18, 21, through s_v and s_q) and the body force G
// (Eq. 9, 13).
//
// One step is f_{t+1} = C(P(f_t)): P pulls the post-collision populations
// (Eq. 5, periodic x, walls Eq. 20), C collides every node (Eq. 4, 6-13).  The
// adjoint runs backwards: mu = J_C(P f_t)^T lambda_{t+1} per node, then
// lambda_t = P^T mu, while r_b, a and G collect lambda_{t+1}^T dC/dtheta and
// mu^T dP/dr.  J_C^T lambda is formed column by column with forward-mode dual
// numbers pushed through the very collision template the sweeps use (one
// tangent per input population, one for a, one for G); P^T is written out by
// hand as a gather (each post-collision population is pulled by one node, or
// by two wall nodes).  The forward keeps a checkpoint every C steps (C ~
// sqrt(N)) and recomputes each segment before walking it backwards.
// Parameter sums are FP64; states and adjoints are FP32 or FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/clb.h"
#include "clb_device.cuh"
#include "clb_internal.h"

namespace clb {

// Forward-mode dual number with one tangent component.
template <class R> struct Dual {
    R v, d;
    __host__ __device__ Dual() : v(0), d(0) {}
    __host__ __device__ Dual(double x) : v(R(x)), d(0) {}
    __host__ __device__ Dual(R x, R dx) : v(x), d(dx) {}
};
template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, Dual<R> b) { return {a.v + b.v, a.d + b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, Dual<R> b) { return {a.v - b.v, a.d - b.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a) { return {-a.v, -a.d}; }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, Dual<R> b) {
    return {a.v * b.v, a.v * b.d + a.d * b.v};
}
template <class R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, Dual<R> b) {
    const R q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
template <class R> __device__ __forceinline__ Dual<R>& operator+=(Dual<R>& a, Dual<R> b) { return a = a + b; }
template <class R> __device__ __forceinline__ Dual<R>& operator-=(Dual<R>& a, Dual<R> b) { return a = a - b; }
template <class R> __device__ __forceinline__ Dual<R> rcp(Dual<R> a) {
    const R q = R(1) / a.v;
    return {q, -a.d * q * q};
}

}  // namespace clb

using namespace clb;

namespace {

// Constants of one adjoint run in compute type R.
template <class R> struct AdjConst {
    KC<R> c;       // collision constants (body-force channel)
    R dsv4_da;     // d(s_v/4)/da
    R dsq4_da;     // d(s_q/4)/da
    R r, rc;       // r_b, 1 - r_b
    R ref;         // reference density of the stored deviations
    int nx, ny;
};

// The 9 pre-collision populations of node (x, y): pull with periodic x and
// the CBBSR walls (Eq. 20 and its mirror), from a state [9][ny][nx].
template <class R>
__device__ __forceinline__ void pull(const R* f, int nx, int ny, int x, int y, R r, R rc, R (&o)[9]) {
    const int nn = nx * ny;
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;
    auto at = [&](int i, int yy, int xx) -> R { return f[i * nn + yy * nx + xx]; };
    o[0] = at(0, y, x);
    o[1] = at(1, y, xm);
    o[3] = at(3, y, xp);
    if (y == 0) {
        o[2] = at(4, 0, x);
        o[5] = r * at(7, 0, x) + rc * at(8, 0, xm);
        o[6] = r * at(8, 0, x) + rc * at(7, 0, xp);
    } else {
        o[2] = at(2, y - 1, x);
        o[5] = at(5, y - 1, xm);
        o[6] = at(6, y - 1, xp);
    }
    if (y == ny - 1) {
        o[4] = at(2, y, x);
        o[7] = r * at(5, y, x) + rc * at(6, y, xp);
        o[8] = r * at(6, y, x) + rc * at(5, y, xm);
    } else {
        o[4] = at(4, y + 1, x);
        o[7] = at(7, y + 1, xp);
        o[8] = at(8, y + 1, xm);
    }
}

template <class R>
__global__ void adj_forward_kernel(const R* fin, R* fout, AdjConst<R> k) {
    const int nn = k.nx * k.ny;
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        R d[9];
        pull(fin, k.nx, k.ny, node % k.nx, node / k.nx, k.r, k.rc, d);
        collide<R, MODE_PERIODIC>(d, k.ref, k.c);
        for (int i = 0; i < 9; ++i) fout[i * nn + node] = d[i];
    }
}

// Collision constants with the tangent of one parameter: which = 0 none,
// 1 a (through s_v and s_q), 2 G.
template <class R>
__device__ __forceinline__ KC<Dual<R>> dual_consts(const AdjConst<R>& k, int which) {
    KC<Dual<R>> c;
    const KC<R>& p = k.c;
    c.s3_12 = Dual<R>(p.s3_12, R(0));
    c.s8_4 = Dual<R>(p.s8_4, R(0));
    c.sv_4 = Dual<R>(p.sv_4, which == 1 ? k.dsv4_da : R(0));
    c.sq_4 = Dual<R>(p.sq_4, which == 1 ? k.dsq4_da : R(0));
    c.hfx = Dual<R>(p.hfx, which == 2 ? R(0.5) : R(0));
    c.fx = Dual<R>(p.fx, which == 2 ? R(1) : R(0));
    c.hfy = Dual<R>(p.hfy, R(0));
    c.fy = Dual<R>(p.fy, R(0));
    c.A = c.B = c.A316 = c.CA = c.r = c.rc = c.slope = c.sha = c.shd = c.drho_in = c.drho_out = Dual<R>(0.0);
    c.ref0 = Dual<R>(p.ref0, R(0));
    c.sc = c.isc = Dual<R>(1.0);
    return c;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double s = sh[0];
    __syncthreads();
    return s;
}

constexpr int kAdjThreads = 128;

// mu = J_C^T lambda_{t+1} at every node (indexed like the pre-collision
// populations), and the parameter terms of step t added to this block's slots
// acc[k * gridDim.x + blockIdx.x], k = 0, 1, 2 (r, a, G).  Each slot has one
// writer and the launches run in stream order, so every slot is summed in a
// fixed order and the gradient is the same bit for bit on every run.
template <class R>
__global__ void __launch_bounds__(kAdjThreads)
    adj_back_kernel(const R* f_t, const R* lam, R* mu, double* acc, AdjConst<R> k) {
    __shared__ double sh[kAdjThreads];
    const int nn = k.nx * k.ny;
    double gr = 0, ga = 0, gg = 0;
    for (int base = blockIdx.x * blockDim.x; base < nn; base += gridDim.x * blockDim.x) {
        const int node = base + threadIdx.x;
        if (node < nn) {
            const int x = node % k.nx, y = node / k.nx;
            R fb[9], l[9];
            pull(f_t, k.nx, k.ny, x, y, k.r, k.rc, fb);
            for (int i = 0; i < 9; ++i) l[i] = lam[i * nn + node];
            const KC<Dual<R>> c0 = dual_consts(k, 0);
            R m[9];
            for (int j = 0; j < 9; ++j) {  // column j of the collision Jacobian
                Dual<R> d[9];
                for (int i = 0; i < 9; ++i) d[i] = Dual<R>(fb[i], i == j ? R(1) : R(0));
                collide<Dual<R>, MODE_PERIODIC>(d, Dual<R>(k.ref, R(0)), c0);
                R s = 0;
                for (int i = 0; i < 9; ++i) s += l[i] * d[i].d;
                m[j] = s;
                mu[j * nn + node] = s;
            }
            for (int which = 1; which <= 2; ++which) {  // dC/da, dC/dG
                const KC<Dual<R>> cp = dual_consts(k, which);
                Dual<R> d[9];
                for (int i = 0; i < 9; ++i) d[i] = Dual<R>(fb[i], R(0));
                collide<Dual<R>, MODE_PERIODIC>(d, Dual<R>(k.ref, R(0)), cp);
                double s = 0;
                for (int i = 0; i < 9; ++i) s += (double)l[i] * (double)d[i].d;
                if (which == 1)
                    ga += s;
                else
                    gg += s;
            }
            // dP/dr at the wall rows (Eq. 20): d fbar5/dr = f7(x) - f8(x-1), ...
            const int xm = x == 0 ? k.nx - 1 : x - 1;
            const int xp = x == k.nx - 1 ? 0 : x + 1;
            auto at = [&](int i, int xx) -> double { return (double)f_t[i * nn + y * k.nx + xx]; };
            if (y == 0) gr += (double)m[5] * (at(7, x) - at(8, xm)) + (double)m[6] * (at(8, x) - at(7, xp));
            if (y == k.ny - 1) gr += (double)m[7] * (at(5, x) - at(6, xp)) + (double)m[8] * (at(6, x) - at(5, xm));
        }
    }
    gr = block_sum(gr, sh);
    ga = block_sum(ga, sh);
    gg = block_sum(gg, sh);
    if (threadIdx.x == 0) {
        acc[0 * gridDim.x + blockIdx.x] += gr;
        acc[1 * gridDim.x + blockIdx.x] += ga;
        acc[2 * gridDim.x + blockIdx.x] += gg;
    }
}

// lambda_t = P^T mu: each post-collision population of step t is pulled by
// the node it streams to, or, at a wall, by the bounce-back and the specular
// terms of Eq. 20 (two nodes of the wall row).
template <class R>
__global__ void adj_transpose_kernel(const R* mu, R* lam, AdjConst<R> k) {
    const int nx = k.nx, ny = k.ny, nn = nx * ny;
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        const int x = node % nx, y = node / nx;
        const int xm = x == 0 ? nx - 1 : x - 1;
        const int xp = x == nx - 1 ? 0 : x + 1;
        auto M = [&](int i, int yy, int xx) -> R { return mu[i * nn + yy * nx + xx]; };
        R o[9];
        o[0] = M(0, y, x);
        o[1] = M(1, y, xp);  // f1 at x is pulled by x+1
        o[3] = M(3, y, xm);
        // moving up (2, 5, 6): pulled by row y+1, or by the top-wall terms
        if (y == ny - 1) {
            o[2] = M(4, y, x);
            o[5] = k.r * M(7, y, x) + k.rc * M(8, y, xp);
            o[6] = k.r * M(8, y, x) + k.rc * M(7, y, xm);
        } else {
            o[2] = M(2, y + 1, x);
            o[5] = M(5, y + 1, xp);
            o[6] = M(6, y + 1, xm);
        }
        // moving down (4, 7, 8): pulled by row y-1, or by the bottom-wall terms
        if (y == 0) {
            o[4] = M(2, 0, x);
            o[7] = k.r * M(5, 0, x) + k.rc * M(6, 0, xm);
            o[8] = k.r * M(6, 0, x) + k.rc * M(5, 0, xp);
        } else {
            o[4] = M(4, y - 1, x);
            o[7] = M(7, y - 1, xm);
            o[8] = M(8, y - 1, xp);
        }
        for (int i = 0; i < 9; ++i) lam[i * nn + node] = o[i];
    }
}

// J = (1/nx) sum u_x of the final post-collision state and lambda_N = dJ/df_N:
// u_x = sum_i e_ix f_i / rho - G/2, so dJ/df_i = (e_ix - u_x - G/2) / (nx rho).
template <class R>
__global__ void __launch_bounds__(kAdjThreads) adj_final_kernel(const R* f, R* lam, double* acc, AdjConst<R> k) {
    __shared__ double sh[kAdjThreads];
    const int nn = k.nx * k.ny;
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    double js = 0;
    for (int base = blockIdx.x * blockDim.x; base < nn; base += gridDim.x * blockDim.x) {
        const int node = base + threadIdx.x;
        if (node < nn) {
            double rho = (double)k.ref, jx = 0;
            for (int i = 0; i < 9; ++i) {
                const double v = (double)f[i * nn + node];
                rho += v;
                jx += ex[i] * v;
            }
            const double ux = jx / rho - 0.5 * (double)k.c.fx;
            js += ux / k.nx;
            for (int i = 0; i < 9; ++i) lam[i * nn + node] = R((ex[i] - ux - 0.5 * (double)k.c.fx) / (k.nx * rho));
        }
    }
    js = block_sum(js, sh);
    if (threadIdx.x == 0) acc[3 * gridDim.x + blockIdx.x] = js;
}

// ------------------------------------------------------ resident engine
//
// For a grid whose two states fit in one block's shared memory, the whole
// checkpointed forward pass is one launch of one block, with block barriers
// between the steps; the backward walk over every segment is one launch of a
// thread-block cluster, with cluster barriers between its phases (the
// arithmetic is that of the kernels above).  In the backward step the 9 + 2
// forward-mode columns of each node's collision are spread over separate
// threads.  The parameter sums stay per thread (FP64, in step order) and are
// added by fixed trees at the end, so the gradient is the same bit for bit on
// every run.
constexpr int kResThreads = 256;  // the dual-number collision needs ~160-250 registers
constexpr int kCols = 11;         // 9 population tangents, then a and G

__device__ __forceinline__ double res_block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kResThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// One step of the whole grid in shared memory, a -> b (and optionally to a
// global copy `out`).
template <class R>
__device__ __forceinline__ void res_step(const R* a, R* b, R* out, const AdjConst<R>& k) {
    const int nn = k.nx * k.ny;
    for (int node = threadIdx.x; node < nn; node += kResThreads) {
        R d[9];
        pull(a, k.nx, k.ny, node % k.nx, node / k.nx, k.r, k.rc, d);
        collide<R, MODE_PERIODIC>(d, k.ref, k.c);
        for (int i = 0; i < 9; ++i) {
            b[i * nn + node] = d[i];
            if (out) out[i * nn + node] = d[i];
        }
    }
}

// Forward pass from f^eq(rho_out, 0): checkpoint s (the state at step s C)
// into ckpt + s state_elems, then J and lambda_N (as adj_final_kernel).
template <class R>
__global__ void __launch_bounds__(kResThreads)
    adj_res_forward_kernel(R* ckpt, size_t state_elems, int every, long long nsteps, R* lam_final, double* J,
                           AdjConst<R> k) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int nn = k.nx * k.ny, n9 = 9 * nn;
    R* a = reinterpret_cast<R*>(sm_raw);
    R* b = a + n9;
    double* red = reinterpret_cast<double*>(sm_raw + ((2 * n9 * sizeof(R) + 15) / 16) * 16);
    for (int e = threadIdx.x; e < n9; e += kResThreads) a[e] = R(0);  // zero deviations
    __syncthreads();
    for (long long t = 0; t < nsteps; ++t) {
        if (t % every == 0) {
            R* c = ckpt + (size_t)(t / every) * state_elems;
            for (int e = threadIdx.x; e < n9; e += kResThreads) c[e] = a[e];
        }
        res_step<R>(a, b, nullptr, k);
        __syncthreads();
        R* t2 = a;
        a = b;
        b = t2;
    }
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    double js = 0;
    for (int node = threadIdx.x; node < nn; node += kResThreads) {
        double rho = (double)k.ref, jx = 0;
        for (int i = 0; i < 9; ++i) {
            const double v = (double)a[i * nn + node];
            rho += v;
            jx += ex[i] * v;
        }
        const double ux = jx / rho - 0.5 * (double)k.c.fx;
        js += ux / k.nx;
        for (int i = 0; i < 9; ++i) lam_final[i * nn + node] = R((ex[i] - ux - 0.5 * (double)k.c.fx) / (k.nx * rho));
    }
    js = res_block_sum(js, red);
    if (threadIdx.x == 0) *J = js;
}

// The backward walk over every segment, spread over one thread-block cluster
// of `gridDim.x` blocks: recompute the segment's states from its checkpoint,
// then per step mu_t = J_C^T lambda_{t+1}, one thread per node and column,
// with lambda_{t+1} = P^T mu_{t+1} gathered on the fly from the previous
// step's mu (lambda_N itself for the first step), so one cluster barrier
// separates the steps.  mu (two buffers) and the segment states are in global
// memory (a few KB each, resident in L2); the cluster barrier (release /
// acquire at cluster scope) orders them.  Every block runs the same loop
// counts, so every barrier is reached by all of them.  Each block's
// parameter sums go to part[rank * 3 + 0..2], added on the host in rank order.
constexpr int kClusterMax = 16;

__device__ __forceinline__ void cluster_barrier() {
    __threadfence();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ int cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}

// lambda_t(node) = (P^T mu)(node): each post-collision population of step t is
// pulled by the node it streams to, or, at a wall, by the bounce-back and the
// specular terms of Eq. 20 (as adj_transpose_kernel).
template <class R>
__device__ __forceinline__ void transpose_at(const R* mu, int nx, int ny, int x, int y, R r, R rc, R (&o)[9]) {
    const int nn = nx * ny;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    auto M = [&](int i, int yy, int xx) -> R { return mu[i * nn + yy * nx + xx]; };
    o[0] = M(0, y, x);
    o[1] = M(1, y, xp);
    o[3] = M(3, y, xm);
    if (y == ny - 1) {
        o[2] = M(4, y, x);
        o[5] = r * M(7, y, x) + rc * M(8, y, xp);
        o[6] = r * M(8, y, x) + rc * M(7, y, xm);
    } else {
        o[2] = M(2, y + 1, x);
        o[5] = M(5, y + 1, xp);
        o[6] = M(6, y + 1, xm);
    }
    if (y == 0) {
        o[4] = M(2, 0, x);
        o[7] = r * M(5, 0, x) + rc * M(6, 0, xm);
        o[8] = r * M(6, 0, x) + rc * M(5, 0, xp);
    } else {
        o[4] = M(4, y - 1, x);
        o[7] = M(7, y - 1, xm);
        o[8] = M(8, y - 1, xp);
    }
}

template <class R>
__global__ void __launch_bounds__(kResThreads)
    adj_cl_backward_kernel(const R* ckpt, R* seg, size_t state_elems, int every, long long nsteps,
                           const R* lam_final, R* mu0, R* mu1, double* part, AdjConst<R> k) {
    __shared__ double red[kResThreads];
    const int nn = k.nx * k.ny, n9 = 9 * nn, nx = k.nx, ny = k.ny;
    const int rank = cluster_rank();
    const int g0 = rank * kResThreads + (int)threadIdx.x, gs = (int)gridDim.x * kResThreads;
    double gr = 0, ga = 0, gg = 0;
    const R* mu_next = nullptr;  // mu of step t + 1 (none before the first backward step)
    R* mu_cur = mu0;
    const long long nseg = (nsteps + every - 1) / every;
    for (long long s = nseg - 1; s >= 0; --s) {
        const long long t0 = s * every;
        const int len = (int)min((long long)every, nsteps - t0);
        const R* c = ckpt + (size_t)s * state_elems;
        for (int e = g0; e < n9; e += gs) seg[e] = c[e];
        cluster_barrier();
        for (int j = 1; j < len; ++j) {  // recompute the segment's states
            const R* a = seg + (size_t)(j - 1) * state_elems;
            R* b = seg + (size_t)j * state_elems;
            for (int node = g0; node < nn; node += gs) {
                R d[9];
                pull(a, nx, ny, node % nx, node / nx, k.r, k.rc, d);
                collide<R, MODE_PERIODIC>(d, k.ref, k.c);
                for (int i = 0; i < 9; ++i) b[i * nn + node] = d[i];
            }
            cluster_barrier();
        }
        for (int j = len - 1; j >= 0; --j) {
            const R* ft = seg + (size_t)j * state_elems;
            for (int it = g0; it < nn * kCols; it += gs) {
                const int node = it / kCols, col = it - node * kCols;
                const int x = node % nx, y = node / nx;
                R lam[9];
                if (mu_next) {
                    transpose_at(mu_next, nx, ny, x, y, k.r, k.rc, lam);
                } else {
                    for (int i = 0; i < 9; ++i) lam[i] = lam_final[i * nn + node];
                }
                R fb[9];
                pull(ft, nx, ny, x, y, k.r, k.rc, fb);
                const KC<Dual<R>> cd = dual_consts(k, col < 9 ? 0 : col - 8);
                Dual<R> d[9];
                for (int i = 0; i < 9; ++i) d[i] = Dual<R>(fb[i], i == col ? R(1) : R(0));
                collide<Dual<R>, MODE_PERIODIC>(d, Dual<R>(k.ref, R(0)), cd);
                if (col < 9) {
                    R m = 0;
                    for (int i = 0; i < 9; ++i) m += lam[i] * d[i].d;
                    mu_cur[col * nn + node] = m;
                    // dP/dr at the wall rows (Eq. 20)
                    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
                    auto at = [&](int i, int xx) -> double { return (double)ft[i * nn + y * nx + xx]; };
                    if (y == 0 && col == 5) gr += (double)m * (at(7, x) - at(8, xm));
                    if (y == 0 && col == 6) gr += (double)m * (at(8, x) - at(7, xp));
                    if (y == ny - 1 && col == 7) gr += (double)m * (at(5, x) - at(6, xp));
                    if (y == ny - 1 && col == 8) gr += (double)m * (at(6, x) - at(5, xm));
                } else {
                    double sum = 0;
                    for (int i = 0; i < 9; ++i) sum += (double)lam[i] * (double)d[i].d;
                    if (col == 9)
                        ga += sum;
                    else
                        gg += sum;
                }
            }
            cluster_barrier();
            mu_next = mu_cur;
            mu_cur = mu_cur == mu0 ? mu1 : mu0;
        }
    }
    gr = res_block_sum(gr, red);
    ga = res_block_sum(ga, red);
    gg = res_block_sum(gg, red);
    if (threadIdx.x == 0) {
        part[rank * 3 + 0] = gr;
        part[rank * 3 + 1] = ga;
        part[rank * 3 + 2] = gg;
    }
}

// Shared memory of the resident forward kernel: two states and the block sum.
size_t res_smem(int nx, int ny, size_t elem) {
    return ((2 * 9 * (size_t)nx * ny * elem + 15) / 16) * 16 + kResThreads * sizeof(double);
}
constexpr size_t kResSmemCap = 200 * 1024;

}  // namespace

struct clb_adjoint {
    int nx = 0, ny = 0, storage = 0;
    int64_t nsteps = 0;
    int every = 0;
    size_t elem = 0, state_elems = 0;
    void* ckpt = nullptr;  // checkpoints: state at steps 0, C, 2C, ...
    int nckpt = 0;
    void* seg = nullptr;   // one recomputed segment: C + 1 states
    void* lam[2] = {nullptr, nullptr};
    void* lam_final = nullptr;  // lambda_N = dJ/df_N, kept for every backward call
    void* mu = nullptr;
    double* acc = nullptr; // per-block partial sums [4][nb]: r, a, G and J
    int nb = 0;            // blocks of every adjoint launch
    bool resident = false; // resident engine: the forward pass in one block, the backward in one cluster
    int cluster = 0;       // blocks of the backward cluster (0: not yet launched)
    AdjConst<float> kf;
    AdjConst<double> kd;
    double J = 0;
    double g = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
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

template <class R> AdjConst<R>& kconst(clb_adjoint* h);
template <> AdjConst<float>& kconst<float>(clb_adjoint* h) { return h->kf; }
template <> AdjConst<double>& kconst<double>(clb_adjoint* h) { return h->kd; }

int blocks_for(size_t n, int t) { return (int)std::min<size_t>((n + t - 1) / t, 1024); }

template <class R> R* state_at(void* base, size_t state_elems, int64_t k) {
    return static_cast<R*>(base) + (size_t)k * state_elems;
}

// Copy the [4][nb] partial sums to the host and add each row in block order.
cudaError_t sum_partials(clb_adjoint* h, int rows, double* out) {
    std::vector<double> part((size_t)rows * h->nb);
    cudaError_t e = cudaMemcpyAsync(part.data(), h->acc, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < rows; ++k) {
        double v = 0;
        for (int b = 0; b < h->nb; ++b) v += part[(size_t)k * h->nb + b];
        out[k] = v;
    }
    return cudaSuccess;
}

template <class R> cudaError_t set_res_smem(size_t bytes) {
    return cudaFuncSetAttribute(adj_res_forward_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Both passes in one block each (resident engine).
template <class R> cudaError_t forward_resident(clb_adjoint* h) {
    const size_t smem = res_smem(h->nx, h->ny, sizeof(R));
    cudaError_t e = set_res_smem<R>(smem);
    if (e != cudaSuccess) return e;
    adj_res_forward_kernel<R><<<1, kResThreads, smem, h->stream>>>(
        static_cast<R*>(h->ckpt), h->state_elems, h->every, (long long)h->nsteps, static_cast<R*>(h->lam_final),
        h->acc, kconst<R>(h));
    e = cudaGetLastError();
    double J = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&J, h->acc, sizeof J, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) h->J = J;
    return e;
}

// Launch the cluster backward kernel with `cl` blocks (16 needs the
// non-portable cluster size, which the device may refuse).
template <class R> cudaError_t launch_cl_backward(clb_adjoint* h, int cl) {
    auto kern = adj_cl_backward_kernel<R>;
    if (cl > 8) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kResThreads);
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<const R*>(h->ckpt), static_cast<R*>(h->seg), h->state_elems,
                              h->every, (long long)h->nsteps, static_cast<const R*>(h->lam_final),
                              static_cast<R*>(h->lam[0]), static_cast<R*>(h->mu), h->acc, kconst<R>(h));
}

template <class R> cudaError_t backward_resident(clb_adjoint* h, double* out3) {
    // the largest cluster the device runs (16 blocks, else the portable 8)
    int cl = h->cluster;
    cudaError_t e = cudaSuccess;
    if (cl == 0) {
        cl = kClusterMax;
        e = launch_cl_backward<R>(h, cl);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cl = 8;
            e = launch_cl_backward<R>(h, cl);
        }
        if (e == cudaSuccess) h->cluster = cl;
    } else {
        e = launch_cl_backward<R>(h, cl);
    }
    double part[3 * kClusterMax];
    if (e == cudaSuccess) e = cudaMemcpyAsync(part, h->acc, 3 * cl * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    for (int q = 0; q < 3; ++q) {
        double v = 0;
        for (int r = 0; r < cl; ++r) v += part[r * 3 + q];  // rank order
        out3[q] = v;
    }
    return cudaSuccess;
}

template <class R> cudaError_t forward_run(clb_adjoint* h) {
    if (h->resident) return forward_resident<R>(h);
    const AdjConst<R>& k = kconst<R>(h);
    const int nb = h->nb;
    R* cur = state_at<R>(h->seg, h->state_elems, 0);
    R* nxt = state_at<R>(h->seg, h->state_elems, 1);
    cudaError_t e = cudaMemsetAsync(cur, 0, h->state_elems * sizeof(R), h->stream);  // f^eq(rho_out, 0)
    for (int64_t t = 0; t < h->nsteps && e == cudaSuccess; ++t) {
        if (t % h->every == 0)
            e = cudaMemcpyAsync(state_at<R>(h->ckpt, h->state_elems, t / h->every), cur, h->state_elems * sizeof(R),
                                cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) break;
        adj_forward_kernel<R><<<nb, kAdjThreads, 0, h->stream>>>(cur, nxt, k);
        e = cudaGetLastError();
        std::swap(cur, nxt);
    }
    if (e != cudaSuccess) return e;
    // final state and J, lambda_N (into lam_final)
    e = cudaMemsetAsync(h->acc, 0, (size_t)4 * nb * sizeof(double), h->stream);
    if (e == cudaSuccess) {
        adj_final_kernel<R><<<nb, kAdjThreads, 0, h->stream>>>(cur, static_cast<R*>(h->lam_final), h->acc, k);
        e = cudaGetLastError();
    }
    double hacc[4];
    if (e == cudaSuccess) e = sum_partials(h, 4, hacc);
    if (e == cudaSuccess) h->J = hacc[3];
    return e;
}

template <class R> cudaError_t backward_run(clb_adjoint* h, double seed, double grad[3]) {
    if (h->resident) {
        double hacc[3];
        cudaError_t e = backward_resident<R>(h, hacc);
        if (e != cudaSuccess) return e;
        grad[0] = seed * hacc[0];
        grad[1] = seed * hacc[1];
        grad[2] = seed * (hacc[2] - 0.5 * h->ny);
        return cudaSuccess;
    }
    const AdjConst<R>& k = kconst<R>(h);
    const int nb = h->nb;
    cudaError_t e = cudaMemsetAsync(h->acc, 0, (size_t)3 * nb * sizeof(double), h->stream);
    R* lam = static_cast<R*>(h->lam[0]);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(lam, h->lam_final, h->state_elems * sizeof(R), cudaMemcpyDeviceToDevice, h->stream);
    R* lam2 = static_cast<R*>(h->lam[1]);
    R* mu = static_cast<R*>(h->mu);
    for (int64_t s = (h->nsteps - 1) / h->every; s >= 0 && e == cudaSuccess; --s) {
        const int64_t t0 = s * h->every;
        const int64_t len = std::min<int64_t>(h->every, h->nsteps - t0);
        // recompute the segment's states t0 .. t0+len-1
        e = cudaMemcpyAsync(state_at<R>(h->seg, h->state_elems, 0), state_at<R>(h->ckpt, h->state_elems, s),
                            h->state_elems * sizeof(R), cudaMemcpyDeviceToDevice, h->stream);
        for (int64_t j = 1; j < len && e == cudaSuccess; ++j) {
            adj_forward_kernel<R><<<nb, kAdjThreads, 0, h->stream>>>(state_at<R>(h->seg, h->state_elems, j - 1),
                                                                     state_at<R>(h->seg, h->state_elems, j), k);
            e = cudaGetLastError();
        }
        for (int64_t j = len - 1; j >= 0 && e == cudaSuccess; --j) {
            adj_back_kernel<R><<<nb, kAdjThreads, 0, h->stream>>>(state_at<R>(h->seg, h->state_elems, j), lam, mu,
                                                                  h->acc, k);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
            adj_transpose_kernel<R><<<nb, kAdjThreads, 0, h->stream>>>(mu, lam2, k);
            e = cudaGetLastError();
            std::swap(lam, lam2);
        }
    }
    double hacc[3];
    if (e == cudaSuccess) e = sum_partials(h, 3, hacc);
    if (e != cudaSuccess) return e;
    // explicit dependence of J on G: u_x = sum e f / rho - G/2, summed over y
    grad[0] = seed * hacc[0];
    grad[1] = seed * hacc[1];
    grad[2] = seed * (hacc[2] - 0.5 * h->ny);
    return cudaSuccess;
}

template <class R> void fill_consts(AdjConst<R>& k, const SweepArgs& sa, const KC<R>& c, double dsv_da, double dsq_da,
                                    int nx, int ny) {
    k.c = c;
    k.dsv4_da = R(dsv_da / 4.0);
    k.dsq4_da = R(dsq_da / 4.0);
    k.r = R(sa.r);
    k.rc = R(1.0 - sa.r);
    k.ref = R(sa.ref0);
    k.nx = nx;
    k.ny = ny;
}

}  // namespace

extern "C" {

clb_status clb_adjoint_destroy(clb_adjoint* h) {
    if (!h) return CLB_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->dfree(h->ckpt);
    h->dfree(h->seg);
    h->dfree(h->lam[0]);
    h->dfree(h->lam[1]);
    h->dfree(h->lam_final);
    h->dfree(h->mu);
    h->dfree(h->acc);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return CLB_OK;
}

clb_status clb_adjoint_forward(int nx, int ny, double kn, double a, double r, double g, int64_t nsteps,
                               int checkpoint_every, const clb_opts* opts, clb_adjoint** out, double* J) {
    clb::TraceRange trace_("clb_adjoint_forward");
    if (!out) return (clb_status)set_error(CLB_EINVAL, "clb_adjoint_forward: out is NULL");
    *out = nullptr;
    clb_opts o;
    clb_opts_default(&o);
    if (opts) o = *opts;
    if (nx < 1 || ny < 1 || (long long)nx * ny > (1 << 22) || nsteps < 1 || !(kn > 0) || !(a >= 0) || r > 1 ||
        !std::isfinite(g) || !(o.rho_out > 0))
        return (clb_status)set_error(CLB_EINVAL, "clb_adjoint_forward: argument out of range");
    if (o.storage != CLB_FP64 && o.storage != CLB_FP32_SHIFTED)
        return (clb_status)set_error(CLB_EINVAL, "clb_adjoint_forward: storage must be FP64 or FP32-shifted");
    if ((o.alloc == nullptr) != (o.free == nullptr))
        return (clb_status)set_error(CLB_EINVAL, "clb_adjoint_forward: alloc and free hooks must be given together");
    clb_adjoint* h = new (std::nothrow) clb_adjoint;
    if (!h) return (clb_status)set_error(CLB_ENOMEM, "clb_adjoint_forward: host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->storage = o.storage;
    h->nsteps = nsteps;
    h->every = checkpoint_every > 0 ? checkpoint_every : (int)std::ceil(std::sqrt((double)nsteps));
    h->elem = o.storage == CLB_FP64 ? 8 : 4;
    h->state_elems = (size_t)9 * nx * ny;
    h->nckpt = (int)((nsteps + h->every - 1) / h->every);
    h->g = g;
    h->alloc = o.alloc;
    h->dealloc = o.free;
    h->alloc_ctx = o.alloc_ctx;
    // constants: s_v, s_q (Eq. 18, 21) and their derivatives with respect to a
    SweepArgs sa{};
    sa.s3 = o.s3;
    sa.s8 = o.s8;
    rates_at(kn, ny, a, o.b2, &sa.sv, &sa.sq);
    sa.rate_A = 1.0;
    sa.r = r >= 0 ? r : r_from_sigma(o.sigma);
    sa.gx = g;
    sa.ref0 = o.rho_out;  // stored values are deviations from w_i rho_out in both precisions
    sa.store_scale = 1.0;
    derive_constants(sa);
    const double c6 = std::sqrt(6.0 / 3.14159265358979323846) * ny;
    const double tau = c6 * kn / (1.0 + a * kn);
    const double dtau_da = -c6 * kn * kn / ((1.0 + a * kn) * (1.0 + a * kn));
    const double dsv_da = -sa.sv * sa.sv * dtau_da;
    const double dinvsq_dtau = -3.0 / (16.0 * tau * tau) + 3.14159265358979323846 * o.b2 / 4.0;
    const double dsq_da = -sa.sq * sa.sq * dinvsq_dtau * dtau_da;
    fill_consts(h->kf, sa, sa.kf, dsv_da, dsq_da, nx, ny);
    fill_consts(h->kd, sa, sa.kd, dsv_da, dsq_da, nx, ny);
    if (o.stream) {
        h->stream = static_cast<cudaStream_t>(o.stream);
    } else if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) == cudaSuccess) {
        h->own_stream = true;
    } else {
        cudaError_t e = cudaGetLastError();
        delete h;
        return (clb_status)set_error(CLB_ECUDA, "clb_adjoint_forward: stream: %s", cudaGetErrorString(e));
    }
    const size_t sb = h->state_elems * h->elem;
    h->ckpt = h->dalloc(sb * h->nckpt);
    h->seg = h->dalloc(sb * (h->every + 1));
    h->lam[0] = h->dalloc(sb);
    h->lam[1] = h->dalloc(sb);
    h->lam_final = h->dalloc(sb);
    h->mu = h->dalloc(sb);
    h->nb = blocks_for((size_t)nx * ny, kAdjThreads);
    // one block per pass when the grid fits in its shared memory, unless
    // opts->pipeline asks for one launch per step (1)
    h->resident = o.pipeline != 1 && res_smem(nx, ny, h->elem) <= kResSmemCap;
    h->acc = static_cast<double*>(h->dalloc(std::max<size_t>(4 * (size_t)h->nb, 3 * kClusterMax) * sizeof(double)));
    if (!h->ckpt || !h->seg || !h->lam[0] || !h->lam[1] || !h->lam_final || !h->mu || !h->acc) {
        clb_adjoint_destroy(h);
        return (clb_status)set_error(CLB_ENOMEM, "clb_adjoint_forward: device allocation failed");
    }
    cudaError_t e = h->storage == CLB_FP64 ? forward_run<double>(h) : forward_run<float>(h);
    if (e != cudaSuccess) {
        clb_adjoint_destroy(h);
        return (clb_status)set_error(CLB_ECUDA, "clb_adjoint_forward: %s", cudaGetErrorString(e));
    }
    if (J) *J = h->J;
    *out = h;
    return CLB_OK;
}

clb_status clb_adjoint_backward(clb_adjoint* h, double seed, double grad[3]) {
    clb::TraceRange trace_("clb_adjoint_backward");
    if (!h || !grad) return (clb_status)set_error(CLB_EINVAL, "clb_adjoint_backward: NULL argument");
    cudaError_t e = h->storage == CLB_FP64 ? backward_run<double>(h, seed, grad) : backward_run<float>(h, seed, grad);
    if (e != cudaSuccess) return (clb_status)set_error(CLB_ECUDA, "clb_adjoint_backward: %s", cudaGetErrorString(e));
    return CLB_OK;
}

// Q = J / (3 G ny^2 sqrt(1/6)): the normalised flow rate of Sec. 3.1 with
// RT = 1/3, p = rho0 RT and F = rho0 G.
static double q_norm_of(const clb_adjoint* h) { return 3.0 * h->g * (double)h->ny * h->ny * std::sqrt(1.0 / 6.0); }

clb_status clb_adjoint_q(const clb_adjoint* h, double* q) {
    if (!h || !q) return (clb_status)set_error(CLB_EINVAL, "clb_adjoint_q: NULL argument");
    if (h->g == 0) return (clb_status)set_error(CLB_EINVAL, "clb_adjoint_q: Q is undefined for G = 0");
    *q = h->J / q_norm_of(h);
    return CLB_OK;
}

clb_status clb_adjoint_q_backward(clb_adjoint* h, double seed, double grad[3]) {
    clb::TraceRange trace_("clb_adjoint_q_backward");
    if (!h || !grad) return (clb_status)set_error(CLB_EINVAL, "clb_adjoint_q_backward: NULL argument");
    if (h->g == 0) return (clb_status)set_error(CLB_EINVAL, "clb_adjoint_q_backward: Q is undefined for G = 0");
    double dj[3];
    cudaError_t e = h->storage == CLB_FP64 ? backward_run<double>(h, 1.0, dj) : backward_run<float>(h, 1.0, dj);
    if (e != cudaSuccess) return (clb_status)set_error(CLB_ECUDA, "clb_adjoint_q_backward: %s", cudaGetErrorString(e));
    // dQ/dtheta = (dJ/dtheta) / norm, and for G also the normalisation's own -Q/G
    const double norm = q_norm_of(h), q = h->J / norm;
    grad[0] = seed * (dj[0] / norm);
    grad[1] = seed * (dj[1] / norm);
    grad[2] = seed * (dj[2] / norm - q / h->g);
    return CLB_OK;
}

}  // extern "C"
