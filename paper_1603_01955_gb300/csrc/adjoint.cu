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

template <class R> cudaError_t forward_run(clb_adjoint* h) {
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
    h->acc = static_cast<double*>(h->dalloc((size_t)4 * h->nb * sizeof(double)));
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
