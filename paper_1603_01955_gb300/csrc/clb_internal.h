// Internal interface between the host runtime (runtime.cu) and the sweep
// kernels (sweep.cu) of the CLB channel library.  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace clb {

enum : int { MODE_PERIODIC = 0, MODE_PRESSURE = 1 };

// Row kinds: the first / last row touches the bottom / top wall.  The kernels
// compute them from the row index (row_kind); the end columns' roles
// (pressure inlet / outlet, or the columns mirrored into the periodic halo
// columns -1 and nx so that the next sweep needs no wrap-around) follow from
// x = 0 and x = nx - 1 in the same way, so no node-type mask is stored.
enum : uint8_t { ROW_BOTTOM = 1, ROW_TOP = 2 };
__host__ __device__ __forceinline__ int row_kind(int y, int ny) {
    return (y == 0 ? ROW_BOTTOM : 0) | (y == ny - 1 ? ROW_TOP : 0);
}

// Launch constants in the compute type of a sweep, derived on the host so
// that no thread spends FP64 instructions on them (GB300's FP64 rate is a
// small fraction of its FP32 rate).
template <typename R> struct KC {
    R s3_12, s8_4;    // s3/12, s8/4
    R sv_4, sq_4;     // constant s_v/4, s_q/4 (body-force channel)
    R A, B, A316, CA; // pressure channel: tau = A/(rho+B); 3/(16A); (pi B2/4) A
    R hfx, hfy;       // F/2
    R fx, fy;         // F
    R r, rc;          // r_b, 1 - r_b
    R ref0, slope;    // deviation reference R(x) = ref0 + slope x
    R sha, shd;       // added to a value pulled from column x-1: -w slope (axis, diagonal)
    R drho_in, drho_out;
    R sc, isc;        // storage scale of the 16-bit formats and its inverse (1 otherwise)
};

// Everything one sweep launch needs (passed by value as a kernel argument).
struct SweepArgs {
    const void* fin;          // populations of the last step (post-collision)
    void* fout;               // populations written by this step
    int nx, ny;
    int pitch;                // elements per stored row
    int xoff;                 // element index of column 0 in a row (column -1 is xoff-1)
    long long plane;          // elements per direction plane (= ny * pitch)
    // collision (Eq. 7, 14, 18, 21)
    double s3, s8;
    double sv, sq;            // constant rates (body-force channel)
    double rate_A, rate_B;    // pressure channel: tau = A / (rho + B)
    double rate_C;            // pi * B2 / 4
    double r;                 // CBBSR bounce-back fraction (Eq. 20)
    double gx, gy;            // body force per unit mass (Eq. 9, 13)
    // Stored values are deviations f - w_i R(x) from a reference density
    // R(x) = ref0 + ref_slope * x (R = 0 for FP64 storage).
    double ref0, ref_slope;
    double drho_in, drho_out; // rho_in - R(0), rho_out - R(nx-1)
    double store_scale;       // stored value = deviation * store_scale (16-bit formats)
    // Centreline Knudsen number (pressure channel, Sec. 3.2): kn_mode 1 takes
    // the rates of column x from the centreline density of the last step,
    // rc_in[x] (rows yc0 and yc1, averaged), and the centre rows write this
    // step's densities to rc_out.  rc arrays hold 2 x rc_stride elements of
    // the compute type (one block per centre row).
    int kn_mode;
    int yc0, yc1;
    int rc_stride;
    const void* rc_in;
    void* rc_out;
    int withhold_tile;        // testing: TMA tile whose inputs are never sent (-1: none)
    int tile_order;           // TMA sweep: 0 = tiles from the first, 1 = from the last
    KC<float> kf;             // the constants above, derived, in FP32
    KC<double> kd;            // ... and in FP64
    // kf in the units of the stored values: every density-like constant times
    // the storage scale (a power of two, so exactly), sc = isc = 1.  The
    // TMA-staged sweeps collide the stored 16-bit values without unscaling
    // them; the collision is homogeneous in the densities, so the results are
    // the scaled results bit for bit.
    KC<float> ks;
};

// Fill a.kf, a.kd and a.ks from the double fields of a.
void derive_constants(SweepArgs& a);

// s_v (Eq. 18) and s_q (Eq. 21) at a Knudsen number, N = ny.
void rates_at(double kn, int ny, double a, double b2, double* sv, double* sq);

// r_b of Eq. 21 from the TMAC sigma, with B1 = 1 - 0.1817 sigma (Sec. 3).
double r_from_sigma(double sigma);

// NVTX range over a host call of the library (Nsight timelines show the
// calls; without an attached tool the push and pop return at once).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Record a failure message for clb_last_error() and return st.
int set_error(int st, const char* fmt, ...);

// Launch one sweep.  storage: clb_storage value; mode: MODE_*; vec: nodes per
// thread along x; block_x: threads per block.
cudaError_t launch_sweep(int storage, int mode, int vec, int block_x, const SweepArgs& a,
                         cudaStream_t stream);

// True if (storage, vec) has a compiled sweep.
bool sweep_supported(int storage, int vec);

// The sweep with TMA-staged inputs (FP32 and 16-bit storage); variant picks
// the tile shape.  sched: two device counters, zero between launches (zero
// them once after allocation; each launch leaves them zero again).  *status
// collects error bits of bounded waits that expired.
cudaError_t launch_sweep_tma(int storage, int mode, int variant, const SweepArgs& a, cudaStream_t stream,
                             unsigned* sched, unsigned* status);
int tma_variant_count();

}  // namespace clb
