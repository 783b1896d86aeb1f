/*
 * clb.h - C ABI of the GB300 (sm_103a) hot path of the cascaded lattice
 * Boltzmann (CLB) method for 2D microchannel gas flow of Liu & He,
 * "Numerical modelling of microchannel gas flows in the transition flow
 * regime using the cascaded lattice Boltzmann method" (arXiv:1603.01955).
 *
 * One call of clb_step(sim, n) advances a straight channel by n time steps of
 * the fused D2Q9 stream-and-collide sweep:
 *   - streaming of the transformed populations fbar = f - S/2 (Sec. 2.1, Eq. 4-5);
 *   - the cascaded central-moment collision with its body-force source
 *     (Eq. 6-13), relaxation rates s3 = 1.1, s8 = 1.2 (Sec. 3);
 *   - a relaxation rate per node from the Bosanquet effective viscosity at the
 *     local Knudsen number (Sec. 2.2, Eq. 16-18; Sec. 3.2 Kn = Kn_out p_out/p);
 *   - combined bounce-back/specular-reflection walls (Eq. 20) with r_b and
 *     s6 = s7 = s_q of the modified second-order slip condition (Eq. 19, 21);
 *   - periodic inlet/outlet (Sec. 3.1) or pressure inlet/outlet columns
 *     rebuilt by linear extrapolation (Sec. 3.2).
 *
 * Geometry: nx nodes along the channel (x), ny across it (y).  The walls sit
 * half a cell below row 0 and above row ny-1, so H = ny (Eq. 18's N).
 *
 * Conventions for every entry point:
 *   - Device state is owned by the library; every host array is owned by the
 *     caller, and a NULL output pointer skips that output.
 *   - All device work is queued on the simulation's stream (the one given in
 *     clb_opts, or one the library creates).  clb_step does not synchronise;
 *     clb_observables, clb_get_state, clb_set_state and clb_sync do.
 *   - Nothing is thrown across the ABI.  Each call returns a clb_status;
 *     clb_last_error() gives a message for the last failure on the calling
 *     thread.
 *   - A simulation may be used from one host thread at a time.
 *   - A simulation (batch, adjoint handle) lives on the device that was
 *     current when it was created, as its stream and buffers do; make that
 *     device current before every call on it.  The library does not switch
 *     devices itself.  The TMA-staged sweep (clb_opts.pipeline >= 2) opts
 *     into its shared-memory size once per process, with the device current
 *     at its first launch; in a process that drives several devices a launch
 *     on another device may be refused (CLB_ECUDA), so give the channels there
 *     pipeline 1, or run one process per device.
 */
#ifndef CLB_H
#define CLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct clb_sim clb_sim; /* opaque */

typedef enum {
    CLB_OK = 0,
    CLB_EINVAL = 1,   /* a parameter is out of range or inconsistent */
    CLB_ENOMEM = 2,   /* device or host allocation failed */
    CLB_ECUDA = 3,    /* a CUDA call failed (message has the CUDA error) */
    CLB_ENUMERIC = 4, /* a NaN or Inf was seen in the fields */
    CLB_ETIMEOUT = 5, /* a bounded device wait gave up (TMA-staged sweep); the results are invalid */
    CLB_EIO = 6       /* a checkpoint file could not be written or read, or is not a valid checkpoint */
} clb_status;

typedef enum {
    CLB_DRIVE_BODY_FORCE = 0, /* periodic in x, constant body force G along x (Sec. 3.1) */
    CLB_DRIVE_PRESSURE = 1    /* pressure inlet/outlet, drive_value = p_in/p_out (Sec. 3.2) */
} clb_drive;

typedef enum {
    CLB_FP64 = 0,         /* populations stored and collided in FP64 (144 B per node update) */
    CLB_FP32_SHIFTED = 1, /* FP32 deviations f - w_i rho_ref(x), FP32 collision (72 B) */
    CLB_FP16_SCALED = 2,  /* FP16 deviations times a field scale 2^14, FP32 collision (36 B) */
    CLB_BF16_SCALED = 3   /* BF16 deviations (scale 1), FP32 collision (36 B) */
} clb_storage;

/* Optional settings; clb_opts_default() fills the paper's values (Sec. 3). */
typedef struct {
    double b2;      /* second-order slip coefficient B2 (Eq. 19, 21); 0.55 */
    double sigma;   /* TMAC sigma, used for r_b when r < 0 (Eq. 19, 21; B1 = 1 - 0.1817 sigma); 1.0 */
    double s3, s8;  /* free relaxation rates; 1.1, 1.2 */
    double rho_out; /* outlet density (pressure drive) or mean density (body force); 1.0 */
    int storage;    /* clb_storage; CLB_FP32_SHIFTED */
    int vec;        /* nodes per thread along x of the direct sweep: FP64 1|2 (default 1),
                       FP32 1|2|4 (default 1 below 196,608 nodes, else 4), 16-bit 4|8 (4);
                       0 = default */
    int block_x;    /* threads per block, a multiple of 32 in 32..256; 0 = default 128 */
    void* stream;   /* cudaStream_t to queue work on; NULL = a stream owned by the library */
    /* Device allocator hooks (e.g. a framework's caching allocator); both NULL
     * = cudaMalloc / cudaFree.  alloc returns NULL on failure. */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* alloc_ctx;
    /* How the sweep reads its inputs (FP32 and 16-bit storage; FP64 and
     * kn_mode 1 always 1): 0 = default (1 for channels below 2^20 nodes;
     * larger ones 2 for FP32_SHIFTED, 3 for FP16_SCALED and BF16_SCALED),
     * 1 = direct vector loads with warp shuffles (the only engine that vec and
     * block_x configure), 2..4 = staged through shared memory by TMA bulk
     * copies, tile shape 0..2 of the table in sweep_tma.cu (2: 512 consumer
     * threads x 2 nodes, 3 stages; 3: 128 x 4 nodes, 2 stages; 4: 256 x 4
     * nodes, 3 stages), tiles claimed dynamically by the blocks of a
     * persistent grid.  All give bit-identical results. */
    int pipeline;
    /* Local Knudsen number of a pressure channel (Sec. 3.2): 0 = from the
     * node's own pressure (default), 1 = from the centreline pressure p(x) of
     * the column, taken one step behind (middle row, or mean of the two middle
     * rows).  1 uses the direct-load sweep. */
    int kn_mode;
    /* Testing only: >= 0 makes the first TMA-staged sweep launch withhold the
     * inputs of that tile, so that its bounded waits expire and the next
     * clb_sync / clb_observables returns CLB_ETIMEOUT.  -1 (default) = off. */
    int test_withhold_tile;
    /* CUDA-graph replay of clb_step for channels whose sweeps are short
     * enough for launch overhead to matter: chunks of this many consecutive
     * sweeps are captured once (per buffer parity) and replayed.  0 =
     * default (64 for channels below 2^20 nodes, off above; off with the
     * testing option), < 0 = off, > 0 = chunk length.
     * Results are identical with or without replay. */
    int graph_steps;
} clb_opts;

void clb_opts_default(clb_opts* opts);

/*
 * Create a channel and set its initial state f = f^eq(rho_init(x), u = 0)
 * (Eq. 11), with rho_init = rho_out (body force) or linear from
 * rho_in = drive_value * rho_out at x = 0 to rho_out at x = nx-1 (pressure).
 *
 *   nx, ny      lattice nodes; nx >= 1 (body force) or nx >= 4 (pressure); 1 <= ny <= 65535
 *   kn          Knudsen number (body force) or outlet Knudsen number Kn_out (pressure), > 0
 *   a           Bosanquet rarefaction factor of Eq. 16 (the paper uses 2), >= 0
 *   r           bounce-back fraction r_b in [0, 1] of Eq. 20; r < 0 = Eq. 21 from opts->sigma
 *   drive       clb_drive
 *   drive_value G (lattice acceleration) or p_in/p_out (> 0)
 *   opts        NULL = defaults
 *   out         receives the new simulation; NULL on failure
 * Errors: CLB_EINVAL (ranges above), CLB_ENOMEM, CLB_ECUDA.
 */
clb_status clb_create(int nx, int ny, double kn, double a, double r, clb_drive drive,
                      double drive_value, const clb_opts* opts, clb_sim** out);

/* Advance n >= 0 time steps (Eq. 4-5 with the boundaries above).  Queued on
 * the stream, returns without waiting.  Errors: CLB_EINVAL (n < 0, sim NULL),
 * CLB_ECUDA (launch failure). */
clb_status clb_step(clb_sim* sim, int64_t n);

/* Scalars of the current state.  Densities and velocities are taken per node
 * from the populations of the last completed step (Eq. 12-13). */
typedef struct {
    double mass_flow;  /* m = mean over x of sum_y rho u_x (Sec. 3.2) */
    double q_norm;     /* Q = sum_y u_x / (F H^2 sqrt(RT/2)/p) (Sec. 3.1, body force),
                          or S = m / m_ns (Sec. 3.2, pressure; m_ns = no-slip isothermal flow
                          with the unreduced viscosity) */
    double u_slip;     /* u_x at the profile column extrapolated linearly from the first two
                          rows to each wall, mean of both walls */
    double residual;   /* |m(t) - m(t_prev)| / |m(t)| against the previous clb_observables
                          call; -1 on the first call */
    double total_mass; /* sum of rho over all nodes */
    double ux_max;     /* max_y u_x at the profile column (Sec. 3.2 u_x,max) */
    int64_t step;      /* time steps completed */
} clb_scalars;

/*
 * Observables (Sec. 3.1, 3.2), reduced on the GPU in FP64 and copied to host
 * arrays.  profile_col: column of the velocity profiles; -1 = outlet
 * (nx-1, pressure) or column 0 (body force).  Outputs (each may be NULL):
 *   s          scalars above
 *   ux_prof    [ny]  u_x(y) at profile_col
 *   uy_prof    [ny]  u_y(y) at profile_col
 *   p_centre   [nx]  centreline pressure p = rho/3 (middle row, or mean of the two middle rows)
 *   dp_nonlin  [nx]  (p_centre - p_l)/p_out, p_l = p_in - (p_in - p_out) x/(nx-1)
 *   m_of_x     [nx]  sum_y rho u_x per column
 * Synchronises the stream.  Errors: CLB_EINVAL, CLB_ECUDA, CLB_ENUMERIC (a
 * NaN/Inf density or velocity was found; outputs are still written).
 */
clb_status clb_observables(clb_sim* sim, int profile_col, clb_scalars* s, double* ux_prof,
                           double* uy_prof, double* p_centre, double* dp_nonlin, double* m_of_x);

/* Copy the populations out / in, as FP64 host arrays [9][ny][nx], index
 * (i*ny + y)*nx + x, holding the post-collision populations f~_i (Eq. 4) of
 * the last completed step, whatever the storage.  Direction i follows Eq. 1:
 * e0 = (0,0), e1..e4 = (1,0), (0,1), (-1,0), (0,-1), e5..e8 = (1,1), (-1,1),
 * (-1,-1), (1,-1).  Synchronises the stream.  A transient device buffer of
 * 72*nx*ny bytes is taken through the allocator for the copy. */
clb_status clb_get_state(clb_sim* sim, double* host_f);
clb_status clb_set_state(clb_sim* sim, const double* host_f);

/* Description of a simulation. */
typedef struct {
    int nx, ny;
    int pitch;            /* elements per stored row (includes halo and padding) */
    int storage;          /* clb_storage */
    int vec, block_x;     /* launch shape of the sweep */
    int drive;            /* clb_drive */
    double bytes_per_node;/* algorithmic HBM bytes per node update: 18 * element size (9 reads + 9 writes) */
    double sv, sq;        /* s_v, s_q (Eq. 18, 21) at Kn (body force) or Kn_out (pressure) */
    double r;             /* r_b in use */
    double kn, a, g, rho_in, rho_out;
    int64_t step;
    void* stream;         /* the cudaStream_t in use */
    int pipeline;         /* sweep engine in use: 1 direct loads, 2.. TMA-staged tile shape (see clb_opts) */
    int kn_mode;          /* local Knudsen number: 0 node pressure, 1 centreline pressure */
} clb_info_t;
clb_status clb_info(const clb_sim* sim, clb_info_t* info);

/* Wait for all queued work of the simulation.  CLB_ETIMEOUT if a sweep
 * recorded an expired wait since the last check. */
clb_status clb_sync(clb_sim* sim);

/* Release everything the simulation owns; NULL is accepted. */
clb_status clb_destroy(clb_sim* sim);

/* Message for the last failing call on this thread ("" if none). */
const char* clb_last_error(void);

/* ------------------------------------------------------------------------
 * Checkpoint and resume.  The paper has no counterpart; a long run (the
 * steady states of Sec. 3.2 take 1e5-1e6 steps) can stop and continue
 * unchanged.
 *
 * clb_save writes the channel's complete state to the file `path`
 * (created or replaced):
 *   - the problem statement (nx, ny, drive and its value, Kn, a, r_b in use,
 *     B2, sigma, s3, s8, rho_out, storage, kn_mode);
 *   - the step counter and the residual history of clb_observables;
 *   - the stored populations of the current time level, bit for bit in the
 *     storage format, halo columns included;
 *   - the centreline densities that the next step's rates use (kn_mode 1).
 * The layout is a 176-byte little-endian header, then the two payloads.  The
 * header holds the magic "CLBCKPT1", the version and the payload sizes, and a
 * 64-bit FNV-1a checksum over the payloads.  clb_save synchronises the stream.
 * The file is only as portable as the byte order: same-endian machines only.
 * Errors: CLB_EINVAL (NULL argument); CLB_ETIMEOUT (an earlier sweep gave
 * up, nothing written); CLB_ECUDA; CLB_EIO (the file cannot be written).
 *
 * clb_load creates a simulation from such a file.  Everything that defines
 * the problem comes from the file, including opts->storage, kn_mode, b2,
 * sigma, s3, s8 and rho_out, which are ignored.  Only the run-time options
 * are taken from `opts` (NULL = defaults): stream, allocator hooks, pipeline,
 * vec, block_x.  Stepping the loaded simulation gives, bit for bit, what
 * stepping the saved one would have given (every sweep engine computes the
 * same values).
 * Errors: CLB_EINVAL (NULL path or out); CLB_EIO (unreadable, truncated, bad
 * magic, version or checksum, or a layout this library version would not
 * create); CLB_ENOMEM / CLB_ECUDA as for clb_create.  *out is NULL on
 * failure.
 * ------------------------------------------------------------------------ */
clb_status clb_save(clb_sim* sim, const char* path);
clb_status clb_load(const char* path, const clb_opts* opts, clb_sim** out);

/* ------------------------------------------------------------------------
 * Batched Knudsen sweep (Sec. 3.1, Fig. 2): many periodic body-force channels
 * of uneven height and Knudsen number advanced together.  Each channel lives
 * in the shared memory of a thread block for many steps (one persistent
 * launch per chunk of steps, replayed from a CUDA graph), so the channel must
 * fit: 9 * nx * ny * element size <= 200 KB.  Every channel uses the same a,
 * r_b, G and opts (s3, s8, B2, sigma, rho_out); its rates s_v, s_q come from
 * its own Kn and ny (Eq. 18, 21).  The arithmetic per node is that of
 * clb_step on a periodic channel.
 *
 * Schedule: each channel is updated by a warp-aligned range of one block's
 * threads, each thread taking 1, 2, 4 or 8 nodes; unpacked, every channel has
 * a block of its own; packed, small channels share blocks (first fit by
 * decreasing width, within 200 KB of shared memory per block).  Every
 * schedule gives the same bits.
 * ------------------------------------------------------------------------ */
typedef struct clb_batch clb_batch; /* opaque */

/* n channels; nx[k], ny[k], kn[k] per channel (host arrays).  opts->storage
 * CLB_FP64 or CLB_FP32_SHIFTED; opts->block_x 0 = schedule autotuned on the
 * first clb_batch_step (or by clb_batch_tune), else that many threads per
 * block (32..512), one channel per block, nodes per thread the fewest of 1,
 * 2, 4, 8 that fit.  Initial state f^eq(rho_out, 0).
 * Errors: CLB_EINVAL, CLB_ENOMEM, CLB_ECUDA. */
clb_status clb_batch_create(int n, const int* nx, const int* ny, const double* kn, double a, double r, double g,
                            const clb_opts* opts, clb_batch** out);

/* Advance every channel n >= 0 steps (queued on the batch's stream). */
clb_status clb_batch_step(clb_batch* b, int64_t n);

/* Autotuner: time every feasible schedule (nodes per thread 1, 2, 4, 8,
 * each unpacked and packed) for 200 steps on a copy of the state and keep
 * the fastest; the state itself does not advance.  *block_x_out (may be NULL)
 * receives the chosen threads per block.  Synchronises. */
clb_status clb_batch_tune(clb_batch* b, int* block_x_out);

/* Use the schedule with nodes_per_thread (1, 2, 4 or 8) and packing
 * (0 = one channel per block, 1 = packed) instead of the tuner's choice.
 * Synchronises.  Errors: CLB_EINVAL (a value out of range, or a channel
 * needs more than 512 threads at that many nodes per thread). */
clb_status clb_batch_set_schedule(clb_batch* b, int nodes_per_thread, int packed);

/* The schedule in use (each output may be NULL): threads per block, nodes
 * per thread, blocks per launch, packed (0/1). */
clb_status clb_batch_schedule(const clb_batch* b, int* threads_per_block, int* nodes_per_thread, int* blocks,
                              int* packed);

/* Per-channel scalars into s[n] (mass_flow, q_norm = Q of Sec. 3.1, u_slip at
 * column 0, total_mass, step; residual and ux_max are not computed: -1, 0).
 * Synchronises.  CLB_ENUMERIC if a channel holds NaN/Inf. */
clb_status clb_batch_observables(clb_batch* b, clb_scalars* s);

/* Channel k's populations as FP64 host arrays [9][ny][nx] (layout of
 * clb_get_state).  Synchronises; takes a transient device buffer. */
clb_status clb_batch_get_state(clb_batch* b, int k, double* host_f);
clb_status clb_batch_set_state(clb_batch* b, int k, const double* host_f);

/* Block size in use, steps done, and the cudaStream_t (each may be NULL). */
clb_status clb_batch_info(const clb_batch* b, int* block_x, int64_t* step, void** stream);

/* Release everything; NULL is accepted. */
clb_status clb_batch_destroy(clb_batch* b);

/* ------------------------------------------------------------------------
 * Discrete adjoint of a periodic body-force channel (Sec. 3.1): the gradient
 * of the flow sum J = (1/nx) sum_{x,y} u_x after nsteps steps from
 * f^eq(rho_out, 0) with respect to r_b (Eq. 20), the Bosanquet factor a
 * (Eq. 16-18, 21: through s_v and s_q) and the body force G (Eq. 9, 13).
 * The normalised flow rate of Sec. 3.1 is Q = J / (3 G ny^2 sqrt(1/6)).
 * ------------------------------------------------------------------------ */
typedef struct clb_adjoint clb_adjoint; /* opaque */

/* Run the forward pass, keeping a checkpoint every checkpoint_every steps
 * (<= 0: ceil(sqrt(nsteps))), and return J.  opts->storage CLB_FP64 or
 * CLB_FP32_SHIFTED (states and adjoints in that precision; the parameter
 * sums are FP64).  r < 0 takes r_b from Eq. 21 with opts->sigma (the gradient
 * is still with respect to r_b).  Device memory: (ceil(nsteps/C) + C + 5)
 * states of 9 nx ny elements.  Synchronises.  nx * ny <= 2^22.
 * Engine: a grid whose two states fit in one block's shared memory
 * (2 * 9 nx ny elements <= about 200 KB: 2800 nodes in FP32) runs the
 * forward pass as one launch of one block and each backward pass as one
 * launch of an 8-block cluster; larger grids, or opts->pipeline = 1, use one
 * launch per step.  Both give the same states; the FP64 sums of J and of the
 * gradient are taken in different orders. */
clb_status clb_adjoint_forward(int nx, int ny, double kn, double a, double r, double g, int64_t nsteps,
                               int checkpoint_every, const clb_opts* opts, clb_adjoint** out, double* J);

/* grad[0..2] = seed * dJ/d(r_b, a, G), walking the checkpointed forward pass
 * backwards (recomputing each segment).  May be called repeatedly; the
 * parameter sums are taken per thread block and added in a fixed order, so
 * repeated calls give the same bits.  Synchronises. */
clb_status clb_adjoint_backward(clb_adjoint* h, double seed, double grad[3]);

/* The normalised flow rate of Sec. 3.1 after the forward pass,
 * Q = J / (F H^2 sqrt(RT/2) / p) with RT = 1/3, p = rho0 RT, F = rho0 G, H = ny,
 * that is Q = J / (3 G ny^2 sqrt(1/6)).  No device work.
 * Errors: CLB_EINVAL (NULL argument, or G = 0). */
clb_status clb_adjoint_q(const clb_adjoint* h, double* q);

/* grad[0..2] = seed * dQ/d(r_b, a, G): the adjoint gradient of J (as
 * clb_adjoint_backward) divided by the normalisation, and for G also the
 * normalisation's own term -Q/G.  May be called repeatedly; synchronises.
 * Errors: CLB_EINVAL (NULL argument, or G = 0), CLB_ECUDA. */
clb_status clb_adjoint_q_backward(clb_adjoint* h, double seed, double grad[3]);

/* Release everything; NULL is accepted. */
clb_status clb_adjoint_destroy(clb_adjoint* h);

/*
 * clb_observables_noalloc - the observables of clb_observables, computed from
 * populations the caller already holds in device memory, without allocating
 * anything.  The paper has no counterpart: this is a library convenience.
 *
 * Who needs it: callers that may not allocate device memory at the time they
 * want the numbers - for instance a program whose device memory is owned by
 * another runtime's allocator or fully budgeted in advance, where cudaMalloc
 * could fail or would stall every stream of the device.  Such a caller passes
 * its own input and output buffers; this call uses no cudaMalloc, cudaFree or
 * allocating library routine, and no allocator hook.
 *
 *   f_dev        device pointer to FP64 post-collision populations [9][ny][nx],
 *                index (i*ny + y)*nx + x (the layout of clb_get_state)
 *   nx, ny       1 <= nx <= 65536, 1 <= ny <= 4096; larger sizes are rejected
 *                with CLB_EINVAL and a message naming the limit
 *   drive, g, rho_in, rho_out, kn
 *                the problem statement needed by the scalars (as in clb_create:
 *                g is the body force, kn the (outlet) Knudsen number)
 *   profile_col  as in clb_observables
 *   stream       cudaStream_t to run on (NULL = legacy default stream); the call
 *                synchronises it before returning
 *   outputs      host arrays as in clb_observables (each may be NULL);
 *                s->residual and s->step are -1 (this call keeps no state)
 *
 * Scratch: a fixed device array of about 1.2 MB inside the library (enough for
 * the maximum sizes above), which every GPU that loads the library holds until
 * the process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  The address is kept for the life of the process:
 * after cudaDeviceReset (or anything else that destroys the device's primary
 * context) it is stale, so do not call this entry point on that device again.
 * All calls on a device share the array: calls that overlap on the GPU (from
 * several streams or threads at once) race and give wrong results; serialise
 * them.  The array keeps the last call's contents, and each call clears the
 * part it uses before reducing.
 * Errors: CLB_EINVAL, CLB_ECUDA, CLB_ENUMERIC (non-finite field, outputs written).
 */
clb_status clb_observables_noalloc(const double* f_dev, int nx, int ny, int drive, double g, double rho_in,
                                   double rho_out, double kn, int profile_col, void* stream, clb_scalars* s,
                                   double* ux_prof, double* uy_prof, double* p_centre, double* dp_nonlin,
                                   double* m_of_x);

/*
 * clb_peak_fma - the GPU's fused multiply-add throughput in FP32
 * (storage = CLB_FP32_SHIFTED) or FP64 (storage = CLB_FP64), in TFLOP/s
 * (2 FLOP per fused multiply-add), measured by a short microbenchmark on the
 * current device: every SM runs many independent chains of fused
 * multiply-adds.  The paper has no counterpart; it is the compute peak the
 * sweeps' measured FLOP rate is reported against.
 *   stream   cudaStream_t to run on (NULL = legacy default stream); the call
 *            synchronises it
 *   tflops   output (host)
 * Takes a few milliseconds (FP32) to some tens of milliseconds (FP64).
 * Errors: CLB_EINVAL (storage not FP32_SHIFTED or FP64, tflops NULL), CLB_ECUDA.
 */
clb_status clb_peak_fma(int storage, void* stream, double* tflops);

#ifdef __cplusplus
}
#endif
#endif /* CLB_H */
