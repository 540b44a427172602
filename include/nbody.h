/*
 * nbody.h -- C ABI of libnbody, the GB300 (sm_103a) differentiable
 * direct-sum N-body library.
 *
 * The method is the one of "Differentiable N-body code for Galactic Dynamics
 * Odisseo" (arXiv 2511.22468):
 *   - softened direct pairwise gravity, no tree or multipole (Sec. 1,
 *     "N-body codes"):  a_i = -G sum_j m_j (x_i - x_j) (|x_i - x_j|^2 + eps^2)^(-3/2)
 *   - external potential of MWPotential2014's NFW halo, Miyamoto-Nagai
 *     disk and power-law bulge (Sec. 2.2.1)
 *   - second-order Velocity-Verlet (kick-drift-kick) with a fixed number of
 *     steps (Sec. 2.2.1)
 *   - reverse-mode gradients of the final state with respect to the initial
 *     conditions, the time step (integration time), the particle masses and
 *     the potential's parameters (Sec. 2; the parameter vector of Sec. 2.2.1
 *     and Fig. 2)
 *   - the inference stages built on them: the mock-stream pipeline with a
 *     binned-density or point-cloud (MMD) loss, batched ensembles and grid
 *     searches (Sec. 2.2.1, Fig. 2), orbit fitting with its Fisher matrix
 *     (Sec. 2.2.2), and a neural surrogate (Sec. 3 outlook).
 *
 * Conventions for every call:
 *   - Return value: NBODY_OK (0) or a negative NBODY_E* code; no call exits,
 *     throws or traps.  nbody_strerror() names a code.
 *   - Layout: per-particle vectors are structure-of-arrays FP64, x[d*n + i]
 *     for d = 0, 1, 2 (3 x n doubles); masses are n doubles.
 *   - Pointers marked "host or device" may be either: the library copies
 *     through unified addressing (cudaMemcpyDefault).  Pinned host memory
 *     keeps copies asynchronous.
 *   - Stream: all device work of a context runs on the CUDA stream given to
 *     nbody_create (0 = legacy default stream).  Calls that return data to
 *     host memory synchronise that stream before returning; the others are
 *     asynchronous with respect to the host.
 *   - Ownership: the library owns the context and its device buffers
 *     (state, staging arrays, partial sums, tape); it never frees or keeps
 *     caller memory beyond the call.
 *   - A context is not thread-safe: one host thread at a time.
 *   - Requires an sm_103a device (GB300); eps must be > 0.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NBODY_API __attribute__((visibility("default")))
#else
#define NBODY_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define NBODY_OK 0
#define NBODY_EINVAL (-1)   /* bad argument: size, pointer, eps <= 0 ... */
#define NBODY_ENOMEM (-2)   /* device or host allocation failed */
#define NBODY_ECUDA (-3)    /* a CUDA runtime call failed */
#define NBODY_ETIMEOUT (-4) /* a bounded device wait expired */
#define NBODY_ENAN (-5)     /* a non-finite value appeared in the state */
#define NBODY_ESTATE (-6)   /* call out of order (e.g. vjp without a tape) */
#define NBODY_ENODEV (-7)   /* no usable sm_103a device */
#define NBODY_ESIZE (-8)    /* problem larger than a fixed-size buffer holds */

/* ---- external potential components (Sec. 2.2.1) ---- */
#define NBODY_EXT_NFW 1u /* NFW halo: Phi = -G M ln(1 + r/r_s) / r          */
#define NBODY_EXT_MN 2u  /* Miyamoto-Nagai: Phi = -G M / sqrt(R^2 + (a + sqrt(z^2 + b^2))^2) */
#define NBODY_EXT_BULGE 4u /* MWPotential2014's bulge (Sec. 2.2.1): density
                              rho_0 (r/r_1)^-alpha exp(-(r/r_c)^2) of total
                              mass M_b, a = -G M_b P(s, r^2/r_c^2) x / r^3,
                              P the regularised incomplete gamma function,
                              s = (3 - alpha)/2; 0 <= alpha < 2             */

/* ---- FP32 recentring origin of the pair sum ---- */
#define NBODY_CENTER_FIXED 0u /* origin = params.center for every step       */
#define NBODY_CENTER_GUIDE 1u /* origin follows a test particle started at
                                 (center, center_vel) in the external
                                 potential with the same steps             */

/* ---- tape modes ---- */
#define NBODY_TAPE_KEEP_LAST 0u /* the forward pass keeps the last segment's
                                   tape, so the reverse sweep recomputes
                                   every segment but the last             */
#define NBODY_TAPE_LEAN 1u      /* keep checkpoints only; the reverse sweep
                                   recomputes every segment               */

typedef struct nbody_params {
  double G;                 /* gravitational constant                        */
  double eps;               /* Plummer softening length, > 0                 */
  double dt;                /* time step; may be negative (backward orbit)   */
  int64_t checkpoint_every; /* K >= 1: integrate() records an adjoint tape
                               with a checkpoint every K steps; 0: no tape   */
  uint32_t ext_flags;       /* NBODY_EXT_NFW | NBODY_EXT_MN | NBODY_EXT_BULGE */
  uint32_t center_mode;     /* NBODY_CENTER_FIXED or NBODY_CENTER_GUIDE      */
  uint32_t tape_mode;       /* NBODY_TAPE_KEEP_LAST or NBODY_TAPE_LEAN       */
  uint32_t reserved;        /* must be 0                                     */
  double nfw_M;             /* NFW scale mass 4 pi rho_0 r_s^3               */
  double nfw_rs;            /* NFW scale radius                              */
  double mn_M;              /* disk mass                                     */
  double mn_a;              /* disk scale length                             */
  double mn_b;              /* disk scale height                             */
  double center[3];         /* FP64 origin subtracted before the FP32 pair
                               sum (fixed) or the guide's start position     */
  double center_vel[3];     /* guide start velocity (CENTER_GUIDE)           */
  double bulge_M;           /* bulge total mass M_b                          */
  double bulge_alpha;       /* bulge inner slope, 0 <= alpha < 2             */
  double bulge_rc;          /* bulge cut-off radius, > 0                     */
} nbody_params;

typedef struct nbody_ctx nbody_ctx; /* opaque, owned by the library */

/* Create a context for n >= 1 particles with the given parameters; work runs
 * on cuda_stream (a cudaStream_t, NULL = legacy default stream) of the
 * current device.  The state is zero until nbody_set_state.
 * Errors: EINVAL (n < 1, p NULL, eps <= 0, reserved != 0), ENODEV, ENOMEM. */
NBODY_API int nbody_create(nbody_ctx **out, int64_t n, const nbody_params *p,
                 void *cuda_stream);

/* Release every device buffer of the context; NULL is a no-op. */
NBODY_API void nbody_destroy(nbody_ctx *c);

/* Replace the parameters (same n).  Invalidates the tape and the cached
 * acceleration.  Errors: EINVAL. */
NBODY_API int nbody_set_params(nbody_ctx *c, const nbody_params *p);

/* Copy positions x (3 x n), velocities v (3 x n) and masses m (n) into the
 * context (host or device pointers; the caller keeps ownership).  Resets
 * the guide to params.center / center_vel and invalidates the tape.
 * Errors: EINVAL (NULL pointer), ECUDA. */
NBODY_API int nbody_set_state(nbody_ctx *c, const double *x, const double *v,
                    const double *m);

/* Copy the current state out (host or device pointers; either may be NULL).
 * Synchronises the context stream.  Errors: ECUDA. */
NBODY_API int nbody_get_state(nbody_ctx *c, double *x, double *v);

/* Advance k >= 0 kick-drift-kick steps of params.dt (Sec. 2.2.1) without
 * recording a tape.  Errors: EINVAL, ECUDA, ENAN (sticky, see get_status). */
NBODY_API int nbody_step(nbody_ctx *c, int64_t k);

/* Advance n_steps >= 1 steps and, when checkpoint_every > 0, record the
 * adjoint tape of exactly this call (checkpoints every K steps).  x_out and
 * v_out (host or device, may be NULL) receive the final state; when either
 * is given the call synchronises.  Errors: EINVAL, ENOMEM, ECUDA, ENAN. */
NBODY_API int nbody_integrate(nbody_ctx *c, int64_t n_steps, double *x_out,
                    double *v_out);

/* Reverse sweep of the last nbody_integrate call (Sec. 2, reverse-mode
 * gradients), discrete adjoint of the kick-drift-kick map with
 * recomputation of tape segments.  Inputs: xbar, vbar = dL/dx_T, dL/dv_T
 * (3 x n, host or device; NULL means zero).  Outputs (host or device):
 * x0bar, v0bar = dL/dx_0, dL/dv_0 (3 x n each, may be NULL); mbar_or_null
 * (n doubles, may be NULL) = dL/dm_j, the per-particle mass gradient
 * (costs four more FP32 operations per pair in the VJP kernel);
 * theta_bar (host, 4 doubles) = { dL/d dt,
 *                                 sum_j m_j dL/dm_j (common mass scale),
 *                                 dL/d nfw_M, dL/d mn_M }.
 * The state after the call is the final state of the integration.
 * Synchronises the context stream.
 * Errors: ESTATE (no tape), EINVAL, ECUDA, ENAN. */
NBODY_API int nbody_vjp(nbody_ctx *c, const double *xbar, const double *vbar,
              double *x0bar, double *v0bar, double *mbar_or_null,
              double theta_bar[4]);

/* Gradient of the same loss with respect to the parameters of the external
 * potential (Sec. 2.2.1; the first five are the parameter set of the Fisher
 * analysis, Sec. 2.2.2), from the last successful nbody_vjp of this context:
 * out (host, 6 doubles) = { dL/d nfw_M, dL/d nfw_rs, dL/d mn_M, dL/d mn_a,
 * dL/d mn_b, dL/d bulge_M }; zero for a component that is switched off.
 * Does not touch the GPU.  Errors: EINVAL (batch context), ESTATE (no
 * gradient yet). */
NBODY_API int nbody_potential_grad(nbody_ctx *c, double out[6]);

/* Diagnostics of the current state: out = { K = sum m v^2 / 2,
 * W_pair = -G sum_{i<j} m_i m_j / sqrt(r_ij^2 + eps^2),
 * W_ext = sum m Phi_ext(x), |P| = |sum m v| } (host).  The pair term uses
 * the FP32 pair kernel with FP64 accumulation.  Synchronises.
 * Errors: ECUDA. */
NBODY_API int nbody_energy(nbody_ctx *c, double out[4]);

/* Total momentum sum m v (host, 3 doubles).  Synchronises. */
NBODY_API int nbody_momentum(nbody_ctx *c, double out[3]);

/* Sticky device status of the context: NBODY_OK, or NBODY_ENAN when a
 * non-finite value was written to the state.  Synchronises. */
NBODY_API int nbody_get_status(nbody_ctx *c);

/* Static text for a status code. */
NBODY_API const char *nbody_strerror(int code);

/* Number of kernels this library has launched in the calling process
 * (all contexts); a monotonically increasing counter for accounting. */
NBODY_API int64_t nbody_launch_count(void);

/* ---- batched ensemble ---- */

/* Create a context holding n_sims >= 1 independent simulations of uneven
 * size: simulation s owns particles offsets[s] .. offsets[s+1]-1 (host
 * array of n_sims + 1 increasing values, offsets[0] = 0) and has its own
 * parameters p[s] (G, eps, dt, potential, centre; tape_mode must be 0;
 * checkpoint_every > 0 for every simulation, or for none, asks the runs to
 * record their trajectories for nbody_vjp_batch).  Every step runs one
 * persistent pair-force launch over all simulations (a work list of
 * (simulation, i-tile, j-chunk) items, largest first, taken through an
 * atomic counter) and one batched update; nbody_integrate replays the whole
 * step loop as one CUDA graph, captured on its first call for a given
 * step count.  On a batch context, nbody_set_params takes an array of
 * n_sims parameter sets; nbody_set_state / nbody_get_state use arrays laid
 * out 3 x offsets[n_sims] (simulations concatenated); the adjoint is
 * nbody_vjp_batch (nbody_vjp, nbody_energy, nbody_momentum and the timing
 * calls return EINVAL).
 * Errors: EINVAL, ENODEV, ENOMEM, ECUDA. */
NBODY_API int nbody_create_batch(nbody_ctx **out, int n_sims,
                                 const int64_t *offsets, const nbody_params *p,
                                 void *cuda_stream);

/* Discrete adjoint of a batch's last nbody_integrate (or nbody_step) run,
 * for every simulation at once (Sec. 2: the reverse of the kick-drift-kick
 * steps with the pair VJP and the external-field Hessian).  The run must
 * have recorded its trajectory (checkpoint_every > 0 when it ran): the
 * batch keeps positions and pair accelerations at every point and the
 * half-step velocities of every step in device memory, 72 B per particle
 * and step (a 1000-step run of 1024 simulations of 1000 particles: 75 GB),
 * so nothing is recomputed.  One persistent launch per point computes the
 * pair VJP of each work item's rows over its simulation's whole j-range
 * (FP32 within a tile, FP64 across tiles, in fixed order) and applies the
 * FP64 adjoint update to those rows; the sweep is captured once as a CUDA
 * graph per step count.  The FP32 copies of the cotangents staged for the
 * pair VJP are rescaled per simulation by an exact power of two (from the
 * simulation's largest |lambda| at the point before), so cotangents of any
 * FP64 size can be propagated.
 * xbar, vbar (3 x offsets[n_sims], the batch's layout; host or device;
 * either may be NULL for zero) are dL/dx_T, dL/dv_T; x0bar, v0bar (same
 * layout, may be NULL) receive dL/dx_0, dL/dv_0; theta_bar (host or device,
 * n_sims x 8, may be NULL) receives per simulation (dL/d dt, sum_j m_j
 * dL/dm_j, dL/dM_NFW, dL/dM_MN, dL/dr_s, dL/da_MN, dL/db_MN, dL/dM_bulge).
 * Synchronises.  Errors: EINVAL, ESTATE (no recorded run), ENOMEM, ECUDA,
 * ENAN. */
NBODY_API int nbody_vjp_batch(nbody_ctx *c, const double *xbar, const double *vbar,
                              double *x0bar, double *v0bar, double *theta_bar);

/* Launch-shape candidates of the batched pair kernel (threads per block,
 * i-particles per thread, j-chunk length). */
#define NBODY_NTUNE 8

/* Time every candidate on the batch's current positions (probe_steps whole
 * steps each: the pair pass and the update, fused into one launch when every
 * simulation takes one j-chunk, run with zero kick and no drift so that the
 * state is not advanced), select the fastest and return its index in *best
 * (may be NULL); ms (host, NBODY_NTUNE entries, may be NULL) receives the
 * time per step of each.  Batch contexts only.
 * Synchronises.  Errors: EINVAL, ENOMEM, ECUDA. */
NBODY_API int nbody_autotune(nbody_ctx *c, int64_t probe_steps, int *best,
                             double ms[NBODY_NTUNE]);

/* Select candidate `choice` (0 .. NBODY_NTUNE-1), e.g. from a cached
 * autotuning result; nbody_get_tuning returns the current one (or a
 * negative code).  Batch contexts only.  Errors: EINVAL, ECUDA. */
NBODY_API int nbody_set_tuning(nbody_ctx *c, int choice);
NBODY_API int nbody_get_tuning(nbody_ctx *c);

/* ---- launch shape of the pair kernels (single-system contexts) ---- */

/* Override the launch shape of the pair-force (vjp = 0) or pair-VJP
 * (vjp = 1) kernel: variant 0 = i-particles in registers and j-tiles in
 * shared memory (threads, per_thread in {128 x 4, 128 x 8, 256 x 4,
 * 256 x 2} forward, {256 x 2, 128 x 4, 128 x 2} VJP), variant 1 = j split
 * over the lanes of a warp (threads 256, per_thread 4 or 8 forward, 2 or 4
 * VJP); chunks = number of j-chunks (1..32), 0 = chosen to fill the GPU.
 * Results change only by the summation order.  Invalidates the tape and
 * the cached acceleration.  Errors: EINVAL. */
NBODY_API int nbody_set_pair_shape(nbody_ctx *c, int vjp, int variant,
                                   int threads, int per_thread, int chunks);

/* Current shape {variant, threads, per_thread, chunks} (host, 4 ints). */
NBODY_API int nbody_get_pair_shape(nbody_ctx *c, int vjp, int out[4]);

/* j-pairs per shared-memory tile of the tile variant (variant 0) of the
 * pair-force (vjp = 0) or pair-VJP (vjp = 1) kernel: the default (512
 * forward, 256 VJP) or 128, whose finer j-chunks suit small systems
 * (128-pair instances: forward 128 x {4, 2, 1} and 64 x {2, 4} threads x
 * per_thread, VJP 128 x {2, 1} and 64 x 2).  Call after nbody_set_pair_shape,
 * which restores the default; the chunk count is kept.  Results change only
 * by the summation order.  Invalidates the tape and the cached
 * acceleration.  nbody_get_pair_tile returns the current tile size.
 * Errors: EINVAL. */
NBODY_API int nbody_set_pair_tile(nbody_ctx *c, int vjp, int tile_pairs);
NBODY_API int nbody_get_pair_tile(nbody_ctx *c, int vjp);

/* Where the chunk sums of a tile-variant pair kernel split into chunks >= 2
 * are added up: mode 1 = by the block of each row tile that finishes last,
 * inside the pair kernel (the consumer then reads one slice); 0 = by the
 * consumer (the update or adjoint kernel reads every chunk's slice); -1 =
 * automatic (1 when chunks >= 8, the default).  Both add the slices in
 * ascending chunk order, so results are bitwise the same; only the time
 * differs.  vjp selects the pair-VJP kernel (1) or the pair-force kernel (0).
 * Errors: EINVAL. */
NBODY_API int nbody_set_pair_finish(nbody_ctx *c, int vjp, int mode);

/* Tune the pair-force and pair-VJP launch shapes of a single-system context
 * on its current state: every supported shape and tile size, each with the
 * chunk count chosen to fill the GPU and the nearest counts that split the
 * j-tiles evenly, and each with its chunk sums added in the pair kernel and
 * by the consumer (nbody_set_pair_finish), is timed together with a consumer
 * of its sums (the update kernel with a zero kick) over at least
 * probe_launches launches (about 2 ms of them); the fastest is kept.
 * fwd_best / vjp_best (host, 4 ints each, may be NULL) receive the chosen
 * {variant, threads, per_thread, chunks}.  The state is not advanced; the
 * tape and the cached acceleration are invalidated.  Synchronises.
 * Errors: EINVAL, ECUDA. */
NBODY_API int nbody_autotune_pair(nbody_ctx *c, int probe_launches,
                                  int fwd_best[4], int vjp_best[4]);

/* ---- per-kernel timing (CUDA events on the context stream) ---- */
#define NBODY_KCLASS_PAIR 0    /* pair-force kernel (forward and recompute)   */
#define NBODY_KCLASS_VJP 1     /* pair VJP kernel                             */
#define NBODY_KCLASS_UPDATE 2  /* kick-drift-kick update kernel               */
#define NBODY_KCLASS_ADJOINT 3 /* adjoint update kernel                       */
#define NBODY_KCLASS_FIELD 4   /* FP64 external field of a forward point (on a
                                  side stream beside the pair kernel)       */
#define NBODY_NKCLASS 5

/* Enable (1) or disable (0) event timing of the context's kernels: when
 * enabled, every launch of the classes above is bracketed by two CUDA
 * events recorded on the context stream, and the external field of a
 * forward point then runs on the context stream as well (not beside the
 * pair kernel), so that its events time the kernel alone.  Errors: EINVAL. */
NBODY_API int nbody_set_timing(nbody_ctx *c, int enable);

/* Sum of the event-timed durations (ms) and launch counts per class since
 * the previous call (or since timing was enabled), then reset.  ms and
 * launches are host arrays of NBODY_NKCLASS entries; launches may be NULL.
 * Synchronises the context stream.  Errors: EINVAL, ECUDA. */
NBODY_API int nbody_kernel_times(nbody_ctx *c, double ms[NBODY_NKCLASS],
                                 int64_t launches[NBODY_NKCLASS]);

/* Throughput probes of the units the kernels use, on the current device:
 * out = { scalar FP32 FMA TFLOP/s, packed f32x2 FMA TFLOP/s, FP64 FMA
 * TFLOP/s, MUFU rsqrt Gop/s, SM count, MUFU ex2 Gop/s } (host, 6
 * doubles).  Each probe runs 8 independent FMA (or MUFU) chains per thread
 * on 8 blocks of 256 threads per SM.  Synchronises.
 * Errors: ENODEV, ENOMEM, ECUDA. */
NBODY_API int nbody_peaks(double out[6], void *cuda_stream);

/* ---- stateless kernels (device pointers only, stream = cuda_stream) ---- */

/* Softened pair acceleration of n particles (Sec. 1), the FP32 hot loop:
 * positions are recentred on center (FP64, 3 doubles, host), rounded to
 * FP32 and summed in FP32 within a j-tile, in FP64 across tiles.
 * x (3 x n) and m (n) in device memory; acc (3 x n, device) receives a_i.
 * Allocates and frees scratch (cudaMallocAsync) on the stream.
 * Errors: EINVAL, ENOMEM, ECUDA. */
NBODY_API int nbody_pair_accel(int64_t n, const double *x, const double *m, double G,
                     double eps, const double center[3], double *acc,
                     void *cuda_stream);

/* External acceleration (NFW halo + Miyamoto-Nagai disk per p->ext_flags,
 * Sec. 2.2.1; G M included) at n >= 1 points x (3 x n SoA, host or device)
 * into acc (3 x n, host or device): the FP64 field the integrator kicks
 * with.  Only the potential fields of p are used (p->eps and p->dt must
 * still be valid).  Synchronises.  Errors: EINVAL, ENODEV, ENOMEM, ECUDA. */
NBODY_API int nbody_ext_accel(const nbody_params *p, int64_t n, const double *x,
                              double *acc, void *cuda_stream);

/* ---- the mock-stream pipeline (Fig. 2, Sec. 2.2.1) ---- */

/* Loss L(Theta), Theta = { t_end, M_Plummer, M_NFW, M_MN } (Sec. 2.2.1):
 *  1. the progenitor's present-day centre of mass (X0, V0) is integrated
 *     backward for t_end as a single particle in the NFW + MN potential
 *     (n_steps kick-drift-kick steps of -t_end/n_steps; Fig. 2 step 2);
 *  2. a unit Plummer sample (xhat, vhat) is scaled and shifted there:
 *     x = a xhat + X, v = sqrt(G M_Plummer / a) vhat + V, m = M_Plummer / n
 *     (Fig. 2 step 3);
 *  3. the n-body system is integrated forward n_steps steps of
 *     t_end/n_steps with pair forces and the potential (Sec. 2.2.1);
 *  4. positions are projected to sky angles seen from `observer` in the
 *     frame e1 = unit(X0 - observer), pole = unit((X0 - observer) x V0),
 *     phi1 = atan2(d.e2, d.e1), phi2 = asin(d.pole / |d|);
 *  5. a Gaussian-smoothed nb1 x nb2 histogram (sigma = half a bin, each bin
 *     receiving the normal-CDF mass between its edges, weights 1/n) is
 *     compared with a target: L = mean_b (rho_b - target_b)^2.
 * The paper compares point clouds with an MMD (Fig. 2 step 4); that loss is
 * selected with nbody_stream_set_target_cloud, the binned density with
 * nbody_stream_set_target. */
typedef struct nbody_stream_cfg {
  int64_t n;                /* progenitor particles, >= 1                    */
  int64_t n_steps;          /* steps of the orbit and of the n-body run      */
  int64_t checkpoint_every; /* adjoint checkpoint spacing K >= 1             */
  double G;                 /* gravitational constant                        */
  double eps;               /* softening length, > 0                         */
  double a_prog;            /* Plummer scale radius of the progenitor, > 0   */
  double nfw_rs;            /* NFW scale radius (fixed)                      */
  double mn_a, mn_b;        /* disk scale length and height (fixed)          */
  double X0[3], V0[3];      /* present-day centre of mass                    */
  double observer[3];       /* observer position                             */
  int32_t nb1, nb2;         /* histogram bins in phi1 and phi2, 1..64        */
  double phi1_lo, phi1_hi;  /* phi1 window (radians)                         */
  double phi2_lo, phi2_hi;  /* phi2 window (radians)                         */
} nbody_stream_cfg;

typedef struct nbody_stream nbody_stream; /* opaque, owned by the library */
typedef struct nbody_mmd nbody_mmd;       /* opaque, owned by the library */

/* Create the pipeline for a unit Plummer sample xhat, vhat (3 x n each,
 * host or device; copied).  The target starts at zero.
 * Errors: EINVAL, ENODEV, ENOMEM, ECUDA. */
NBODY_API int nbody_stream_create(nbody_stream **out,
                                  const nbody_stream_cfg *cfg,
                                  const double *xhat, const double *vhat,
                                  void *cuda_stream);

/* Replace the target density (nb1 * nb2 doubles, row-major [b1][b2], host
 * or device) and use the density loss of step 5.  Errors: EINVAL, ECUDA. */
NBODY_API int nbody_stream_set_target(nbody_stream *s, const double *target);

/* Use the point-cloud loss instead (the paper's comparison, Fig. 2 step 4):
 * L = MMD^2 between the final phase-space cloud (x_T, v_T) and a target
 * cloud tx, tv (3 x m each, host or device), with the standardisation and
 * bandwidths of nbody_mmd_create (declared below).  The gradient then flows
 * through both x_T and v_T.  Errors: as nbody_mmd_create. */
NBODY_API int nbody_stream_set_target_cloud(nbody_stream *s, int64_t m,
                                            const double *tx, const double *tv,
                                            const double *scale_or_null,
                                            int n_sigma, const double *sigma);

/* Run steps 1-5 at theta (host, 4 doubles, all > 0).  loss (host, may be
 * NULL) receives L; density (host or device, nb1 * nb2, may be NULL) the
 * histogram.  Records what nbody_stream_grad needs.  Synchronises.
 * Errors: EINVAL, ENOMEM, ECUDA, ENAN. */
NBODY_API int nbody_stream_forward(nbody_stream *s, const double theta[4],
                                   double *loss, double *density);

/* dL/dTheta at the theta of the last nbody_stream_forward (host, 4
 * doubles), by the discrete adjoint of every step: head, n-body reverse
 * sweep (nbody_vjp), Plummer shift and backward orbit.  Synchronises.
 * Errors: ESTATE (no forward), ECUDA, ENAN. */
NBODY_API int nbody_stream_grad(nbody_stream *s, double theta_bar[4]);

/* Steps 1-2 alone: the initial state at theta (host, 4 doubles) -- x0, v0
 * (3 x n) and m (n), device pointers -- and the recovered centre of mass
 * (host, 6 doubles: X, V; may be NULL).  Synchronises.
 * Errors: EINVAL, ECUDA. */
NBODY_API int nbody_stream_initial_state(nbody_stream *s, const double theta[4],
                                         double *x0, double *v0, double *m,
                                         double com[6]);

/* Tune the launch shapes of the pipeline's n-body kernels (as
 * nbody_autotune_pair) on the initial state at theta (host, 4 doubles).
 * The next nbody_stream_forward keeps the chosen shapes; a recorded forward
 * is dropped.  Synchronises.  Errors: EINVAL, ECUDA. */
NBODY_API int nbody_stream_autotune(nbody_stream *s, const double theta[4],
                                    int probe_launches);

/* Launch shape {variant, threads, per_thread, chunks} (host, 4 ints) of the
 * pipeline's pair-force (vjp = 0) or pair-VJP (vjp = 1) kernel, as chosen by
 * the default rule or by nbody_stream_autotune (see nbody_get_pair_shape).
 * Errors: EINVAL. */
NBODY_API int nbody_stream_get_pair_shape(nbody_stream *s, int vjp, int out[4]);

/* Steps 1-2 for `count` parameter vectors at once (host or device, count x 4
 * doubles, all > 0), one backward orbit per GPU thread: x0, v0 (device,
 * 3 x (count n) SoA, member b in columns b n .. b n + n - 1: the layout of
 * a batch context of count simulations of n particles), m (device,
 * count n) and com (host or device, count x 6, may be NULL).  The same
 * arithmetic as nbody_stream_initial_state.  Synchronises.
 * Errors: EINVAL, ENOMEM, ECUDA. */
NBODY_API int nbody_stream_initial_states(nbody_stream *s, int64_t count,
                                          const double *thetas, double *x0,
                                          double *v0, double *m, double *com);

/* Steps 4-5 alone: the histogram (nb1 * nb2, host or device) of positions x
 * (3 x n, device) and, when loss is not NULL, their loss against the target.
 * Does not change what nbody_stream_grad uses.  Synchronises.
 * Errors: EINVAL, ECUDA. */
NBODY_API int nbody_stream_head(nbody_stream *s, const double *x,
                                double *density, double *loss);

/* Release the pipeline; NULL is a no-op. */
NBODY_API void nbody_stream_destroy(nbody_stream *s);

/* ---- the pipeline for many parameter vectors at once ----
 *
 * The point-cloud form of the pipeline above for `count` parameter vectors
 * theta_b = (t_end, M_Plummer, M_NFW, M_MN) together, member b scored by
 * MMD^2 against its own target cloud: the gradient refinement of many grid
 * points or of many bootstrap realisations of the observation (Sec. 2.2.1).
 * Steps 1-2 run one thread per member; step 3 is one batch context of
 * count simulations of n particles (nbody_create_batch) recording its
 * trajectories, its reverse sweep nbody_vjp_batch; the MMD terms of all
 * members take one launch each way. */
typedef struct nbody_stream_batch nbody_stream_batch; /* opaque */

/* cfg as for nbody_stream_create (checkpoint_every and the histogram
 * fields are not used: the batch keeps whole trajectories); xhat, vhat the
 * unit Plummer sample (3 x n, host or device); the targets tx, tv (3 x
 * count m, target b in columns b m .. b m + m - 1, host or device), all
 * compared in the units `scale` (host, 6 standard deviations) with the
 * bandwidths sigma (host, n_sigma in 1..4).  1 <= count <= 65535.  Device
 * memory: about 72 B per particle and step for the recorded trajectories
 * (count n (3 n_steps + 2) x 24 B).  Errors: EINVAL, ENODEV, ENOMEM, ECUDA. */
NBODY_API int nbody_stream_batch_create(nbody_stream_batch **out,
                                        const nbody_stream_cfg *cfg, int64_t count,
                                        const double *xhat, const double *vhat, int64_t m,
                                        const double *tx, const double *tv,
                                        const double *scale, int n_sigma,
                                        const double *sigma, void *cuda_stream);

/* losses[b] = MMD^2 of member b's final cloud at thetas[b] (host or device,
 * count x 4) against target b, and when theta_bars is not NULL (host or
 * device, count x 4) its gradient dL_b/dtheta_b.  A member whose run or
 * gradient leaves the finite range gets loss +inf and a NaN gradient; the
 * members are independent, so the others are unaffected and the call still
 * succeeds.  When the reverse sweep raised the NaN flag but no member's loss
 * or gradient shows a non-finite value (the failure cannot be attributed to
 * a member), the call returns NBODY_ENAN.  The first call tunes the batch's
 * pair-kernel launch shape.  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA,
 * ENAN. */
NBODY_API int nbody_stream_batch_loss_grad(nbody_stream_batch *s, const double *thetas,
                                           double *losses, double *theta_bars);

/* The two parts of every gradient component of the last
 * nbody_stream_batch_loss_grad call with gradients, parts (host or device,
 * count x 8): parts[b][0..3] the n-body run's parts of dL/d(t_end, M_NFW,
 * M_MN) and the velocity scaling's part of dL/dM_Plummer (in the order t_end,
 * M_Plummer, M_NFW, M_MN), parts[b][4..7] the backward orbit's parts and the
 * masses' part; theta_bars[b][q] = parts[b][q] + parts[b][4 + q].  The parts
 * of t_end, M_NFW and M_MN cancel to first order (the centre of mass returns
 * to its present-day point), so each part is the well-conditioned quantity
 * to check.  Synchronises.  Errors: EINVAL, ESTATE (no gradient yet), ECUDA. */
NBODY_API int nbody_stream_batch_grad_parts(nbody_stream_batch *s, double *parts);

/* Release; NULL is a no-op. */
NBODY_API void nbody_stream_batch_destroy(nbody_stream_batch *s);

/* ---- maximum mean discrepancy between phase-space point clouds ----
 *
 * The paper's first inference method (Sec. 2.2.1; Fig. 2, step 4) compares
 * the simulated and the observed stream as point clouds with the MMD and
 * ranks the 10^4 points of its grid search by it.  A point is
 * q = (x, y, z, vx, vy, vz); coordinates are standardised per dimension,
 * u = (q - mu) / s, mu and s the target's mean and standard deviation (or
 * the caller's scale), and the kernel is
 *   k(a, b) = sum_l exp(-|u_a - u_b|^2 / (2 sigma_l^2)),  1 <= l <= 4.
 * The estimator is the biased V-statistic
 *   MMD^2 = 1/n^2 sum k(x, x') + 1/m^2 sum k(y, y') - 2/(n m) sum k(x, y).
 * Pair sums run in FP32 within 512-point tiles and in FP64 across tiles,
 * in fixed order (bitwise reproducible).  All arrays are FP64 SoA: a cloud
 * of c points is x (3 x c) and v (3 x c). */

/* Evaluator for clouds of n points against the target (tx, tv: 3 x m each,
 * host or device; copied and staged).  max_sets bounds the sets of one
 * batched call.  scale_or_null (host, 6) replaces the target's standard
 * deviations; sigma (host, n_sigma in 1..4, all > 0) are the bandwidths in
 * standardised units.  The target's own term is computed here, once.
 * Errors: EINVAL, ENODEV, ENOMEM, ECUDA. */
NBODY_API int nbody_mmd_create(nbody_mmd **out, int64_t n, int64_t max_sets,
                               int64_t m, const double *tx, const double *tv,
                               const double *scale_or_null, int n_sigma,
                               const double *sigma, void *cuda_stream);

/* MMD^2 of one cloud (x, v: 3 x n, host or device) into *loss (host), and
 * when xbar / vbar are not NULL its gradient dMMD^2/dx, dMMD^2/dv (3 x n
 * each, host or device).  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA,
 * ENAN. */
NBODY_API int nbody_mmd_eval(nbody_mmd *h, const double *x, const double *v,
                             double *loss, double *xbar, double *vbar);

/* MMD^2 of `sets` clouds at once (1 <= sets <= max_sets): x, v are 3 x
 * (sets * n) SoA, cloud b in columns b*n .. b*n+n-1 (the layout of a batch
 * context whose simulations all hold n particles); losses (host or device,
 * `sets` doubles).  One launch for all clouds.  Synchronises.
 * Errors: EINVAL, ENOMEM, ECUDA, ENAN. */
NBODY_API int nbody_mmd_eval_batch(nbody_mmd *h, int64_t sets, const double *x,
                                   const double *v, double *losses);

/* MMD^2 of each of `sets` clouds against each of `targets` other clouds of
 * m2 points (the bootstrap realisations of an observation, Sec. 2.2.1),
 * with this evaluator's standardisation and bandwidths (those of its own
 * target: MMD^2 depends on differences only, so every realisation is
 * compared in the same units).  x, v: 3 x (sets n) as in
 * nbody_mmd_eval_batch; ty, tv: 3 x (targets m2), target t in columns
 * t m2 .. t m2 + m2 - 1 (host or device); losses[t * sets + b] (host or
 * device, sets * targets doubles).  Every cloud's own term and every
 * target's own term is computed once; the cross terms take one launch per
 * group of targets.  1 <= sets, targets <= 65535.  Device scratch: 24 B
 * per point of the clouds and targets, and up to 256 MB of block sums;
 * allocated and freed by the call.  Synchronises.
 * Errors: EINVAL, ENOMEM, ECUDA, ENAN. */
NBODY_API int nbody_mmd_eval_cross(nbody_mmd *h, int64_t sets, const double *x,
                                   const double *v, int64_t targets, int64_t m2,
                                   const double *ty, const double *tv, double *losses);

/* The standardisation in use: mu and s (host, 6 each; either may be NULL). */
NBODY_API int nbody_mmd_target_stats(nbody_mmd *h, double mu[6], double scale[6]);

/* Release the evaluator; NULL is a no-op. */
NBODY_API void nbody_mmd_destroy(nbody_mmd *h);

/* ---- orbit fitting and the Fisher matrix (Sec. 2.2.2) ----
 *
 * The progenitor, a single particle, is integrated from its present-day
 * point (X0, V0) forward and backward with kick-drift-kick steps of dt in
 * the NFW + Miyamoto-Nagai field of theta = (M_NFW, r_s, M_MN, a_MN, b_MN),
 * projected onto the stream frame (e1 towards X0 from the observer, pole
 * along (X0 - observer) x V0): phi1, phi2 (rad), mu_phi1 cos phi2, mu_phi2
 * (mas/yr, relative to the observer's velocity), v_h (km/s); interpolated
 * linearly along phi1 at the observed phi1 values (an observation beyond
 * the arc's end takes the end point) and compared by
 *   chi^2 = sum_obs sum_q (model_q - obs_q)^2 / sigma_q^2,
 * q = (phi2, mu_phi1 cos phi2, mu_phi2, v_h).  The arc runs forward while
 * phi1 stays in [phi1_lo, phi1_hi] and increases, backward while it stays
 * in the window and decreases, at most t_max each way.  Derivatives are
 * exact (forward-mode dual numbers through orbit, projection and
 * interpolation) with respect to xi = ln theta.  One GPU thread per
 * parameter vector; all arithmetic FP64. */
typedef struct nbody_orbitfit_cfg {
  double G;                  /* gravitational constant                        */
  double X0[3], V0[3];       /* present-day progenitor position, velocity     */
  double observer[3];        /* observer position                             */
  double observer_vel[3];    /* observer velocity                             */
  double phi1_lo, phi1_hi;   /* window (rad), phi1_lo < 0 < phi1_hi           */
  double dt;                 /* step, > 0                                     */
  double t_max;              /* longest integration each way, >= dt           */
  double sigma[4];           /* errors of phi2 (rad), mu1, mu2 (mas/yr), v_h (km/s) */
} nbody_orbitfit_cfg;

typedef struct nbody_orbitfit nbody_orbitfit; /* opaque, owned by the library */

/* obs: n_obs rows (phi1, phi2, mu_phi1 cos phi2, mu_phi2, v_h), host, any
 * order (copied, sorted by phi1).  Errors: EINVAL, ENODEV, ENOMEM, ECUDA. */
NBODY_API int nbody_orbitfit_create(nbody_orbitfit **out, const nbody_orbitfit_cfg *cfg,
                                    int64_t n_obs, const double *obs, void *cuda_stream);

/* chi^2 at count parameter vectors theta (host, count x 5, all > 0) into
 * chi2 (host, count); grad (count x 5, may be NULL) = d chi^2 / d ln theta;
 * gn (count x 25, may be NULL) = the Gauss-Newton matrix
 * sum (dr/d ln theta)(dr/d ln theta)^T of the scaled residuals r (half the
 * Gauss-Newton Hessian of chi^2: the Fisher matrix of a Gaussian
 * likelihood).  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA. */
NBODY_API int nbody_orbitfit_eval(nbody_orbitfit *h, int64_t count, const double *theta,
                                  double *chi2, double *grad, double *gn);

/* Levenberg-Marquardt on ln theta from count starts at once (one GPU thread
 * each; max_iter in 1..10000): step (A + lambda diag A) delta = -grad/2,
 * lambda divided by 10 on success and multiplied by 10 on failure; stops
 * when an accepted step lowers chi^2 by less than 1e-10 of itself or when,
 * at lambda <= 1e-3, the step's predicted decrease -grad.delta/2 is below
 * 1e-6.  theta_lo, theta_hi (host,
 * 5 each, both or neither) bound the trial points (projection onto the box
 * in ln theta).  theta_out (count x 5), chi2_out (count), iters_out (count,
 * may be NULL), host.  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA. */
NBODY_API int nbody_orbitfit_lm(nbody_orbitfit *h, int64_t count, const double *theta0,
                                int max_iter, const double *theta_lo,
                                const double *theta_hi, double *theta_out,
                                double *chi2_out, int *iters_out);

/* Fisher matrix at theta: F = (1/2) d^2 chi^2 / d ln theta^2, exact
 * (second-order forward-mode dual numbers through orbit, projection and
 * interpolation); F_gn (may be NULL) the Gauss-Newton matrix at theta.  Both
 * host, 5 x 5 row-major.  Errors: EINVAL, ENOMEM, ECUDA. */
NBODY_API int nbody_orbitfit_fisher(nbody_orbitfit *h, const double *theta, double F[25],
                                    double F_gn[25]);

/* The model arc at theta: *n_pts rows (phi1, phi2, mu1, mu2, v_h) by
 * increasing phi1 into arc (host, max_pts x 5).  Errors: EINVAL, ESIZE
 * (*n_pts > max_pts; *n_pts is set), ENOMEM, ECUDA. */
NBODY_API int nbody_orbitfit_arc(nbody_orbitfit *h, const double *theta, int64_t max_pts,
                                 double *arc, int64_t *n_pts);

/* Release; NULL is a no-op. */
NBODY_API void nbody_orbitfit_destroy(nbody_orbitfit *h);

/* ---- density surrogate (the paper's outlook, Sec. 3: a neural network
 *      coupled to the solver) ---- */

/* y = W3 GELU(W2 GELU(W1 u + b1) + b2) + b3, GELU(z) = z Phi(z) with the
 * exact normal CDF, FP32 (the contractions on the tensor cores as three
 * TF32 products per FP32 product: a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi).  Parameters are one flat FP32 array in the order
 * W1 (h x in), b1 (h), W2 (h x h), b2 (h), W3 (out x h), b3 (out), weight
 * matrices row-major (one row per output unit).  Inputs u are (batch x in)
 * and outputs y, targets t (batch x out), row-major, in device memory.
 * Used to map the four stream parameters to a binned density and to
 * warm-start the simulator's gradient descent. */
typedef struct nbody_mlp nbody_mlp; /* opaque, owned by the library */

/* Create a network with the given widths for batches of at most max_batch
 * rows; parameters start at zero (set them with nbody_mlp_set_params).
 * Errors: EINVAL, ENODEV, ENOMEM. */
NBODY_API int nbody_mlp_create(nbody_mlp **out, int n_in, int n_hidden,
                               int n_out, int max_batch, void *cuda_stream);

/* Number of FP32 parameters (the length of the flat array). */
NBODY_API int64_t nbody_mlp_num_params(const nbody_mlp *m);

/* Copy the flat parameter array in or out (host or device pointers);
 * set_params also resets the Adam moments and step count.
 * Errors: EINVAL, ECUDA. */
NBODY_API int nbody_mlp_set_params(nbody_mlp *m, const float *params);
NBODY_API int nbody_mlp_get_params(nbody_mlp *m, float *params);

/* y = MLP(u) for `batch` rows (1 .. max_batch).  Errors: EINVAL, ECUDA. */
NBODY_API int nbody_mlp_forward(nbody_mlp *m, const float *u, int batch,
                                float *y);

/* Mean squared error L = mean (MLP(u) - t)^2 over batch x out, and its
 * gradients: with respect to the parameters (kept inside the network for
 * nbody_mlp_adam_step and copied to grads, device, when not NULL) and to
 * the inputs (du, device, batch x in, when not NULL).  loss (host) may be
 * NULL.  Synchronises when loss is requested.  Errors: EINVAL, ECUDA. */
NBODY_API int nbody_mlp_loss_grad(nbody_mlp *m, const float *u, const float *t,
                                  int batch, float *loss, float *grads,
                                  float *du);

/* One Adam update (Kingma & Ba, bias-corrected) of every parameter with the
 * gradient of the last nbody_mlp_loss_grad.  Errors: EINVAL, ESTATE, ECUDA. */
NBODY_API int nbody_mlp_adam_step(nbody_mlp *m, float lr, float beta1,
                                  float beta2, float eps);

/* Invert the network: from `starts` initial inputs u (starts x n_in,
 * device; overwritten with the results) run `iters` Adam steps (learning
 * rate lr, inputs clamped to [lo, hi]) on each row's squared error
 * mean_o (MLP(u)_o - target_o)^2 against target (n_out, device).  loss
 * (device, starts floats, may be NULL) receives each row's final error.
 * Requires starts <= max_batch.  Errors: EINVAL, ECUDA. */
NBODY_API int nbody_mlp_invert(nbody_mlp *m, const float *target, int starts,
                               float *u, int iters, float lr, float lo, float hi,
                               float *loss);

/* Sticky device status of the network's tensor-core GEMMs: NBODY_OK, or
 * NBODY_ETIMEOUT when a bounded wait for the tensor cores' completion
 * expired (that GEMM's output was not written; each wait gives up after 1 s).
 * For failure-detection tests only, the environment variable
 * NBODY_MLP_TEST_NO_MMA=1 at nbody_mlp_create makes that network's GEMMs
 * issue no tensor-core work, so that every wait expires.  Synchronises the
 * network's stream.  Errors: EINVAL, ECUDA. */
NBODY_API int nbody_mlp_get_status(nbody_mlp *m);

/* Release the network; NULL is a no-op. */
NBODY_API void nbody_mlp_destroy(nbody_mlp *m);

/* ---- allocation-free variant (no counterpart in the paper) ---- */

/* Largest n accepted by nbody_pair_accel_noalloc. */
#define NBODY_NOALLOC_MAX_N 32768

/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they need forces -- an application
 * that reserves all of its device memory up front under a fixed budget, or
 * a hot loop that must not take the allocator's locks or pay its latency.
 *
 * Same result, kernels and launch shapes as nbody_pair_accel, but the
 * call makes no device allocation (no cudaMalloc, cudaMallocAsync or
 * cudaFree, no allocating library routine): its scratch is one 4 MiB
 * device array inside the library, which every GPU that loads the library
 * holds until the process exits.  x (3 x n), m (n) and acc (3 x n) are
 * caller-owned device memory; center is 3 host doubles, read by value
 * during the call (the caller may reuse them as soon as the call returns).
 *
 * - n must be in [1, NBODY_NOALLOC_MAX_N]; a larger n returns NBODY_ESIZE
 *   and launches nothing.
 * - The first call on a device looks up the device address of the array
 *   (cudaGetSymbolAddress) with that device current, and looks it up again
 *   after the device's context has been re-created (cudaDeviceReset); make
 *   that first call before any stream capture on the device.
 * - Asynchronous: acc is complete when cuda_stream reaches the end of the
 *   call.  Every call on a device shares the one array, so calls that may
 *   overlap on the GPU (issued to different streams without ordering)
 *   race and give undefined results; calls on one stream are safe.
 * Errors: EINVAL, ESIZE, ENODEV, ECUDA. */
NBODY_API int nbody_pair_accel_noalloc(int64_t n, const double *x,
                                       const double *m, double G, double eps,
                                       const double center[3], double *acc,
                                       void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* NBODY_H */
