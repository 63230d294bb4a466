/*
 * pml.h -- C ABI of the GB300 (sm_103a) implementation of the reflectionless discrete
 * perfectly matched layer of A. Chern, "A Reflectionless Discrete Perfectly Matched
 * Layer" (arXiv 1804.01390).
 *
 * What the library computes
 * -------------------------
 * The semi-discrete PML system eq:DiscretePML (Sec. 1.1.2, Eq. 3a-3c) on a periodic box
 * (the paper truncates the layer periodically, Sec. 1.1.3), written in first-order form
 * with V = dU/dt:
 *
 *   dU/dt     = V
 *   dV/dt     = sum_a (U(i+e_a) - 2U(i) + U(i-e_a)) / h^2
 *             + sum_a (sigma_a[i_a] Psi_a(i+e_a) - sigma_a[i_a - 1] Phi_a(i-e_a)) / h   + sources
 *   dPhi_a/dt = -(sigma_a[i_a-1] Phi_a(i-e_a) + sigma_a[i_a] Phi_a(i)) / 2 - (U(i+e_a) - U(i-e_a)) / (2h)
 *   dPsi_a/dt = -(sigma_a[i_a-1] Psi_a(i) + sigma_a[i_a] Psi_a(i+e_a)) / 2 - (U(i+e_a) - U(i-e_a)) / (2h)
 *
 * advanced in time by the classic four-stage Runge-Kutta method (RK4, Sec. 1.1.3).
 * Phi_a lives where sigma_a[i_a] != 0 and Psi_a where sigma_a[i_a - 1] != 0 (the support
 * statement after Eq. 3); elsewhere both are identically zero.
 *
 * Geometry
 * --------
 * Axis a has N[a] physical ("interior") vertices and a layer of w vertices on each side:
 * T[a] = N[a] + 2w vertices indexed 0..T[a]-1, periodic.  Physical vertices are
 * w..w+N[a]-1.  sigma_a[e] is edge-centred: it belongs to the edge (e, e+1 mod T[a])
 * (the vertical gap s_j of eq:VertexPositions; the factors of eq:IntroSolution).  The
 * depth of edge e in the layer is d_e = max(w-1-e, e-(w+N-1), 0).
 *
 * Dense field arrays exchanged through this ABI are row-major [T2][T1][T0] (x fastest),
 * of the context's precision (float for 32, double for 64).  In 2D T2 = 1.
 *
 * Conventions of every call
 * -------------------------
 *  - Every call returns a pml_status and never aborts; pml_last_error() gives text.
 *  - The caller owns every buffer it passes in.  "on_device" = 1 means the pointer is
 *    device memory of the context's device, 0 means host memory.
 *  - Work is enqueued on the CUDA stream given at creation.  Calls that return data to
 *    the host (pml_read_field with a host pointer, pml_norms, pml_sync) synchronise that
 *    stream; the others return as soon as the work is enqueued.  Errors of enqueued
 *    kernels are reported by the next synchronising call.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef PML_H_
#define PML_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pml_ctx pml_ctx;

typedef enum {
    PML_OK = 0,
    PML_EINVAL = 1,      /* invalid argument                                          */
    PML_ENOMEM = 2,      /* allocation failed or workspace too small                   */
    PML_ECUDA = 3,       /* a CUDA runtime/driver call failed                          */
    PML_ESTATE = 4,      /* call not valid in the context's current state              */
    PML_EUNSTABLE = 5,   /* dt beyond the RK4 stability limit sqrt(2/d) h              */
    PML_ENONFINITE = 6,  /* non-finite input (a source amplitude), or the periodic scan of
                            the state found a non-finite value (pml_set_check_interval)   */
    PML_ETIMEOUT = 7     /* a bounded device-side wait gave up (kernel error flag set) */
} pml_status;

typedef struct {
    int ndim;        /* 2 or 3                                                    */
    int64_t n[3];    /* physical (interior) vertices per axis; n[2] ignored in 2D */
} pml_grid;

enum {
    PML_SIGMA_CONSTANT = 0, /* sigma_max * [d_e > 0]             (Fig. HalfSpaceGauss)   */
    PML_SIGMA_POWER = 1,    /* sigma_max * (d_e / w)^order       (order 2: quadratic ramp) */
    PML_SIGMA_RANDOM = 2,   /* sigma_max * u_e * [d_e > 0], u_e = user[a][e] in [0,1)
                               (Fig. HalfSpaceRand)                                       */
    PML_SIGMA_USER = 3      /* sigma_a[e] = user[a][e] as given; must be >= 0, finite and
                               zero on the physical edges w-1 .. w+N-1                   */
};

typedef struct {
    int kind;                /* PML_SIGMA_*                                    */
    double sigma_max;        /* in units of 1/h times h, i.e. the paper's sigma */
    double order;            /* exponent of PML_SIGMA_POWER                     */
    const double *user[3];   /* host arrays of length T[a] for RANDOM / USER    */
} pml_sigma_profile;

/* fields of pml_read_field */
enum { PML_FIELD_U = 0, PML_FIELD_V = 1 };
#define PML_FIELD_PHI(a) (2 + 2 * (a))
#define PML_FIELD_PSI(a) (3 + 2 * (a))

/* flags of pml_create */
enum {
    PML_FLAG_ADJOINT = 1,    /* also allocate the adjoint state (pml_adjoint_*) */
    PML_FLAG_WALL = 2        /* end every axis with a reflecting wall instead of the periodic
                                wrap: U, V, Phi, Psi are zero at the vertices -1 and T[a]
                                (the layer backed by a reflecting boundary, Sec. 1.1.4).
                                sigma_a[T[a]-1] (the wrap edge) is set to 0. */
};

/*
 * Bytes of device workspace pml_create needs for this problem.  Pass a buffer of at
 * least that size (256-byte aligned, e.g. a torch uint8 tensor) to pml_create, or pass
 * NULL there to let the library cudaMalloc (and later cudaFree) it.
 */
pml_status pml_workspace_bytes(const pml_grid *grid, int pml_width, int precision, int flags,
                               size_t *bytes);

/*
 * Create a solver for eq:DiscretePML on the periodic box N + 2w (Sec. 1.1.3).
 *   grid       physical vertices per axis (2D or 3D)
 *   h, dt      grid spacing and RK4 time step; dt must satisfy dt <= sqrt(2/ndim) h, the
 *              RK4 stability limit of the undamped discrete wave equation (else
 *              PML_EUNSTABLE)
 *   pml_width  w >= 0 layer vertices per side (w = 0: plain periodic wave equation)
 *   profile    damping profile (see PML_SIGMA_*); applied on every axis
 *   precision  32 (FP32 state, FP32 arithmetic) or 64 (FP64)
 *   cuda_stream  cudaStream_t the library enqueues on (NULL = legacy default stream)
 *   workspace, workspace_bytes  caller-owned device buffer (see pml_workspace_bytes) or
 *              NULL/0 for library-owned memory
 *   flags      PML_FLAG_*
 * The state is zero after creation and the step counter is 0.
 */
pml_status pml_create(const pml_grid *grid, double h, double dt, int pml_width,
                      const pml_sigma_profile *profile, int precision, void *cuda_stream,
                      void *workspace, size_t workspace_bytes, int flags, pml_ctx **out);

/*
 * Set the state: U = u0, V = v0 (NULL -> 0), Phi = Psi = 0, step counter = 0
 * (the paper's runs start at rest in the layer, Sec. 1.1.3).  u0 / v0 are dense
 * T-grids of the context's precision (host memory for on_device = 0, else device).
 * Asynchronous on the context's stream; the clearing of the fields the copies do not fill
 * runs on a side stream the library creates at the first call, joined back before the
 * call's last work on the context's stream.
 */
pml_status pml_set_initial(pml_ctx *ctx, const void *u0, const void *v0, int on_device);

/*
 * Point sources: dV/dt(x_s) += amp[s] * g(t) with the Ricker wavelet
 * g(t) = (1 - 2 pi^2 f^2 (t - t_delay)^2) exp(-pi^2 f^2 (t - t_delay)^2), evaluated at the
 * RK4 stage times t_n, t_n + dt/2, t_n + dt (t_n = n dt).  coords: host [ns][ndim]
 * (x, y[, z]); each source must lie where no layer term reaches it within one step
 * (the interior run of every axis, see pml_query_layout), else PML_EINVAL.  ns = 0
 * removes all sources.  Not part of the paper (its runs are source-free).
 */
pml_status pml_set_sources(pml_ctx *ctx, int ns, const int64_t *coords, const double *amp,
                           double f_peak, double t_delay);

/*
 * Receivers: after every pml_step step k (counted from this call), U at each receiver
 * is written to trace_buf[k * nr + r] (device, context precision), for k < capacity.
 * nr = 0 removes the receivers.
 */
pml_status pml_set_receivers(pml_ctx *ctx, int nr, const int64_t *coords, void *trace_buf,
                             int64_t capacity);

/*
 * Advance n RK4 steps (asynchronous).  With a two-step kernel variant selected (see
 * pml_set_variant; 2D FP32 contexts), consecutive steps with no sources and no receiver
 * row to record advance two per pass (temporal blocking depth 2); the state after each
 * pair equals that of two single steps up to rounding (the first step's values near the
 * layer are then formed by the layer's operator form instead of the closed form).
 */
pml_status pml_step(pml_ctx *ctx, int64_t n);

/* Copy field PML_FIELD_* of the current state into a dense T-grid (host or device). */
pml_status pml_read_field(pml_ctx *ctx, int field, void *dst, int on_device);

/*
 * FP64 reductions over the physical window w..w+N-1 of every axis (synchronising):
 *   out[0] = E, the energy eq:Energy (Sec. 1.1.5):
 *            1/2 sum V^2 + 1/2 sum_i sum_a ((U(i+e_a) - U(i)) / h)^2
 *   out[1] = max |U|, out[2] = sqrt(sum U^2),
 *   out[3] = sqrt(sum (U - ref)^2), out[4] = max |U - ref|
 * ref: NULL, or a device FP64 array of the window shape [N2][N1][N0].
 */
pml_status pml_norms(pml_ctx *ctx, const double *ref, double out[5]);

/* Current step counter (number of RK4 steps since pml_set_initial). */
pml_status pml_get_step(const pml_ctx *ctx, int64_t *step);

/* Wait for all enqueued work and report any device-side error. */
pml_status pml_sync(pml_ctx *ctx);

/*
 * Failure detection.  The device-side error word of a context is sticky: once a kernel
 * has set it, every synchronising call reports it, until pml_set_initial or
 * pml_load_state replaces the state (and clears the word).
 *
 * pml_set_check_interval: every `steps` steps of pml_step (and of pml_adjoint_step, on
 *   the adjoint state) the library scans U and V of the current state for NaN and Inf
 *   (one read of both fields, about 0.05 % of the step time at the default); the first
 *   non-finite value makes the next synchronising call return PML_ENONFINITE, naming the
 *   field and the step.  A blow-up shows up in U or V within one step wherever it starts,
 *   since every Phi_a / Psi_a feeds dV/dt.  The scan runs when the step counter crosses a
 *   multiple of `steps`; 0 turns it off; the default is 1000.  Batches (pml_batch_step)
 *   do not scan.
 * pml_set_wait_limit: the limit in nanoseconds of every bounded device wait (a kernel
 *   waiting for its own tile copies; 0 restores the default of 2 s).  A wait that runs out
 *   records its site, lets the copies in flight land (0.1 s at most each) and ends its
 *   work; the next synchronising call returns PML_ETIMEOUT.  Limits below 1000 ns make
 *   every wait give up at once, which exercises that error path on purpose (for tests of
 *   a caller's error handling).  Takes effect for work
 *   enqueued afterwards; a batch keeps the limits its contexts had at pml_batch_create.
 */
pml_status pml_set_check_interval(pml_ctx *ctx, int64_t steps);
pml_status pml_set_wait_limit(pml_ctx *ctx, uint64_t ns);

/*
 * Integer layout tables of axis `axis` (host arrays of length T[axis]):
 *   phi_active[i] = sigma[i] != 0, psi_active[i] = sigma[i-1] != 0 (supports, Sec. 1.1.2)
 *   interior[i]   = 1 on the run of vertices where sigma vanishes on edges i-2..i+1, the
 *                   run containing the centre vertex: there one RK4 step of Eq. 3 equals
 *                   one RK4 step of eq:DiscreteWaveEquation, and the library uses its
 *                   interior (layer-free) kernel.
 * Any pointer may be NULL.
 */
pml_status pml_query_layout(const pml_ctx *ctx, int axis, uint8_t *phi_active,
                            uint8_t *psi_active, uint8_t *interior);

/* Edge-centred damping of axis `axis` as used (host, length T[axis], FP64). */
pml_status pml_query_sigma(const pml_ctx *ctx, int axis, double *sigma);

/*
 * Layer work items of a box, planned on the host without a GPU or a context.  The paper
 * has no counterpart: how the layer frame (every vertex outside the layer-free run of
 * pml_query_layout) is cut into work items is this library's choice; this query lets a
 * caller (or a test) inspect the items the layer kernels of such a box would take.
 *   grid, pml_width, profile, precision, flags  as for pml_create
 *   sm_count   streaming multiprocessors the plan assumes (2D frames that give fewer items
 *              than 8 per SM get proportionally shorter ones), >= 1
 *   which      0: the frame of one step (2D); 1 / 2: the first / second layer pass of a
 *              two-step block, the frames of the run shrunk by 6 / by 2 (2D FP32);
 *              3: the slab tiles of the 3D frame (3D FP32); 4: the items of this box in
 *              a batch's one-step layer launch (2D FP32)
 *   out        NULL or a host int32 array [cap][10]: x0, y0, z0 (region origin), xlo, xhi,
 *              ylo, yhi, zlo, zhi (inclusive output range; y (2D) and z (3D) ranges of
 *              the band across the periodic seam run past T - 1 and wrap), flags (bit a:
 *              the aux fields of axis a are active within the item's reach); the first
 *              min(cap, count) items are written
 *   count      number of items of the set
 * PML_EINVAL for invalid arguments or an item set that does not belong to the box.
 */
pml_status pml_plan_layer_items(const pml_grid *grid, int pml_width, const pml_sigma_profile *profile,
                                int precision, int flags, int sm_count, int which, int32_t *out, int64_t cap,
                                int64_t *count);

/*
 * Discrete adjoint of the RK4 scheme (the transpose of one step is P(dt A)^T =
 * P(dt A^T), A^T written out from the entries of Eq. 3).  Requires PML_FLAG_ADJOINT.
 *
 * pml_adjoint_reset: adjoint state := 0, adjoint clock := current forward step count,
 *   source-amplitude gradient accumulators := 0.
 * pml_adjoint_step: for k = 0..n-1, with m = adjoint clock:
 *     1. dJ/dU_m at the receivers += residual[k * nr + r] (device, context precision,
 *        [n][nr]; NULL = no injection)
 *     2. accumulate dJ/da_s of the step m-1 -> m
 *     3. adjoint state := P(dt A)^T adjoint state;  adjoint clock := m - 1
 *   For a misfit J = 1/2 sum_{m>=1} sum_r (U_m(x_r) - d_{m,r})^2 the residual row of
 *   step m is U_m(x_r) - d_{m,r}.  Afterwards, if grad_u is not NULL the U part of the
 *   adjoint state (dJ/dU at the adjoint clock) is copied to grad_u (device dense T-grid,
 *   context precision), and if grad_amp is not NULL the accumulated dJ/da (host, FP64,
 *   [ns]) is copied there (synchronising).
 *   With a two-step variant selected and neither a residual nor sources (nothing injected
 *   or accumulated between steps), the transposed steps advance two per pass, as pml_step
 *   does.
 */
pml_status pml_adjoint_reset(pml_ctx *ctx);
pml_status pml_adjoint_step(pml_ctx *ctx, int64_t n, const void *residual, void *grad_u,
                            double *grad_amp);
/*
 * Gradient of the receiver misfit with respect to the damping profile (not in the paper:
 * the derivative of eq:DiscretePML's sigma entries carried through the discrete adjoint
 * of the RK4 step).  Requires PML_FLAG_ADJOINT.
 *
 * From the current forward state (step s0) the call runs n RK4 steps, recording the
 * receiver traces as pml_step does (the receiver buffer needs n free rows), and forms
 *   J = 1/2 sum_{m=1..n} sum_r (U_{s0+m}(x_r) - target[(m-1) nr + r])^2
 * (target: device array [n][nr] of the context precision).  Alternatively `residual`
 * (same layout) gives dJ/dU_{s0+m}(x_r) directly, for any misfit of the traces; then
 * *misfit is set to 0.  With receivers exactly one of the two must be given; without
 * receivers both are ignored and the gradient is 0.
 * It then runs the adjoint backwards and accumulates, per step, sum over the four RK4
 * stages of kbar_i^T (dA/dsigma) Y_i, with Y_i the stage inputs of the forward step and
 * kbar_i the stage cotangents, in FP64.  Forward states are recomputed from checkpoints
 * taken every `interval` steps (0: ceil(sqrt(n))), so the call holds about
 * n/interval + interval + 7 states in device memory (cudaMalloc for its duration).  The
 * stage vectors are formed only where the contraction needs them: within three stencil
 * steps of the edges with nonzero sigma.  Periodic boxes and boxes with walls
 * (PML_FLAG_WALL: fields zero beyond the ends) alike.
 *
 * Outputs: grad_sigma (host FP64, T[0] + T[1] (+ T[2]) values, axis by axis, indexed by
 * edge): dJ/dsigma_a[e] with the supports of Phi/Psi held fixed; edges with sigma = 0
 * report 0.  *misfit = J.  grad_amp (optional, host FP64 [ns]): dJ/da_s.  Afterwards the
 * forward state is the one after step s0 + n (as after pml_step(n)) and the adjoint
 * state holds dJ/dy at step s0 (pml_adjoint_read_field(PML_FIELD_U) gives dJ/dU_{s0}).
 * Synchronising.
 */
pml_status pml_sigma_gradient(pml_ctx *ctx, int64_t n, const void *target, const void *residual,
                              int64_t interval, double *grad_sigma, double *misfit, double *grad_amp);
/* Device bytes pml_sigma_gradient(ctx, n, ..., interval, ...) allocates for its duration
 * (checkpoints, the states of one segment, six stage states and small tables), with the
 * context's current receivers. */
pml_status pml_sigma_gradient_bytes(const pml_ctx *ctx, int64_t n, int64_t interval, size_t *bytes);

/* Copy field PML_FIELD_* of the adjoint state into a dense T-grid (host or device). */
pml_status pml_adjoint_read_field(pml_ctx *ctx, int field, void *dst, int on_device);

/*
 * Checkpoints: the complete forward state (U, V, Phi_a, Psi_a in the library's padded
 * layout) plus the step counter.  pml_state_bytes gives the size; dst/src may be host or
 * device memory.
 */
pml_status pml_state_bytes(const pml_ctx *ctx, size_t *bytes);
pml_status pml_save_state(pml_ctx *ctx, void *dst, int on_device);
pml_status pml_load_state(pml_ctx *ctx, const void *src, int on_device);

/*
 * Kernel timing.  With enable = 1 every kernel the context launches is bracketed by CUDA
 * events recorded on the context's stream (kinds: 0 interior, 1 layer, 2 point kernels
 * for sources / receivers and the finiteness scan).  pml_profile_read synchronises, returns the summed
 * durations in milliseconds and the launch counts per kind, and clears them.
 */
pml_status pml_profile_enable(pml_ctx *ctx, int enable);
pml_status pml_profile_read(pml_ctx *ctx, double ms[3], int64_t launches[3]);

/*
 * Kernel variants and autotuning.  The layer-free (interior) kernel of a 2D context
 * exists in several shapes (columns per lane, rows per TMA box, pipeline depth,
 * resident CTAs per SM).  In 3D the variants are the kernels of the layer frame: 0 the
 * z-streaming tile kernel, 1 level passes, 2 (FP32 only, the default there) slab tiles
 * whose halo is 4 along axes with damping within reach and 2 along the others.  Variants 0 .. n1-1 advance one step per
 * pass; 2D FP32 contexts add variants n1 .. count-1 that advance two steps per pass
 * (temporal blocking depth 2, see pml_step), selecting one of those keeps the one-step
 * variant last selected for single steps and the adjoint.  pml_get_variant reports the
 * current one and how many exist; pml_set_variant selects one (synchronising);
 * pml_get_time_block reports the steps per pass of the current variant (1 or 2).
 * pml_autotune times every variant for `steps` steps on the current state (sources and
 * receivers are suspended while it runs; the state advances by
 * (steps + 2) * count steps, so tune before pml_set_initial), keeps the fastest (and the
 * fastest one-step variant for single steps), writes its index to *chosen and, if
 * times_ms is not NULL, each variant's milliseconds per step to times_ms[0..count-1].
 */
pml_status pml_get_variant(const pml_ctx *ctx, int *variant, int *count);
pml_status pml_set_variant(pml_ctx *ctx, int variant);
pml_status pml_get_time_block(const pml_ctx *ctx, int *depth);
pml_status pml_autotune(pml_ctx *ctx, int steps, double *times_ms, int *chosen);

/*
 * FP64 energy and norms of a dense field pair, computed without allocating any device
 * memory.  The paper has no counterpart: this serves callers that cannot allocate device
 * memory when they need the numbers, such as services that reserve all their memory at
 * start-up and must not allocate afterwards, or processes whose device memory is owned by
 * another allocator or capped by a fixed budget.
 *
 *   ndim, T      2 or 3 axes, T[a] vertices per axis; U, V are dense row-major
 *                [T2][T1][T0] device arrays of the given precision (32 or 64)
 *   wlo, whi     inclusive window per axis, 0 <= wlo <= whi < T
 *   h            grid spacing; ref: NULL or a device FP64 array of the window shape
 *   cuda_stream  stream the two reduction kernels run on; the call synchronises it
 *   out          host double[5]: the energy over the window,
 *                  1/2 sum_i (V(i)^2 + sum_a ((U(i + e_a) - U(i)) / h)^2),
 *                with the forward differences wrapping periodically at the box edge;
 *                max |U|, ||U||_2, ||U - ref||_2, max |U - ref|, exactly as pml_norms
 *                reports them
 *
 * The per-row partial sums live in one fixed array of this library's device memory
 * (16384 rows x 5 doubles, 640 KB, held on every device that uses it until the process
 * exits).  A window with more than 16384 rows (y extent times z extent) is rejected with
 * PML_EINVAL.  The array's device address is looked up once per device and context (again
 * after a device reset).  The call copies the results to host memory and synchronises the
 * stream, so it must never be made while that stream is being captured into a CUDA graph.
 * Every call reuses the same array and overwrites the partials it reads, so results never
 * mix across calls; but two calls whose kernels overlap on the GPU (other streams, other
 * host threads) race for it: serialise them.
 */
pml_status pml_norms_dense_static(int ndim, const int64_t *T, int precision, const void *U, const void *V,
                                  const int64_t *wlo, const int64_t *whi, double h, const double *ref,
                                  void *cuda_stream, double *out);

/*
 * Batched stepping of many independent 2D grids ("shots" of uneven sizes).  The paper
 * has no counterpart: each grid is an ordinary context (pml_create) and keeps its own
 * sizes, layer width, damping, h and dt; a batch advances all of them together with one
 * layer-kernel launch and one interior-kernel launch per step, both spanning every grid
 * (work items of all grids share one queue), and replays runs of 32 steps from a CUDA
 * graph it captures once per kernel variant.  Each step of each grid is the same RK4
 * step of Eq. 3 as pml_step computes.
 *
 * pml_batch_create: the contexts must all be 2D, of one precision, on one stream, and
 *   distinct; they must outlive the batch.  The batch allocates its own device tables
 *   (one descriptor of about 2.6 KB per grid plus the layer tile list) with cudaMalloc.
 * pml_batch_step: n steps of every grid (asynchronous on the contexts' stream).  All
 *   contexts must be at the same ping-pong parity (as after pml_set_initial, or after
 *   equal numbers of steps) and have no sources or receivers (PML_ESTATE otherwise).
 *   Each context's step counter advances by n; pml_step, pml_read_field, pml_norms and
 *   the rest keep working on each context between batch steps.
 * pml_batch_get_variant / pml_batch_set_variant / pml_batch_autotune: as for a single
 *   context, over the batched interior kernel's variants (columns per lane, rows per TMA
 *   box, pipeline depth, resident CTAs per SM, rows per work item); autotuning advances
 *   every grid by (steps + 2) * count steps.  FP32 batches add two-step variants (two
 *   steps per pass, as for a single context: a layer pass into each context's mid buffer,
 *   a second one from it, and the two-step interior kernel, all grids per launch; the graph
 *   then replays 16 pairs); an odd last step uses the one-step variant last selected.
 *   pml_batch_get_time_block reports the steps per pass of the current variant.
 * pml_batch_profile_enable / pml_batch_profile_read: event timing of every launch
 *   (kinds 0 interior, 1 layer); while enabled, steps are launched one by one without the
 *   graph and without overlap.
 * pml_batch_info: info[0] grids, info[1] interior work items, info[2] layer tiles,
 *   info[3] CTAs of the interior launch.
 * Errors of batch calls are described by pml_last_error(NULL).
 */
typedef struct pml_batch pml_batch;
pml_status pml_batch_create(int count, pml_ctx *const *ctxs, pml_batch **out);
pml_status pml_batch_step(pml_batch *batch, int64_t n);
pml_status pml_batch_get_variant(const pml_batch *batch, int *variant, int *count);
pml_status pml_batch_set_variant(pml_batch *batch, int variant);
pml_status pml_batch_get_time_block(const pml_batch *batch, int *depth);
pml_status pml_batch_autotune(pml_batch *batch, int steps, double *times_ms, int *chosen);
pml_status pml_batch_profile_enable(pml_batch *batch, int enable);
pml_status pml_batch_profile_read(pml_batch *batch, double ms[2], int64_t launches[2]);
pml_status pml_batch_info(const pml_batch *batch, int64_t info[4]);
void pml_batch_destroy(pml_batch *batch);

/*
 * Layer design (host only, no device work).  The amplitude factor of the residual wave a
 * layer lets back into the physical domain, from the one-edge decay rate rho of
 * eq:IntroDecayRate (Sec. 1.1.2) multiplied over the edges the wave crosses (Sec. 1.1.4):
 *   backed = 0: prod_e |rho(s_e, k, w)|            (a layer truncated periodically, as here:
 *                                                 the wave crosses every layer edge once)
 *   backed = 1: prod_e |rho(s_e, k, w)| / |rho(s_e, -conj(k), w)|   (a layer backed by a
 *                                                 reflecting wall, crossed there and back)
 * pml_residual_factor: sigma_h[e] = sigma * h of the m edges crossed; k h = kh_re + i kh_im
 * the wave number normal to the layer (traveling waves: kh_im = 0), omega_h = omega * h
 * (omega from the discrete dispersion relation (omega h)^2 = sum_a 4 sin^2(k_a h / 2)).
 * pml_design_width: the smallest w in 1..w_max for which the library's profile of `kind`
 * (PML_SIGMA_CONSTANT or PML_SIGMA_POWER with `order`, peak sigma_max * h = sigma_max_h)
 * keeps the factor at or below eps for every omega h in (0, omega_h_max] and incidence with
 * cos(theta) = Re(k)/omega in [cos_min, 1] (grazing waves are not damped at all, Sec. 1.1.4:
 * they take w / cos(theta) to cross the layer).  *w_out = -1 when none does;
 * *worst_out = the largest factor of the sweep at the returned (or last) width.
 */
pml_status pml_residual_factor(int m, const double *sigma_h, double kh_re, double kh_im, double omega_h,
                               int backed, double *factor);
pml_status pml_design_width(int kind, double sigma_max_h, double order, double cos_min, double omega_h_max,
                            double eps, int backed, int w_max, int *w_out, double *worst_out);

/*
 * Arithmetic peak of the current device, measured by the library's own kernel (the paper
 * has no counterpart: it is the denominator of the FP64 step's roofline, since that path
 * is bound by the FP64 pipe rather than by memory).  Every thread of 4 x 512-thread
 * blocks per SM runs eight independent fused multiply-add chains for `iters` iterations
 * (a positive multiple of 16) in `precision` (32 or 64); one warm-up launch, then one
 * timed launch bracketed by CUDA events on `cuda_stream` (synchronising).
 *   tflops  2 x FMAs / elapsed time, in 10^12 flop/s
 *   ms      elapsed time of the timed launch (may be NULL)
 * Allocates nothing.  Errors are described by pml_last_error(NULL).
 */
pml_status pml_fma_peak(int precision, void *cuda_stream, int64_t iters, double *tflops, double *ms);

void pml_destroy(pml_ctx *ctx);
const char *pml_last_error(const pml_ctx *ctx);
const char *pml_status_string(pml_status s);

#ifdef __cplusplus
}
#endif

#endif /* PML_H_ */
