/*
 * swkb.h -- C ABI of libswkb.so, a single-GPU (sm_103a) screened-WKB
 * propagator (Bruno & Maas, "WKB Across Caustics: The Screened-WKB Method").
 *
 * The library advances a 2-D Helmholtz field u(x, z) of the model problem
 * Laplace(u) + k^2 eps(x, z) u = 0 (Sec. 2, Eq. helmholtz_3D) from one flat
 * screen x = x_q to the next (Sec. 2, Eq. ray_bundle; Algorithm 1):
 *   (a) DFT of the screen field into plane-wave modes (Eqs. fft_eq, ifft_eq,
 *       fourier_psi), keeping |n| <= n_max;
 *   (b) each mode's ray family marched across the slab by classical RK4 on the
 *       characteristics of the eikonal / transport equations (Eqs. charsys,
 *       charsys_s, transport_xt) with x as the ray parameter; the amplitude is
 *       A = A0 sqrt(P0 / (P1 Z_s)), the corrected form of Eq.
 *       delta_psi_eq_jac (J = X_t Z_s - Z_t X_s, Delta psi = J_t / (2 J));
 *   (c) 4-point Lagrange interpolation of each mode's phase and amplitude from
 *       the ray landings onto the grid of the next screen (Eq.
 *       ray_bundle_q_plus_1);
 *   (d) the modal sum u(z_m) = sum_n A_n(z_m) exp(i k psi_n(z_m)).
 * Ground boundaries (Neumann / Dirichlet) use the paper's reflection (Sec.
 * 2.3): the library solves on the mirrored period and projects the field onto
 * even / odd functions after each screen.
 *
 * Conventions for every entry point:
 *   - No C++ exception crosses this boundary; every call returns swkb_status.
 *     On failure a message is available from swkb_last_error() (thread-local).
 *   - Inputs passed by pointer are copied before the call returns; the caller
 *     keeps ownership.  Outputs are written only when the call returns SWKB_OK
 *     (device outputs may have been overwritten in part on error).
 *   - Complex fields are complex128, interleaved (re, im) doubles.  A field on
 *     n_z points holds the values at z_m = z_a + m (z_b - z_a) / n_z,
 *     m = 0 .. n_z - 1 (for grounded domains: the physical half z >= z_a).
 *   - A plan is not thread-safe; use one plan per host thread.  The server
 *     (swkb_server_*) is thread-safe.
 *   - No entry point forks, traps or spins without a bound.
 */
#ifndef SWKB_H
#define SWKB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swkb_plan swkb_plan;      /* opaque, library-owned */
typedef struct swkb_server swkb_server;  /* opaque, library-owned */

typedef enum {
  SWKB_OK = 0,
  SWKB_ERR_INVALID_ARG = 1,  /* bad argument; nothing was changed            */
  SWKB_ERR_OOM = 2,          /* device memory could not be allocated          */
  SWKB_ERR_CAUSTIC = 3,      /* a ray family folded between two screens:
                                Z_s <= 0 or ray landings not increasing (the
                                Remark after Eq. ray_bundle_q_plus_1: choose a
                                smaller screen spacing)                      */
  SWKB_ERR_TURNING = 4,      /* eps - Q^2 <= 0 on a ray (turning point in x) */
  SWKB_ERR_RANGE = 5,        /* a ray left the permittivity table, or the
                                ghost rays did not cover the screen          */
  SWKB_ERR_CUDA = 6,         /* a CUDA runtime call failed                   */
  SWKB_ERR_TIMEOUT = 7,      /* a bounded wait gave up                       */
  SWKB_ERR_AGAIN = 8,        /* server queue full; retry later               */
  SWKB_NOT_READY = 9,        /* swkb_poll: request still in flight           */
  SWKB_ERR_CANCELLED = 10    /* request cancelled                            */
} swkb_status;

/* SWKB_BC_OPEN: the overlapping Fourier-continuation method of Sec. 2.2 (Eq.
 * ifft_eq_phi_patches): [z_a, z_b) is not periodic, the field must vanish
 * near both ends, and each screen expands it patch by patch (fc_patch grid
 * points per patch, fc_overlap shared by neighbours; see swkb_options). */
enum { SWKB_BC_PERIODIC = 0, SWKB_BC_NEUMANN = 1, SWKB_BC_DIRICHLET = 2, SWKB_BC_OPEN = 3 };
enum { SWKB_FP64 = 0, SWKB_MIXED = 1 };

/*
 * Permittivity eps(x, z) = n(x, z)^2 and its first two z-derivatives, sampled
 * on n_cols range columns x_cols[c] (non-decreasing; two equal positions
 * encode a jump: left limit first, then right limit) and n_p uniform nodes
 * z0_p + i dz_p.  Arrays are row-major [n_cols][n_p] float64, caller-owned,
 * copied by swkb_plan_create.  The library evaluates eps by quintic Hermite
 * interpolation in z (C^2) and linearly in x between the columns that bracket
 * x; at the start of a screen the right limit is taken, at its end the left.
 * For grounded domains (SWKB_BC_NEUMANN / _DIRICHLET) the table describes
 * z >= z_a only, must start at z0_p == z_a and must have eps_z == 0 there;
 * the library evaluates the reflected permittivity eps(z_a + |z - z_a|)
 * (Sec. 2.3).
 */
typedef struct {
  int32_t n_cols;
  const double* x_cols;
  int32_t n_p;
  double z0_p, dz_p;
  const double* eps;
  const double* eps_z;
  const double* eps_zz;
} swkb_profile;

/* Physical vertical extent [z_a, z_b), first screen x0, boundary condition. */
typedef struct {
  double z_a, z_b, x0;
  int32_t bc;
} swkb_domain;

typedef struct {
  int32_t precision;      /* SWKB_FP64 or SWKB_MIXED (FP32 arithmetic with an
                             FP64 range-phase carry)                          */
  double theta_max;       /* radians; keeps |n| <= floor(sin(theta_max) L/lambda) */
  int32_t n_max;          /* > 0 overrides theta_max                          */
  int32_t ray_stride;     /* R: one ray every R grid points (R | N_fft)       */
  int32_t rk4_steps;      /* N_t: RK4 steps per screen                        */
  double absorber_frac;   /* top absorber over this fraction of the height
                             (grounded domains only; 0 = off)                  */
  int32_t autotune;       /* 1: at plan creation, time the candidate launch
                             shapes (resummation tile and CTAs per SM, DFT
                             split) on the plan's buffers and keep the
                             fastest; cached per shape for the process       */
  void* cuda_stream;      /* cudaStream_t to run on; NULL = a library stream.
                             The plan also owns a second stream for the ray
                             march (unless SWKB_OVERLAP=0 or reuse_rays):
                             within every call it forks from this stream and
                             joins back into it, so results are ordered on
                             this stream as if one stream ran everything     */
  int32_t device;         /* CUDA device ordinal                              */
  int32_t reuse_rays;     /* 1: for a range-independent medium (one table
                             column) march the rays once per propagate call
                             and reuse them on every screen: the ray data
                             depend only on the medium slab, not on the
                             field, so results are identical (0 = march every
                             screen, the default)                             */
  int32_t planes;         /* P > 1 (dividing rk4_steps): allocate ray buffers
                             for P - 1 planes inside each screen, enabling
                             swkb_propagate_planes with up to P planes per
                             screen (0 or 1 = none)                           */
  /* Fixed launch shapes, e.g. those an autotuned plan reported in
     swkb_plan_info.  All three > 0 replaces the default and the autotuned
     shapes (autotune is then skipped): tile_points in {64, 128, 256, 512}
     and at most the summed period (n_fft, or n_fft / 2 when grounded);
     ctas_per_sm >= 1; fft_n1 a power of two, at most 64 and n_fft / 32.
     Otherwise SWKB_ERR_INVALID_ARG.  All three 0 = default or autotuned
     shapes.  The shapes change the launch layout and the order of some
     sums (the DFT split, the mode groups' partial sums), so fields differ
     between shapes by rounding only. */
  int32_t tile_points;    /* grid points per resummation tile                 */
  int32_t ctas_per_sm;    /* resummation CTAs per SM the mode groups target   */
  int32_t fft_n1;         /* DFT split N = fft_n1 * (N / fft_n1)              */
  /* SWKB_BC_OPEN only (ignored otherwise).  Patch p holds the grid points
     p (fc_patch - fc_overlap) .. p (fc_patch - fc_overlap) + fc_patch - 1;
     the patches must tile the n_z points exactly, with 2 <= fc_overlap,
     2 fc_overlap <= fc_patch, 16 <= fc_patch and fc_patch + 25 <= 2048.
     Each patch's samples are continued by FC-Gram (5 matching points, 25
     continuation points) to a sequence of N_p = fc_patch + 25 points whose
     DFT gives the patch's modes (kappa_n = 2 pi n / (k N_p dz), |n| <=
     floor(sin(theta_max) N_p dz / lambda) or n_max); the partition of unity
     S^p rises and falls over fc_overlap points (a C-infinity step), also at
     the interval's two ends; every ray of mode n launched at z_j carries
     sum_p S^p(z_j) w_n^p / N_p.  No absorber and no autotune; inner planes
     (swkb_propagate_planes) as for the other plans; swkb_debug_screen and the
     batch kernel refuse these plans. */
  int32_t fc_patch;
  int32_t fc_overlap;
} swkb_options;

typedef struct {
  int32_t n_fft;          /* N: period points (n_z, or 2 n_z when grounded)   */
  int32_t n_max, n_modes; /* kept modes n = -n_max .. n_max                   */
  int32_t n_rays;         /* N / R                                            */
  int32_t n_ghost;        /* ghost rays per side                              */
  int32_t n_rays_total;   /* n_rays + 2 n_ghost (per mode)                    */
  int32_t tile_points;    /* grid points per resummation tile                 */
  int32_t mode_groups;    /* mode groups of the resummation                   */
  int32_t march_modes;    /* modes whose rays are marched (grounded domains:
                             n >= 0 only -- mode -n is the mirror image)      */
  int32_t resum_points;   /* grid points summed per screen (grounded domains:
                             the physical half plus one tile)                 */
  int32_t fft_n1;         /* DFT split N = fft_n1 * (N / fft_n1)              */
  double dz, period;      /* grid spacing, period length                      */
  double eps_ref;         /* reference permittivity of the phase carry        */
  size_t device_bytes;    /* device memory held by the plan                   */
  int32_t medium_pieces;  /* FP32 plans: cubic pieces per permittivity-table
                             interval the march evaluates (0: the quintic
                             itself; always 0 for FP64 plans)                 */
  int32_t ctas_per_sm;    /* resummation CTAs per SM the mode groups target  */
  int32_t fc_patches;     /* SWKB_BC_OPEN: patches (else 0); n_fft is then n_z
                             rounded up to a multiple of 64 (the points the
                             rays cover and the sum runs over; the permittivity
                             table must cover their reach) and period the
                             patches' N_p dz */
  int32_t fc_period_points; /* SWKB_BC_OPEN: N_p = fc_patch + 25 (else 0)     */
} swkb_plan_info;

/* Fill *opt with defaults: FP64, theta_max 30 deg, R 1, N_t 8, no absorber. */
void swkb_options_default(swkb_options* opt);

/*
 * Build a plan: validates the arguments, derives the mode set and the ray
 * layout, uploads the permittivity table and allocates every device buffer
 * (all allocation happens here).  n_z physical points; screen_dx the screen
 * spacing.  The FFT length (n_z, or 2 n_z when grounded) must be a power of
 * two between 64 and 2^20 (SWKB_BC_OPEN: any n_z in [64, 2^20 - 256] that the
 * patches tile).  Returns SWKB_ERR_INVALID_ARG on bad shapes, on a
 * table that does not cover the rays' reach, or on a mode evanescent at the
 * reference permittivity.
 */
swkb_status swkb_plan_create(const swkb_profile* profile, double k, const swkb_domain* domain,
                             int32_t n_z, double screen_dx, const swkb_options* options,
                             swkb_plan** out);

swkb_status swkb_plan_get_info(const swkb_plan* plan, swkb_plan_info* info);

/*
 * Propagate: u0 on screen q0 (x = x0 + q0 dx) -> u_out on screen
 * q0 + n_screens.  u0 / u_out hold n_z complex128 values; with on_device = 0
 * they are host pointers (the library copies in and out), with on_device = 1
 * device pointers on the plan's stream.  When snapshot_every > 0, u_out holds
 * n_screens / snapshot_every consecutive fields (after screens q0 +
 * snapshot_every, q0 + 2 snapshot_every, ...) instead of the last one only.
 * Restarting from a returned field at the matching q0 gives the same result
 * as one longer call (checkpoint / resume).  Blocks until the plan's stream
 * has finished (the status of every ray is read back).
 */
swkb_status swkb_propagate(swkb_plan* plan, const double* u0, int32_t q0, int32_t n_screens,
                           double* u_out, int32_t snapshot_every, int32_t on_device);

/*
 * Fields between screens (Sec. 2.1: further interpolation points may be
 * added for visualisation).  Like swkb_propagate, but u_out receives
 * n_screens * planes fields of n_z complex128 values, rows ordered (screen,
 * plane): row (q - q0) planes + j - 1 is the field on x_q + j dx / planes,
 * j = 1..planes.  The last row of each screen is the screen's field (the
 * snapshot swkb_propagate returns, absorber applied); the rows before it are
 * the ray field inside the screen: the screen's modes, its rays stopped after
 * j rk4_steps / planes RK4 steps, interpolated and summed like the screen,
 * with the range phase of that plane and no absorber.  planes must divide
 * rk4_steps and be at most the plan's swkb_options.planes (1 always works).
 * Pointers and blocking as in swkb_propagate; runs without a CUDA graph.
 * Errors: SWKB_ERR_INVALID_ARG (NULL, counts, planes), the ray statuses of
 * swkb_propagate.
 */
swkb_status swkb_propagate_planes(swkb_plan* plan, const double* u0, int32_t q0,
                                  int32_t n_screens, int32_t planes, double* u_out,
                                  int32_t on_device);

/*
 * One screen with every intermediate exposed, for testing (host pointers;
 * any output may be NULL).  u_full: N complex128 values on the whole period
 * (z_lo + m dz; z_lo = 2 z_a - z_b when grounded; a grounded plan expects
 * the even (Neumann) or odd (Dirichlet) field every grounded screen carries,
 * and forms c_{-n} = +-c_n from it).  Outputs: c [n_modes]
 * complex128 mode coefficients w_n / N (step a); delta, r, a [n_modes]
 * [n_rays_total] float64 ray landing (grid units from z_lo), residual phase
 * r = psi - kappa_n (z - z_lo) and amplitude factor sqrt(P0 / (P1 Z_s))
 * (step b); u_next N complex128: the modal sum times the absorber, before the
 * reflection step (steps c, d).  Grounded plans march modes n >= 0 and sum
 * the physical half only: their rays of mode -n are returned as the mirror
 * images of mode n's (ray 0, which has no mirror partner, as NaN) and the
 * other half of u_next as the reflection of the physical half.
 */
swkb_status swkb_debug_screen(swkb_plan* plan, int32_t q, const double* u_full, double* c,
                              double* delta, double* r, double* a, double* u_next);

void swkb_plan_destroy(swkb_plan* plan);

/* Kernel kinds of the per-kernel accounting (swkb_plan_stats). */
enum {
  SWKB_KERNEL_INIT = 0,     /* field -> full period (extension)              */
  SWKB_KERNEL_REDUCE = 1,   /* partial sums, absorber, reflection            */
  SWKB_KERNEL_FFT = 2,      /* step (a), both FFT passes                     */
  SWKB_KERNEL_MARCH = 3,    /* step (b)                                      */
  SWKB_KERNEL_BRACKET = 4,  /* landing checks, tile brackets                 */
  SWKB_KERNEL_RESUM = 5,    /* steps (c) + (d)                               */
  SWKB_KERNEL_OUTPUT = 6,   /* full period -> n_z complex128                 */
  SWKB_KERNEL_KINDS = 7
};

typedef struct {
  uint64_t launches;                         /* kernel launches since reset    */
  uint64_t screens;                          /* screens advanced since reset   */
  uint64_t kernel_launches[SWKB_KERNEL_KINDS];
  uint64_t kernel_timed[SWKB_KERNEL_KINDS];  /* launches that were timed      */
  double kernel_ms[SWKB_KERNEL_KINDS];       /* device time of the timed
                                                launches per kind, from CUDA
                                                events recorded on the plan's
                                                stream around each of them     */
} swkb_plan_stats;

/* kinds: bit mask of kernel kinds (1 << SWKB_KERNEL_*; SWKB_TIME_ALL for
   every kind, 0 to stop) whose launches get CUDA events recorded around them
   on the plan's stream, accumulating per-kind device time; every >= 1 times
   one launch in `every` of each selected kind (each timed launch adds two
   event records to the stream).  Resets the counters.  With SWKB_TIME_SERIAL
   or'ed into kinds, swkb_propagate runs the ray march on the plan's stream
   as well (no second stream), so that each event pair brackets its own
   kernel alone instead of a kernel sharing the GPU with the march; the
   results are bit-identical either way. */
#define SWKB_TIME_ALL ((1 << SWKB_KERNEL_KINDS) - 1)
#define SWKB_TIME_SERIAL (1 << 30)
swkb_status swkb_plan_set_timing(swkb_plan* plan, int32_t kinds, int32_t every);
swkb_status swkb_plan_get_stats(const swkb_plan* plan, swkb_plan_stats* stats);

/*
 * Step (a) -- the pruned DFT of one screen field, c_n = w_n / N for
 * |n| <= n_max (FP64) -- without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, such as host frameworks that own and pre-partition all device
 * memory and forbid other allocators, or latency-critical loops in which an
 * allocation would synchronise the device and stall other work.
 *
 * u: device pointer, n_fft complex128 values of the screen field on its whole
 * period; c: device pointer, 2 n_max + 1 complex128 outputs (n = -n_max ..
 * n_max).  Both stay owned by the caller.  n_fft must be a power of two in
 * [64, 65536] and 1 <= n_max <= n_fft / 2 - 1; anything larger is rejected
 * with SWKB_ERR_INVALID_ARG, as are host pointers.  The call is asynchronous
 * on cuda_stream (NULL = the default stream).
 *
 * The working storage is a fixed set of file-scope device arrays (3 MB:
 * the pass-1 intermediate, the twiddles and one unit phase per mode, each
 * 65536 complex128 values) that every GPU loading this library holds until
 * the process exits.
 * The first call on a device performs a one-time set-up on that device (it
 * resolves the arrays' device addresses, initialises one of them and
 * synchronises the device); make that first call before any stream capture.
 * All calls on a device share the arrays and leave the last call's contents
 * in them (each call rewrites everything it reads, so nothing needs
 * clearing); calls that overlap on the GPU -- e.g. on two streams at once --
 * race on the arrays and must be serialised by the caller.
 */
swkb_status swkb_modes_noalloc(const double* u, int32_t n_fft, int32_t n_max, double* c,
                               void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching request loop.  Requests (each a whole
 * propagation job) are admitted while their device footprint fits the HBM
 * budget and a slot is free; every admitted request keeps its field and ray
 * state resident on the device and advances one screen per scheduler round,
 * interleaved with the other resident requests on separate streams, so that
 * requests of different sizes overlap on the GPU.  Arrivals wait in a FIFO.
 * ------------------------------------------------------------------------- */
typedef struct {
  const swkb_profile* profile;
  double k;
  const swkb_domain* domain;
  int32_t n_z;
  double screen_dx;
  const swkb_options* options;  /* cuda_stream is ignored (the server owns streams) */
  const double* u0;             /* host, n_z complex128, copied at submit     */
  int32_t q0, n_screens;
} swkb_request;

typedef struct {
  uint64_t submitted, completed, failed, rejected;
  int32_t resident, queued;
  size_t hbm_in_use;
} swkb_server_stats;

/* hbm_budget_bytes: device bytes the resident requests may hold; max_slots:
   requests resident at once; queue_cap: waiting requests (0 = unbounded). */
swkb_status swkb_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t queue_cap,
                               int32_t device, swkb_server** out);
/* Copies the request; SWKB_ERR_AGAIN when the queue is full; *ticket > 0. */
swkb_status swkb_submit(swkb_server* server, const swkb_request* req, uint64_t* ticket);
/* SWKB_NOT_READY while in flight; on completion copies the n_z complex128
   result to host u_out (may be NULL) and releases the ticket; a failed
   request returns its error status once.  timeout_ms < 0 waits without
   limit, 0 polls. */
swkb_status swkb_poll(swkb_server* server, uint64_t ticket, double* u_out, int32_t timeout_ms);
swkb_status swkb_cancel(swkb_server* server, uint64_t ticket);
swkb_status swkb_server_get_stats(swkb_server* server, swkb_server_stats* stats);
/* Cancels queued requests, waits for resident ones, frees everything. */
void swkb_server_destroy(swkb_server* server);

/* ---------------------------------------------------------------------------
 * Batched propagation in one persistent launch.  Many requests of uneven
 * size (frequency, N_z, range, medium) are advanced screen by screen by ONE
 * cooperative kernel launch (captured in a CUDA graph and replayed per run):
 * every step of every screen of every request (Algorithm 1: the ray march,
 * the two DFT passes, the landing brackets, the fused interpolation and modal
 * sum; the extension of the input before the first screen and the final
 * reduction and output) is a job of work items in one device queue, ordered
 * so that each job's producers come earlier; persistent CTAs claim items in
 * queue order and wait -- bounded -- on per-request counters of finished
 * items.  Rays depend on the medium only, so each request's march runs one
 * screen ahead of its field into three rotating ray buffers.  Each request
 * keeps its own plan's arithmetic, launch shapes and summation orders: its
 * field equals the one its plan computes alone, bit for bit.
 * ------------------------------------------------------------------------- */
typedef struct swkb_batch swkb_batch;   /* opaque, library-owned */

typedef struct {
  int32_t ctas_per_sm;    /* persistent CTAs per SM (0 = as many as fit)      */
  int32_t wait_limit_ms;  /* bound of every wait of a work item on its
                             producers (0 = 2000 ms); a wait that runs out
                             abandons the launch with SWKB_ERR_TIMEOUT       */
  int32_t device;         /* CUDA device ordinal                              */
  void* cuda_stream;      /* cudaStream_t to run on; NULL = a library stream */
} swkb_batch_options;

typedef struct {
  int32_t instances, precision;
  int32_t grid, ctas_per_sm, threads;   /* the persistent launch's shape      */
  int32_t jobs;                         /* jobs in the queue                  */
  int64_t items;                        /* work items over all jobs           */
  int32_t steps;                        /* screen steps (the longest request) */
  size_t shared_bytes;                  /* dynamic shared memory per CTA      */
  size_t device_bytes;                  /* device memory held by the batch    */
} swkb_batch_info;

/* Zeroes *opt (every field's default). */
void swkb_batch_options_default(swkb_batch_options* opt);

/*
 * Build a batch of n requests (swkb_request as for the server: profile,
 * wavenumber, domain, n_z, spacing, options, incident field u0 (host), q0,
 * n_screens >= 1).  All requests share one precision (options->precision);
 * each gets a plan with its own options (fixed launch shapes or autotune as
 * requested; reuse_rays and planes are ignored; fft_n1 must be >= 2), its
 * input field is copied to the device, and the batch allocates its queue,
 * counters and a third ray-buffer set per request.  Errors: those of
 * swkb_plan_create (message prefixed with the request index),
 * SWKB_ERR_INVALID_ARG (n < 1, NULL, mixed precisions, n_screens < 1),
 * SWKB_ERR_OOM, SWKB_ERR_CUDA.
 */
swkb_status swkb_batch_create(int32_t n, const swkb_request* reqs,
                              const swkb_batch_options* opt, swkb_batch** out);

/*
 * Run every request of the batch, each from its input field on screen q0 to
 * screen q0 + n_screens, in one persistent launch.  u_in: NULL (the fields
 * given at creation, or those of the last run's u_in) or the requests'
 * inputs concatenated in request order (sum of n_z complex128 values);
 * u_out: the outputs, concatenated the same way (NULL: not returned).  Both
 * are device pointers when on_device = 1, else host memory.  Blocks until
 * done.  Errors: SWKB_ERR_TIMEOUT (a wait ran out; nothing else is wrong
 * with the device, the batch can be run again), the ray statuses of
 * swkb_propagate (message prefixed with the request index), SWKB_ERR_CUDA.
 */
swkb_status swkb_batch_run(swkb_batch* batch, const double* u_in, double* u_out,
                           int32_t on_device);

swkb_status swkb_batch_get_info(const swkb_batch* batch, swkb_batch_info* info);
void swkb_batch_destroy(swkb_batch* batch);

/* ---------------------------------------------------------------------------
 * Separation-of-variables reference (Sec. 3.1).  For a permittivity that
 * does not depend on x, the exact one-way field is u(x, z) = sum_i a_i
 * exp(i alpha_i x) phi_i(z) (Eq. series_sol), with (phi_i, alpha_i^2) the
 * eigenpairs of the Sturm-Liouville problem phi'' + k^2 eps phi =
 * alpha^2 phi (Eq. phi_equation) and a_i the projections of the field at
 * x = 0 (Eqs. series_init, sl_expansion).  The library discretises it by
 * Galerkin on the Fourier modes |n| <= K of the period, split by parity about
 * a symmetry point z_c of eps: in the orthonormal bases 1, sqrt(2)
 * cos(kappa_n s) (n = 1..K) and sqrt(2) sin(kappa_n s) (n = 1..K),
 * s = z - z_c, kappa_n = 2 pi n / L, the operator is the real symmetric
 * matrix A_nm = -kappa_n^2 delta_nm + k^2 w_n w_m (eh_|n-m| +- eh_(n+m)) / 2
 * (w_0 = 1, w_n = sqrt(2); + cosines, - sines; eh_j the period mean of
 * eps cos(kappa_j s)), whose eigenpairs come from a batched FP64 Jacobi
 * eigen-solver.  alpha_i is the principal square root (evanescent modes
 * decay).
 * ------------------------------------------------------------------------- */

/*
 * Batched eigen-decomposition of real symmetric matrices, FP64, by the
 * parallel cyclic Jacobi method (round-robin pairing: every sweep rotates
 * each index pair once, n/2 disjoint pairs at a time, on the device).
 * A: batch matrices of n x n, row-major; (A + A^T) / 2 is decomposed.
 * lambda_out: batch x n eigenvalues, in no particular order.
 * vectors_out: batch x n x n, row j the unit eigenvector of lambda_out[j]
 * (NULL: not returned).  sweeps_out (NULL: not returned): sweeps used, the
 * largest over the batch; the iteration stops once the off-diagonal
 * Frobenius norm of every matrix is at most 1e-15 of its Frobenius norm.
 * on_device = 1: A, lambda_out and vectors_out are device pointers, ordered
 * on cuda_stream (NULL = the legacy default stream); 0: host pointers.  The
 * call allocates its workspace (about 2 batch n^2 doubles, 3 with vectors)
 * per call, blocks until done, and leaves A unchanged.  Errors: SWKB_ERR_INVALID_ARG (NULL,
 * batch < 1, n < 1 or n > 8192, non-finite entries: no convergence),
 * SWKB_ERR_OOM, SWKB_ERR_CUDA.
 */
swkb_status swkb_sym_eig(int32_t batch, int32_t n, const double* A, double* lambda_out,
                         double* vectors_out, int32_t* sweeps_out, int32_t on_device,
                         void* cuda_stream);

typedef struct {
  int32_t bc;      /* SWKB_BC_NEUMANN / SWKB_BC_DIRICHLET: grounded at z_a, field
                      on z_a + m (z_b - z_a) / n_z, the period that of the S-WKB
                      mirror, [2 z_a - z_b, z_b), z_c = z_a, one parity (cosines
                      / sines); SWKB_BC_PERIODIC: period [z_a, z_b), field on
                      z_a + m (z_b - z_a) / n_z, eps even about z_sym, both
                      parities                                                */
  double z_a, z_b;
  double z_sym;    /* SWKB_BC_PERIODIC only: the symmetry point z_c, a grid
                      point of the field                                      */
  int32_t n_z;     /* field points                                             */
  int32_t K;       /* modes kept: 1 <= K < N_period / 2                        */
  int32_t n_q;     /* eps samples: n_q + 1 values at z_c + i L / (2 n_q),
                      i = 0..n_q (the half period from z_c); n_q >= 2 K       */
} swkb_hill_desc;

/*
 * The separation-of-variables field of `batch` problems sharing one
 * swkb_hill_desc, each with its own wavenumber k[b] (host array) and
 * permittivity eps[b][n_q + 1]: u0[b] (n_z complex128, the field at x = 0)
 * -> u_out[b][r] (n_z complex128) at every range x[r], r < n_x (host array,
 * x >= 0).  The projections are period means over the field points (exact for
 * fields band-limited to |n| <= K; grounded fields are mirrored onto the
 * period with zero at its top point).  lambda_out (NULL: not returned):
 * batch x n_eig eigenvalues alpha_i^2, cosine block (K + 1) first, then sine
 * block (K), each in no particular order; n_eig = K + 1 (Neumann), K
 * (Dirichlet), 2 K + 1 (periodic).  on_device = 1: eps, u0, u_out and
 * lambda_out are device pointers, ordered on cuda_stream; 0: host.
 * Allocates its workspace per call (per parity block and problem the matrix
 * and the log of its rotations, about 10 K^2 doubles) and blocks until
 * done.  Errors:
 * SWKB_ERR_INVALID_ARG (NULL, sizes, K or n_q out of range, z_sym off the
 * grid, k <= 0, x < 0, non-finite eps), SWKB_ERR_OOM, SWKB_ERR_CUDA.
 */
swkb_status swkb_hill_propagate(const swkb_hill_desc* desc, int32_t batch, const double* k,
                                const double* eps, const double* u0, int32_t n_x,
                                const double* x, double* u_out, double* lambda_out,
                                int32_t on_device, void* cuda_stream);

const char* swkb_last_error(void);
const char* swkb_status_string(swkb_status s);

#ifdef __cplusplus
}
#endif
#endif /* SWKB_H */
