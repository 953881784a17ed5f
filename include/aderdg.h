/*
 * aderdg.h -- C ABI of the GB300 (sm_103a) ADER-DG predictor/corrector.
 *
 * The library advances hyperbolic systems Q_t + div F(Q) = 0 on periodic
 * uniform Cartesian meshes with the unlimited ADER discontinuous Galerkin
 * scheme of Dumbser, Fambri, Tavelli, Bader and Weinzierl (2018):
 *   - nodal tensor-product basis on N+1 Gauss-Legendre nodes per direction
 *     (Sec. 2.1),
 *   - element-local space-time predictor solved by a discrete Picard
 *     iteration (Sec. 2.2, eq. pde.st2; derivative matrix eq. D_kl),
 *   - corrector: diagonal mass, volume integral and Rusanov face fluxes on
 *     the time-averaged predictor (Sec. 2.1, eq. pde.nc.gw2, pc.scheme with
 *     B = 0, rusanov),
 *   - CFL time step dt = alpha / sum_d lambda_d^max / dx_d (Sec. 3).
 *
 * Conventions shared by every entry point
 *   - Status: every function returns int; ADERDG_OK (0) on success, a
 *     negative ADERDG_E_* code on failure, ADERDG_PENDING (> 0) only from
 *     aderdg_poll.  aderdg_last_error() returns a thread-local message for
 *     the last failure of the calling thread.  No C++ exception crosses the
 *     ABI.
 *   - State layout ("AoS", Sec. 2.2): u[e][s][v], double, variable index v
 *     fastest, then the spatial node s = sx + n*sy + n^2*sz (n = N+1), then
 *     the element e = ex + Cx*(ey + Cy*ez).  Node sx of element ex sits at
 *     x = lo_x + (ex + xi_sx) * dx, xi the Gauss-Legendre nodes of [0,1]
 *     returned by aderdg_gl_nodes.
 *   - Memory: "where" = ADERDG_HOST for host pointers, ADERDG_DEVICE for
 *     device pointers of the current CUDA device.  Host buffers are copied
 *     before the call returns; device buffers are read on the handle's
 *     stream and must stay valid until the next aderdg_sync on it.
 *   - Handles are opaque and owned by the library; all device memory of a
 *     handle comes from the allocator given at creation (NULL: cudaMalloc)
 *     and is released by aderdg_destroy.
 *   - All device work of a handle is issued on its CUDA stream; calls are
 *     asynchronous unless documented as synchronising.
 *   - There is no CPU fallback: on a machine without a usable CUDA device,
 *     aderdg_create fails with ADERDG_E_CUDA.
 */
#ifndef ADERDG_H
#define ADERDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define ADERDG_OK 0
#define ADERDG_PENDING 1          /* aderdg_poll: not finished yet */
#define ADERDG_E_INVAL (-1)       /* bad argument (sizes, N, pde, pointers) */
#define ADERDG_E_NOMEM (-2)       /* allocation failed / admission impossible */
#define ADERDG_E_CUDA (-3)        /* CUDA runtime error (message has details) */
#define ADERDG_E_NONFINITE (-4)   /* a non-finite value appeared in the state */
#define ADERDG_E_TIMEOUT (-5)     /* a bounded device wait gave up */
#define ADERDG_E_BUSY (-6)        /* queue full */
#define ADERDG_E_UNSUPPORTED (-7) /* valid but not compiled (e.g. N too large) */
#define ADERDG_E_CANCELLED (-8)   /* request cancelled */

/* ---- PDE systems -------------------------------------------------------
 * ADVECTION   m = 1,   F_d = a_d u, source S = -kappa u (eq. pde);
 *             p = (a_x, a_y, a_z, kappa), kappa >= 0 (0: pure advection)
 * EULER       m = d+2, Q = (rho, rho v, rho E), ideal gas
 *             p = (gamma-1)(rho E - rho |v|^2 / 2)  (Sec. 3.1, eq. euler);
 *             p[0] = gamma
 * ELASTICITY  m = 9,   Q = (sxx, syy, szz, sxy, syz, sxz, u, v, w),
 *             velocity-stress form of Sec. 3.2 with alpha = 1 and constant
 *             material; p = (rho, lambda, mu); d = 3 only                */
/* DIFFUSE_ELASTICITY  the diffuse-interface linear elasticity system of
 *             Sec. 3.2 (purely non-conservative: B(Q) . grad Q, no flux):
 *             Q = (sigma, w = alpha v, alpha, lambda, mu, rho) with sigma =
 *             (xx, yy, zz, xy, yz, xz), m = 13, in 3D, and the plane-strain
 *             (xx, yy, xy), m = 9, in 2D; alpha (volume fraction of the
 *             solid, > 0; a vacuum is a small positive value) and the
 *             material fields lambda, mu, rho are part of the state and
 *             never change; faces use the path-conservative Rusanov
 *             scheme (eq. pc.scheme, three-point Gauss-Legendre path
 *             integral).  No parameters.                                 */
#define ADERDG_PDE_ADVECTION 1
#define ADERDG_PDE_EULER 2
#define ADERDG_PDE_ELASTICITY 3
#define ADERDG_PDE_DIFFUSE_ELASTICITY 4

/* ---- precision modes ---------------------------------------------------
 * FP64        everything in double
 * MIXED_FP32  predictor, face fluxes and lift in float; the update
 *             u += dt*(...), the CFL reduction and the totals in double   */
#define ADERDG_FP64 0
#define ADERDG_MIXED_FP32 1

#define ADERDG_HOST 0
#define ADERDG_DEVICE 1

/* ---- initial guess of the Picard iteration (Sec. 2.2) ------------------
 * TRIVIAL  q0 = u(t^n)                                    (default)
 * ORDER2   q0 = u + tau L(u)                              (second order)
 * ORDER3   q0 = u + tau k1 + tau^2 (k2 - k1) / (2 dt),    (third order)
 *          k1 = L(u), k2 = L(u + dt k1)
 * EXTRAP   the previous step's predictor q_prev, extrapolated in time
 *          past its interval and shifted to start at u:
 *          q0(t^n + tau) = u + q_prev(1 + tau / dt_prev) - q_prev(1)
 *          (time in units of the previous step).  A step without a
 *          previous predictor (the first after aderdg_set_state, or a
 *          predictor call with an explicit dt) takes ORDER3 with its
 *          default count.  Holds n^(d+1) m values per element more.
 * CERK     dense output of a continuous explicit Runge-Kutta scheme (the
 *          CERK schemes Sec. 2.2 names): k_i = L(u + dt sum_{j<i} a_ij k_j),
 *          q0 = u + dt sum_i b_i(tau/dt) k_i, of uniform order k in time.
 *          N <= 4: the classical fourth-order method (k2 = L(u + dt k1/2),
 *          k3 = L(u + dt k2/2), k4 = L(u + dt k3)) with the cubics
 *          b1 = th - 3th^2/2 + 2th^3/3, b2 = b3 = th^2 - 2th^3/3,
 *          b4 = -th^2/2 + 2th^3/3 (k = 3).  N = 5: a six-stage scheme
 *          with quartic weights (k = 4); N >= 6: an eleven-stage scheme
 *          with quintic weights (k = 5) -- degree N - 1 at N = 5 and 6,
 *          where one Picard iteration suffices.
 * with tau = t - t^n and L(w) = -div F(w), the element-local nodal
 * derivative of the flux (plus -B(w) grad w + S(w) where the PDE has
 * them).  The default Picard count after a guess of degree k in time is
 * max(1, N + 1 - k): N+1 for TRIVIAL, N for ORDER2, N-1 for ORDER3, N-2
 * (N <= 4), N-3 (N = 5) or N-4 (N >= 6) for CERK (the paper notes N - k iterations
 * suffice), and 2 for EXTRAP (degree N). */
#define ADERDG_GUESS_TRIVIAL 0
#define ADERDG_GUESS_ORDER2 1
#define ADERDG_GUESS_ORDER3 2
#define ADERDG_GUESS_EXTRAP 3
#define ADERDG_GUESS_CERK 4

/* ---- tile shapes -------------------------------------------------------
 * The predictor is compiled in ADERDG_NUM_PRED_SHAPES launch variants and
 * the corrector in ADERDG_NUM_CORR_SHAPES (shape 0 is the default).
 * Shapes 0-2 of both are CTA sizes (default, half, double).  Corrector
 * shape 3 gives every warp one element of its own (a shared-memory slice
 * per warp and no CTA-wide barrier between the staging, face-flux and
 * update phases); corrector shape 4 is a quarter-size CTA (64 threads:
 * more independent CTAs per SM); corrector shape 5 is the half-size CTA
 * taking four groups of elements per tile, staging the next group's inputs
 * while it computes the current one.  Predictor
 * shapes 3 and 4 are, for 2D FP32 solves whose n x n x m space-time plane
 * fits the registers, a kernel in which each thread owns that plane (about
 * 128 and 256 threads per CTA); elsewhere they repeat shapes 0 and 2.
 * Predictor shapes 5 and 6 are shapes 0 and 1 with the derivative
 * contractions of the Picard iterations on the tensor cores (mma.sync
 * TF32 with three split products, FP32 accumulation) on the FP32 path; in
 * FP64 they repeat shapes 0 and 1.  Predictor shapes 7 and 8 are shapes 0
 * and 1 on the FP32 path of a conservative system with the state, not the
 * fluxes, exchanged through shared memory (each pencil owner evaluates its
 * flux component); bit-identical to shapes 0-2; elsewhere repeats of
 * shapes 0 and 1.  For a given (PDE, d, N, precision) every shape computes
 * bit-identical results within each of the three kernel families (shapes
 * 0-2 and 7-8, 3-4, 5-6); the families round differently (all within the
 * path's tolerance); only the speed differs.  ADERDG_SHAPE_AUTOTUNE picks the
 * shapes measured fastest on the current device. */
#define ADERDG_NUM_PRED_SHAPES 9
#define ADERDG_NUM_CORR_SHAPES 6
#define ADERDG_SHAPE_DEFAULT 0
#define ADERDG_SHAPE_AUTOTUNE (-1)

typedef struct {
    int dim;            /* 2 or 3 */
    int64_t cells[3];   /* elements per direction (> 0); unused entries ignored */
    double lo[3], hi[3];/* box; periodic in every direction */
} aderdg_mesh_t;

typedef struct {
    int kind;           /* ADERDG_PDE_* */
    double p[8];        /* parameters, see above */
} aderdg_pde_t;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc returns a device pointer of at least `bytes` bytes, 256-byte
 * aligned, or NULL; free releases it. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} aderdg_alloc_t;

typedef struct {
    int precision;              /* ADERDG_FP64 / ADERDG_MIXED_FP32 */
    int picard_iters;           /* Picard iterations P after the initial guess;
                                   0 -> max(1, N + 1 - degree of the guess) */
    double cfl_alpha;           /* CFL coefficient; 0 -> library default
                                   (0.9 x the von Neumann limit of the scheme) */
    void *cuda_stream;          /* cudaStream_t; NULL -> the legacy stream */
    const aderdg_alloc_t *alloc;/* NULL -> cudaMalloc / cudaFree */
    int pred_shape;             /* predictor shape: 0 .. ADERDG_NUM_PRED_SHAPES-1
                                   or ADERDG_SHAPE_AUTOTUNE */
    int corr_shape;             /* corrector shape: 0 .. ADERDG_NUM_CORR_SHAPES-1
                                   or ADERDG_SHAPE_AUTOTUNE */
    const char *tune_cache;     /* text file of autotuned shapes, read and
                                   appended; NULL -> process memory only */
    int initial_guess;          /* ADERDG_GUESS_* (0: trivial) */
    int limiter;                /* 1: the a posteriori subcell finite-volume
                                   limiter (Sec. 2.3, eq. pde.nc.fv) after
                                   every aderdg_step / aderdg_advance step:
                                   both precisions, every PDE
                                   (non-conservative products and sources
                                   included); not with the EXTRAP guess;
                                   ADERDG_E_UNSUPPORTED for that and for an
                                   instance whose subcell arrays do not fit
                                   a CTA (3D elasticity N = 4, 3D
                                   diffuse-interface elasticity N = 3).
                                   2: the same limiter with the subcell data
                                   of limited elements kept between steps:
                                   an element the last step limited takes
                                   the subcell averages its subcell scheme
                                   produced as its subcell data at t^n
                                   (eq. subcellaverage; not the averages of
                                   the reconstructed polynomial) for the
                                   maximum-principle bounds, the subcell
                                   scheme and the coupling, and its wave
                                   speeds for the CFL step come from those
                                   averages; an initial state can be given
                                   as subcell averages
                                   (aderdg_set_subcell_state).  Handles
                                   only: aderdg_batch_create returns
                                   ADERDG_E_UNSUPPORTED.  Other values:
                                   ADERDG_E_INVAL.
                                   With either mode the subcell scheme keeps
                                   the face fluxes of the troubled elements
                                   for their neighbours' coupling: up to 256
                                   MB per solve, fewer if the environment
                                   variable ADERDG_LIMITER_FLUX_SLOTS (read
                                   when the handle or batch is created) sets
                                   a lower number of elements; the coupling
                                   forms the others' fluxes itself, with the
                                   same results */
} aderdg_config_t;

typedef struct aderdg_s aderdg_t;

/* Sizes and cost model of a handle (algorithmic counts per step). */
typedef struct {
    int dim, N, nvar, precision, picard_iters;
    int64_t elements;           /* E */
    int64_t dofs;               /* E (N+1)^d, the paper's DOF count (Sec. 3.1) */
    double cfl_alpha;
    double flops_predictor;     /* algorithmic flops of one predictor launch */
    double flops_corrector;     /* algorithmic flops of one corrector launch */
    double bytes_predictor;     /* algorithmic HBM bytes of one predictor launch */
    double bytes_corrector;     /* algorithmic HBM bytes of one corrector launch */
    size_t device_bytes;        /* device memory held by the handle */
    int pred_shape, pred_threads, pred_epb;  /* predictor shape in use: index,
                                                CTA threads, elements per CTA */
    int corr_shape, corr_threads, corr_epb;  /* corrector, likewise */
    int initial_guess;                       /* ADERDG_GUESS_* */
} aderdg_info_t;

/* Thread-local message of the last failure (never NULL). */
const char *aderdg_last_error(void);

/* ABI version (major*10000 + minor*100 + patch). */
int aderdg_version(void);

/* The library's N+1 Gauss-Legendre nodes x[] and weights w[] on [0,1]
 * (Sec. 2.1), increasing.  1 <= N <= 9.  Host pointers, n = N+1 entries. */
int aderdg_gl_nodes(int N, double *x, double *w);

/* Default CFL coefficient for degree N (0.9 x the von Neumann limit of the
 * scheme for 1D linear advection; the paper's Sec. 3 only bounds it by
 * 1/(2N+1), and 0.9/(2N+1) is unstable for N >= 3). */
double aderdg_default_alpha(int N);

/* Create a solver for one periodic mesh, degree N, nVar variables.
 * Supported: d = 2 with N = 1..7 for ADVECTION and EULER; d = 3 with
 * N = 1..4 for ADVECTION, EULER and ELASTICITY; DIFFUSE_ELASTICITY with
 * N = 2..4 in 2D and N = 2, 3 in 3D (other (PDE, d, N): ADERDG_E_UNSUPPORTED).
 * The subcell limiter (cfg->limiter) is available for all of them except
 * 3D ELASTICITY N = 4 and 3D DIFFUSE_ELASTICITY N = 3, whose subcell
 * arrays do not fit a CTA, and not with the EXTRAP guess.  Limits:
 * 1 <= cells[d] <= 2^30, E = prod cells[d] <= 2^31, hi > lo, and the
 * parameter ranges above (Euler gamma > 1; elasticity rho > 0, mu > 0,
 * lambda + 2 mu > 0; advection kappa >= 0): ADERDG_E_INVAL otherwise.
 * nVar must equal the PDE's m.  The state is zero and t = 0 until
 * aderdg_set_state.  On failure *out is set to NULL. */
int aderdg_create(const aderdg_mesh_t *mesh, int N, int nVar, const aderdg_pde_t *pde,
                  const aderdg_config_t *cfg, aderdg_t **out);

/* Release all device memory of the handle (synchronises its stream). */
int aderdg_destroy(aderdg_t *h);

int aderdg_get_info(const aderdg_t *h, aderdg_info_t *info);

/* Upload a state (layout above, E n^d m doubles) at time t; computes the
 * wave-speed maxima the next CFL step needs and clears the step counter
 * and the error flags. */
int aderdg_set_state(aderdg_t *h, const double *u, int where, double t);

/* Download the state.  Synchronising.  t and step may be NULL.  Returns
 * ADERDG_E_NONFINITE if a non-finite value was produced since set_state. */
int aderdg_get_state(aderdg_t *h, double *u, int where, double *t, int64_t *step);

/* Space-time predictor (Sec. 2.2) of every element with time step dt:
 * Picard iterations, time averages, volume integral and face traces (kept
 * on the device for aderdg_corrector).  dt > 0. */
int aderdg_predictor(aderdg_t *h, double dt);

/* Corrector (eq. pde.nc.gw2) with time step dt: Rusanov fluxes on every
 * face from the predictor's traces, surface lift, u += dt*(volume -
 * surface), and the new wave-speed maxima.  Must follow aderdg_predictor
 * with the same dt.  Does not advance t. */
int aderdg_corrector(aderdg_t *h, double dt);

/* Predictor outputs in the oracle's layout, for checking:
 *   volume[e][s][v]               (E n^d m)    volume term / diagonal mass
 *   qface[e][d][side][p][v],
 *   fface[e][d][side][p][v]       (E d 2 n^(d-1) m) time-averaged traces,
 * side 0 = face xi_d = 0, p = the other spatial indices in increasing order.
 * fface is zero for a purely non-conservative system (no flux).  The
 * volume term includes the non-conservative product and the source.
 * Any pointer may be NULL.  Synchronising. */
int aderdg_get_predictor_outputs(aderdg_t *h, double *volume, double *qface, double *fface,
                                 int where);

/* Troubled elements of the last limited step (Sec. 2.3): flags[e] = 1 for
 * an element that the subcell scheme replaced (host array of E ints, may be
 * NULL), *count their number (may be NULL).  ADERDG_E_INVAL on a handle
 * without the limiter.  Synchronising. */
int aderdg_troubled(aderdg_t *h, int *flags, int64_t *count);

/* Kept subcell data (cfg->limiter = 2; Sec. 2.3, eq. subcellaverage and the
 * least-squares reconstruction that follows eq. pde.nc.fv).
 *
 * aderdg_set_subcell_state sets the state from the subcell averages avg of
 * every element, avg[e][a][v] ((2N+1)^d subcells a per element, x fastest,
 * then y, z; E (2N+1)^d nVar doubles), in host or device memory (where),
 * at time t: each element's nodal state becomes the least-squares
 * reconstruction of its averages, every element is marked as limited
 * (aderdg_troubled then reports all of them), so that the next step takes
 * avg as the subcell data at t^n, and the CFL wave speeds of the state are
 * those of avg.  A discontinuous initial state given this way needs no
 * admissible nodal interpolant.  The library copies avg; the caller keeps
 * ownership.  Synchronising.
 *
 * aderdg_get_subcell_state copies out the kept subcell averages in the same
 * layout: rows of the elements that aderdg_troubled marks hold their
 * averages; the other rows are unspecified.  Synchronising.
 *
 * Both return ADERDG_E_INVAL for a NULL argument, a non-finite t, or a
 * handle that does not keep subcell data. */
int aderdg_set_subcell_state(aderdg_t *h, const double *avg, int where, double t);
int aderdg_get_subcell_state(aderdg_t *h, double *avg, int where);

/* One full step: dt from the CFL condition on the current state, clipped so
 * that t does not pass t_end (the clipped step sets t = t_end exactly),
 * then predictor and corrector.  No step is taken once t >= t_end.  dt is
 * computed and kept on the device; if dt_taken is non-NULL the call
 * synchronises and returns it (0 if no step was taken). */
int aderdg_step(aderdg_t *h, double t_end, double *dt_taken);

/* Steps until t_end or max_steps, as a replayed CUDA graph of steps;
 * synchronises every few steps to read the device time. */
int aderdg_advance(aderdg_t *h, double t_end, int64_t max_steps);

/* The CFL time step of the current state (synchronising). */
int aderdg_cfl_dt(aderdg_t *h, double *dt);

/* Conserved totals M_v = sum_e |Omega_e| sum_s w_s u[e][s][v] (nVar doubles,
 * host), by a fixed-order reduction (deterministic).  Synchronising. */
int aderdg_mass(aderdg_t *h, double *per_var);

/* Wait for all work of the handle; reports a pending device error flag. */
int aderdg_sync(aderdg_t *h);

/* Kernel timing for measurement tools.  With enable != 0, every step
 * records CUDA events on the handle's stream around its predictor and
 * corrector launches; aderdg_profile_read waits for the most recent step
 * and returns the two durations in milliseconds.  Disabled by default. */
int aderdg_profile(aderdg_t *h, int enable);
int aderdg_profile_read(aderdg_t *h, float *ms_predictor, float *ms_corrector);

/* ---- many independent solves in one launch per step ----------------------
 * A batch holds independent solves of any mix of meshes, degrees and PDEs.
 * Each step computes every solve's own CFL dt on the device, then launches
 * one predictor and one corrector per (PDE, dimension, degree, parameters)
 * group, each covering all solves of that group (tiles of consecutive
 * elements numbered solve after solve); aderdg_batch_advance replays the
 * step sequence as one CUDA graph per step.  A solve's arithmetic does not
 * depend on the batch it is in: its results are bitwise the same alone and
 * in any mix. */
typedef struct aderdg_batch_s aderdg_batch_t;

typedef struct {
    aderdg_mesh_t mesh;
    int N;
    aderdg_pde_t pde;
} aderdg_solve_spec_t;

/* Create a batch of `count` solves (state zero, t = 0).  cfg applies to all
 * of them (precision, initial guess, Picard count: 0 -> the default rule per
 * solve's N, CFL alpha: 0 -> default per N, stream, allocator, tile shapes,
 * the subcell limiter). */
int aderdg_batch_create(const aderdg_solve_spec_t *specs, int count, const aderdg_config_t *cfg,
                        aderdg_batch_t **out);
int aderdg_batch_destroy(aderdg_batch_t *b);

/* Upload / download the state of solve i (layout as for a single solve). */
int aderdg_batch_set_state(aderdg_batch_t *b, int i, const double *u, int where, double t);
int aderdg_batch_get_state(aderdg_batch_t *b, int i, double *u, int where, double *t, int64_t *step);

/* One step of every solve that has not reached its t_end (t_end: `count`
 * host doubles, or NULL to keep the previous ones). */
int aderdg_batch_step(aderdg_batch_t *b, const double *t_end);

/* Steps until every solve reaches t_end[i] (host array, or NULL to keep
 * the previous ones) or max_steps; the step sequence is a replayed CUDA
 * graph.  Synchronises every few steps.  Returns ADERDG_E_NONFINITE if any
 * solve produced a non-finite value (the others keep going). */
int aderdg_batch_advance(aderdg_batch_t *b, const double *t_end, int64_t max_steps);

/* Totals: DOFs (sum over solves of E (N+1)^d), device bytes, groups. */
int aderdg_batch_info(const aderdg_batch_t *b, int64_t *dofs, size_t *device_bytes, int *groups);

/* Troubled elements of solve i in the last limited step (a batch created
 * with cfg->limiter: every solve runs the subcell limiter; the rules of the
 * single-solve handle apply).  flags: E host ints or NULL, *count or NULL.
 * ADERDG_E_INVAL for a batch without the limiter.  Synchronising. */
int aderdg_batch_troubled(aderdg_batch_t *b, int i, int *flags, int64_t *count);

/* Per-solve status after a synchronising call: 0 running, 1 done (t >=
 * t_end), ADERDG_E_NONFINITE.  status: `count` ints (host). */
int aderdg_batch_status(aderdg_batch_t *b, int *status);

/* ---- serving: continuous batching of incoming solves --------------------
 * A server owns a device-memory budget and a background scheduler thread.
 * aderdg_submit copies a request (mesh, N, PDE, initial state, t_end) and
 * returns a ticket at once.  The scheduler admits queued requests while
 * their device memory fits the budget (oldest first), keeps admitted
 * states resident, advances all of them together in batched steps (new
 * requests join between steps, finished ones leave), and copies each
 * finished state back to host memory.  aderdg_poll reports PENDING until
 * then, after which the result stays readable until aderdg_release. */
typedef struct aderdg_server_s aderdg_server_t;

typedef struct {
    size_t device_budget_bytes;  /* 0: 90 % of the free device memory */
    int max_queue;               /* queued (not yet admitted) requests; 0: 100000 */
    int steps_per_round;         /* steps between admission rounds; 0: 8 */
    int precision;               /* ADERDG_FP64 / ADERDG_MIXED_FP32: requests' default */
    void *cuda_stream;           /* NULL: a stream of the server's own */
    int pred_shape, corr_shape;  /* tile shapes, as in aderdg_config_t */
    const char *tune_cache;      /* as in aderdg_config_t */
    int initial_guess;           /* ADERDG_GUESS_* (requests' default), Picard count by
                                    the default rule */
} aderdg_server_config_t;

typedef struct {
    aderdg_solve_spec_t spec;
    const double *u0;            /* host, E (N+1)^d m doubles, copied */
    double t_end;
    int precision;               /* ADERDG_FP64 / ADERDG_MIXED_FP32; -1: the server's */
    int initial_guess;           /* ADERDG_GUESS_*; -1: the server's */
} aderdg_request_t;

typedef struct {
    int status;                  /* ADERDG_OK, ADERDG_PENDING or an error */
    double latency_s;            /* submit -> result on the host */
    double queue_s;              /* submit -> admission */
    double t;                    /* final time */
    int64_t steps;
    const double *u;             /* final state (library-owned until release) */
    size_t n_values;
} aderdg_result_t;

int aderdg_server_create(const aderdg_server_config_t *cfg, aderdg_server_t **out);
/* Stops the scheduler, drops unfinished requests, frees everything. */
int aderdg_server_destroy(aderdg_server_t *s);
/* ADERDG_E_BUSY if the queue is full, ADERDG_E_NOMEM if the request could
 * never fit the budget, ADERDG_E_INVAL / UNSUPPORTED for bad specs. */
int aderdg_submit(aderdg_server_t *s, const aderdg_request_t *req, uint64_t *ticket);
int aderdg_poll(aderdg_server_t *s, uint64_t ticket, aderdg_result_t *res);
int aderdg_release(aderdg_server_t *s, uint64_t ticket);
int aderdg_cancel(aderdg_server_t *s, uint64_t ticket);
/* Server counters: queued, active, finished, device bytes in use. */
int aderdg_server_stats(aderdg_server_t *s, int64_t *queued, int64_t *active, int64_t *finished,
                        size_t *bytes_in_use);

/* ---- domain decomposition --------------------------------------------------
 * The distributed-memory structure of the scheme (Sec. 2.2, the closing
 * remarks on MPI; Sec. 4): the periodic mesh is split into a
 * parts[0] x parts[1] (x parts[2]) grid of blocks; each step, every block
 * runs the predictor on its boundary elements first (those with a face on
 * a split block boundary), sends their time-averaged face traces to the
 * neighbouring blocks while the predictor of its interior elements runs,
 * and then runs the corrector on the received traces; the time step comes
 * from one global max-reduction of the per-direction wave speeds, so every
 * block takes the dt of the undivided mesh.
 *
 * Plan (host logic, no device needed).  Blocks are numbered x-fastest over
 * the block grid; along a direction of C cells and p blocks, the first
 * C mod p blocks take one cell more.  1 <= parts[d] <= cells[d], at most
 * 4096 blocks.  Elements inside a block are numbered x-fastest. */
typedef struct {
    int rank;                 /* block index */
    int coords[3];            /* position in the block grid */
    int64_t offset[3];        /* first global cell per direction */
    int64_t cells[3];         /* cells per direction (1 beyond dim) */
    int neighbour[3][2];      /* block across face (d, side: 0 lower, 1 upper);
                                 -1 if direction d is not split (it then wraps
                                 periodically inside the block) */
    int64_t elements;         /* cells[0] cells[1] cells[2] */
    int64_t boundary_elements;/* elements with a face on a split boundary */
    int64_t face_chunks[3][2];/* face-trace chunks sent across (and received
                                 on) face (d, side): elements / cells[d], or 0 */
} aderdg_dd_block_t;

int aderdg_dd_plan(const aderdg_mesh_t *mesh, const int parts[3], int rank, aderdg_dd_block_t *block);

/* The elements of block `rank` on its face (d, side), in the order of the
 * chunks it sends across that face: j = the element's index over the other
 * directions, lowest fastest (the receiver stores chunk j at the same
 * transverse position).  elements: face_chunks[d][side] entries (host). */
int aderdg_dd_face_elements(const aderdg_mesh_t *mesh, const int parts[3], int rank, int d, int side,
                            int64_t *elements);

/* The boundary elements (boundary_elements entries) and the interior ones
 * (elements - boundary_elements) of block `rank`, each increasing; either
 * pointer may be NULL (host). */
int aderdg_dd_element_lists(const aderdg_mesh_t *mesh, const int parts[3], int rank, int64_t *boundary,
                            int64_t *interior);

/* A partitioned solver with every block on the current GPU: the exchange
 * stores each block's boundary chunks into its neighbours' halo buffers
 * (on a second stream that overlaps the interior predictor) and the
 * reduction runs over the blocks' control blocks.  The results are bitwise
 * those of aderdg_create + aderdg_step on the undivided mesh.  Arguments as
 * for aderdg_create (cfg->limiter: ADERDG_E_UNSUPPORTED); states are passed
 * in the global layout and scattered to / gathered from the blocks. */
typedef struct aderdg_dd_s aderdg_dd_t;
int aderdg_dd_create(const aderdg_mesh_t *mesh, int N, int nVar, const aderdg_pde_t *pde,
                     const aderdg_config_t *cfg, const int parts[3], aderdg_dd_t **out);
int aderdg_dd_destroy(aderdg_dd_t *dd);
int aderdg_dd_set_state(aderdg_dd_t *dd, const double *u, int where, double t);
int aderdg_dd_get_state(aderdg_dd_t *dd, double *u, int where, double *t, int64_t *step);
/* as aderdg_step / aderdg_advance on the undivided mesh */
int aderdg_dd_step(aderdg_dd_t *dd, double t_end, double *dt_taken);
int aderdg_dd_advance(aderdg_dd_t *dd, double t_end, int64_t max_steps);
/* blocks, boundary elements over all blocks, bytes exchanged per step,
 * device bytes held; any pointer may be NULL */
int aderdg_dd_info(const aderdg_dd_t *dd, int *blocks, int64_t *boundary_elements, size_t *halo_bytes_per_step,
                   size_t *device_bytes);

/* ---- a step that allocates nothing ---------------------------------------
 * The paper has no counterpart; this is an integration aid of the library.
 *
 * One ADER-DG step with the given dt -- predictor then corrector, the same
 * kernels and result as aderdg_predictor + aderdg_corrector on a handle --
 * from u_in to u_out, caller-owned device buffers in the state layout above
 * (they may be the same buffer).  No handle is created.
 *
 * For callers that cannot call cudaMalloc: frameworks whose device memory
 * must all come from their own allocator, code paths where cudaMalloc's
 * implicit device synchronisation is not acceptable, and real-time or
 * embedded hosts that forbid allocation after start-up.  This call
 * allocates no memory at all: the volume term, the face traces, the FP32
 * path's reference states, the step's descriptor and its control block
 * live in one fixed device array of ADERDG_NOALLOC_SCRATCH_BYTES (32 MiB),
 * part of the library module, which every GPU that loads the library
 * holds until the process exits.  The mesh and PDE limits of
 * aderdg_create apply (ADERDG_E_INVAL); meshes whose scratch would exceed
 * the array are rejected with ADERDG_E_INVAL too (the message gives the
 * size needed).
 *
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress, once per device, with that device current); make
 * that first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents (each call clears the parts that
 * must start at zero): calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it, so serialise them.  Work is
 * queued on cuda_stream (NULL: the legacy stream); the call does not
 * synchronise and does not check for non-finite values.  Errors are
 * reported through aderdg_last_error. */
#define ADERDG_NOALLOC_SCRATCH_BYTES (32u << 20)
int aderdg_step_noalloc(const aderdg_mesh_t *mesh, int N, int nVar, const aderdg_pde_t *pde,
                        int precision, int picard_iters, const double *u_in, double *u_out,
                        double dt, void *cuda_stream);

/* ---- tile-shape autotuning ---------------------------------------------
 * Not part of the paper's method (its kernels are tuned offline by its
 * code generator); a performance aid of this library.
 *
 * Times every compiled predictor and corrector shape of spec's (PDE, d, N)
 * at `precision` on a synthetic periodic mesh of about 2^21 nodes (the
 * spec's mesh and state are not used; the cost of a step does not depend
 * on the data) and returns the fastest shape indices in shapes[0]
 * (predictor) and shapes[1] (corrector).  The choice is kept for the
 * process and, if tune_cache is not NULL, appended to that text file; a
 * later call finds it there without timing unless flags has
 * ADERDG_TUNE_FORCE.  ms (NULL or ADERDG_NUM_PRED_SHAPES +
 * ADERDG_NUM_CORR_SHAPES floats) receives the measured milliseconds per
 * launch, predictor shapes first (-1 where nothing was timed).  Synchronising; allocates and frees device memory
 * (about 2^21 x m x 40 bytes). */
#define ADERDG_TUNE_FORCE 1
int aderdg_autotune(const aderdg_solve_spec_t *spec, int precision, const char *tune_cache, int flags,
                    int shapes[2], float *ms);

/* Measurement utility: the FMA throughput this GPU sustains, in TFLOP/s
 * (FMA = 2 flops), from independent FMA chains on every SM.  kind 0: FP64
 * (DFMA), kind 1: FP32 (FFMA).  Synchronising; runs for ~0.1 s.  Used as
 * the denominator of the ALU rooflines. */
int aderdg_peak_tflops(int kind, double *tflops);

/* Check utility: y[i] = 1 / x[i] as the kernels compute it on the device
 * (the flux's reciprocal of the density and of volume fractions, in the
 * compute type: precision ADERDG_FP64, or ADERDG_MIXED_FP32 for the FP32
 * path, where x is rounded to float and the result widened).  x and y are
 * n doubles in host memory (caller-owned, n <= 2^26); x must hold normal,
 * finite, nonzero numbers.  The result is within one ulp of the correctly
 * rounded 1/x in the compute type.  Synchronising; allocates and frees
 * 16 n bytes of device memory.  ADERDG_E_INVAL on bad arguments. */
int aderdg_device_recip(const double *x, double *y, long long n, int precision);

#ifdef __cplusplus
}
#endif
#endif /* ADERDG_H */
