/*
 * rswr.h -- C ABI of librswr: Relative Schwarz Waveform Relaxation (RSWR) for
 * the 1-D wave equation on NVIDIA GB300 (sm_103a).
 *
 * Method: F. Wei and A. Zhao, "A Non-iterative Overlapping Schwarz Waveform
 * Relaxation Algorithm for Wave Equation", arXiv 2203.10477.
 *
 * Problem (paper Sec. 2.1, Eq. (2.1)-(2.3)):
 *     u_tt = a^2 u_xx on [xa, xb], a > 0,
 *     u(x, 0) = 0, u_t(x, 0) = 0   (or a caller-supplied state),
 *     u(xa, t) = f_A(t),  u(xb, t) = f_B(t).
 * Discretisation (the paper fixes none): grid x_j = xa + j dx, j = 0..nx-1,
 * dx = (xb - xa)/(nx - 1); level n is t = n dt; second-order central leapfrog
 * with Courant number c = a dt / dx <= 1, c2 = c*c, k = 2 - 2 c2:
 *     canonical form:  u^{n+1}_j = fma(c2, u^n_{j-1} + u^n_{j+1}, fma(k, u^n_j, -u^{n-1}_j))
 *     increment form:  v^{n+1}_j = fma(c2, (u^n_{j+1} - u^n_j) - (u^n_j - u^n_{j-1}), v^n_j),
 *                      u^{n+1}_j = u^n_j + v^{n+1}_j            (v^n = u^n - u^{n-1})
 * Both are evaluated in exactly this operation order with correctly rounded
 * IEEE arithmetic, so results are reproducible bit for bit.  Coefficients are
 * computed once in double (c = a*dt/dx, c2 = c*c, k = 2 - 2*c2,
 * inv2dx = 1/(2 dx)); an F32 plan rounds c2 and inv2dx to float and computes
 * k = 2 - 2*c2 in float.
 *
 * A state is a pair of arrays (q0, q1) of nx points each:
 *     canonical form: q0 = u^n, q1 = u^{n-1};   increment form: q0 = u^n, q1 = v^n.
 * At level 0 the boundary entries are always overwritten with the Dirichlet
 * samples (q0) and "at rest" values (q1 = q0 canonical, q1 = 0 increment).
 *
 * Decomposition (paper Sec. 2.2, Sec. 3): n_sub overlapping subdomains in a
 * row.  Core i is [b_i, b_{i+1} - 1] with b_i = floor(i * nx / n_sub); its
 * window extends ceil(ov/2) points to the left and floor(ov/2) points to the
 * right (clipped to the grid), so neighbours share exactly `overlap` points.
 * One time span is S steps with S <= floor(overlap/2): the discrete form of the
 * Waveform Time Span Theorem (Sec. 2.4) for a scheme whose domain of dependence
 * grows one point per step.  Each span runs predict (Sec. 2.3, zero input flux
 * guess), select (Sec. 2.4, index mask) and update (Sec. 2.5, core write-back),
 * and the loop restarts from the combined state (Sec. 2.6).  The combined state
 * equals the monolithic leapfrog bit for bit.
 *
 * Conventions
 *   - All data pointers are DEVICE pointers owned by the caller unless a
 *     function says otherwise; the library never frees them.
 *   - Element type of every data array is float for RSWR_F32 plans and double
 *     for RSWR_F64 plans.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream; host arguments are
 *     consumed before the call returns.
 *   - A plan or batch may be used by one stream at a time; it is not
 *     thread-safe.
 *   - No exception crosses the ABI.  Every call returns an rswr_status; the
 *     detail of the last failure on the calling thread is in
 *     rswr_last_error_message().  Device-side failures (a bounded wait that
 *     expired) are latched on the device and reported by rswr_plan_check /
 *     rswr_batch_check.
 */
#ifndef RSWR_H
#define RSWR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rswr_status {
    RSWR_OK = 0,
    RSWR_EINVAL = 1,     /* bad argument: NULL where required, size out of range, T < 0 */
    RSWR_ECFL = 2,       /* Courant number a*dt/dx > 1: the leapfrog would be unstable */
    RSWR_EOVERLAP = 3,   /* overlap < 2, a core shorter than the overlap, or S > floor(ov/2) */
    RSWR_ENOMEM = 4,     /* device or host allocation failed */
    RSWR_ECUDA = 5,      /* a CUDA runtime call failed (message has the CUDA error) */
    RSWR_ETIMEOUT = 6,   /* a bounded device-side wait expired (kernel returned early) */
    RSWR_ENOTSUP = 7     /* unsupported dtype / form / device */
} rswr_status;

typedef enum rswr_dtype { RSWR_F32 = 0, RSWR_F64 = 1 } rswr_dtype;

/* RSWR_FORM_DEFAULT = canonical for F64, increment for F32 (the canonical form
 * accumulates too much rounding in float over 10^4 steps). */
typedef enum rswr_form { RSWR_FORM_DEFAULT = 0, RSWR_FORM_CANONICAL = 1, RSWR_FORM_INCREMENT = 2 } rswr_form;

/* How the spans of a run are scheduled on the GPU. */
typedef enum rswr_mode {
    RSWR_MODE_PERSISTENT = 0, /* one launch for all spans; per-tile neighbour flags (default) */
    RSWR_MODE_PER_SPAN = 1    /* one launch per span (the span loop of Sec. 2.6 on the host) */
} rswr_mode;

/* The name of a status code ("RSWR_OK", ...); a static string. */
const char* rswr_status_string(rswr_status s);
/* A description of the last error this thread's calls returned (static
 * storage, valid until the thread's next failing call; "" when none). */
const char* rswr_last_error_message(void);
/* Library version, major * 100 + minor. */
int32_t rswr_version(void);

/* ------------------------------------------------------------------------ */
/* Plans: one problem                                                        */
/* ------------------------------------------------------------------------ */

typedef struct rswr_plan_s* rswr_plan_t;

/* Creates a plan for one problem (paper Sec. 2.1 problem, Sec. 2.2 / Sec. 3
 * decomposition into n_sub subdomains sharing `overlap` points).
 * Allocates the plan's device workspace (two ping-pong state pairs of the
 * padded grid) on the current device.  flags: reserved, pass 0.
 * Errors: EINVAL (nx < 3, n_sub < 1, a <= 0, dt <= 0, xb <= xa, bad dtype or
 * form), ECFL, EOVERLAP (overlap < 2 or floor(nx/n_sub) < overlap), ENOMEM,
 * ECUDA.  On error *plan is NULL. */
rswr_status rswr_plan_create(rswr_plan_t* plan, double xa, double xb, double a, int64_t nx, double dt,
                             int32_t n_sub, int32_t overlap, int32_t dtype, int32_t form, uint32_t flags);

/* Creates a plan for the part [lo, hi) of the grid of (xa, xb, nx): the
 * building block of one problem split over several GPUs (paper Sec. 3: the
 * subdomains in a row; a GPU keeps a block of them plus halo points).  The
 * part has hi - lo points with the spacing and the stencil coefficients of
 * the whole grid (c = a dt / dx, dx = (xb - xa)/(nx - 1)), decomposed into its
 * own n_sub subdomains sharing `overlap` points.  Its two end nodes are
 * Dirichlet nodes of rswr_run: fA drives point lo, fB point hi - 1.  At
 * lo = 0 / hi = nx they are the problem's own boundary nodes; at a cut they
 * hold a guess, whose influence travels one point per step, so a run of s
 * steps from the true state is exact on [lo + s, hi - 1 - s] (the Waveform
 * Time Span Theorem, Sec. 2.4, applied to the part as a window).  Results of
 * a part equal the whole grid's on those points bit for bit.
 * rswr_run_paper is not available on a part (RSWR_ENOTSUP).
 * Errors: as rswr_plan_create, and EINVAL unless 0 <= lo, hi <= nx and
 * hi - lo >= 3; ECFL is checked on the whole grid. */
rswr_status rswr_plan_create_part(rswr_plan_t* plan, double xa, double xb, double a, int64_t nx, double dt,
                                  int64_t lo, int64_t hi, int32_t n_sub, int32_t overlap, int32_t dtype, int32_t form,
                                  uint32_t flags);

/* Frees the plan and its workspace (synchronises the device first). NULL is a no-op. */
void rswr_plan_destroy(rswr_plan_t plan);

typedef struct rswr_plan_info {
    int64_t nx;
    int32_t dtype, form, n_sub, overlap;
    double c, c2, k, inv2dx;         /* double coefficients */
    float c2f, kf, inv2dxf;          /* F32 coefficients */
    int32_t span_steps;              /* S */
    int32_t halo;                    /* H >= S: halo of a CTA window */
    int32_t core;                    /* owned points per CTA tile */
    int32_t window;                  /* points per CTA window = core + 2H */
    int32_t points_per_thread, threads_per_cta, variant, mode;
    int64_t ntiles;                  /* CTA tiles covering the grid */
    int64_t state_len;               /* elements of one padded state array */
    int64_t workspace_bytes;
} rswr_plan_info;

/* Fills *info (host struct): the problem, its coefficients (Sec. 2.1 on the
 * grid, both precisions), the span S and the CTA tiling of the current
 * variant.  Errors: EINVAL for NULL arguments. */
rswr_status rswr_plan_get_info(rswr_plan_t plan, rswr_plan_info* info);

/* Steps per span, 1 <= S <= floor(overlap/2) (else EOVERLAP). */
rswr_status rswr_plan_set_span(rswr_plan_t plan, int32_t S);

/* Kernel variant (points per thread x threads per CTA) for the plan's dtype
 * and form; see rswr_variant_count / rswr_variant_get.  Re-tiles the grid.
 * RSWR_EINVAL when the variant cannot run the plan's span (its max_span,
 * rswr_variant_get_tiling).  rswr_plan_set_span moves a plan whose variant
 * cannot run the new span to the default variant for it. */
rswr_status rswr_plan_set_variant(rswr_plan_t plan, int32_t variant);
rswr_status rswr_plan_set_mode(rswr_plan_t plan, int32_t mode);

/* Upper bound, in seconds, of every device-side wait (default 5 s). */
rswr_status rswr_plan_set_wait_limit(rswr_plan_t plan, double seconds);

/* Adjoint checkpoint spacing (rswr_adjoint with grad_a): a checkpoint every
 * `spans` spans (1 keeps every span state; the whole adjoint sweep is then one
 * persistent launch); 0 (default) chooses automatically.  RSWR_EINVAL for
 * spans < 0. */
rswr_status rswr_plan_set_checkpoint_spacing(rswr_plan_t plan, int64_t spans);

/* Point sources (the pulse sources of the paper's Sec. 4 experiments), used
 * by rswr_run, rswr_run_host and rswr_mono until replaced.  Source q sits at
 * grid point j[q] (host array, 0 <= j[q] < nx) and has the samples
 * samples[q * pitch + n], n = 0..T (DEVICE memory in the plan's dtype, owned
 * by the caller and kept alive while the set is active; pitch >= T+1 of
 * every run, else that run fails with RSWR_EINVAL).  When level n+1 is formed
 * (n = 0..T-1) the sample of level n+1 is added at j[q]: to u^{n+1} in the
 * canonical form; to the increment v^{n+1}, after which u^{n+1} = u^n +
 * v^{n+1}, in the increment form.  Several sources at one point apply in list
 * order; a source on a Dirichlet node (j = 0 or nx-1) never applies.  Every
 * RSWR window containing j (halo included) applies the source, so rswr_run
 * stays bit-identical to rswr_mono.  nsrc = 0 clears the set.  rswr_adjoint
 * and rswr_run_paper return RSWR_ENOTSUP while a set is active.
 * Errors: EINVAL (point outside the grid, pitch < 1, NULL arrays, samples not
 * aligned to the element size). */
rswr_status rswr_plan_set_sources(rswr_plan_t plan, int64_t nsrc, const int64_t* j, const void* samples,
                                  int64_t pitch);

/* Failure-injection hook for tests: in persistent mode, CTA tile `tile` does
 * not publish completion of span `span`, so its neighbours' bounded waits
 * expire and the run reports RSWR_ETIMEOUT.  tile = -1 disables. */
rswr_status rswr_plan_inject_missing_flag(rswr_plan_t plan, int32_t tile, int32_t span);

/* Timing hook: when set, every run records `start` (a cudaEvent_t passed as
 * void*) on its stream right before its first span (or step) kernel and
 * `stop` right after its last one, so a caller can time the kernels alone.
 * NULL, NULL clears the hook.  The events stay owned by the caller. */
rswr_status rswr_plan_set_kernel_events(rswr_plan_t plan, void* start, void* stop);

/* Autotuner: times every kernel variant of the plan's dtype/form (window
 * width and CTA mapping), both scheduling modes and the spans S = floor(ov/2)
 * and S/2 on `probe_steps` steps of a zero-data run, and keeps the fastest;
 * returns its variant index in *variant (may be NULL).  The choice is
 * remembered per (dtype, form, size class, S) for the process and, when the
 * environment variable RSWR_AUTOTUNE_CACHE names a file, persisted there and
 * reused without timing.  Synchronous; uses the plan's workspace. */
rswr_status rswr_plan_autotune(rswr_plan_t plan, int64_t probe_steps, int32_t* variant, void* stream);

/* Runs are captured into a CUDA graph (on a private stream) the first time a
 * set of arguments is seen and replayed on `stream` while the arguments stay
 * the same (default on).  enable = 0 launches every kernel directly. */
rswr_status rswr_plan_set_graph(rswr_plan_t plan, int32_t enable);

/* Waits for `stream`, then reports a device-side failure latched by the last
 * run (RSWR_ETIMEOUT) or RSWR_OK.  code/tile/span may be NULL. */
rswr_status rswr_plan_check(rswr_plan_t plan, void* stream, int32_t* code, int32_t* tile, int32_t* span);

/*
 * THE HOT PATH.  Advances the problem T steps (t_end = T dt) by RSWR spans.
 *   fA, fB   Dirichlet samples f_A(n dt), f_B(n dt), n = 0..T (T+1 values);
 *            NULL means identically 0.
 *   q0, q1   initial state pair (nx each) or NULL: q0 = NULL gives zero data
 *            (paper Sec. 2.1); q1 = NULL with q0 given starts at rest.
 *   out0,out1  final state pair (nx each); required.
 *   traces   NULL, or (n_sub-1) x 2 x (T+1) values: the boundary output
 *            waveforms (paper Sec. 2.2 definitions) of every interface i
 *            between subdomains i and i+1 at every level:
 *              traces[(2i+0)(T+1)+n] = flux of subdomain i at the left end of subdomain i+1,
 *              traces[(2i+1)(T+1)+n] = flux of subdomain i+1 at the right end of subdomain i,
 *            flux = (u_{j+1} - u_{j-1}) * inv2dx.
 *   j_r, recv  receiver: recv[n] = u^n_{j_r}, n = 0..T (recv may be NULL; j_r
 *            ignored then).
 * Errors: EINVAL, ECUDA.  Device-side timeouts: see rswr_plan_check.
 */
rswr_status rswr_run(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, const void* q0, const void* q1,
                     void* out0, void* out1, void* traces, int64_t j_r, void* recv, void* stream);

/* Same as rswr_run with every pointer a HOST pointer: the call copies the
 * inputs to plan-owned device buffers, runs, copies the outputs back and
 * synchronises `stream` before returning.  Page-locked host memory makes the
 * copies asynchronous DMA. */
rswr_status rswr_run_host(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, const void* q0,
                          const void* q1, void* out0, void* out1, void* traces, int64_t j_r, void* recv,
                          void* stream);

/* RSWR exactly as the paper states it (Sec. 2.3-2.6, Sec. 3), with the span
 * chosen from the data every time: each interface predicts both neighbours
 * over the predictive span tau with a zero input-flux guess; the pair's span
 * is the largest number of leading steps over which the two predictions agree
 * exactly at some overlap point; the global span is the minimum over pairs,
 * capped by the Waveform Time Span Theorem (steps < (overlap - 1)/(2c)); each
 * subdomain is then solved again over that span with the neighbour's
 * predicted output flux as Neumann data, u = p_i on Omega_i minus the windows
 * left of it, and the next predictive span is ceil(1.1 * span) (beta = 0.1;
 * first span tau = overlap).  Equal to the monolithic solve up to rounding
 * (the flux round trip g = (u+ - u-)/(2dx), ghost = u + 2dx g).
 * Same arguments as rswr_run (no traces or receiver); spans (host, capacity
 * spans_cap, may be NULL) receives the selected spans, *nspans their count.
 * Synchronous.  The span is chosen on the device: the call queues the kernels
 * of as many spans as the run needs at the least (each span advances at most
 * the Theorem's cap), reads the run's progress back, and repeats until T is
 * reached — usually one read-back per run. */
rswr_status rswr_run_paper(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, const void* q0,
                           const void* q1, void* out0, void* out1, int64_t* spans, int64_t spans_cap,
                           int64_t* nspans, void* stream);

/* The monolithic comparator: the same arguments and results as rswr_run,
 * computed by one whole-grid leapfrog step per launch (no decomposition, the
 * paper's true solution of Sec. 2.1).  Bit-identical to rswr_run. */
rswr_status rswr_mono(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, const void* q0, const void* q1,
                      void* out0, void* out1, void* traces, int64_t j_r, void* recv, void* stream);

/*
 * A forward run kept for the gradient that follows it (not in the paper; the
 * training pattern of the gradient workload): zero initial data, Dirichlet
 * samples fA, fB (T+1 each, NULL = 0), final state pair into out0/out1 and,
 * when recv is not NULL, the receiver trace u^n_{j_r}, n = 0..T, into recv --
 * the same values as rswr_run, bit for bit.  It runs the sweep that
 * rswr_adjoint with dL/da needs first (spans of the adjoint's length, every
 * span-boundary state stored in the plan's workspace) and keeps those states:
 * a following rswr_adjoint with grad_a on the same plan, with the same fA and
 * fB pointers and the same T, skips its own forward sweep.  The caller must
 * not change the contents of fA or fB in between.  A call with other
 * pointers, another T, a changed span, variant or checkpoint spacing, or a
 * paper-literal run in between discards the kept states; rswr_adjoint then
 * sweeps again (same results).  When the states do not fit in device memory
 * this is a plain rswr_run and nothing is kept.
 * Errors: as rswr_run; ENOTSUP while user point sources are set.
 */
rswr_status rswr_run_keep(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, int64_t j_r, void* recv,
                          void* out0, void* out1, void* stream);

/*
 * Discrete adjoint (not in the paper; the gradient workload of this library).
 * For the receiver trace y^n = u^n_{j_r} of a zero-data run with Dirichlet
 * samples fA, fB, and a cotangent wbar = dL/dy (T+1 values), computes
 *   grad_fA[n] = dL/dfA[n]   (T+1 values, required),
 *   grad_a[0]  = dL/da       (one double, device pointer; NULL skips it).
 * The adjoint variables obey the leapfrog backward in time with zero
 * Dirichlet data and the source wbar at j_r; they run through the same span
 * kernel.  dL/da pairs them with the forward levels, recomputed on chip
 * from span-boundary states (the levels' Laplacians kept in shared memory,
 * or in tensor memory by the persistent FP32 sweep): by default every span
 * state is kept when they fit in half of the free device memory (one forward
 * sweep -- one resident launch when the plan's variant is a resident one and
 * its tiles fit -- then one persistent adjoint launch over all spans), else
 * one checkpoint every ceil(sqrt(#spans)) spans with the states of each
 * segment recomputed before its spans are processed
 * (rswr_plan_set_checkpoint_spacing overrides).
 * Canonical plans give grad_fA bit-identical to a plain FP64 discrete adjoint
 * of the canonical leapfrog.
 */
rswr_status rswr_adjoint(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, int64_t j_r,
                         const void* wbar, void* grad_fA, double* grad_a, void* stream);

/* ------------------------------------------------------------------------ */
/* Batches: many independent problems in one launch                          */
/* ------------------------------------------------------------------------ */

typedef struct rswr_problem {
    int64_t nx;
    double xa, xb, a, dt;
    int32_t n_sub, overlap;
} rswr_problem;

typedef struct rswr_batch_s* rswr_batch_t;

/* A batch of nprob independent problems with one dtype and form.  Every
 * problem is validated like rswr_plan_create.  The span S of the batch is the
 * smallest floor(overlap/2) over its problems (global maximum span, paper
 * Sec. 3).  Packed arrays: problem p occupies [off[p], off[p+1]) of a packed
 * state array (off[0] = 0, off[p+1] = off[p] + nx_p) and rows p*(T+1) ..
 * p*(T+1)+T of a packed waveform array. */
rswr_status rswr_batch_create(rswr_batch_t* batch, int32_t nprob, const rswr_problem* problems, int32_t dtype,
                              int32_t form, uint32_t flags);
void rswr_batch_destroy(rswr_batch_t batch);

/* Writes the nprob+1 packed offsets (host array). */
rswr_status rswr_batch_offsets(rswr_batch_t batch, int64_t* offsets);
/* The rswr_plan_* setters and queries of the same names, for a batch (info
 * describes problem 0 and the batch's shared tiling: span, variant, mode,
 * total tiles and workspace). */
rswr_status rswr_batch_get_info(rswr_batch_t batch, rswr_plan_info* info);
rswr_status rswr_batch_set_mode(rswr_batch_t batch, int32_t mode);
rswr_status rswr_batch_set_variant(rswr_batch_t batch, int32_t variant);
rswr_status rswr_batch_set_wait_limit(rswr_batch_t batch, double seconds);
rswr_status rswr_batch_set_checkpoint_spacing(rswr_batch_t batch, int64_t spans);
rswr_status rswr_batch_set_kernel_events(rswr_batch_t batch, void* start, void* stop);
/* rswr_plan_set_sources for a batch: source q belongs to problem problem[q]
 * (host array) and sits at its grid point j[q]; used by rswr_batch_run. */
rswr_status rswr_batch_set_sources(rswr_batch_t batch, int64_t nsrc, const int32_t* problem, const int64_t* j,
                                   const void* samples, int64_t pitch);
rswr_status rswr_batch_set_graph(rswr_batch_t batch, int32_t enable);
/* As rswr_plan_autotune, over the batch's own problems. */
rswr_status rswr_batch_autotune(rswr_batch_t batch, int64_t probe_steps, int32_t* variant, void* stream);
rswr_status rswr_batch_check(rswr_batch_t batch, void* stream, int32_t* code, int32_t* tile, int32_t* span);

/* All problems advance T steps in one persistent launch (default mode).
 *   fA, fB   packed waveforms nprob x (T+1), or NULL (zero)
 *   q0, q1   packed initial states or NULL; out0, out1 packed final states (required)
 *   j_r      HOST array of nprob receiver indices (-1 = none) or NULL
 *   recv     packed receiver traces nprob x (T+1), or NULL */
rswr_status rswr_batch_run(rswr_batch_t batch, const void* fA, const void* fB, int64_t T, const void* q0,
                           const void* q1, void* out0, void* out1, const int64_t* j_r, void* recv, void* stream);

/* Per-problem gradients of the receiver-trace functional (see rswr_adjoint):
 *   j_r      HOST array of nprob receiver indices (required, 0 <= j_r < nx_p)
 *   wbar     packed cotangents nprob x (T+1)
 *   grad_fA  packed nprob x (T+1) outputs
 *   grad_a   device double[nprob] or NULL */
rswr_status rswr_batch_adjoint(rswr_batch_t batch, const void* fA, const void* fB, int64_t T, const int64_t* j_r,
                               const void* wbar, void* grad_fA, double* grad_a, void* stream);

/* ------------------------------------------------------------------------ */
/* Running without any allocation                                            */
/* ------------------------------------------------------------------------ */

/*
 * The paper has no counterpart of this call; it exists for callers that may
 * not allocate device memory where they solve -- for instance code running
 * under a framework whose caching allocator already holds the memory the
 * process may use, or latency-critical loops in which cudaMalloc/cudaFree,
 * which synchronise the device, are not acceptable.
 *
 * Same problem, decomposition and results as rswr_plan_create + rswr_run
 * (default form, no traces or receiver), but no plan: the call allocates
 * nothing and works in a 32 MiB scratch area compiled into the library (every
 * GPU that loads it keeps it until the process exits).  It needs
 * 4 * (nx + about 2 CTA windows) * sizeof(element) bytes plus small tables:
 * about nx <= 1.0e6 for RSWR_F64 and nx <= 2.0e6 for RSWR_F32; larger
 * problems are rejected with RSWR_EINVAL and a message.
 *   fA, fB   device, T+1 Dirichlet samples each, or NULL (zero)
 *   q0, q1   device initial state pair or NULL (zero data / at rest)
 *   out0, out1  device final state pair (required)
 *   stream   a cudaStream_t of the CURRENT device, or NULL (legacy stream);
 *            a stream of another device is rejected with RSWR_EINVAL
 * The first call on each device looks up the scratch area's device address
 * (with that device current) and remembers it; make that first call before
 * any stream capture.  After cudaDeviceReset on a device the remembered
 * address is stale: load the library again before calling this on that
 * device.  All calls share the scratch area and each clears what must start
 * at zero; calls whose work overlaps on the GPU race and give wrong results.
 * The call returns once its work on `stream` has finished: it reads the
 * device error record back, and a bounded device wait that ran out of time
 * is reported as RSWR_ETIMEOUT.
 */
rswr_status rswr_run_noalloc(double xa, double xb, double a, int64_t nx, double dt, int32_t n_sub, int32_t overlap,
                             int32_t dtype, const void* fA, const void* fB, int64_t T, const void* q0,
                             const void* q1, void* out0, void* out1, void* stream);

/* ------------------------------------------------------------------------ */
/* Measurement utility                                                       */
/* ------------------------------------------------------------------------ */

/*
 * Arithmetic-pipe throughput probe (not a step of the paper's method): the
 * denominator of the span kernels' roofline.  Launches `blocks` x `threads`
 * threads (threads a multiple of 32, at most 1024) on `stream`; each thread
 * runs 8 independent chains of `iters` fused multiply-adds of `dtype`
 * (RSWR_F64: the FP64 pipe, RSWR_F32: the FP32 pipe; 2: packed pairs of FP32
 * values, fma.rn.f32x2, two FMA lanes per instruction; 3: packed adds,
 * add.rn.f32x2) and writes one value
 * to sink[thread] (device, blocks * threads elements of FP64 for RSWR_F64,
 * else FP32, caller-owned).  The call is asynchronous and changes no device
 * setting; the caller times it with events on `stream`: FMA lanes per second
 * = 8 * iters * blocks * threads / seconds (twice that for dtypes 2, 3).
 * Errors: EINVAL (bad sizes, NULL sink, dtype), ECUDA (launch failed).
 */
rswr_status rswr_fma_probe(int32_t dtype, int64_t iters, int32_t blocks, int32_t threads, void* sink, void* stream);

/* ------------------------------------------------------------------------ */
/* Kernel variants                                                           */
/* ------------------------------------------------------------------------ */

int32_t rswr_variant_count(void);
/* dtype, form (RSWR_FORM_CANONICAL / RSWR_FORM_INCREMENT), points per thread
 * and threads per CTA of variant v. */
rswr_status rswr_variant_get(int32_t v, int32_t* dtype, int32_t* form, int32_t* points_per_thread,
                             int32_t* threads_per_cta);
/* Tiling of variant v: warp halo (0: warps exchange neighbour values every
 * step; > 0: warp windows overlap by twice this many points), points per CTA
 * window, longest span the variant runs (0: any span whose halo fits the
 * window; > 0: at most this many steps, because its warps never exchange data
 * inside a span) and threads per CTA at launch (threads_per_cta compute
 * threads, plus 32 for variants with a producer warp that moves the windows).
 * Any pointer may be NULL.  RSWR_EINVAL for v out of range. */
rswr_status rswr_variant_get_tiling(int32_t v, int32_t* warp_halo, int32_t* window, int32_t* max_span,
                                    int32_t* threads_launched);

/* How a variant runs its CTAs (*kind):
 *   RSWR_VARIANT_SINGLE_ROLE      every thread loads, steps and stores windows;
 *   RSWR_VARIANT_WARP_SPECIALISED compute warps plus one producer warp that
 *                                 moves the windows (tickets, TMA, flags);
 *   RSWR_VARIANT_RESIDENT         one CTA per tile for the whole run, the
 *                                 window kept on chip and only halo strips
 *                                 exchanged between spans; a grid whose tiles
 *                                 do not all fit on the GPU at once is refused
 *                                 by rswr_run with RSWR_ENOTSUP (never a
 *                                 default variant; the autotuner tries it).
 * RSWR_EINVAL for v out of range or kind NULL. */
typedef enum {
    RSWR_VARIANT_SINGLE_ROLE = 0,
    RSWR_VARIANT_WARP_SPECIALISED = 1,
    RSWR_VARIANT_RESIDENT = 2
} rswr_variant_kind;
rswr_status rswr_variant_get_kind(int32_t v, int32_t* kind);

#ifdef __cplusplus
}
#endif

#endif /* RSWR_H */
