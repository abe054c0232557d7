/*
 * pgdto.h -- C ABI of the GB300 (sm_103a) PGD-TO optimizer step.
 *
 * Method: projected gradient descent for topology optimisation with a regularised
 * dual projection (arXiv 2511.13905).  One step (Alg. 3) computes
 *   1. the step size alpha_t: the fallback alpha_fb / ||grad f||_inf at t = 0 or after
 *      the warm-up when a constraint is violated by more than tol_N (Sec. 3.4), else the
 *      spectral step of eq. final_alpha (BB1 when s^T y > eps_alpha, else eq. alpha);
 *   2. the PR+ conjugate-gradient direction d_t of eq. CG;
 *   3. the trial point z = x_t + omega alpha_t d_t;
 *   4. the projection of z onto lo <= x <= hi and the rows linearised about x_t,
 *      a_j^T x <= b_j with b_j = G_j - g_j(x_t) + a_j^T x_t (Sec. 3.2, eq. linearized),
 *      regularised as in Sec. 3.2.3 and solved in its dual:
 *        x(lam) = clip(z - A^T lam, lo, hi),  lam >= 0 (lam = -y of Thm 2),
 *        r_j(lam) = a_j^T x(lam) - b_j - 2 lam_j / C <= 0,  lam_j r_j = 0   (eq. h);
 *      single and independent rows by a per-row root search (Alg. 1, Sec. 3.2.2),
 *      coupled rows by Alg. 2 (single-row candidates, then semismooth Newton on the
 *      m x m Jacobian A D A^T + (2/C) I of eq. reg_jacobian);
 *   5. x_{t+1} = x(lam*) and the ratio ||x_{t+1} - x_t|| / ||x_{t+1}||.
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA global-memory pointers valid in the current context;
 *     FP32 arrays are dense, element i at offset i.  Pointers 16-byte aligned take the
 *     vectorised path; others work but are slower.
 *   - A holds the constraint gradients.  Dense layout (modes SINGLE, COUPLED): m rows
 *     of n floats, row j at A + j*n.  Segmented layout (mode INDEPENDENT): one float
 *     per variable, the coefficient of the row whose segment contains it.
 *   - Work is enqueued on the handle's CUDA stream and runs asynchronously.  When an
 *     info pointer is non-NULL the call waits for the stream and fills it.
 *   - No entry point aborts, traps or prints.  Errors come back as pgdto_status;
 *     device-side conditions (a grid barrier that timed out, non-finite input, an
 *     iteration limit) are reported through the status returned by the call that
 *     waits (info != NULL, pgdto_last_info, pgdto_poll).
 *   - Caller-owned buffers must stay valid until the stream work completes.
 */
#ifndef PGDTO_H
#define PGDTO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PGDTO_OK = 0,
    PGDTO_ERR_ARG = 1,          /* invalid argument; nothing was enqueued */
    PGDTO_ERR_OOM = 2,          /* device or pinned allocation failed */
    PGDTO_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    PGDTO_ERR_NONFINITE = 4,    /* NaN or Inf in an input reduction; outputs not meaningful */
    PGDTO_ERR_TIMEOUT = 5,      /* a device-side wait ran out of its budget; outputs not meaningful */
    PGDTO_ERR_BUSY = 6,         /* server full or request still running */
    PGDTO_NOT_CONVERGED = 7,    /* iteration limit reached; best iterate returned and flagged */
    PGDTO_ERR_UNSUPPORTED = 8   /* combination not available on this device */
} pgdto_status;

typedef enum {
    PGDTO_AUTO = 0,         /* SINGLE if m == 1, INDEPENDENT if segments given, else COUPLED */
    PGDTO_SINGLE = 1,       /* one row (Alg. 1) */
    PGDTO_INDEPENDENT = 2,  /* rows with disjoint supports (Sec. 3.2.2), segmented layout */
    PGDTO_COUPLED = 3       /* general rows, m <= 4 (Alg. 2) */
} pgdto_mode;

/* Parameters; pgdto_params_default fills the paper's defaults. */
typedef struct {
    double C;               /* regularisation, 1e12 (Sec. 3.2.3, Sec. 3.5) */
    double alpha_max;       /* step cap, 1e2 (Sec. 3.5) */
    double alpha_fallback;  /* fallback step numerator, 0.2 (Sec. 3.3) */
    double tol_B;           /* Alg. 1 tolerance, 1e-8; used relative to the bracket here */
    double tol_N;           /* Alg. 2 / fallback tolerance, 1e-6 (Sec. 3.5) */
    double omega;           /* global relaxation, 1.0 (Sec. 3.4) */
    double eps_alpha;       /* BB1 threshold on s^T y, 1e-6 (Sec. 3.4) */
    double c1;              /* Armijo constant of the Newton line search, 1e-4 (App. A.3.3) */
    double c2;              /* curvature constant, 0.9 (App. A.3.3; recorded, not enforced) */
    double tol_lambda;      /* relative width at which a dual root search stops, 1e-10; a row
                               search also stops once both Newton predictions agree to 1000
                               tol_lambda and to 1e-8 / max_i |a_i| (the final pass takes one
                               exact Newton step from there, and runs again if that step moves
                               lam by more than 1e-7 lam or some free x_i by more than 1e-7) */
    int t_warmup;           /* steps before the fallback rule applies, 50 (Sec. 3.4) */
    int maxiter_newton;     /* Alg. 2 maxiter (the paper gives none), 50 */
    int max_passes;         /* cap on root-search passes per projection, 64 */
    int barrier_timeout_ms; /* budget of each device-side wait, 2000 */
    pgdto_mode mode;        /* PGDTO_AUTO */
    int fault_inject;       /* tests only: 1 = block 0 leaves before the first grid reduction,
                               so the others' waits run out and the call reports
                               PGDTO_ERR_TIMEOUT (no fault, trap or hang); 0 = off */
    int engine;             /* 0 auto, 1 grid (all SMs, grid-wide reductions), 2 cluster (one
                               thread-block cluster, reductions in distributed shared memory;
                               single and independent rows only).  Auto: cluster for n up to
                               131072, grid above it */
    int cluster_elems;      /* cluster engine: variables per thread block; a problem's cluster
                               has ceil(n / cluster_elems) blocks rounded up to a power of two,
                               at most 16.  It depends on n alone, so a problem's result is the
                               same alone and in any batch.  0 = the share pgdto_autotune_batch
                               chose for this device and n's bucket, else 8192 (the cluster
                               engine runs two 256-thread blocks per SM; 8192 variables of a
                               block fit its share of shared memory) */
    int eq_mask;            /* bit j set: row j is an equality g_j(x) = G_j (Sec. 3.2.4), always
                               active, lambda_j of either sign, and its violation for the
                               fallback rule is |g_j - G_j|; bits at or above m must be 0 */
    int compaction;         /* single/independent rows: 1 = free-set compaction (Sec. 4.2.1) -- once
                               the bracket is within 50% of the root, elements whose clip state it
                               fixes are summed once and later passes visit the rest (shares that
                               stream from global memory only); 0 (default) = every pass visits
                               every element, which measured faster on the shipped workloads */
    int stage1;             /* coupled rows, cold start: 1 = Alg. 2's stage 1 first (the m
                               single-row searches, then the test of each candidate against
                               every row); 0 (default) = stage 2's Newton iteration from
                               lam = 0.  Both reach the same optimum; on the 4-row workload
                               stage 1 cost more passes than it saved.  A warm start (the
                               handle's previous step) begins at the previous lam either way */
} pgdto_params;

/* Per-call report. */
typedef struct {
    double alpha;           /* step size taken (omega not applied) */
    double beta;            /* PR+ coefficient */
    double lambda[4];       /* dual solution, lam = -y >= 0 */
    double b[4];            /* right-hand sides used, b_j = G_j - g_j(x_t) + a_j^T x_t */
    double viol[4];         /* a_j^T x_{t+1} - b_j (regularised optimum: 2 lam_j / C) */
    double rel_change;      /* ||x_{t+1} - x_t||_2 / ||x_{t+1}||_2 (Alg. 3 stopping ratio) */
    double phi_inf;         /* max_j |Phi_j| at exit (coupled) or max_j |r_j| (root search) */
    int passes;             /* passes over the projection data after the trial-point pass */
    int newton_iters;       /* Alg. 2 stage 2 iterations */
    int stage;              /* 0 root search, 1 Alg. 2 stage 1 accepted, 2 Newton */
    int branch;             /* step-size rule: 0 fallback, 1 BB1, 2 Lipschitz */
    int status;             /* pgdto_status of the device work */
    int t;                  /* iteration index the step used */
    double visited;         /* element evaluations of the root-search passes (n per row and
                               pass without compaction; fewer once its lists are in use) */
} pgdto_info;

typedef struct pgdto_handle pgdto_handle;

/* Fill *p with the defaults listed above.  PGDTO_ERR_ARG if p is NULL. */
pgdto_status pgdto_params_default(pgdto_params* p);

/*
 * Create a handle for problems with n variables and m constraint rows.
 *   n >= 1; 1 <= m <= 4; lo < hi, both finite.
 *   seg_offsets: host array of m + 1 offsets, 0 = s_0 < s_1 < ... < s_m = n, for the
 *     segmented INDEPENDENT layout (row j owns variables [s_j, s_{j+1})); NULL for
 *     dense rows.  Copied; the caller keeps ownership.
 *   params: NULL for defaults.  cuda_stream: the cudaStream_t to enqueue on (NULL =
 *     legacy default stream).
 * The handle owns the optimizer state (x_prev, g_prev, d_prev, the iteration index t)
 * and a device workspace, about 4 n floats plus a fixed part.  Allocation failure
 * returns PGDTO_ERR_OOM and leaves *h NULL.
 */
pgdto_status pgdto_create(pgdto_handle** h, int64_t n, int m, const int64_t* seg_offsets,
                          float lo, float hi, const pgdto_params* params, void* cuda_stream);

/* Free the handle after waiting for its stream.  NULL is ignored. */
void pgdto_destroy(pgdto_handle* h);

/* Replace the stream the handle enqueues on. */
pgdto_status pgdto_set_stream(pgdto_handle* h, void* cuda_stream);

/*
 * Load optimizer state (checkpoint resume, or a prior step computed elsewhere):
 * x_prev = rho_{t-1}, g_prev = grad f(rho_{t-1}), d_prev = d_{t-1}, device pointers of
 * n floats, copied on the stream; NULL means zeros.  t is the iteration index the next
 * pgdto_step takes (t = 0 starts Alg. 3 from scratch and ignores the arrays).
 */
pgdto_status pgdto_set_state(pgdto_handle* h, const float* x_prev, const float* g_prev,
                             const float* d_prev, int t);

/* Copy the state out to device buffers (each may be NULL); *t receives the next index. */
pgdto_status pgdto_get_state(pgdto_handle* h, float* x_prev, float* g_prev, float* d_prev, int* t);

/*
 * One Alg. 3 iteration (steps 1-5 above) at index t = the handle's counter, which then
 * advances.
 *   x       device, n floats: rho_t on entry, rho_{t+1} on return (in place).
 *   grad_f  device, n floats: grad f(rho_t).
 *   A       device constraint gradients grad g_j(rho_t), layout of the handle's mode.
 *   g_val   host, m doubles: g_j(rho_t) (for linear rows a_j^T rho_t).
 *   G       host, m doubles: the bounds G_j.
 *   info    NULL for an asynchronous call; otherwise filled after the stream is waited on.
 * The state moves to (rho_t, grad f(rho_t), d_t).  Returns PGDTO_ERR_ARG for NULL
 * pointers, or the device status when info is non-NULL.
 */
pgdto_status pgdto_step(pgdto_handle* h, float* x, const float* grad_f, const float* A,
                        const double* g_val, const double* G, pgdto_info* info);

/*
 * The same step with HOST buffers (for callers whose sensitivities live on the host):
 * x, grad_f and A are copied to handle-owned device buffers on the stream, the step
 * runs, and rho_{t+1} is copied back into x.  Page-locked host memory gives the fastest
 * copies.  Always waits for the stream before returning.
 */
pgdto_status pgdto_step_host(pgdto_handle* h, float* x, const float* grad_f, const float* A,
                             const double* g_val, const double* G, pgdto_info* info);

/*
 * The regularised projection alone (Alg. 1 / Alg. 2 on given data, Sec. 3.2):
 *   z       device, n floats, the point to project.
 *   A       device, layout of the handle's mode.
 *   b       host, m doubles, right-hand sides.
 *   x_out   device, n floats: x(lam*) = clip(z - A^T lam*, lo, hi).  May alias z.
 *   lambda_out  host, m doubles or NULL; written only when info is non-NULL or after
 *           pgdto_last_info (it is read back from the device).
 * Does not touch the optimizer state.
 */
pgdto_status pgdto_project(pgdto_handle* h, const float* z, const float* A, const double* b,
                           float* x_out, double* lambda_out, pgdto_info* info);

/*
 * Batched form: `count` independent steps, each on a thread-block cluster of its own
 * whose size follows from its n (params.cluster_elems), so a problem's result is the same
 * alone and in any batch.  Problems of one cluster size share one launch, largest first;
 * launches of different sizes (at most five) run side by side on streams forked from and
 * joined back into the first handle's stream.  Handles must be in SINGLE or INDEPENDENT
 * mode and share the first handle's stream.  Per handle k: x[k], grad_f[k], A[k] as for
 * pgdto_step; g_val[4k + j], G[4k + j] its row scalars.  Each handle's state advances as
 * after pgdto_step.  infos: NULL for an asynchronous call, else `count` reports (waits
 * for the stream).  The list of problems is uploaded through pinned and device buffers
 * owned by the first handle (grown on demand).
 */
pgdto_status pgdto_step_many(int count, pgdto_handle* const* hs, float* const* x, const float* const* grad_f,
                             const float* const* A, const double* g_val, const double* G, pgdto_info* infos);

/* Batched projections, same conventions: z[k], A[k], b[4k + j], x_out[k]; lambda_out[4k + j]. */
pgdto_status pgdto_project_many(int count, pgdto_handle* const* hs, const float* const* z,
                                const float* const* A, const double* b, float* const* x_out,
                                double* lambda_out, pgdto_info* infos);

/*
 * pgdto_autotune_batch -- choose, on the current device, the cluster engine's block share
 * for batches of `count` single-row problems of n variables.  It builds that batch from a
 * counter-based hash on the device (its own buffers and handles, freed before it returns),
 * times 3 + 5 batched steps (pgdto_step_many, from the same starting state each time) for
 * each share in {1024, 2048, 4096, 8192} with CUDA events on `cuda_stream`, and records the
 * share with the lowest median time for this device and n's power-of-two bucket
 * (2^(b-1) < n <= 2^b).  Handles created afterwards with params.cluster_elems = 0 and n in
 * that bucket take it; handles that exist keep theirs, so a problem's result is the same
 * alone and in any batch only among handles created under the same table.
 *   n: 1 .. 131072 (the cluster engine's range under engine = auto); count: 1 .. 4096.
 *   best_out, ms_out: host, the share chosen and its median batched-step time in ms, or NULL.
 * Synchronises `cuda_stream`.  Errors: PGDTO_ERR_ARG for sizes outside those ranges,
 * PGDTO_ERR_OOM / PGDTO_ERR_CUDA from the device; the table is left as it was.
 * Not thread-safe against concurrent calls on one device.  The paper has no counterpart.
 */
pgdto_status pgdto_autotune_batch(int64_t n, int count, int* best_out, double* ms_out, void* cuda_stream);

/* Forget every share pgdto_autotune_batch recorded, on every device (handles created
 * afterwards use params.cluster_elems, or 8192 when it is 0). */
void pgdto_autotune_reset(void);

/* ------------------------------------------------------------------ serving
 * A server runs optimizer steps for many concurrent design sessions with continuous
 * batching: every session keeps its design x and optimizer state on the device between
 * its steps; a submitted step's inputs are copied by DMA from the caller's buffers on a
 * copy stream and, while one cycle runs on the GPU, newly arrived steps queue for the
 * next.  A cycle launches every queued single/independent session small enough for one
 * thread-block cluster as one batched step (pgdto_step_many), then each coupled-row
 * session and each larger session in a whole-GPU launch of its own, smallest first; a
 * completion thread delivers each launch's results as soon as that launch completes,
 * while the next cycle is already being launched.  Sessions are admitted while their device memory fits the HBM budget;
 * otherwise submit returns PGDTO_ERR_BUSY and the caller retries after sessions close.
 * The paper has no serving layer; the step each request runs is Alg. 3 as above.
 */
typedef struct pgdto_server pgdto_server;

typedef struct {
    uint64_t session;            /* design id; its first request creates the session */
    int64_t n;                   /* size of the design (fixed per session) */
    int m;                       /* rows (fixed per session) */
    const int64_t* seg_offsets;  /* as pgdto_create (NULL = dense rows); read on the first request */
    float lo, hi;                /* box (fixed per session) */
    const float* x0;             /* host, n floats: the starting design; first request only */
    const float* grad_f;         /* host, n floats: grad f(rho_t), copied during submit */
    const float* A;              /* host, constraint gradients (mode layout), copied during submit */
    double g_val[4], G[4];       /* row scalars of this step */
    float* x_out;                /* host, n floats: receives rho_{t+1} when the step completes */
    int close_session;           /* 1: release the session's device memory after this step */
    int eq_mask;                 /* equality rows as pgdto_params.eq_mask; read on the first request */
} pgdto_request;

/* budget_bytes: device memory the sessions may hold; max_sessions: open sessions at most;
 * params: for every session (NULL = defaults); cuda_stream: stream of the launches. */
pgdto_status pgdto_server_create(pgdto_server** srv, uint64_t budget_bytes, int max_sessions,
                                 const pgdto_params* params, void* cuda_stream);

/* Queue one step; *ticket identifies it.  Returns once the inputs (grad_f, A, and x0 on a
 * session's first request) have been copied to the device, so those buffers are free on
 * return; x_out must stay valid until the step is reported.  PGDTO_ERR_BUSY: budget or
 * session limit reached, or this session already has a step queued or running.
 * PGDTO_ERR_CUDA: an upload failed (a new session is not kept). */
pgdto_status pgdto_submit(pgdto_server* srv, const pgdto_request* req, uint64_t* ticket);

/* Open a session without a step: admission (session limit, HBM budget), the session's
 * device state, and the upload of its starting design req->x0 (host, n floats; copied
 * before the call returns).  Only req->session, n, m, seg_offsets, lo, hi, x0 and eq_mask
 * are read.  Its first pgdto_submit then needs no x0.  PGDTO_ERR_ARG if the session is
 * already open, PGDTO_ERR_BUSY if it would not fit, PGDTO_ERR_CUDA if the upload failed. */
pgdto_status pgdto_server_open(pgdto_server* srv, const pgdto_request* req);

/* Non-blocking: *done = PGDTO_ERR_BUSY while the step is queued or running, else its final
 * status (x_out written, info filled when non-NULL).  A finished ticket is forgotten after
 * the first poll that reports it. */
pgdto_status pgdto_poll(pgdto_server* srv, uint64_t ticket, pgdto_status* done, pgdto_info* info);

/* Blocking form of pgdto_poll: waits up to timeout_ms for the step.  *done as for
 * pgdto_poll (PGDTO_ERR_BUSY when the wait ran out); completed_us (nullable) receives the
 * moment the result was published, on the server's clock (pgdto_server_clock_us).
 * PGDTO_ERR_ARG for an unknown or already reported ticket. */
pgdto_status pgdto_wait(pgdto_server* srv, uint64_t ticket, int timeout_ms, pgdto_status* done, pgdto_info* info,
                        int64_t* completed_us);

/* Microseconds since the server was created (steady clock); -1 for NULL. */
int64_t pgdto_server_clock_us(const pgdto_server* srv);

/* Counters: launches (batches), steps completed, sessions open, bytes in use. */
pgdto_status pgdto_server_stats(pgdto_server* srv, int64_t* batches, int64_t* steps, int* sessions,
                                uint64_t* bytes_in_use);

/* Wait for queued steps, stop the service thread, free every session. */
void pgdto_server_destroy(pgdto_server* srv);

/* Wait for the handle's stream and report the last step or projection. */
pgdto_status pgdto_last_info(pgdto_handle* h, pgdto_info* info, double* lambda_out);

/*
 * Phase timeline of the last step or projection (tracing): waits for the stream, writes
 * up to max_marks times in microseconds since the kernel started, one per grid-wide
 * reduction in order (step: step-size pass, trial-point pass, each root-search pass or
 * Newton iteration, final pass), and returns how many marks there were (or -1 on error).
 * Taken from the device's global timer; resolution is that timer's.
 */
int pgdto_trace(pgdto_handle* h, double* us_out, int max_marks);

/* Number of the library's kernels launched by this handle so far (for accounting). */
int64_t pgdto_kernel_launches(const pgdto_handle* h);

/*
 * pgdto_project_noalloc -- the projection of pgdto_project for callers that cannot
 * allocate device memory.  The paper has no counterpart; this is a deployment variant.
 * Callers that cannot call cudaMalloc include processes whose device memory belongs to
 * another allocator (a framework's caching allocator that has reserved the GPU's memory,
 * or a pool fixed at start-up, where a cudaMalloc would fail or fragment it) and loops
 * with a latency budget that must never block in the driver's allocator.  No handle is
 * involved (creating one allocates); the call allocates nothing and frees nothing.
 *   n, m, seg_offsets, lo, hi as for pgdto_create (m > 1 needs the segmented layout:
 *     rows with disjoint supports; coupled rows are not served here); C > 0 the
 *     regularisation of eq. h (1e12 in the paper).  Other parameters are the defaults.
 *   z, A, x_out: device, as for pgdto_project (x_out may alias z); b: host, m doubles.
 *   lambda_out / info: host or NULL; when either is non-NULL the call waits for the stream
 *     (cudaStreamSynchronize) and reads the result back, otherwise it returns as soon as
 *     the work is enqueued and the result's status is not observed.
 * Workspace: a file-scope device array of about 2.3 MB (the reduction partials of two
 * alternating rounds for up to 1024 blocks and 4 rows, plus the control block and the
 * report) that every GPU loading the library holds until the process exits.  Sizes
 * beyond what it holds, m > 4, return PGDTO_ERR_ARG; n has no limit of its own.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture.  Every call
 * shares the one array: calls whose device work overlaps (two streams, two host threads)
 * race and give wrong results, so serialise them.  Before its kernel runs, each call
 * clears the barrier counters, the sticky status and the abort flag, and marks the report
 * unpublished, so a device wait that ran out returns PGDTO_ERR_TIMEOUT (lambda_out then
 * NaN), never the previous call's result.
 */
pgdto_status pgdto_project_noalloc(int64_t n, int m, const int64_t* seg_offsets, float lo, float hi, double C,
                                   const float* z, const float* A, const double* b, float* x_out,
                                   double* lambda_out, pgdto_info* info, void* cuda_stream);

/* Tests only: make the following pgdto_project_noalloc calls leave block 0 before the first
 * grid reduction (fault_inject = 1) with a device-wait budget of timeout_ms (0 = the
 * default), so that the other blocks' waits run out and the call reports
 * PGDTO_ERR_TIMEOUT; nothing faults, traps or hangs.  (0, 0) restores normal calls. */
pgdto_status pgdto_noalloc_set_test_fault(int fault_inject, int timeout_ms);

/*
 * Read-bandwidth probe (measurement tooling; the paper has no counterpart).  Enqueues one
 * kernel that reads the n floats at buf once with 128-bit loads (n a multiple of 4, buf
 * 16-byte aligned, both device) and writes one partial sum per block to out (device,
 * `blocks` floats).  Timing repeated launches with CUDA events gives the L2 read rate for
 * a buffer well under the L2 size and the HBM read rate for one far above it: the two
 * bounds of the projection passes.  PGDTO_ERR_ARG on bad arguments, PGDTO_ERR_CUDA if the
 * launch fails.
 */
pgdto_status pgdto_probe_read(const float* buf, int64_t n, float* out, int blocks, void* cuda_stream);

/* Library version string, e.g. "pgdto-gb300 0.1 sm_103a". */
const char* pgdto_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PGDTO_H */
