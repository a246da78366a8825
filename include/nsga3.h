/*
 * nsga3.h -- C ABI of the GB300 NSGA-III environmental-selection engine.
 *
 * The method is the per-generation NSGA-III step of arXiv 2504.06067
 * (Alg. 1, in its tensorized form Alg. 2): variation of the parents, merge
 * R_t = P_t u Q_t, non-dominated sorting into F_s, F_l, F_drop,
 * normalization and association with reference points (Eq. 2), niche
 * counts and niche selection of the last front.  All objectives are
 * minimised (Eq. 1).
 *
 * Conventions for every call:
 *   - Objective matrices are FP32, row-major, one row per individual.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous and stream-ordered unless stated.
 *   - Pointers documented as "any" may point to device memory or to host
 *     memory (pinned or pageable); the library copies with cudaMemcpyDefault.
 *     Pointers documented as "device" must be device memory.  The caller
 *     owns every pointer it passes; the context owns all its workspace.
 *   - A return value other than NSGA3_OK means the call enqueued nothing
 *     (argument errors) or that a CUDA call failed; nsga3_last_error()
 *     describes it.  Errors detected on the device (non-finite objectives,
 *     timeouts, internal invariant failures) are sticky in the context and
 *     returned by nsga3_sync().  Nothing aborts the process.
 *   - One context must not be used from two host threads at once.
 */
#ifndef NSGA3_H
#define NSGA3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nsga3_ctx nsga3_ctx;

typedef enum {
    NSGA3_OK = 0,
    NSGA3_EINVAL = 1,     /* bad argument */
    NSGA3_ENOMEM = 2,     /* device allocation failed */
    NSGA3_ECUDA = 3,      /* a CUDA runtime call failed */
    NSGA3_ENONFINITE = 4, /* NaN or Inf in the objectives given to nsga3_select */
    NSGA3_ETIMEOUT = 5,   /* a bounded device wait expired */
    NSGA3_ESTATE = 6,     /* call not valid in this context state */
    NSGA3_EINTERNAL = 7   /* a device-side invariant failed */
} nsga3_status;

/* Options of a context.  Initialise with nsga3_default_opts(). */
typedef struct {
    uint64_t seed;          /* Philox key (seed lo, seed hi) */
    int p2;                 /* inner-layer Das-Dennis divisions, 0 = single layer */
    double tau;             /* inner-layer shrink factor (z_in = (1-tau)/m + tau z) */
    float eta_c;            /* SBX distribution index (default 20) */
    float eta_m;            /* polynomial-mutation distribution index (default 20) */
    float p_c;              /* crossover probability per pair (default 1) */
    float p_m;              /* mutation probability per variable; < 0 -> 1/d (default) */
    int full_sort;          /* 1: rank every front (F_drop gets its real front index) */
    int debug_recheck_all;  /* 1: association rechecks every reference in FP64 */
    const float* W;         /* host, m x (m-1) row-major weights of the softmax-simplex
                               objective f = (1+g) softmax(W x[:m-1]); NULL: the context
                               only serves nsga3_select / nsga3_set_population */
    int streaming;          /* 1: no dominance matrix; the peel recomputes the dominance
                               of each front's members on the fly (device memory O(N)
                               instead of (2N)^2 / 8 bytes; same results); m <= 10 */
    int norm_history;       /* 1: normalization keeps a running ideal point (minimum over
                               every merged population so far) and remembers the extreme
                               points, which stay candidates in later generations; the
                               history starts empty at nsga3_create and nsga3_init and is
                               updated by every selection that normalizes.  0: stateless
                               (ideal and extremes of the current S u F_l only) */
    int problem;            /* 0: softmax-simplex objective (needs W); 1: 0-1 multi-objective
                               knapsack over d items (needs the kp_* arrays): binary
                               variables, uniform crossover, bit-flip mutation, repair;
                               m <= 10 */
    const int32_t* kp_profit;   /* host, m x d profits (> 0), read during create only */
    const int32_t* kp_weight;   /* host, m x d weights (> 0), read during create only */
    const int32_t* kp_capacity; /* host, m capacities, read during create only */
    int wait_ms;            /* budget of every device-side wait (the grid barriers of the
                               cooperative kernels), in ms of device time; past it the
                               kernel records NSGA3_ETIMEOUT and returns (default 20,000;
                               <= 0: the default) */
    int phase_timing;       /* CUDA events recorded inside the graphs for nsga3_phase_times:
                               0 (default) none; 1 around the dominance build and the
                               front peel only; 2 around every phase.  Each event node
                               adds a few microseconds to every replay */
    int dom_ctas_per_sm;    /* launch shape of the dominance build (m <= 10): persistent
                               CTAs per SM, 0 (default) = as many as are resident at once;
                               larger values are clamped to that.  Results do not depend
                               on it (a tuning knob, swept by bench.py --workload shapes) */
    int peel_ctas_per_sm;   /* launch shape of the cooperative front peel: CTAs per SM,
                               0 (default) = as many as are resident at once; larger values
                               are clamped to that.  Results do not depend on it */
} nsga3_opts;

/* Fills *o with the defaults above (seed 0, single layer, tau 0.5). */
void nsga3_default_opts(nsga3_opts* o);

/*
 * Creates a context for populations of N individuals (merged 2N), m
 * objectives (2 <= m <= 512; the objective sweep of the paper's Table II
 * reaches 512; kernels are specialised for each m <= 10 and take m at run
 * time above; with m > 32 the intercept system is eliminated by a
 * cooperative grid), d variables (d >= m - 1 when W is given) and
 * Das-Dennis divisions ref_divisions >= 1 (Sec. II-C: w points uniform on
 * the unit simplex; opts->p2 > 0 adds an inner layer).  N must be even,
 * 2 <= N and 2N <= 2^21.  Allocates all device workspace (about
 * (2N)^2 / 8 bytes for the dominance matrix) on the current device and
 * builds the reference directions.  *out receives the context.
 * Errors: EINVAL (sizes), ENOMEM, ECUDA.
 */
nsga3_status nsga3_create(int m, int d, int N, int ref_divisions, const nsga3_opts* opts,
                          nsga3_ctx** out);

/* Frees the context and its device memory (synchronises its work). */
void nsga3_destroy(nsga3_ctx* ctx);

/*
 * Self-test of the device-side wait budget (no counterpart in the paper):
 * enqueues one single-CTA kernel that waits, with the same bounded wait as
 * the grid barriers, on a control word that nothing sets.  When opts.wait_ms
 * of device time have passed it records NSGA3_ETIMEOUT in the context and
 * returns; the next nsga3_sync reports (and clears) it and the context stays
 * usable.  Asynchronous on `stream`; never faults or traps.
 * Errors: EINVAL (null context), ECUDA (launch).
 */
nsga3_status nsga3_wait_probe(nsga3_ctx* ctx, void* stream);

/* Device bytes nsga3_create allocates for these arguments (each buffer
 * rounded up to 256 bytes); no allocation and no device work.  Without a
 * device the per-SM buffers are sized for 256 SMs (an upper bound).
 * Errors: EINVAL as nsga3_create. */
nsga3_status nsga3_workspace_bytes(int m, int d, int N, int ref_divisions, const nsga3_opts* opts,
                                   uint64_t* bytes);

/* Human-readable description of the last error of ctx (or of the last failed
 * nsga3_create on this thread when ctx is NULL).  Never NULL. */
const char* nsga3_last_error(const nsga3_ctx* ctx);

/* Number w of reference directions. */
int nsga3_num_refs(const nsga3_ctx* ctx);

/* Copies the w x m FP64 reference directions (Das-Dennis, lexicographic order
 * of the compositions, outer layer first) to Z (any).  Synchronous. */
nsga3_status nsga3_get_refs(nsga3_ctx* ctx, double* Z);

/*
 * Environmental selection of N out of the merged 2N individuals (Alg. 1
 * from the non-dominated sort on, Alg. 2).
 *   objs      any, 2N x m FP32 objectives (minimised); read before return
 *             on the stream.
 *   ranks     any, 2N int32 out: 0-based front index for fronts F_1..F_l,
 *             -1 for F_drop (with opts.full_sort every front is ranked).
 *   selected  any, N int32 out: indices of P_{t+1} in ascending order.
 * Random choices of the niche selection use this context's generation
 * counter (nsga3_set_counter); nsga3_select does not advance it.
 * Non-finite objectives set NSGA3_ENONFINITE, reported by nsga3_sync().
 */
nsga3_status nsga3_select(nsga3_ctx* ctx, const float* objs, int32_t* ranks, int32_t* selected,
                          void* stream);

/* Initial population: x ~ U[0,1]^d from Philox(i*d+v, 0, 6, 0), evaluated;
 * parent ranks 0; generation counter 0.  Needs opts.W. */
nsga3_status nsga3_init(nsga3_ctx* ctx, void* stream);

/* Variation + objective only (Alg. 1, the crossover and mutation step): children of the current
 * parents into rows N..2N-1 of the merged population (see
 * nsga3_get_children).  Does not advance the counter.  Needs opts.W. */
nsga3_status nsga3_vary(nsga3_ctx* ctx, void* stream);

/* One generation (Alg. 1): variation, merge, selection, next population;
 * advances the counter by one.  One CUDA-graph launch of plain kernel nodes
 * (every front is peeled inside one cooperative kernel). Needs opts.W. */
nsga3_status nsga3_step(nsga3_ctx* ctx, void* stream);

/* `generations` calls of nsga3_step. */
nsga3_status nsga3_run(nsga3_ctx* ctx, int generations, void* stream);

/* Advances every context in ctxs[0..n) by `generations` generations with
 * batched CUDA graphs: one graph holds 4 consecutive generations of every
 * run as parallel branches (a second graph one generation, for the
 * remainder), so the runs' kernels overlap on the device and small runs run
 * ahead of large ones between launches.  Results equal each run stepped
 * alone.  Every context needs opts.W and must live on the current device.
 * The graphs are kept by ctxs[0] and rebuilt whenever the list differs from
 * the one they were built for; lists are compared by the contexts' creation
 * serials (unique for the life of the process), not by address, so a
 * context created where a destroyed one lived never inherits its graphs.
 * Errors: EINVAL (n < 1, a NULL context or one without an objective, a
 * context listed twice, generations < 0), ECUDA. */
nsga3_status nsga3_run_batch(nsga3_ctx** ctxs, int n, int generations, void* stream);

/* How many times ctx (as ctxs[0] of nsga3_run_batch) has built its batched
 * graphs (diagnostics; no device work).  Errors: EINVAL (NULL argument). */
nsga3_status nsga3_batch_graph_builds(const nsga3_ctx* ctx, int64_t* builds);

/* Copies the N parents out: X (any, N x d), F (any, N x m), rank (any, N).
 * Any pointer may be NULL to skip it. */
nsga3_status nsga3_get_population(nsga3_ctx* ctx, float* X, float* F, int32_t* rank, void* stream);

/* Replaces the N parents: X (any, N x d), F (any, N x m), rank (any, N).
 * Any pointer may be NULL to keep the current values. */
nsga3_status nsga3_set_population(nsga3_ctx* ctx, const float* X, const float* F,
                                  const int32_t* rank, void* stream);

/* Copies the N children of the last nsga3_vary / nsga3_step variation:
 * X (any, N x d), F (any, N x m); either may be NULL. */
nsga3_status nsga3_get_children(nsga3_ctx* ctx, float* X, float* F, void* stream);

/* Sets / reads the Philox generation counter (counter word 1). */
nsga3_status nsga3_set_counter(nsga3_ctx* ctx, uint64_t gen, void* stream);
nsga3_status nsga3_get_counter(nsga3_ctx* ctx, uint64_t* gen, void* stream); /* synchronous */

/* Waits for `stream`, then returns and clears the context's sticky device
 * status (NSGA3_OK, NSGA3_ENONFINITE, NSGA3_ETIMEOUT or NSGA3_EINTERNAL). */
nsga3_status nsga3_sync(nsga3_ctx* ctx, void* stream);

/*
 * Diagnostics of the last selection (synchronous): info[0..12] =
 *   l, |S|, K, |F_l|, niching needed, normalization fallback,
 *   peel passes, |S u F_l|, level L*, refs taken at L*, list overflows,
 *   debug recheck misses, dominator word-rows read by the peel (each row
 *   is 2N 32-bit words).  info must hold 13 entries.
 */
nsga3_status nsga3_get_selection_info(nsga3_ctx* ctx, int32_t* info);

/* Capacity paths the niching kernels took in the last selection
 * (synchronous; diagnostics for tests of the paths that only large or
 * skewed inputs reach): a bit mask of
 *   NSGA3_PATH_UNSTAGED  more than 12,288 references: the level kernel reads
 *                        the niche counts from global memory
 *   NSGA3_PATH_DEEP      the level threshold L* is 4,096 or more (binary
 *                        search instead of the level histogram)
 *   NSGA3_PATH_CKOVER    more than 4,096 references hold a level-L* member
 *                        (with NSGA3_PATH_UNSTAGED)
 *   NSGA3_PATH_BINOVER   a radix bin of the level kernel held more than
 *                        1,024 reference keys
 *   NSGA3_PATH_LARGE     a partial take from a reference of more than 32
 *                        members (block-wide member selection)
 *   NSGA3_PATH_RADIX     the block-wide selection ran an 8-bit radix pass
 *   NSGA3_PATH_RADIX2    ... and a second one.
 * Errors: EINVAL (NULL argument), ECUDA. */
#define NSGA3_PATH_UNSTAGED 1u
#define NSGA3_PATH_DEEP 2u
#define NSGA3_PATH_CKOVER 4u
#define NSGA3_PATH_BINOVER 8u
#define NSGA3_PATH_LARGE 16u
#define NSGA3_PATH_RADIX 32u
#define NSGA3_PATH_RADIX2 64u
nsga3_status nsga3_get_selection_paths(nsga3_ctx* ctx, uint32_t* paths);

/* Work of the dominance build in the last selection (synchronous;
 * diagnostics, m <= 10, zeros above): stats[0..7] = block pairs (32 x 32
 * points, upper triangle) ruled out without a test, tested in one direction
 * with objectives 1..m-1 (every row f_0 below every column f_0), tested in
 * the "row dominates column" direction only, in the "column dominates row"
 * direction only, tested both ways, 256 x 256 tiles with no block pair to
 * test, the (lane, column) point pairs the kernel compared (one-direction
 * block pairs compare only their live rows and columns), and the pairs of
 * a live row and a live column among them.  stats must hold 8 values.
 * Errors: EINVAL (NULL argument), ECUDA. */
nsga3_status nsga3_get_dominance_stats(nsga3_ctx* ctx, int64_t* stats);

/* Self-test of the block-wide selection routine that the niching kernels
 * use to take the smallest (priority, index) keys (Alg. 2's random pick of
 * references and members, read as the smallest Philox priorities): one
 * CTA marks the `need` smallest of n unique 64-bit keys.
 *   keys   device, n unique uint64 keys
 *   marks  device, n uint32 outputs: 1 for the need smallest keys, else 0
 *   paths  device, one uint32 output: NSGA3_PATH_RADIX / _RADIX2 bits of
 *          the radix passes the routine ran
 * Asynchronous on `stream`; allocates nothing.  Errors: EINVAL (NULL
 * pointer, n < 1, need outside [0, n]), ECUDA (launch).  Sets no message
 * for nsga3_last_error. */
nsga3_status nsga3_select_smallest_probe(const uint64_t* keys, int n, int need, uint32_t* marks,
                                         uint32_t* paths, void* stream);

/* Measured instruction-issue ceiling of the dominance build (no counterpart
 * in the paper; used as the denominator of its roofline): a kernel issues
 * the dominance test's instruction mix -- two FP32 subtractions and one
 * 3-input logic operation on their sign bits per step, eight independent
 * chains per thread, no memory traffic -- on blocks_per_sm x (SM count)
 * CTAs of 256 threads, `iters` steps per chain, `reps` timed launches after
 * one warm-up launch (CUDA events on `stream`).  *instr_per_s receives the
 * thread-instructions per second of the fastest launch, *best_ms (may be
 * NULL) its time.  in_scratch: device, at least 256 bytes the caller owns
 * (the kernel reads 32 floats from its start and may write one word at
 * byte 128).  Synchronous.  Errors: EINVAL (NULL pointer, blocks_per_sm
 * outside [1, 64], iters or reps < 1), ECUDA.  Sets no message for
 * nsga3_last_error. */
nsga3_status nsga3_issue_probe(int blocks_per_sm, int iters, int reps, double* instr_per_s, float* best_ms,
                               void* in_scratch, void* stream);

/* Normalization of the last niching selection (synchronous): ideal point
 * zstar[m], intercepts a[m] (FP64), extreme-point indices ext[m] (with
 * opts.norm_history an index 2N + r names the r-th remembered extreme
 * vector); any may be NULL. */
nsga3_status nsga3_get_normalization(nsga3_ctx* ctx, double* zstar, double* a, int32_t* ext);

/* Association of the last niching selection (synchronous): pi (any, 2N
 * int32, -1 outside S u F_l) and dist (any, 2N FP64). */
nsga3_status nsga3_get_association(nsga3_ctx* ctx, int32_t* pi, double* dist);

/*
 * Device times (ms) of the phases of the last replayed generation or
 * selection, measured by CUDA events recorded inside the graph:
 *   ms[0] variation+objective, ms[1] per-selection reset (+ finite check),
 *   ms[2] dominance matrix kernel, ms[3] front peel (all passes),
 *   ms[4] normalization + association + niching, ms[5] compaction + gather,
 *   ms[6] whole graph.  Synchronous; n is the capacity of ms (up to 7).
 * Phases that opts.phase_timing does not time read -1 (with phase_timing
 * 1 only ms[2] and ms[3] are measured).  Errors: EINVAL with phase_timing 0 (eager
 * execution, NSGA3_EAGER=1, times every phase whatever the option).
 */
nsga3_status nsga3_phase_times(nsga3_ctx* ctx, float* ms, int n);

/* Kernel launches made by the last replayed generation or selection (the
 * peel is one launch whatever the number of fronts).  Synchronous. */
nsga3_status nsga3_last_launches(nsga3_ctx* ctx, int32_t* launches);

/* Kernel launches made on behalf of ctx since nsga3_create (the set-up
 * kernels excluded): initialisation, variation and every replayed generation
 * or selection.  Synchronous. */
nsga3_status nsga3_total_launches(nsga3_ctx* ctx, int64_t* launches);

/* ------------------------------------------------------------------------
 * Run server: continuous batching of independent runs on one GPU.
 *
 * Requests arrive at any time (any host thread).  A worker thread admits
 * them in arrival order while a slot is free and the memory budget holds the
 * run's workspace (nsga3_workspace_bytes), carving contexts out of one
 * arena allocated at creation, so admission and release never call
 * cudaMalloc or cudaFree.  Admitted runs advance concurrently, each on its
 * own stream, `gens_per_launch` generations per launch batch; a finished
 * run's population is copied to host memory and its slot and memory are
 * reused at once.  A run's result depends only on its request (Philox
 * counters), never on the other runs in flight.
 * ------------------------------------------------------------------------ */
typedef struct nsga3_server nsga3_server;

typedef struct {
    int m, d, N, ref_divisions;  /* as nsga3_create */
    int generations;             /* >= 0 */
    nsga3_opts opts;             /* opts.W (host, m x (m-1)) is required and is
                                    copied by nsga3_server_submit */
} nsga3_request;

typedef struct {
    int32_t status;              /* nsga3_status of the run */
    int32_t m, d, N, generations;
    uint64_t workspace_bytes;
    double t_submit, t_admit, t_done;  /* seconds on the server clock; t_admit < 0 if never admitted */
    char message[256];           /* error text when status != NSGA3_OK */
} nsga3_run_info;

typedef struct {
    int64_t submitted, admitted, completed, active, pending, peak_active;
    int64_t launches;            /* kernels launched for the completed runs */
    uint64_t budget_bytes, bytes_in_use, peak_bytes;
} nsga3_server_stats;

/* Creates a server on the current device: one cudaMalloc of memory_budget
 * bytes, max_active slot streams (1..1024) and the worker thread.
 * max_active = 1 serves one run at a time (the plain path).  The slot
 * streams share the device's hardware work queues (8 unless the process sets
 * CUDA_DEVICE_MAX_CONNECTIONS, up to 32, before CUDA is initialised); with
 * more slots than queues, kernels of unrelated runs can wait on one another.
 * Errors: EINVAL, ENOMEM (the budget cannot be allocated), ECUDA. */
nsga3_status nsga3_server_create(uint64_t memory_budget, int max_active, int gens_per_launch,
                                 nsga3_server** out);

/* Queues a request; *id receives its id (0, 1, ... in submission order).
 * Thread-safe, never blocks on the device.  Errors: EINVAL (arguments as
 * nsga3_create, generations < 0, no opts.W), ESTATE (server shutting down).
 * A request whose workspace exceeds the budget completes with ENOMEM. */
nsga3_status nsga3_server_submit(nsga3_server* srv, const nsga3_request* req, int64_t* id);

/* Waits up to timeout_ms (< 0: forever) for a completed run not yet
 * returned by an earlier wait; *id = -1 on timeout. */
nsga3_status nsga3_server_wait(nsga3_server* srv, int timeout_ms, int64_t* id);

/* Copies a completed run's final population to host memory (X: N x d,
 * F: N x m, rank: N; any may be NULL), fills *info (may be NULL) and
 * releases the result.  Returns the run's status; EINVAL for an unknown or
 * already fetched id. */
nsga3_status nsga3_server_fetch(nsga3_server* srv, int64_t id, float* X, float* F, int32_t* rank,
                                nsga3_run_info* info);

nsga3_status nsga3_server_get_stats(nsga3_server* srv, nsga3_server_stats* stats);

/* Seconds since the server was created (the clock of nsga3_run_info). */
double nsga3_server_now(const nsga3_server* srv);

/* Description of the last failed nsga3_server_submit. */
const char* nsga3_server_last_error(const nsga3_server* srv);

/* Stops the server: pending requests complete with ESTATE, active runs are
 * stopped after their queued work; frees the arena and the streams. */
void nsga3_server_destroy(nsga3_server* srv);

/*
 * Largest n accepted by nsga3_rank_noalloc. */
#define NSGA3_NOALLOC_MAX_N 2048

/*
 * Non-dominated sorting ranks of n points, with no device allocation and no
 * context.  The paper has no counterpart: it is a convenience for callers
 * that cannot allocate device memory -- code enqueueing work while a stream
 * is captured into a CUDA graph (allocation is not a stream operation),
 * real-time loops whose allocator use is forbidden, and plug-ins that a host
 * application only gives pre-reserved memory.  nsga3_create allocates its
 * workspace, so none of them can use nsga3_select.
 *
 *   objs   device, n x m FP32 objectives, row-major, minimised
 *   n      1 <= n <= NSGA3_NOALLOC_MAX_N
 *   m      2 <= m <= 10
 *   ranks  device, n int32 outputs: 0 for the first non-dominated front,
 *          1 for the next, ... (the front index of every point, as
 *          nsga3_select gives it with full_sort = 1).  Comparisons are IEEE:
 *          a NaN objective makes a point neither dominate nor be dominated.
 *   stream cudaStream_t as void* (NULL = legacy default stream); the call is
 *          asynchronous and stream-ordered.
 *
 * Workspace: one statically sized __device__ array (about 530 KB) that every
 * GPU on which this library is loaded holds until the process exits.  The
 * first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  The address is cached per device for the life of the
 * process: after cudaDeviceReset (or any other reset of the device's primary
 * context) the library's device symbols may be reloaded elsewhere, so this
 * entry point must not be called again in that process.  Every call on a
 * device shares the array, which keeps the
 * last call's contents; each call clears what must start at zero itself.
 * Calls whose executions overlap on the GPU (other streams, other host
 * threads) race on the array: order them on one stream or with events.
 *
 * Returns NSGA3_EINVAL, enqueuing nothing, when a pointer is NULL, n is out
 * of [1, NSGA3_NOALLOC_MAX_N] or m out of [2, 10]; NSGA3_ECUDA when there is
 * no usable device or the address lookup or the launch fails.  The call sets
 * no message for nsga3_last_error.
 */
nsga3_status nsga3_rank_noalloc(const float* objs, int n, int m, int32_t* ranks, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NSGA3_H */
