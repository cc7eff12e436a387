/*
 * dope.h -- C-ABI of the GB300 DOPE ADMM hot path.
 *
 * DOPE (Dolz, Ben Ayed, Desrosiers, "DOPE: Distributed Optimization for
 * Pairwise Energies", arXiv 1704.03116) minimises the binary pairwise energy
 *
 *     E(y) = sum_i u_i y_i + lambda sum_{edges ij} w_ij |y_i - y_j|       (Eq. 1)
 *
 * by splitting the grid into sub-regions (blocks) and running the ADMM of
 * Algorithm 1: every block solves its own graph-cut sub-problem with unaries
 * shifted by the consistency variable y and the multipliers a (Eq. 8), then y
 * (Eq. 10) and a (Eq. 11) are updated, mu grows by mu_fact, until every block
 * satisfies ||yhat_k - S_k y||_2 <= eps.  This library runs that loop on one
 * GPU: one CTA per block with the block's residual graph in shared memory
 * (push-relabel + BFS, canonical minimal cut), and a fused elementwise kernel
 * for the y / a updates.  Partitions are non-overlapping (Q = I, the paper's
 * Size00) unless dope_params.grow asks for the overlapping ones of Section 3
 * (Size10 / Size25); connectivities 24 / 48 / 80 / 32 select Section 3's
 * larger kernels, and dope_params.lsa_steps > 0 admits non-submodular
 * weights (blocks solved by LSA-TR, Section 3.4).
 *
 * Conventions
 *  - Grids: 2-D (H, W) or 3-D (D, H, W), row-major, pixel index
 *    i = (z*H + y)*W + x.  N = number of pixels.  N < 2^31.
 *  - Connectivity 4 or 8 (2-D), 6 (3-D).  Forward offsets, in this order:
 *      4-conn (dy,dx): (0,+1) (+1,0);  8-conn adds (+1,+1) (+1,-1);
 *      6-conn (dz,dy,dx): (0,0,+1) (0,+1,0) (+1,0,0).
 *  - Weights: int32 wq[conn/2][N]; wq[k][i] is the pairwise weight of the
 *    edge from pixel i to its forward neighbour along offset k, already in
 *    fixed point x1024 (wq = rne(1024 w)).  Entries whose neighbour lies
 *    outside the grid must be 0.  All entries must be >= 0 (submodular, the
 *    condition in the footnote of Section 1 for |y_i - y_j| terms).
 *  - Quantised instance: U_i = rne(1024 u_i) (int32, |U_i| < 2^30),
 *    Wl_ij = rne(lambda * wq_ij) (int32, < 2^24); E_int(y) = sum U_i y_i +
 *    sum over undirected edges Wl_ij |y_i - y_j| (each edge once, Eq. 3);
 *    E = E_int / 1024 exactly.
 *  - Labels: uint8, 1 = foreground (y_i = 1).  Among minimisers of a block
 *    sub-problem the pointwise-minimal one is returned (unique), so labels
 *    are deterministic and bit-exact.
 *  - Memory: `where` = DOPE_HOST (0) for host pointers or DOPE_DEVICE (1) for
 *    device pointers of the current device.  The caller owns every buffer it
 *    passes; the library only reads / writes it during the call, ordered on
 *    `stream` (a cudaStream_t, NULL = legacy default stream).  Calls that
 *    return results to the host synchronise `stream`.  Device state is owned
 *    by the context.
 *  - Every function returns a DOPE_* status; no exception crosses the ABI.
 *    A context is not thread-safe; use one context per stream.
 */
#ifndef DOPE_H
#define DOPE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DOPE_OK            0
#define DOPE_EINVAL        1   /* bad shape / connectivity / block / pointer / order of calls */
#define DOPE_EUNSUPPORTED  2   /* negative weight (non-submodular) on the submodular path */
#define DOPE_ENOMEM        3   /* device or host allocation failed */
#define DOPE_EOVERFLOW     4   /* |U_i| >= 2^30 or Wl_ij >= 2^24, non-finite u */
#define DOPE_ENOTCONV      5   /* max_iter reached before the stop test held; outputs valid */
#define DOPE_ETIMEOUT      6   /* a bounded device loop or wait ran out; outputs not valid */
#define DOPE_ECUDA         7   /* a CUDA runtime call failed */
#define DOPE_ECANCELED     8   /* the request was cancelled (dope_server_cancel) */

#define DOPE_HOST   0
#define DOPE_DEVICE 1

typedef struct dope_ctx dope_ctx;

/* Algorithm 1 inputs (lambda, eps, mu0, mu_fact) plus solver knobs.
 * Defaults (dope_default_params): mu0 = 0 -> 100 for 2-D grids and 500 for
 * 3-D grids (the paper's settings, Section 3), mu_fact = 1.05, eps = 1e-3,
 * max_iter = 1000, relabel_period = 0 (automatic), threads = 0 (automatic),
 * max_pulses = 0 (automatic: 64 * block volume + 4096), fold_rounds = 0
 * (automatic: 3), launch_mode = 0 (persistent, when the device can run it).
 * relabel_period 0 means 8.  The knobs change speed only, never results: the
 * block cut is exact for any of them. */
typedef struct {
    double mu0;
    double mu_fact;
    double eps;
    int max_iter;
    int relabel_period;  /* push-relabel pulses between global relabels */
    int threads;         /* threads per block-solver CTA (multiple of 32; 0: one per node up
                            to 512, a quarter of the nodes for non-submodular blocks) */
    int max_pulses;      /* bound on push-relabel pulses per block and iteration */
    int fold_rounds;     /* bound on exact-folding rounds per block and iteration */
    int launch_mode;     /* 0: one persistent cooperative launch per solve / iterate call,
                               with run-ahead windows once labels stop moving (on grids
                               with more blocks than co-resident CTAs the windows run in
                               a second launch queued right behind the first);
                            1: two launches per iteration (solve, update);
                            2: persistent launch without run-ahead windows */
    int grow[3];         /* overlapping partition (Section 2: blocks "can overlap"; Section 3's
                            Size10 / Size25): every block grown by grow[a] pixels on both sides
                            along axis a (first ndim entries, same order as the grid), clipped to
                            the grid; 2 grow[a] <= block_shape[a].  All 0 (default): the
                            non-overlapping partition, Q = I.  Overlapping contexts run three
                            launches per iteration; the batched calls and the server take only
                            Q = I contexts. */
    int lsa_steps;       /* 0 (default): submodular weights only (negative weights are
                            DOPE_EUNSUPPORTED).  > 0: weights of any sign (non-submodular pairwise
                            terms, Section 3.4); every block's Eq. 8 is solved by LSA-TR (trust-region
                            local submodular approximation, each step an exact block cut) with at
                            most lsa_steps steps per block and iteration.  Such contexts run two
                            launches per iteration, Q = I only. */
    int barrier_timeout_us;  /* longest wait at a grid barrier of the one-launch solve before the
                            launch gives up: every CTA leaves, the call returns DOPE_ETIMEOUT and
                            the context stays usable.  0 (default): about 2 s. */
} dope_params;

/* Statistics of the last dope_solve / dope_iterate call. */
typedef struct {
    int iterations;             /* ADMM iterations run (Algorithm 1 loop count) */
    int converged;              /* 1 if the stop test held */
    int64_t pulses_total;       /* push-relabel pulses summed over blocks and iterations */
    int pulses_max;             /* most pulses one block took in one iteration */
    int64_t free_nodes_total;   /* nodes left for push-relabel after exact folding */
    double rmax_last;           /* max_k ||yhat_k - S_k y||_2 after the last iteration */
    int64_t kernel_launches;    /* kernels this library launched during the call */
    int64_t bfs_levels_total;   /* BFS levels (barrier rounds) summed over blocks */
    int bfs_levels_max;         /* longest single BFS of one block */
    int fold_rounds_max;        /* most folding rounds one block took */
    double phase_cycles[4];     /* SM cycles of the block solver, summed over CTAs:
                                   capacity build, folding, push-relabel pulses, BFS */
    double loop_cycles[4];      /* persistent launch, summed over CTAs and ordinary iterations:
                                   solve phase, first barrier wait, update phase, second
                                   barrier wait (k_admm_resident: the last entry is its
                                   run-ahead windows) */
    int windows;                /* run-ahead windows run (launch_mode 0) */
    int window_iterations;      /* iterations committed from run-ahead windows */
    double window_cycles[8];    /* run-ahead windows, summed over CTAs.  k_admm_resident: build,
                                   block solve, label check, own update, halo update, window
                                   set-up, wait at the closing barrier, rest of the resolution.
                                   k_admm_persistent: SM cycles of its three phases and the
                                   barrier wait after each (state stepping, wait, certificates,
                                   wait, commit, wait), then two counts: face slots certified
                                   and exact unaries evaluated where a certificate was too weak */
    int solver_kernel;          /* kernel that ran the iterations: 0 k_block_solve + k_face_update
                                   (two launches per iteration), 1 k_admm_persistent, 2 k_admm_resident,
                                   3 k_admm_batch (dope_iterate_batch) */
    int reserved;
    int64_t blocks_solved;      /* k_admm_persistent with worklists: block solves run from the
                                   worklists (after each launch's first iteration, which does
                                   every block); 0 on the other kernels */
    int64_t blocks_updated;     /* likewise, block updates (Eq. 10 / 11) run from the worklists */
    int64_t blocks_solved_partial;  /* of blocks_solved, those whose nodes were all still forced, so
                                   that only their active and changed chunks of face pixels were
                                   evaluated (no capacity build, no cut); after a launch's first
                                   iteration, blocks whose every pixel was found forced that way */
} dope_stats;

/* Device time of the hot-path kernels, measured with CUDA events on the
 * caller's stream while profiling is on (dope_set_profiling).  Only launches
 * that did work are counted (launches issued past convergence return at
 * once and are excluded).  launch_mode 1: index 0 = block solver (steps
 * a4-a6), index 1 = face update (steps a2-a3).  launch_mode 0: index 0 = the
 * persistent kernel (all steps, one launch per call), index 1 unused. */
typedef struct {
    int64_t launches[2];
    double ms[2];
    int64_t first_iteration_launches;   /* block-solver launches that were iteration 1 */
    double first_iteration_ms;          /* their device time */
    int64_t iterations;                 /* ADMM iterations the timed launches covered */
} dope_profile;

/* Fill *p with the defaults above. */
void dope_default_params(dope_params *p);

/* Create a context for one grid / partition / lambda (Algorithm 1 inputs,
 * Section 2 "Block partition scheme").
 *   grid[ndim]        ndim = 2: (H, W); ndim = 3: (D, H, W)
 *   connectivity      4 or 8 for ndim = 2, 6 for ndim = 3
 *   block_shape[ndim] sub-region shape in pixels; must divide grid exactly;
 *                     block volume in [1, 4096]
 *   lambda            >= 0 (Eq. 1)
 *   p                 NULL for defaults
 * Allocates the device state on the current device.  *out receives the
 * context (NULL on error). */
int dope_create(const int64_t *grid, int ndim, int connectivity, const int32_t *block_shape,
                double lambda, const dope_params *p, dope_ctx **out);

/* Unaries u[N] (float32, image order), Eq. 2: u_i = log p(y_i=0|x_i) -
 * log p(y_i=1|x_i), so u_i < 0 favours foreground.  Quantised on the device
 * to U_i = rne(1024 u_i).  Returns DOPE_EOVERFLOW if some |U_i| >= 2^30 or
 * u_i is not finite.  Synchronises `stream`. */
int dope_set_unaries(dope_ctx *ctx, const float *u, int64_t n, int where, void *stream);

/* Pairwise weights wq[conn/2][N] (int32, image order, x1024), Eq. 1.
 * Quantised on the device to Wl = rne(lambda * wq).  DOPE_EUNSUPPORTED if
 * some wq < 0, DOPE_EINVAL if a weight toward a pixel outside the grid is
 * non-zero, DOPE_EOVERFLOW if some Wl >= 2^24.  Synchronises `stream`. */
int dope_set_weights(dope_ctx *ctx, const int32_t *wq, int64_t n, int where, void *stream);

/* Unaries (Eq. 2) and weights (Eq. 1) together, asynchronously: u [n] and
 * wq [conn/2][n] in the layouts above, the same copies and quantisation as
 * dope_set_unaries + dope_set_weights, with no
 * synchronisation.  The quantisers' status (DOPE_EOVERFLOW,
 * DOPE_EUNSUPPORTED, DOPE_EINVAL for the inputs) is reported by the next call
 * on the context that synchronises (dope_solve reads it with its results, in
 * its one synchronisation); after such an error both inputs count as unset.
 * Host inputs are copied on `stream`: they must stay valid and unchanged
 * until the next synchronising call on the context. */
int dope_set_inputs(dope_ctx *ctx, const float *u, const int32_t *wq, int64_t n, int where, void *stream);

/* Algorithm 1 from its initial state (y = 1/2, a = 0, mu = mu0) until every
 * block has ||yhat_k - S_k y||_2 <= eps (tested after each iteration, so at
 * least one runs) or max_iter iterations.  Writes labels[N] (image order;
 * the yhat of the last iteration), *energy_int = E_int(labels) (may be NULL)
 * and *iterations (may be NULL).  Returns DOPE_OK, or DOPE_ENOTCONV with
 * valid outputs when max_iter was reached.  Synchronises `stream`. */
int dope_solve(dope_ctx *ctx, uint8_t *labels, int where, int64_t *energy_int,
               int *iterations, void *stream);

/* dope_solve (Algorithm 1 to its stop test) in two halves, so that several
 * solves (on one or more contexts) can be queued before the host waits.  dope_solve_begin issues the solve on
 * `stream` and returns without synchronising when the solve is one launch
 * (the default launch mode on a partition without overlap, submodular
 * weights); other contexts solve inside it.  dope_solve_end synchronises
 * `stream` and returns what dope_solve returns (status, E_int, iterations);
 * the labels are in `labels` once it has returned.  Between the two calls the
 * context takes no other call; host labels and inputs must stay valid until
 * dope_solve_end.  DOPE_EINVAL: a second begin without an end, or an end
 * without a begin. */
int dope_solve_begin(dope_ctx *ctx, uint8_t *labels, int where, void *stream);
int dope_solve_end(dope_ctx *ctx, int64_t *energy_int, int *iterations, void *stream);

/* Reset the ADMM state to y = 1/2, a = 0, mu = mu0, t = 0 (Algorithm 1,
 * Initialization). */
int dope_reset(dope_ctx *ctx);

/* Run up to n_iter further iterations of Algorithm 1 from the current state,
 * stopping early when the stop test holds.  *iterations_done = total
 * iterations since the last reset, *converged = 1 if the stop test held
 * after the last iteration run.  Synchronises `stream`. */
int dope_iterate(dope_ctx *ctx, int n_iter, int *iterations_done, int *converged, void *stream);

/* Overlapping contexts (grow != 0): the per-block state, box-major -- block k
 * is the box of (block_shape + 2 grow) pixels around its tile, node l at
 * k * V + l (V = box volume; nodes outside the grid are 0): a (Eq. 11, one
 * multiplier per block copy of a pixel) and yhat (the block labels of the last
 * iteration).  cap = entries available in each array (K * V needed); *count =
 * K * V.  DOPE_EINVAL for non-overlapping contexts. */
int dope_get_block_state(dope_ctx *ctx, double *a, uint8_t *yhat, int64_t cap, int64_t *count,
                         void *stream);

/* Copy the ADMM state out (host buffers of N entries, image order):
 * y (Eq. 10), a (Eq. 11, one multiplier per pixel since Q = I), yhat (block
 * labels of the last iteration; 0 before the first), mu (value the next
 * iteration will use), t (iterations done).  Any pointer may be NULL.
 * Overlapping contexts give y, mu and t here (a and yhat must be NULL; they
 * are per block copy: dope_get_block_state). */
int dope_get_state(dope_ctx *ctx, double *y, double *a, uint8_t *yhat, double *mu, int *t,
                   void *stream);

/* Load an ADMM state (host buffers, image order; checkpoint / resume and
 * parity tests).  t = 0 requires y = 1/2 and a = 0 everywhere.  For t >= 1
 * the state must be one Algorithm 1 can reach with Q = I: every pixel with no
 * neighbour in another block must have y_i = yhat_i and a_i = 0 exactly
 * (Eq. 10 / 11 keep them so), else DOPE_EINVAL. */
int dope_set_state(dope_ctx *ctx, const double *y, const double *a, const uint8_t *yhat,
                   double mu, int t, void *stream);

/* Step a4 alone (test hook): the Eq. 8 unaries of the next iteration for the
 * current state, 1024 c_i rounded half-to-even, as int64 C[N] (host, image
 * order).  Values whose magnitude exceeds 2^62 are clamped to +-2^62. */
int dope_shifted_caps(dope_ctx *ctx, int64_t *C, void *stream);

/* Step a5 alone (test hook): solve every block's Eq. 8 min-cut for the given
 * int64 unaries C[N] (host, image order) with the block's n-links Wl, and
 * write the canonical block labels yhat[N] (host, image order).  Leaves the
 * ADMM state unchanged. */
int dope_block_cuts(dope_ctx *ctx, const int64_t *C, uint8_t *yhat, void *stream);

/* E_int of arbitrary labels[N] (image order) on the context's instance,
 * Eq. 1 in int64 (x1024). */
int dope_energy(dope_ctx *ctx, const uint8_t *labels, int where, int64_t *energy_int,
                void *stream);

/* Per-iteration max_k ||yhat_k - S_k y||_2 of the last solve / iterate
 * calls since the reset (host, up to cap entries); *count = entries written. */
int dope_trace(dope_ctx *ctx, double *rmax, int cap, int *count);

/* Statistics of the last dope_solve / dope_iterate call. */
int dope_get_stats(dope_ctx *ctx, dope_stats *st);

/* Turn per-kernel CUDA-event timing on (1) or off (0); turning it on clears
 * the accumulated profile. */
int dope_set_profiling(dope_ctx *ctx, int enable);

/* Accumulated per-kernel device times since profiling was turned on. */
int dope_get_profile(dope_ctx *ctx, dope_profile *out);

/* Number of blocks K and block volume of the context. */
int dope_get_geometry(dope_ctx *ctx, int64_t *n_pixels, int64_t *n_blocks, int *block_volume,
                      int *face_size);

/* Checked build (libdope_checked.so, compiled with DOPE_CHECKED; a test tool,
 * the paper has no counterpart).  Every shared-memory index
 * of the block solver and of the resident kernel is tested against its array
 * before the access; an index outside it is recorded (the first one since the
 * last clear) and the access goes to a scratch cell, so the kernel neither
 * faults nor writes outside the array, and the solve's results are then not
 * valid.  *first_bad (host) receives 0 if no index was outside, else
 * ((array length << 32) | index) + 1; clear != 0 resets the record
 * afterwards.  Synchronises the current device.  Returns DOPE_EUNSUPPORTED on
 * the ordinary library (which has no checks), DOPE_ECUDA if the record
 * cannot be read. */
int dope_check_status(uint64_t *first_bad, int clear);

/* Size of the device scratch array behind dope_solve_noalloc. */
#define DOPE_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Allocation-free variant of dope_solve, for callers that cannot allocate
 * device memory: code running while a framework's caching allocator holds
 * the GPU's memory, plugins whose host forbids cudaMalloc after start-up,
 * and latency-critical loops that cannot afford an allocation or the
 * synchronisation of cudaFree.  The paper has no counterpart; this is a
 * deployment entry point.
 *
 * It runs the same Algorithm 1 solve as dope_create + dope_set_unaries +
 * dope_set_weights + dope_solve (same kernels, same results), without a
 * context.  Arguments are those of dope_create plus: u[N] (float32, image
 * order) and wq[conn/2][N] (int32, image order) as DEVICE pointers on the
 * current device, labels[N] a DEVICE pointer on the current device receiving
 * the labels (image order), *energy_int and *iterations (host, may be NULL).
 * N is the product of grid[]; the function takes no lengths, so the caller
 * must supply buffers of at least these element counts (the Python binding
 * checks them).  Calls no cudaMalloc / cudaFree and no allocating library
 * routine: all device state lives in one static device array of
 * DOPE_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits.  The state takes about (5 + 4 conn/2) N + 16 K F bytes
 * (K blocks of F face pixels) plus 8 bytes per iteration of max_iter, each
 * part rounded up to 256 bytes: 8-connected 32x32 blocks cost about 23 bytes
 * per pixel (832 x 832 fits, 864 x 864 does not), 4-connected 16x16 blocks
 * about 16.  Problems that do not fit, and max_iter above
 * DOPE_NOALLOC_SCRATCH_BYTES / 8, are rejected with DOPE_EINVAL before any
 * GPU work.  The array's memory is taken when this library's device code is
 * first loaded on a device (the first call of an entry point that runs device
 * code there); a caller whose allocator reserves the device's memory should
 * make one call first.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current, and only a
 * successful lookup is kept (a failed one returns DOPE_ECUDA and is retried
 * by the next call); make that first call before any stream capture.  Every call
 * shares the array and it keeps the last call's contents (each call clears
 * what must start at zero itself): calls that overlap on the GPU -- on two
 * streams, or from two host threads -- race and corrupt each other; issue
 * them one after another.  Synchronises `stream`.  Returns what dope_solve
 * returns (DOPE_ENOTCONV with valid outputs at max_iter). */
int dope_solve_noalloc(const int64_t *grid, int ndim, int connectivity, const int32_t *block_shape,
                       double lambda, const dope_params *p, const float *u, const int32_t *wq,
                       uint8_t *labels, int64_t *energy_int, int *iterations, void *stream);

/* ---------------------------------------------------------------------------
 * Batched solves.  The paper runs the blocks of one problem in parallel
 * (Algorithm 1, "in parallel" over k); these calls run the blocks of many
 * problems in one persistent launch.  Each problem still runs its own
 * Algorithm 1 (own iteration count, mu and stop test) with the per-block
 * arithmetic of the single-problem path, so its iterates, labels and energy
 * are bit-identical to running it alone.
 * ------------------------------------------------------------------------- */
#define DOPE_BATCH_MAX 256

/* Advance n (1 .. DOPE_BATCH_MAX) distinct contexts together in one
 * cooperative launch: each runs up to n_iter more iterations of Algorithm 1
 * from its current state (never beyond its max_iter), stopping when its own
 * stop test holds.  The contexts may differ in grid, connectivity, block
 * shape, lambda and parameters; each must have its unaries and weights set.
 * Per context (arrays of n, any may be NULL): iterations[i] = iterations done
 * since its reset, converged[i] = its stop test held after its last
 * iteration, status[i] = its status.  Read labels with dope_labels.
 * Synchronises `stream`.  Returns DOPE_OK, the first nonzero per-context
 * status, DOPE_ETIMEOUT if a bounded grid-barrier wait gave up, or
 * DOPE_EUNSUPPORTED if the device cannot run cooperative launches. */
int dope_iterate_batch(dope_ctx *const *ctxs, int n, int n_iter, int *iterations, int *converged,
                       int *status, void *stream);

/* Labels of the last iteration run (Algorithm 1 output for Q = I: yhat;
 * image order, N bytes at `labels` in `where` memory) and *energy_int =
 * E_int of them (may be NULL), without running further iterations.
 * Synchronises `stream`. */
int dope_labels(dope_ctx *ctx, uint8_t *labels, int where, int64_t *energy_int, void *stream);

/* ---------------------------------------------------------------------------
 * Autotuner.  Picks, for one instance, the solver settings with the shortest
 * device time to convergence: block shape (optional), relabel frequency,
 * CTA width (256 threads: 3 CTAs per SM; 512 threads: 2 per SM), folding
 * rounds and launch mode.  Only the block shape changes the decomposition
 * (Section 2) and so the iterates and the final energy; the other settings
 * change speed only (the block cut is exact and canonical), so their labels
 * are bit-identical.  The paper fixes its block sizes by hand; this is a
 * deployment tool.
 * ------------------------------------------------------------------------- */
#define DOPE_TUNE_BLOCK 1     /* also try block shapes that tile the grid */

typedef struct {
    int32_t block_shape[3];   /* first ndim entries used */
    dope_params params;
    double ms;                /* best device time of one solve (CUDA events) */
    int iterations;
    int converged;
    int64_t energy_int;
    int status;
    int reserved;
} dope_tune_result;

/* Stage-wise search from (block_shape, base): block shapes when flags has
 * DOPE_TUNE_BLOCK, then relabel_period in {2,4,8,16,32}, threads in {auto,
 * 256, 512}, fold_rounds in {1,2,3,4}, launch_mode in {0,2}; each candidate
 * is created, given u[N] / wq[conn/2][N] (`where` memory), solved once to
 * warm up and `reps` (>= 1) times timed.  Every candidate tried goes to
 * out[] (up to cap entries; *count = entries written); *best = the fastest
 * converged one.  Synchronises `stream`. */
int dope_autotune(const int64_t *grid, int ndim, int connectivity, const int32_t *block_shape,
                  double lambda, const dope_params *base, const float *u, const int32_t *wq,
                  int where, int flags, int reps, dope_tune_result *out, int cap, int *count,
                  dope_tune_result *best, void *stream);

/* ---------------------------------------------------------------------------
 * Request server (continuous batching on one GPU).  The paper has no
 * counterpart; this is the serving layer around the batched launch.
 *
 * A worker thread owns one device memory arena.  A submitted request is
 * admitted (first come, first served) when its device state fits in the
 * arena's free memory and fewer than max_batch requests are admitted; its
 * inputs are uploaded on a side stream while the GPU works on the others;
 * the running persistent launch is asked to end at its next iteration
 * boundary, and the next launch takes the new request in.  A launch also
 * ends when one of its requests finishes, whose labels and energy are then
 * written out and whose memory returns to the arena.  Grids need not be
 * whole numbers of blocks: the server pads them with isolated zero-cost
 * pixels, which changes no label or energy of the caller's pixels.
 * mode 1 solves admitted requests one at a time through the single-problem
 * path (dope_solve's kernels), for comparison.
 * ------------------------------------------------------------------------- */
typedef struct dope_server dope_server;

typedef struct {
    uint64_t hbm_bytes;   /* arena size (0: 3/4 of the device's free memory at creation) */
    int max_batch;        /* most admitted requests (0: DOPE_BATCH_MAX) */
    int mode;             /* 0: continuous batching (up to max_batch requests at once),
                             1: one request at a time, 2: continuous batching only as wide
                             as the backlog (at least 2, at most max_batch) */
    int launch_iters;     /* most iterations of one batched launch (0: no bound) */
    int reserved;
} dope_server_params;

typedef struct {
    int ndim;                 /* 2 or 3 */
    int connectivity;         /* 4 / 8 (2-D), 6 (3-D) */
    int64_t grid[3];          /* first ndim entries used; need not be a multiple of the block */
    int32_t block_shape[3];   /* first ndim entries used */
    double lambda;
    dope_params params;       /* as for dope_create (used when use_params != 0) */
    int use_params;
    int where_inputs;         /* DOPE_HOST or DOPE_DEVICE, for unaries and weights */
    const float *unaries;     /* [N] image order */
    const int32_t *weights;   /* [conn/2][N] image order */
    uint8_t *labels;          /* [N] image order, receives the labels */
    int where_labels;         /* DOPE_HOST or DOPE_DEVICE */
    int reserved;
    uint64_t tag;             /* returned in the result */
    const void *image_request;  /* NULL: unaries / weights as above.  Otherwise a
                                   const dope_image_request* (dope_potentials.h):
                                   the server computes the potentials on the GPU
                                   from the image, and unaries / weights are
                                   ignored (may be NULL). */
} dope_request;

typedef struct {
    uint64_t id, tag;
    int status;               /* DOPE_OK, DOPE_ENOTCONV (labels valid), or an error */
    int iterations;
    int converged;
    int reserved;
    int64_t energy_int;       /* E_int of the labels */
    double t_submit, t_admit, t_done;   /* seconds on dope_server_clock */
} dope_result;

typedef struct {
    int64_t submitted, admitted, completed, launches, yields;
    int64_t queued, in_flight;          /* now */
    int64_t max_in_flight;
    uint64_t bytes_limit, bytes_in_use, bytes_peak;
    double gpu_launch_s;                /* summed device time of the solve launches */
} dope_server_stats;

/* Start a server on the current device (p may be NULL for defaults). */
int dope_server_create(const dope_server_params *p, dope_server **out);

/* Queue a request; *id (may be NULL) receives its id.  The request struct is
 * copied; the buffers it points to must stay valid, and unchanged, until its
 * result has been polled.  Returns DOPE_EINVAL for a malformed request. */
int dope_server_submit(dope_server *srv, const dope_request *req, uint64_t *id);

/* Completed results, oldest first: waits up to timeout_s seconds for at
 * least one, then returns up to cap of them (*count may be 0 on timeout). */
int dope_server_poll(dope_server *srv, dope_result *out, int cap, int *count, double timeout_s);

/* Cancel a submitted request.  A queued or admitted request is dropped and
 * its result published with status DOPE_ECANCELED.  One inside a running
 * batched launch makes the launch end at its next iteration boundary (the
 * other requests continue in the next launch, unchanged).  In mode 1 the
 * request being solved finishes first.  A request that has already finished
 * keeps its result.  Its memory returns to the arena; its buffers are no
 * longer written once the result is polled.  DOPE_EINVAL for an id never
 * issued. */
int dope_server_cancel(dope_server *srv, uint64_t id);

/* Seconds since the server was created (the clock of dope_result). */
double dope_server_clock(const dope_server *srv);

int dope_server_get_stats(dope_server *srv, dope_server_stats *st);

/* Stop the worker (requests not yet completed are dropped) and free
 * everything (NULL is ignored). */
void dope_server_destroy(dope_server *srv);

/* Free the context and its device memory (NULL is ignored). */
void dope_destroy(dope_ctx *ctx);

/* Static description of a status code. */
const char *dope_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* DOPE_H */
