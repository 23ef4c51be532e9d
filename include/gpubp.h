/*
 * gpubp: GB300-native bound propagation, double probing and fix-and-propagate for MILP.
 *
 * C ABI.  Plain pointers and sizes; no C++ or framework types cross it.  Every entry point
 * returns an int status: BP_OK (0) or a negative BP_ERR_* code; on error,
 * bp_last_error() returns a thread-local message.  Infeasibility of a problem is a RESULT
 * (a status field of the result struct), never an error code.
 *
 * Problem form (paper, Section 1): minimise c.x subject to
 *     sum_i a_ki x_i <= g_k   for every row k,
 *     l_i <= x_i <= u_i,      x_i integer where is_int[i] != 0.
 * Only "<=" rows exist; an equality is passed as two rows (a.x <= b, -a.x <= -b).
 * |value| >= 1e20 means infinite.  Feasibility tolerance: 1e-6 absolute (Section 3).
 *
 * Streams: every call is enqueued on the caller's cudaStream_t (passed as void*, NULL means
 * the legacy default stream) and returns without a host synchronisation unless stated.
 * One problem handle must not be used by two streams at the same time.
 * Device pointers must be device-accessible addresses on the current CUDA device.
 */
#ifndef GPUBP_H
#define GPUBP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define BP_OK 0
#define BP_ERR_INVALID (-1)   /* malformed input: see bp_last_error() */
#define BP_ERR_CUDA (-2)      /* a CUDA runtime call failed */
#define BP_ERR_OOM (-3)       /* device allocation failed */
#define BP_ERR_CAPACITY (-4)  /* an output buffer is too small; the needed size is reported */
#define BP_ERR_TIMEOUT (-5)   /* a device-side wait gave up (co-residency lost); no hang */

/* result statuses of a propagation */
#define BP_FIXPOINT 0         /* worklist empty: no bound changes any more */
#define BP_INFEASIBLE 1       /* a row's minimal activity exceeds g + tol, or bounds cross */
#define BP_ROUND_LIMIT 2      /* max_rounds rounds were run */

/* memory kinds for caller arrays */
#define BP_MEM_HOST 0
#define BP_MEM_DEVICE 1

typedef struct mip_problem mip_problem;

/* ----------------------------------------------------------------- parameters */

/* Bound-propagation parameters (Section 2.1).  theta: minimum relative improvement for a
 * continuous bound to move (new bound accepted iff old - new > theta * max(1, |old|), or
 * the old bound is infinite); the paper's "threshold" whose value it does not give.
 * Integer bounds move on any improvement after rounding floor(c + 1e-6) / ceil(c - 1e-6).
 * max_rounds: stop after this many rounds (status BP_ROUND_LIMIT).
 * bounds_mem: BP_MEM_DEVICE if lb/ub are device arrays, BP_MEM_HOST if host arrays (the
 * library then copies them in and out on the stream; pinned host memory keeps it async). */
typedef struct {
    double theta;
    int32_t max_rounds;
    int32_t bounds_mem;
    int64_t *trace;      /* optional DEVICE array of 4 * max_rounds int64 (NULL: none): per round
                            the worklist rows, their nonzeros, the variables changed and the
                            device time in ns (globaltimer) when the round ended */
} bp_params;

/* Result of one propagation.  rounds: rounds that processed a non-empty worklist.
 * nnz_updates: sum over rounds of the nonzeros of the rows processed (the work unit of
 * the throughput metric).  first_infeasible_row / _var: the smallest infeasible row index
 * and the smallest crossing variable index in the final round, -1 if none.
 * n_changed: variables whose output bounds differ from the (normalised) input bounds. */
typedef struct {
    int32_t status;
    int32_t rounds;
    int32_t first_infeasible_row;
    int32_t first_infeasible_var;
    int64_t nnz_updates;
    int64_t n_changed;
    int32_t error;        /* BP_OK, or BP_ERR_TIMEOUT when a device wait gave up */
    int32_t reserved;
} bp_result;

void bp_params_default(bp_params *p);   /* theta 1e-3, max_rounds 10000, device bounds, no trace */

/* ------------------------------------------------------------- problem handle */

/*
 * mip_load_csr -- copy a MILP into library-owned device memory and build its layouts.
 *
 * Cites: Section 1 (problem form); Section 2.1 (rows and their transpose are both needed:
 * activities per row, worklist of rows per changed variable).
 *
 * m, n:      rows and variables (0 <= m, n < 2^31).
 * row_ptr:   int64[m+1], row_ptr[0] = 0, nondecreasing, nnz = row_ptr[m] < 2^31.
 * col:       int32[nnz], 0 <= col < n, strictly increasing within a row.
 * val:       double[nnz], finite, |val| >= 1e-12.
 * g:         double[m], finite or >= 1e20 (a free row); NaN or <= -1e20 is invalid.
 * lb, ub:    double[n] default bounds (kept on the handle; normalised: +-1e20 -> +-inf,
 *            integer bounds rounded inward with tol 1e-6).  lb may not be +inf, ub not -inf.
 * is_int:    uint8[n], nonzero = integer variable.
 * c:         double[n] objective, or NULL (zeros).
 * mem_kind:  BP_MEM_HOST or BP_MEM_DEVICE for all the arrays above.
 * stream:    cudaStream_t used for the copies and the layout kernels.
 * out:       receives the handle.  The caller keeps ownership of its arrays.
 * Returns BP_OK; BP_ERR_INVALID (malformed input, message in bp_last_error()),
 * BP_ERR_OOM or BP_ERR_CUDA.  The call synchronises the stream once (validation result).
 */
int mip_load_csr(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col,
                 const double *val, const double *g, const double *lb, const double *ub,
                 const uint8_t *is_int, const double *c, int32_t mem_kind, void *stream,
                 mip_problem **out);

/* Releases every device resource of the handle (after synchronising its last stream). */
int mip_free(mip_problem *p);

/* Sizes of a loaded problem. */
int mip_dims(const mip_problem *p, int32_t *m, int32_t *n, int64_t *nnz);

/* Copies the handle's normalised default bounds into lb/ub (device arrays of n doubles). */
int mip_default_bounds(const mip_problem *p, double *lb, double *ub, void *stream);

/* ------------------------------------------------------------ bound propagation */

/*
 * bp_propagate -- bound propagation to a fixpoint (Section 2.1).
 *
 * Every round computes, for each row k of the round's worklist, the minimal activity
 * L_min^k = sum_{a>0} a l + sum_{a<0} a u (finite part plus a count of infinite terms),
 * declares the row infeasible if L_min^k > g_k + 1e-6, and proposes for each of its
 * variables u_i <= (g_k - L_min^k + a_ki l_i) / a_ki (a_ki > 0) or
 * l_i >= (g_k - L_min^k + a_ki u_i) / a_ki (a_ki < 0), rounded for integers and tested
 * against the bounds at the START of the round (Jacobi rounds).  The next round's
 * worklist holds the rows of every variable changed in this round ("propagation on changed
 * constraints", Section 1); round 0 holds every row.
 *
 * lb, ub:  n doubles each, in: start bounds (normalised by the call), out: bounds after the
 *          last round (on BP_INFEASIBLE: after the round that found the infeasibility).
 *          Device or host memory per params->bounds_mem.
 * params:  NULL for defaults.
 * result:  host pointer.  The library enqueues a copy of the result into it; it is valid
 *          once the stream is synchronised (at return when it is pageable memory).  May be
 *          NULL, then the result stays on the device (see bp_result_device).
 * Returns BP_OK (then check result->error and result->status), BP_ERR_INVALID or
 * BP_ERR_CUDA.  Device-side errors arrive in result->error: BP_ERR_TIMEOUT when a device wait
 * gave up (the bounds are then unspecified).
 */
int bp_propagate(mip_problem *p, double *lb, double *ub, const bp_params *params,
                 bp_result *result, void *stream);

/*
 * bp_propagate_from -- bp_propagate whose round 0 holds only the rows of the given variables
 * (for bounds that are a fixpoint except for those variables, e.g. after fixing them; a probe
 * run one launch at a time).  vars: DEVICE int32[nvars], 0 <= vars[i] < n, duplicates
 * allowed.  The range is checked on the device: an out-of-range index is never dereferenced,
 * the launch stops after its set-up and result->error is BP_ERR_INVALID (bounds unspecified).
 * Other arguments as for bp_propagate (device bounds only).
 */
int bp_propagate_from(mip_problem *p, double *lb, double *ub, const int32_t *vars, int32_t nvars,
                      const bp_params *params, bp_result *result, void *stream);

/*
 * bp_propagate_noalloc -- bp_propagate on device bounds that allocates nothing.  The paper has
 * no counterpart: this call serves callers that may not allocate device memory while they run
 * (a solver that reserves its whole device budget at start-up, or a host framework whose caching
 * allocator holds the free memory, where a cudaMalloc/cudaFree from the library could fail or
 * stall every stream of the device mid-search).
 *
 * The per-call scratch is a fixed array of BP_NOALLOC_SCRATCH_BYTES (32 MiB) in the library's
 * static device memory, one per device, instead of the handle's own buffers.  A problem needs
 * 44 n + 12 m + 32 P bytes, P the pieces of its long rows (about nnz / 256 + rows longer than
 * 256 nonzeros at the default piece length), plus at most 10 KB of control block and alignment;
 * a larger problem is rejected with BP_ERR_CAPACITY before anything is enqueued (bp_last_error
 * gives the exact bytes needed).  Each call clears the part of the scratch that must start at
 * zero.
 *
 * Set-up: mip_load_csr looks up the array's device address on the handle's device
 * (cudaGetSymbolAddress), which loads the module holding it and so reserves its 32 MiB there,
 * together with the handle's own memory.  This entry point then allocates nothing, on its first
 * call as on every later one.  Calls that overlap in time on one device, from any handle,
 * stream or thread, share the one array and race: order them.  The handle must not be used by
 * another call meanwhile either.
 *
 * Arguments and results as for bp_propagate, with params->bounds_mem == BP_MEM_DEVICE.  The
 * handle's device must be current (BP_ERR_INVALID otherwise).  result may be NULL.
 */
#define BP_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int bp_propagate_noalloc(mip_problem *p, double *lb, double *ub, const bp_params *params,
                         bp_result *result, void *stream);

/* Device address of the handle's result slot written by the last bp_propagate. */
const bp_result *bp_result_device(const mip_problem *p);

/* ------------------------------------------------------- batches of instances */

/*
 * mip_set_instances -- declare the loaded problem a batch of independent instances laid out
 * block-diagonally: instance i owns rows [row_off[i], row_off[i+1]) and variables
 * [col_off[i], col_off[i+1]), and no row has a nonzero outside its instance's variables.
 * row_off, col_off: int32[ninst+1] in host or device memory (mem_kind), row_off[0] = 0,
 * row_off[ninst] = m, col_off[0] = 0, col_off[ninst] = n, nondecreasing; 1 <= ninst <= 1024.
 * The layout is validated on the device and kept on the handle.  Synchronises the stream.
 * Returns BP_OK or BP_ERR_INVALID.
 */
int mip_set_instances(mip_problem *p, int32_t ninst, const int32_t *row_off, const int32_t *col_off,
                      int32_t mem_kind, void *stream);

/*
 * bp_propagate_batch -- bound propagation of every instance of the batch in one persistent
 * launch (the batched form; Section 2.1 per instance).  Each instance is propagated exactly
 * as bp_propagate would propagate it alone (its own status, round count, work count and
 * first infeasible indices); an infeasible instance stops without stopping the others.
 * lb, ub:   DEVICE double[n], in/out, as for bp_propagate.
 * results:  DEVICE bp_result[ninst]; first infeasible row / variable are indices of the whole
 *           (concatenated) problem.  No host synchronisation: the call can be captured in a
 *           CUDA graph.
 * Returns BP_OK, BP_ERR_INVALID (no batch declared) or BP_ERR_CUDA.
 */
int bp_propagate_batch(mip_problem *p, double *lb, double *ub, const bp_params *params,
                       bp_result *results, void *stream);

/* -------------------------------------------------------------------- probing */

/*
 * probe_split -- the two branch boxes of an integer variable (Section 2.2).
 * Boxed [l, u]: c = ceil((l + u) / 2), down = [l, c - 1], up = [c, u] (binary: [0,0], [1,1]).
 * Only l finite: [l, l] and [l + 1, +inf).  Only u finite: [u, u] and (-inf, u - 1].
 * Writes box4 = {down_l, down_u, up_l, up_u}; returns 1 if the variable is probed, 0 for a
 * continuous, fixed or free variable.  Pure host function.
 */
int probe_split(int32_t is_int, double l, double u, double *box4);

/* Probing cache (Section 2.2).  For branch e = 2*i + b of pair i (b = 0 down, 1 up):
 * status[e], rounds[e], nnz_updates[e]; offsets[e] .. offsets[e+1] index the implied
 * bounds (var, l, u) of that branch: every variable whose bounds differ from the root,
 * ascending by variable; nothing for an infeasible branch.  All arrays are caller-owned
 * DEVICE memory: status/rounds int32[2P], nnz_updates int64[2P], offsets int64[2P+1],
 * ent_var int32[cap], ent_l/ent_u double[cap]. */
typedef struct {
    int32_t *status;
    int32_t *rounds;
    int64_t *nnz_updates;
    int64_t *offsets;
    int32_t *ent_var;
    double *ent_l;
    double *ent_u;
    int64_t cap;
    int64_t needed;   /* out: entries needed (set also on BP_ERR_CAPACITY) */
} probe_cache;

/*
 * bp_probe_batch -- double probing of P variables in one launch (Section 2.2).
 *
 * Branch b of pair i starts from root ∩ box (box = boxes[4i+2b], boxes[4i+2b+1] for
 * variable var[i]) and runs bp_propagate's rounds with round 0 holding the rows of var[i].
 * Both branches of a pair are propagated together so that they share every row load.
 * root_lb/root_ub: device, n doubles (normally a bp_propagate fixpoint).
 * var: device int32[P]; boxes: device double[4P] (see probe_split).
 * Returns BP_OK, BP_ERR_CAPACITY (cache->needed holds the required entry count; the status,
 * rounds, nnz_updates and offsets arrays are complete), BP_ERR_INVALID (also for a variable
 * index outside [0, n): the kernel skips such a pair and flags it; the other arrays are then
 * incomplete) or BP_ERR_TIMEOUT (a bounded device wait ran out).  Scratch: each block of the
 * launch keeps the variables a pair touches in a table of 2,048 slots (about 0.2 MB per block
 * plus 16 bytes per row); a pair whose branches touch more variables than that is re-run by
 * the blocks that own a dense scratch (104 bytes per variable each, at most 1 GB in total, at
 * least one).  The call synchronises the stream once, at its end: the copy into the cache is
 * launched before the host knows the entry count and checks the capacity on the device, and
 * the count and the index flag are read back together (it is bp_probe_batch_async followed by
 * that read).
 */
int bp_probe_batch(mip_problem *p, const double *root_lb, const double *root_ub, int32_t P,
                   const int32_t *var, const double *boxes, const bp_params *params,
                   probe_cache *cache, void *stream);

/*
 * bp_probe_batch_async -- bp_probe_batch without any host synchronisation, so that the whole
 * batch (bound keys, row caps, the persistent probe launch, offsets and the copy into the
 * cache) can be captured in a CUDA graph and replayed.  Arguments as for bp_probe_batch, plus
 * status_dev: caller-owned DEVICE int64[2] written by the call's last operation: [0] the
 * entries the batch needs (the cache holds min(needed, cache->cap) of them; offsets are always
 * complete), [1] 1 when a variable index was outside [0, n) (that pair was skipped), 2 when a
 * bounded device wait ran out (the batch's results are not valid; BP_ERR_TIMEOUT).  The
 * caller reads them after the stream work (a graph replay) completes; cache->needed is not set.
 * The handle's probing scratch grows on the first call for a given pair count and capacity:
 * make one call of that size before capturing (inside a capture a call that would have to
 * allocate returns BP_ERR_INVALID).  Returns BP_OK or BP_ERR_INVALID (arguments).
 */
int bp_probe_batch_async(mip_problem *p, const double *root_lb, const double *root_ub, int32_t P,
                         const int32_t *var, const double *boxes, const bp_params *params,
                         probe_cache *cache, int64_t *status_dev, void *stream);

/* Result of probe_cache_apply.  status: BP_FIXPOINT, or BP_INFEASIBLE when a pair has both
 * branches infeasible (first_infeasible_pair) or the derived bounds of a variable cross
 * (first_infeasible_var: integer l > u, continuous l > u + 1e-6); fixed_pairs: pairs with exactly
 * one infeasible branch; tightened: variables whose bounds changed. */
typedef struct {
    int32_t status;
    int32_t first_infeasible_pair;
    int32_t first_infeasible_var;
    int32_t fixed_pairs;
    int64_t tightened;
} probe_apply_result;

/*
 * probe_cache_apply -- bounds valid for every solution, derived from a probing cache
 * (Section 2.2: the cache serves early infeasibility detection).  The two branch boxes of a
 * pair cover the probed variable's integer domain (see probe_split), so every feasible point
 * lies in a feasible branch, inside that branch's implied box (the root bounds where the branch
 * lists nothing).  For every pair the bounds are intersected with the hull of its feasible
 * branches' boxes: one infeasible branch fixes the variable to the other branch together with
 * all of that branch's implied bounds; two feasible branches tighten the variables both list to
 * (min of the lower bounds, max of the upper bounds); two infeasible branches leave nothing, and
 * the problem is infeasible.
 * lb, ub:  DEVICE double[n]: in = the root bounds the cache was computed from, out = the
 *          intersection (normalised as bp_propagate normalises bounds).  Follow with
 *          bp_propagate to propagate what was derived.
 * npairs, cache: the P pairs and the cache arrays of a bp_probe_batch call (status, offsets and
 *          the entries; rounds and nnz_updates are not read).
 * result:  HOST pointer, valid at return (the call synchronises the stream).
 * Returns BP_OK or BP_ERR_INVALID; infeasibility is reported in result->status.
 */
int probe_cache_apply(mip_problem *p, double *lb, double *ub, int32_t npairs, const probe_cache *cache,
                      probe_apply_result *result, void *stream);

/*
 * bp_probe_priority -- probe priority keys (Section 2.2) under bounds lb/ub (device):
 * key1 int32[n] = rows violated when the variable's contribution flips from its minimising
 * to its maximising bound (variables with coefficients of both signs only, else 0; -1 for a
 * variable that is not probed), key2 double[n] = largest such violation, key3 double[n] =
 * smallest unit slack (g - L_min) / |a| over its rows.  order int32[n] receives the probed
 * variables sorted by key1 desc, key2 desc, key3 asc, index asc; *count their number
 * (host pointer, valid at return: the call synchronises the stream).
 */
int bp_probe_priority(mip_problem *p, const double *lb, const double *ub, int32_t *key1,
                      double *key2, double *key3, int32_t *order, int32_t *count, void *stream);

/* ------------------------------------------------------------------ autotuning */

/* Split points of the row classes and grid shape of the propagation engine.  Rows are binned
 * by length (Section 2.1): rows with fewer than warp_min nonzeros are handled one per thread,
 * rows of warp_min .. block_min-1 one per warp, and rows of block_min or more nonzeros (every
 * row longer than 256) in pieces of chunk_len nonzeros, one warp each, whose partial
 * activities are summed after a grid-wide phase barrier.  blocks_per_sm: thread blocks per SM
 * of the persistent grid.  Valid: 2 <= warp_min <= 9, warp_min <= block_min <= 257,
 * 1 <= blocks_per_sm <= the number that can be resident (2 on GB300), chunk_len in
 * {32, 64, 128, 256}.  Defaults: 2, 257, all resident, 256 (on GB300 a warp per row beat a
 * thread per row for rows of 2..8 nonzeros on every workload measured). */
typedef struct {
    int32_t warp_min;
    int32_t block_min;
    int32_t blocks_per_sm;
    int32_t chunk_len;
} bp_tuning;

/* What bp_autotune measured.  best_ms / default_ms: median launch time of the chosen and the
 * default configuration; tried: configurations timed; rejected: configurations skipped because
 * some instance's result (status, rounds, nnz-updates, changed variables, first infeasible
 * indices) differed from the defaults'. */
typedef struct {
    bp_tuning best;
    float best_ms;
    float default_ms;
    int32_t tried;
    int32_t rejected;
} bp_tune_report;

/* The handle's current configuration. */
int bp_get_tuning(const mip_problem *p, bp_tuning *out);

/* Sets the configuration (re-bins the rows on the device; synchronises the stream).
 * Returns BP_ERR_INVALID for a configuration outside the valid ranges. */
int bp_set_tuning(mip_problem *p, const bp_tuning *t, void *stream);

/*
 * bp_autotune -- times every configuration of a small grid (warp_min in {2, 9}, block_min in
 * {65, 257}, every valid blocks_per_sm, every valid chunk_len) with one warm-up and `reps`
 * (<= 0: 3) propagations from lb/ub (DEVICE, n doubles each, not modified; the handle's
 * staging buffers hold the working bounds), and keeps the fastest configuration whose results equal the defaults'.  A
 * handle with an instance batch (mip_set_instances) is tuned on bp_propagate_batch, otherwise
 * on bp_propagate.  report (host, may be NULL) receives the measurements.  The call synchronises
 * the stream; on an error the defaults are restored.
 */
int bp_autotune(mip_problem *p, const double *lb, const double *ub, const bp_params *params,
                int32_t reps, bp_tune_report *report, void *stream);

/* ------------------------------------------------------------ fix-and-propagate */

#define FP_BULK_SQRT 0        /* bulk size ceil(sqrt(remaining unfixed integer variables)) */
#define FP_BULK_FRACTION 1    /* bulk size ceil(fraction * integer variables) */
#define FP_FEASIBLE 0
#define FP_INFEASIBLE 1

/* Parameters of fix_and_propagate.  seed: key of the counter-based random draws.
 * last_single: the last variables are fixed one at a time (36 in the paper, Section 2.3).
 * theta, max_rounds: as in bp_params, for every propagation.
 * order_score (DEVICE double[n] or NULL): when given, the integer variables are ranked by
 *   class (binary, ternary, rest), then descending score, then fractionality, then index, and
 *   every bulk takes the unfixed variables in that order: the score replaces the per-bulk
 *   implied-slack sort (NULL keeps the paper's order).
 * up_prob (DEVICE double[n] or NULL): when given, replaces the rounding distribution's
 *   probability of rounding up for fractions strictly between 0.25 and 0.75 (the random band);
 *   outside the band the nearest value is always drawn.  Propagation still judges every fix.
 * repair_max: repairs a run may attempt (Section 2.3, the repair branch of Algorithm 1); 0, the
 *   default, turns the repair off, as in the paper's experiments.  Not with a probing cache.
 * repair_cycles: propagations one repair may run (default 8). */
typedef struct {
    uint64_t seed;
    int32_t bulk_rule;
    int32_t last_single;
    double fraction;
    double theta;
    int32_t max_rounds;
    int32_t repair_max;
    const double *order_score;
    const double *up_prob;
    int32_t repair_cycles;
    int32_t reserved;
} fp_params;

/* A probing cache (bp_probe_batch's layout, all DEVICE arrays): the pairs' variables and
 * branch boxes, and per branch its status, entry offsets and implied bounds. */
typedef struct {
    int32_t npairs;
    int32_t reserved;
    const int32_t *var;
    const double *boxes;
    const int32_t *status;
    const int64_t *offsets;
    const int32_t *ent_var;
    const double *ent_l;
    const double *ent_u;
} fp_cache;

/* Result of fix_and_propagate.  bulks: iterations (bulk and single); bp_runs: propagations
 * (the start one and every candidate vector with at least one kept fixing); recoveries: bulks
 * that failed both ways and were retried one variable at a time; fixed_by_choice: kept
 * fixings of the chosen vectors; refuted: 1 when every integer variable was fixed but the final
 * check (a propagation of the caller's bounds with the integer variables fixed) was infeasible,
 * so the status is FP_INFEASIBLE; nnz_updates: summed over the rounding's propagations (bp_runs;
 * the final check is not counted); repairs: repairs that ended with a feasible propagation;
 * repair_runs: propagations run by repairs (included in bp_runs and nnz_updates). */
typedef struct {
    int32_t status;
    int32_t bulks;
    int32_t bp_runs;
    int32_t recoveries;
    int32_t fixed_by_choice;
    int32_t refuted;
    int64_t nnz_updates;
    int32_t repairs;
    int32_t repair_runs;
} fp_result;

void fp_params_default(fp_params *p);   /* seed 1, sqrt rule, last_single 36, fraction 0.01, repair off
                                          * (repair_max 0, repair_cycles 8) */

/*
 * pdhg_solve -- the approximate LP (Sections 1 and 2.5: the paper's GPU PDLP, warm-started).
 *
 * Primal-dual hybrid gradient for min c^T x s.t. A x <= g, lb <= x <= ub (c: the handle's
 * objective, or params->objective when given; rows with g = +inf are free), with row duals
 * y >= 0:
 *     x+ = proj_[lb, ub](x - tau (c + A^T y)),  y+ = max(0, y + sigma (A (2 x+ - x) - g)),
 *     tau = step / primal_weight,  sigma = step * primal_weight,
 * and with restart_period R > 0 every R iterations the iterate is replaced by the mean of the
 * period's R iterates.  step 0: 0.9 / sqrt(max column |a| sum * max row |a| sum) (a bound on
 * ||A||_2); primal_weight 0: ||c||_2 / ||g||_2 over the finite rows (1 if either is zero).
 * With scaling_iterations K > 0 (PDLP's diagonal preconditioning): K passes of Ruiz
 * equilibration, each dividing every row factor D_r and column factor D_c by the square root of
 * the largest scaled |a| = (D_r |a|) D_c of its row or column (both from the same factors); the
 * iteration then runs on D_r A D_c, D_c c, D_r g, lb / D_c, ub / D_c from x / D_c, y / D_r (the
 * default step and weight taken on the scaled data), and returns x = D_c x~, y = D_r y~.
 * Approximate by design: the caller chooses the iterations (the paper limits each projection by
 * time) and reads the KKT measures (of the original problem).
 *
 * lb, ub:  DEVICE double[n] box (not modified).
 * x:       DEVICE double[n], the primal warm start on entry, the final iterate on return.
 * y:       DEVICE double[m], the dual warm start on entry (>= 0), the final iterate on return.
 * result:  HOST pointer, valid at return (the call synchronises the stream): iterations,
 *          restarts, the step and primal weight used, primal residual ||max(Ax - g, 0)||_2
 *          (finite rows), dual residual (norm of the reduced costs c + A^T y that push a
 *          variable toward an infinite bound), primal objective c^T x, dual objective
 *          -g^T y + sum_j min over [lb_j, ub_j] of r_j x_j (finite parts).
 * Scratch: 3 n + 2 m + pieces doubles (plus n + m with restarts, plus 2 nnz + 5 n + 4 m with
 * scaling), stream-ordered, freed at return.
 * Returns BP_OK, BP_ERR_INVALID (null pointers, negative counts or steps), BP_ERR_OOM or BP_ERR_CUDA.
 */
typedef struct {
    int32_t iterations;
    int32_t restart_period;
    double step;
    double primal_weight;
    const double *objective;   /* DEVICE double[n] in place of the handle's objective, or NULL */
    int32_t scaling_iterations; /* Ruiz preconditioning passes, 0 for none (0) */
    int32_t reserved;
} pdhg_params;

typedef struct {
    int32_t iterations;
    int32_t restarts;
    double step;
    double primal_weight;
    double primal_residual;
    double dual_residual;
    double primal_obj;
    double dual_obj;
} pdhg_result;

void pdhg_params_default(pdhg_params *p);   /* 1000 iterations, restart period 100, defaults */
int pdhg_solve(mip_problem *p, const double *lb, const double *ub, double *x, double *y,
               const pdhg_params *params, pdhg_result *result, void *stream);

/*
 * local_search_mtm -- the local search's move scoring (Section 2.4, the paper's GPU Local-MIP):
 * the mixed-tight-move core under a weighted violation F = sum_k w_k max(0, (A x)_k - g_k)
 * (rows with g = +inf are free).
 *
 * Each iteration forms, for every violated row and every variable in it, the value that alone
 * satisfies the row (integer variables by the smallest integer step: x - ceil(v / a) for
 * a > 0, x + ceil(v / |a|) for a < 0; continuous ones exactly), clamped to [lb, ub], and
 * scores every such move by the drop of F over the variable's column (rows ascending), all
 * scores recomputed each iteration.  The best move (largest score; ties: smallest variable,
 * then smallest value) is applied when its score is positive; otherwise every violated row's
 * weight grows by 1.  Lift and breakthrough moves (objective improvement): local_search_objective.
 * The row activities follow the moves as compensated (Kahan) sums, one compensation term per
 * row, and are summed afresh in row order every recompute_period iterations (0: never), at the
 * start of the iteration (Local-MIP's numerics).
 * Deterministic: the same inputs give the same moves bit for bit.
 *
 * lb, ub:  DEVICE double[n] bounds (not modified).
 * x:       DEVICE double[n], the start point on entry, the final point on return.
 * w:       DEVICE double[m], the weights (1 for a fresh search), updated in place.
 * params:  iterations >= 0, recompute_period >= 0.
 * result:  HOST pointer, valid at return (the call synchronises the stream): moves applied,
 *          weight bumps, violated rows at the end, sum of w_k v_k, and c^T x (the handle's
 *          objective).
 * Scratch: m doubles and a few KB, stream-ordered, freed at return.
 * Returns BP_OK, BP_ERR_INVALID, BP_ERR_OOM or BP_ERR_CUDA.
 */
typedef struct {
    int32_t iterations;
    int32_t recompute_period;   /* activities summed afresh every this many iterations (0: never) */
} ls_params;

typedef struct {
    int32_t iterations;
    int32_t moves;
    int32_t bumps;
    int32_t violated;
    double weighted_violation;
    double objective;
} ls_result;

int local_search_mtm(mip_problem *p, const double *lb, const double *ub, double *x, double *w,
                     const ls_params *params, ls_result *result, void *stream);

/*
 * local_search_objective -- the local search with its objective moves (Section 2.4: Local-MIP's
 * lift and breakthrough moves, the weighted objective), for min c^T x with c the handle's
 * objective.  It extends local_search_mtm's iteration:
 *   - at the start of an iteration, a point with no violated row becomes the incumbent x* when
 *     it is the first such point or its objective is lower; the search keeps D = c x - c x*
 *     through every move (D restarts at 0 with each incumbent);
 *   - lift: at a point with no violated row, every variable with c_j != 0 may move against the
 *     sign of c_j as far as every row of its column stays satisfied (steps (g_r - L_r) / |a|,
 *     floored for integer variables; no limiting row: to the bound), clamped to its bounds; the
 *     largest gain -c_j dx > 0 (ties: smallest variable) is applied and ends the iteration;
 *   - once an incumbent exists, the objective row c x <= c x* - delta joins the weighted
 *     violation with weight w0: every candidate's score adds
 *     w0 (max(0, D + delta) - max(0, D + c_j dx + delta)) to the column's drop, and while the
 *     row is violated its tight values (breakthrough moves) are candidates too; ties between a
 *     mixed tight and a breakthrough move of the same variable and value go to the former;
 *   - with no positive move, the violated rows' weights grow by 1, or, with no violated row,
 *     w0 grows by 1.
 * delta = 1 when every variable with a nonzero cost is integer with an integral cost, else 1e-4.
 * With c = 0 the iterations are local_search_mtm's.  Deterministic: the same inputs give the
 * same moves bit for bit.
 *
 * lb, ub:  DEVICE double[n] bounds (not modified).
 * x:       DEVICE double[n], the start point on entry, the final point on return.
 * w:       DEVICE double[m], the row weights, updated in place.
 * x_best:  DEVICE double[n], written with each incumbent (untouched when none is found).
 * params:  iterations >= 0; recompute_period >= 0 (as local_search_mtm's); obj_weight = w0 at
 *          the start (finite, >= 0).
 * result:  HOST pointer, valid at return (the call synchronises the stream): local_search_mtm's
 *          fields, then lift moves, breakthrough moves (applied), incumbents recorded, found (an
 *          incumbent exists), c^T x_best (+inf when none), w0 at the end, and delta.
 * Scratch: m doubles and a few KB, stream-ordered, freed at return.
 * Returns BP_OK, BP_ERR_INVALID, BP_ERR_OOM or BP_ERR_CUDA.
 */
typedef struct {
    int32_t iterations;
    int32_t recompute_period;   /* as in ls_params */
    double obj_weight;
} ls_obj_params;

typedef struct {
    int32_t iterations;
    int32_t moves;
    int32_t bumps;
    int32_t violated;
    double weighted_violation;
    double objective;
    int32_t lifts;
    int32_t breakthroughs;
    int32_t improvements;
    int32_t found;
    double best_objective;
    double obj_weight;
    double delta;
} ls_obj_result;

int local_search_objective(mip_problem *p, const double *lb, const double *ub, double *x, double *w,
                           double *x_best, const ls_obj_params *params, ls_obj_result *result, void *stream);

/*
 * extended_fp -- the extended feasibility pump's orchestration (Section 2.5, Algorithm 2), in
 * generation mode (it stops at the first feasible point) or improvement mode (improve = 1: the
 * objective cut at each feasible point).
 *
 * Start: the approximate LP from zero (pdhg_solve, lp_iterations), snapped to multiples of
 * 2^-20, rounded by fix_and_propagate (seed), then local_search_mtm (ls_iterations, fresh
 * weights); failing that, local_search_mtm from the all-zero point; the loop starts from the
 * end point with fewer violated rows and keeps its weights.  Each round: project (pdhg_solve
 * warm-started from the previous primal and dual iterates, objective +1 / -1 for an integer
 * variable at its lower / upper bound, 0 otherwise), snap, distance = sum over integer
 * variables of |projection - point|, fix_and_propagate from the projection (seed + round + 1),
 * local_search_mtm for ls_iterations / 5 (a feasible point ends the pump); a cycle (at least
 * cycle_window earlier distances, and the distance improving on their mean by no more than
 * cycle_ratio of it) is broken by local_search_mtm from the point with the kept weights
 * (ls_iterations), otherwise the next point is the projection rounded to the nearest integers.
 *
 * Improvement mode: a feasible point (from the start or a round) becomes the incumbent x*
 * instead of ending the pump.  The loop then works on the problem with one more row, the cut
 * c x <= c x* - delta (delta = 1 when every variable with a nonzero cost is integer with an
 * integral cost, else 1e-4; c x* summed in index order), a handle built on the device and
 * rebuilt at each incumbent; it continues from x* with an empty distance history, the LP's dual
 * iterate extended by 0 and the kept weights by 1 for the cut row.  A point satisfying every row
 * of the cut problem is a better incumbent.  The round budget ends the pump.  Costs of magnitude
 * below 1e-12 are rejected by the cut row's load (BP_ERR_INVALID).  With polish = 1 each new
 * incumbent is first searched by local_search_objective (ls_iterations, fresh weights, objective
 * weight 1) on the problem without the cut, and that search's best replaces it when the search
 * recorded a later incumbent than its start (Section 1: Local-MIP searching the neighbourhood
 * of an integer point).
 *
 * x_out:   DEVICE double[n]: the feasible point found (improvement mode: the last incumbent),
 *          else the loop's last point.
 * result:  HOST pointer (the call synchronises the stream): status FP_FEASIBLE / FP_INFEASIBLE,
 *          found_at (-2 the start rounding, -1 the all-zero start, r >= 0 round r, -3 none) of
 *          the first feasible point, rounds run, cycle breaks, the last distance; improvement
 *          mode: incumbents recorded, how many the polish replaced, and c x* of the last (+inf
 *          when none).
 * Returns BP_OK, BP_ERR_INVALID, BP_ERR_OOM, BP_ERR_CUDA or BP_ERR_TIMEOUT.
 */
typedef struct {
    int32_t rounds;            /* FP rounds at most (20) */
    int32_t lp_iterations;     /* PDHG iterations of the LP and of each projection (500) */
    int32_t ls_iterations;     /* local search iterations (200) */
    int32_t cycle_window;      /* N (3) */
    double cycle_ratio;        /* (0.1) */
    uint64_t seed;             /* fix_and_propagate's seed of the start; round r uses seed + r + 1 */
    int32_t improve;           /* 0: generation mode, 1: improvement mode (0) */
    int32_t polish;            /* improvement mode: 1 to polish each incumbent (0) */
} efp_params;

typedef struct {
    int32_t status;
    int32_t found_at;
    int32_t rounds;
    int32_t cycles;
    double last_distance;
    int32_t improvements;
    int32_t polished;
    double best_objective;
} efp_result;

void efp_params_default(efp_params *p);
int extended_fp(mip_problem *p, const double *lb, const double *ub, double *x_out, const efp_params *params,
                efp_result *result, void *stream);

/*
 * fix_and_propagate -- bulk rounding with bound propagation (Section 2.3, Algorithm 1; LP
 * polish off; the repair optional and off by default, as in the paper's experiments).
 *
 * Propagates the start bounds, sorts the integer variables (binary, ternary, rest; then
 * fractionality of x), and fixes them in bulks: per bulk a stable implied-slack sort
 * (S_i = sum over rows of (a / slack)^2, descending), two candidate values per variable drawn
 * from the rounding distribution, the probing cache's conflict filter and warm start (when a
 * cache is given), a propagation of each candidate vector from the rows of the variables it
 * changes, and the first feasible result kept.  A bulk failing both ways is retried one
 * variable at a time; a single variable failing both ways ends the search and the remaining
 * integer variables are rounded to the nearest value inside their bounds (FP_INFEASIBLE).
 * Repair (repair_max > 0): before giving up on such a variable, up to repair_cycles times,
 * the caller's bounds are propagated with every fixing made by choice so far and the variable
 * at its drawn value; if infeasible, the infeasible row (or, when only a crossing variable is
 * reported, its smallest row whose minimal activity under the final bounds exceeds g + tol)
 * is made feasible by moving the one fixed variable whose move lowers the minimal activity
 * most: by ceil((L_min - g) / |a|) against its coefficient's sign, within the caller's bounds
 * (ties to the smallest index).  A feasible propagation continues the rounding from its bounds.
 * Once every integer variable is fixed, one more propagation starts from the caller's bounds
 * with the integer variables at their values: under the continuous-bound threshold (Section
 * 2.1) the incremental propagations can stop short of a contradiction that this one reaches,
 * and then the result is FP_INFEASIBLE with refuted = 1.
 *
 * x:        DEVICE double[n], the point to round (e.g. an LP relaxation solution).
 * lb, ub:   DEVICE double[n] start bounds (not modified).
 * cache:    NULL or a probing cache (see fp_cache).
 * x_out:    DEVICE double[n]: integer variables at their fixed values, continuous variables
 *           x clamped to their final bounds.
 * result:   HOST pointer, valid at return (the call synchronises the stream: every bulk's
 *           control decision reads a few words back; without a cache, the one-variable
 *           retries of a failed bulk run in one device-driven launch and report back once).
 * Memory: the first call on a handle also loads a second copy of the problem, as two
 * instances of a block-diagonal pair, so that each bulk's two candidate vectors propagate in
 * one launch; the handle keeps it until mip_free (about twice the handle's own device memory).
 * The pair's indices are 32-bit, so m, n and nnz must each be below 2^30 (BP_ERR_CAPACITY
 * otherwise).
 * Returns BP_OK, BP_ERR_INVALID, BP_ERR_CAPACITY, BP_ERR_OOM, BP_ERR_CUDA or BP_ERR_TIMEOUT.
 */
int fix_and_propagate(mip_problem *p, const double *x, const double *lb, const double *ub,
                      const fp_cache *cache, const fp_params *params, double *x_out,
                      fp_result *result, void *stream);

/* ------------------------------------------------------------ learned scorer */
/*
 * A 16-64-64-2 multilayer perceptron (ReLU) that re-ranks the integer variables of
 * fix_and_propagate and proposes the rounding direction of ambiguous fractions.  The paper
 * has no counterpart; it only changes the order and the draw probabilities that
 * fix_and_propagate already takes (fp_params.order_score, fp_params.up_prob), and propagation
 * still judges every fixing.
 *
 * Arithmetic: BF16 operands on the tensor cores (tcgen05) with FP32 accumulation.  Features,
 * hidden activations and back-propagated pre-activation gradients are rounded to BF16 (nearest,
 * ties to even); weights are FP32 masters rounded to BF16 for the products; biases, logits,
 * the output-layer gradient and all sums stay FP32.
 *
 * Parameters (SCORER_NPARAM floats): W1 [64 x 16], b1 [64], W2 [64 x 64], b2 [64], W3 [2 x 64],
 * b3 [2]; each weight matrix [out x in], row-major.  Output 0 is the order score (a logit:
 * larger = fixed earlier within its class), output 1 the logit of rounding up.
 * A scorer lives on the device that was current at scorer_create; one scorer must not be used
 * by two calls at once.
 */
#define SCORER_IN 16
#define SCORER_HIDDEN 64
#define SCORER_OUT 2
#define SCORER_NPARAM 5378
typedef struct scorer scorer;

/* Creates a scorer with He-uniform weights (parameter i of matrix L: (2u - 1) sqrt(6 / fan_in),
 * u the splitmix64 uniform of (seed, 1000 + L, i, 0)) and zero biases.  Only in=16, hidden=64,
 * out=2 is built (BP_ERR_INVALID otherwise). */
int scorer_create(int32_t in, int32_t hidden, int32_t out, uint64_t seed, scorer **out_scorer);
void scorer_free(scorer *s);

/* Host copies of the parameter vector; set_params also resets the Adam state. */
int scorer_get_params(const scorer *s, float *host_params);
int scorer_set_params(scorer *s, const float *host_params);

/*
 * scorer_features -- the 16 features of variables vars[0..nvars) (DEVICE int32), standardised
 * over those variables (mean 0, population standard deviation 1; a constant feature becomes 0)
 * and rounded to BF16, into feat (DEVICE, nvars x 16 BF16 bit patterns, row-major).  In order:
 * degree, log(1 + degree), objective coefficient, up locks (positive coefficients), down locks,
 * log(1 + min(u - l, 1e9)), binary (integer with u - l <= 1), integer, frac(x), |frac(x) - 0.5|,
 * probing-cache implications of the down and up branch, down and up branch infeasible, the
 * implied slack sum S_i of the Section 2.3 rounding order (rows with no infinite term,
 * slack = max(g - L_min, 1e-6)) and the sum of |a| over the column.  x, lb, ub: DEVICE double[n];
 * cache: NULL or a probing cache (its first pair of a variable counts).  Asynchronous.
 */
int scorer_features(mip_problem *p, const double *x, const double *lb, const double *ub,
                    const fp_cache *cache, const int32_t *vars, int32_t nvars, uint16_t *feat,
                    void *stream);

/* Logits of rows x 16 BF16 features (DEVICE) into out (DEVICE float, rows x 2).  Asynchronous. */
int scorer_forward(scorer *s, const uint16_t *feat, int32_t rows, float *out, void *stream);

/* scorer_forward into logits (DEVICE float, rows x 2), then order_score[vars[r]] = logit 0
 * and up_prob[vars[r]] = sigmoid(logit 1) (DEVICE double[n] each, either may be NULL): the
 * fp_params inputs of fix_and_propagate.  Asynchronous. */
int scorer_scores(scorer *s, const uint16_t *feat, const int32_t *vars, int32_t rows, float *logits,
                  double *order_score, double *up_prob, void *stream);

/*
 * Loss of a batch and its gradient: binary cross-entropy with logits per output, averaged over
 * that output's labels; labels: DEVICE float, rows x 2, NaN = no label.  scorer_gradient copies
 * the gradient (SCORER_NPARAM floats) and the loss to host memory (either may be NULL) and
 * synchronises; scorer_train_step then takes one Adam step (beta 0.9 / 0.999, eps 1e-8,
 * bias-corrected, learning rate lr > 0) and, when loss is not NULL, synchronises to return it.
 * Returns BP_ERR_TIMEOUT if a tensor-core wait gave up.
 */
int scorer_gradient(scorer *s, const uint16_t *feat, const float *labels, int32_t rows,
                    float *grad, float *loss, void *stream);
int scorer_train_step(scorer *s, const uint16_t *feat, const float *labels, int32_t rows, float lr,
                      float *loss, void *stream);

/*
 * scorer_labels -- training labels from fix_and_propagate trajectories (no counterpart in the
 * paper).  Adds the outcome of one run that ended FP_FEASIBLE, with weight `weight` (1 / the
 * number of such runs gives shares), to labels (DEVICE float, nvars x 2) of the variables
 * vars[0..nvars) (DEVICE int32): column 0 += weight when the run fixed the variable to the
 * nearest integer of x, floor(x + 1/2) (the order label), column 1 += weight when it fixed it
 * above x (the rounding-direction label).  first != 0 starts the sums: column 0 at 0, column 1
 * at 0, or at NaN (no label) where x is integral.  x, x_out: DEVICE double[n] (x_out as written
 * by fix_and_propagate).  Asynchronous; BP_ERR_INVALID for null or negative arguments.
 */
int scorer_labels(const double *x, const double *x_out, const int32_t *vars, int32_t nvars, float weight,
                  int32_t first, float *labels, void *stream);

/* Parameters and Adam state to / from a file, so that training resumes where it stopped
 * (magic "GPUBPML2", the three sizes and the parameter count as int32, the Adam step count as
 * int64, then the parameters and Adam's first and second moments as floats, little-endian).
 * scorer_load also reads the parameters-only layout "GPUBPML1" and then starts a fresh Adam
 * state.  The calls synchronise the device. */
int scorer_save(const scorer *s, const char *path);
int scorer_load(scorer *s, const char *path);

/* ------------------------------------------------------------------- errors */

/* bp_fp64_rate -- measures the current device's FP64 fused multiply-add throughput in TFLOP/s
 * (2 flops per FMA; the best of five timed launches of independent FMA chains), the denominator
 * of the FP64 pipe fraction reported beside the HBM fraction.  No paper counterpart: a
 * measurement helper.  Synchronises the stream; returns BP_OK, BP_ERR_INVALID or BP_ERR_CUDA. */
int bp_fp64_rate(double *tflops, void *stream);

/* Thread-local message of the last error ("" if none). */
const char *bp_last_error(void);

/* Library version string. */
const char *bp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GPUBP_H */
