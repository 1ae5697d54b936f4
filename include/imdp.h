/*
 * imdp.h — C ABI of the GB300 robust value-iteration library for Interval
 * Markov Decision Processes (IMDPs), after arXiv 2401.04068 (IntervalMDP.jl).
 *
 * Model (Sec. 2): M = (S, A, P_up, P_lo). For every state-action pair (s, a)
 * the transition probability to s' lies in [P_lo(s,a,s'), P_up(s,a,s')], with
 * sum P_lo <= 1 <= sum P_up. Gamma_{s,a} is the set of feasible distributions.
 *
 * Storage (Sec. 3.1 and Sec. 5: compressed sparse column, source/action/
 * destination indices stored sequentially): one CSC matrix whose columns are
 * the (state, action) pairs of all states in order and whose rows are the
 * destination states; `stateptr` maps each state to its range of columns
 * (Appendix A lists the same arrays: colptr, rowval, nzval, stateptr).
 * All indices are 0-based (the paper's Julia is 1-based).
 *
 * Computation (Eq. 2 / Eq. 3): robust value iteration
 *   V_0 = 1_G,  V_k(s) = 1_G(s) + 1_{S\G}(s) opt^pi_a opt^eta_{p in Gamma_{s,a}} sum_s' V_{k-1}(s') p(s'),
 * with the inner problem solved by O-maximization (Sec. 4). The discounted-reward
 * property (Sec. 3.2, whose recursion the paper leaves to the reader) is taken as
 *   V_0 = r,  V_k(s) = r(s) + gamma opt^pi_a opt^eta_p sum_s' V_{k-1}(s') p(s').
 *
 * Conventions for every entry point:
 *   - Errors are returned as imdp_status; nothing is thrown across the ABI.
 *     imdp_last_error() gives a one-line detail for the calling thread.
 *   - The caller owns every pointer it passes; the library copies what it keeps.
 *   - "host or device" pointers are told apart with cudaPointerGetAttributes;
 *     device pointers must be on the current CUDA device.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Every call
 *     returns after its results are written (it synchronizes the stream).
 *   - Outputs are written only when the call returns IMDP_OK (or IMDP_ENOCONV
 *     for V/k/residual of an infinite horizon that hit its iteration cap).
 *   - The library never falls back to the CPU: without a usable CUDA device
 *     every compute call returns IMDP_EDEVICE.
 */
#ifndef IMDP_H
#define IMDP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define IMDP_API __attribute__((visibility("default")))
#else
#define IMDP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IMDP_OK = 0,
  IMDP_EINVAL = 1,       /* malformed arguments or CSC structure */
  IMDP_EINFEASIBLE = 2,  /* some column violates 0 <= lo <= up <= 1, sum lo <= 1 <= sum up (Sec. 2) */
  IMDP_ENOMEM = 3,       /* device or host allocation failed, or the server's HBM budget is too small */
  IMDP_EDEVICE = 4,      /* CUDA error or no CUDA device */
  IMDP_ETIMEOUT = 5,     /* a bounded device-side or host-side wait gave up */
  IMDP_EBUSY = 6,        /* the server has no free slot; retry later */
  IMDP_ENOCONV = 7,      /* infinite horizon: residual still >= eps at the iteration cap */
  IMDP_ENOTFOUND = 8,    /* unknown server ticket */
  IMDP_EPENDING = 9,     /* server ticket not finished yet */
  IMDP_EIO = 10          /* a model file cannot be opened, read or written */
} imdp_status;

/* Storage precision of the transition bounds. IMDP_F64 keeps 64 bits per bound
 * (stored as unsigned fixed point with 63 fractional bits, which resolves
 * probabilities in [0, 1] to 1.1e-19 absolute, finer than binary64 near 1).
 * IMDP_F32 is the fast path: 32 bits per bound (per column, mantissas scaled to
 * the column's largest upper bound, resolution ~2^-31 of it), 12 bytes per
 * transition instead of 20, values kept at 32 bits and 32-bit arithmetic in the
 * hot loop, with a correction stage: a column whose rounding would move a
 * Bellman step by more than a per-iteration budget (default 5e-9, i.e. 1e-6
 * over K = 200 iterations; see imdp_create_csc_f32) keeps its exact 64-bit
 * bounds and runs the 64-bit routines. imdp_model_error_bound gives the
 * resulting guaranteed bound. */
typedef enum { IMDP_F64 = 0, IMDP_F32 = 1 } imdp_dtype;

/* Property types of the specification JSON schema (Appendix A). */
typedef enum { IMDP_REACH = 0, IMDP_REACH_AVOID = 1, IMDP_REWARD = 2 } imdp_property;

/* Specification (Sec. 3.2 and Appendix A): property, horizon, and the
 * satisfaction (adversary) and strategy modes. All pointers are host pointers. */
typedef struct {
  int32_t property;      /* imdp_property */
  int32_t infinite_time; /* 0: fixed horizon `horizon` (FiniteTime*); 1: iterate until max|V_k - V_{k-1}| < eps */
  int32_t horizon;       /* K >= 0 for a finite horizon; iteration cap for an infinite one (0 = 1,000,000) */
  double eps;            /* convergence tolerance on the maximum Bellman residual (infinite_time only) */
  int32_t pessimistic;   /* 1: opt^eta = min (pessimistic); 0: opt^eta = max (optimistic) */
  int32_t maximize;      /* 1: opt^pi = max; 0: opt^pi = min */
  const int32_t* reach;  int32_t n_reach;  /* target set G (reach / reach-avoid) */
  const int32_t* avoid;  int32_t n_avoid;  /* avoid set (reach-avoid); must not meet G */
  const double* reward;  /* n_states rewards (reward property) */
  double discount;       /* reward property: (0, 1] finite horizon, (0, 1) infinite */
} imdp_spec;

typedef struct imdp_model imdp_model;

/* Human-readable name of a status code (static storage). */
IMDP_API const char* imdp_status_string(imdp_status s);

/* One-line detail of the last error raised on the calling thread ("" if none). */
IMDP_API const char* imdp_last_error(void);

/* Library version as "major.minor.patch" (static storage). */
IMDP_API const char* imdp_version(void);

/*
 * Create a device-resident model from CSC arrays (Sec. 3.1, Appendix A).
 *   n_states       |S| >= 1
 *   n_cols         number of (state, action) columns, >= n_states
 *   nnz            number of stored transitions, 0 <= nnz < 2^31
 *   stateptr       int32[n_states + 1]: columns of state s are [stateptr[s], stateptr[s+1]);
 *                  stateptr[0] = 0, strictly increasing (every state has >= 1 action),
 *                  stateptr[n_states] = n_cols
 *   colptr         int32[n_cols + 1]: entries of column j are [colptr[j], colptr[j+1]);
 *                  colptr[0] = 0, nondecreasing, colptr[n_cols] = nnz
 *   rowval         int32[nnz]: destination states, strictly increasing within a column
 *   lower, upper   double[nnz]: P_lo and P_up of each stored transition
 *   dtype          storage precision (IMDP_F64; IMDP_F32 halves the bound storage)
 *   stream         cudaStream_t used for the upload and checks
 *   out            receives the model handle (freed with imdp_model_destroy)
 * Inputs may be host or device pointers; the model keeps its own converted copy
 * (the caller keeps ownership and may free them after the call). Bounds in device
 * or pinned host memory, or in pageable host memory on systems where the GPU
 * reads it (Grace), are converted in place without a staging copy. The call
 * synchronizes `stream`. Returns IMDP_EINVAL for broken structure,
 * IMDP_EINFEASIBLE when a column is infeasible beyond an absolute tolerance of
 * 1e-12 on the sums, IMDP_ENOMEM when device memory runs out.
 */
IMDP_API imdp_status imdp_create_csc(int32_t n_states, int32_t n_cols, int64_t nnz, const int32_t* stateptr,
                            const int32_t* colptr, const int32_t* rowval, const double* lower,
                            const double* upper, imdp_dtype dtype, void* stream, imdp_model** out);

/*
 * imdp_create_csc with IMDP_F32 storage and a chosen per-iteration error budget
 * (no counterpart in the paper, which computes in binary64 only). Every column
 * whose 32-bit rounding error, sum |dlower| + |dupper|, plus 2^-32 for the
 * rounding of the values, exceeds `budget_per_iteration` is a correction column
 * and keeps its exact bounds (20 bytes per transition instead of 12).
 * budget 0 keeps every column exact; a large budget (e.g. 1) none. IMDP_EINVAL
 * for a negative or NaN budget; other arguments and errors as imdp_create_csc.
 */
IMDP_API imdp_status imdp_create_csc_f32(int32_t n_states, int32_t n_cols, int64_t nnz, const int32_t* stateptr,
                                         const int32_t* colptr, const int32_t* rowval, const double* lower,
                                         const double* upper, double budget_per_iteration, void* stream,
                                         imdp_model** out);
/* Correction columns of an IMDP_F32 model: how many, their transitions, and the
 * budget they were chosen by (all 0 for IMDP_F64). Any output may be NULL. */
IMDP_API imdp_status imdp_model_exact_columns(const imdp_model* m, int32_t* n_exact, int64_t* exact_entries,
                                              double* budget_per_iteration);
/*
 * Create a model from dense bounds (Sec. 3.1: IntervalProbabilities with rows =
 * destination states and columns = actions, concatenated over source states).
 *   n_actions      int32[n_states]: number of actions of each state (>= 1)
 *   lower, upper   double[n_states * n_cols], column-major (entry (s', j) at j*n_states + s'),
 *                  n_cols = sum n_actions. Entries with upper == 0 (and lower == 0) are
 *                  structural zeros and are not stored. Host pointers only.
 */
IMDP_API imdp_status imdp_create_dense(int32_t n_states, const int32_t* n_actions, const double* lower,
                              const double* upper, imdp_dtype dtype, void* stream, imdp_model** out);

/* Free a model and its device memory (waits for the device first, as work in
 * flight may still read it). NULL is ignored. */
IMDP_API void imdp_model_destroy(imdp_model* m);

/* Model dimensions and the device bytes it holds. Any output may be NULL. */
IMDP_API imdp_status imdp_model_info(const imdp_model* m, int32_t* n_states, int32_t* n_cols, int64_t* nnz,
                            size_t* device_bytes, int32_t* max_col_nnz);

/*
 * Guaranteed per-iteration error bound of IMDP_F32 storage: the largest sum over
 * one 32-bit column of |lower - stored lower| + |upper - stored upper| (how far
 * the stored intervals move one column's optimum), plus 2^-32 (values kept at
 * 32 bits, rounded to nearest), plus (k_max + 1) 2^-62 (truncated products).
 * Correction columns contribute no rounding. Values lie in [0, 1] and the
 * Bellman operator is non-expansive, so K iterations of a reachability problem
 * stay within K * bound of exact value iteration on the given intervals (scale
 * by the reward map's range for rewards). 0 for IMDP_F64.
 */
IMDP_API imdp_status imdp_model_error_bound(const imdp_model* m, double* per_iteration);

/* Launch plan of a model (no counterpart in the paper; host-only query): the
 * number of tiles the tiled kernel streams, the number of wide states (a state
 * whose entries exceed one tile or that has a column of 1280 entries or more,
 * run by a whole CTA) and the entries of those wide states. Any output may be
 * NULL. IMDP_EINVAL for a NULL model. */
IMDP_API imdp_status imdp_model_plan(const imdp_model* m, int32_t* n_tiles, int32_t* n_wide, int64_t* wide_entries);

/* TEST-ONLY hook for failure detection (no counterpart in the paper; never
 * call it in production code). While `on` is nonzero, step launches of the
 * ring kernel (launch configuration kernel 1) issue no tile copies: every
 * consumer wait runs into its bound
 * (about 2 s), the kernel records the error and returns, and the next read of
 * the session reports IMDP_ETIMEOUT; the CUDA context stays usable. The switch
 * is process-wide; imdp_session_reset turns it off again (and drops the
 * session's captured graph, which may hold stalled launches), so a session
 * that is reset after a timeout runs normally. */
IMDP_API void imdp_debug_stall_producer(int32_t on);

/*
 * value_iteration / control_synthesis (Sec. 3.2) on one model.
 *   V_out         double[n_states] (host or device): V_k after the last iteration
 *   k_out         (host, nullable) iterations performed
 *   residual_out  double[n_states] (host or device, nullable): V_k - V_{k-1} state-wise
 *   policy_out    int32 (host or device, nullable): finite horizon K x n_states,
 *                 entry [t * n_states + s] = local action index for state s at time t
 *                 (time 0 is the first step, the argmax of iteration K - t);
 *                 infinite horizon n_states (stationary policy of the last iteration).
 *                 States held fixed by the property (reach / avoid targets) get -1.
 *                 Ties between actions go to the lowest local index.
 */
IMDP_API imdp_status imdp_value_iteration(imdp_model* m, const imdp_spec* spec, double* V_out, int32_t* k_out,
                                 double* residual_out, int32_t* policy_out, void* stream);


/*
 * Run `count` independent problems (models[i], specs[i]) together: every
 * Bellman iteration of every problem that is still running is one kernel
 * launch for the whole batch. Results are identical to running each problem
 * alone (integer accumulation; no cross-problem reduction).
 *   V_out[i]   double[n_states of models[i]] (host or device)
 *   k_out      int32[count] (host, nullable)
 * A model may appear more than once (e.g. with different specs).
 */
IMDP_API imdp_status imdp_value_iteration_batch(imdp_model* const* models, const imdp_spec* specs, int32_t count,
                                       double* const* V_out, int32_t* k_out, void* stream);

/*
 * Value iteration that allocates no device memory (the paper has no counterpart;
 * this is a deployment aid). For callers that create their models once at
 * start-up and may not allocate afterwards: a controller re-planning every cycle
 * under a fixed memory budget, or code whose device memory belongs to another
 * framework's allocator. Instead of per-call buffers it uses one fixed scratch
 * array compiled into the library (about 3.7 MB, held by every GPU that loads
 * the library until the process exits).
 *   m, spec   as for imdp_value_iteration (reach / reach-avoid properties);
 *             at most 131072 states and 131072 reach + avoid indices, else
 *             IMDP_EINVAL with a message naming the limit; a model of at most
 *             262144 columns keeps its threshold hints from one iteration to
 *             the next as a session does (a larger one searches every column
 *             every iteration: slower, equal up to the products' truncation)
 *   V_out     double[n_states], DEVICE memory on the model's device (current)
 *   k_out     (host, nullable) iterations performed
 * The first call on a device looks up the scratch array's device address; make
 * that first call before any stream capture. Every call synchronizes `stream`
 * before it returns (it reads the iteration state back). All calls share the one array:
 * calls that overlap on the GPU (other streams or host threads) race. Policy and
 * residual outputs are not offered here.
 */
IMDP_API imdp_status imdp_value_iteration_noalloc(imdp_model* m, const imdp_spec* spec, double* V_out,
                                                  int32_t* k_out, void* stream);

/*
 * Resident solver session: the device state of value iteration for `count`
 * problems kept between calls (value buffers, iteration counters, policy
 * storage), so repeated runs and step-by-step control need no re-setup.
 * imdp_value_iteration(_batch) is create + step-until-done + read + destroy.
 *   want_policy   int32[count] (nullable): 1 to record the policy of problem i
 * The models must outlive the session. Sessions are not thread-safe.
 */
typedef struct imdp_session imdp_session;

IMDP_API imdp_status imdp_session_create(imdp_model* const* models, const imdp_spec* specs, int32_t count,
                                         const int32_t* want_policy, void* stream, imdp_session** out);

/* Reset every problem to V_0 and iteration 0 (asynchronous on `stream`). */
IMDP_API imdp_status imdp_session_reset(imdp_session* s, void* stream);

/* Launch `n_iters` Bellman iterations (one kernel each; problems that are done
 * or past their horizon are skipped on the device). Asynchronous on `stream`;
 * chunks of iterations are replayed from a captured CUDA graph when `stream`
 * is not the legacy default stream. */
IMDP_API imdp_status imdp_session_step(imdp_session* s, int32_t n_iters, void* stream);

/* Run until every problem is done (finite: its horizon; infinite: residual < eps
 * or the cap), checking completion every `check_every` iterations (<= 0: 32). */
IMDP_API imdp_status imdp_session_run(imdp_session* s, int32_t check_every, void* stream);

/* Read problem `index`: outputs as in imdp_value_iteration; any may be NULL.
 * Synchronizes `stream`. Returns IMDP_ENOCONV if that problem hit its cap. */
IMDP_API imdp_status imdp_session_read(imdp_session* s, int32_t index, double* V_out, int32_t* k_out,
                                       double* residual_out, int32_t* policy_out, void* stream);

/* Bellman iterations launched by the session so far (one kernel launch each,
 * except on the single-CTA kernel, which runs a step call's iterations in one). */
IMDP_API int64_t imdp_session_launches(const imdp_session* s);

IMDP_API void imdp_session_destroy(imdp_session* s);

/*
 * Launch configuration of a session's Bellman step (no counterpart in the
 * paper, whose GPU kernels have one fixed shape). Every configuration computes
 * the same words; they differ in speed only. Zero fields mean "by rule".
 *   kernel        0 by rule: the single-CTA kernel for a session of one small
 *                 problem; else, from the shape of the session's problems (the
 *                 autotuner's choices on GB300 for the benchmark shapes), direct
 *                 with 3 CTAs per SM and 1024-entry tiles when their columns hold
 *                 256 or more transitions on average, otherwise slice with 3 CTAs
 *                 per SM (4 when every problem has 32-bit storage) when every
 *                 model already has its slice layout (see 4 below: building it
 *                 costs about as many iterations' time as a few hundred save),
 *                 otherwise ring (the server's rule is the single-CTA kernel or
 *                 ring);
 *                 1 ring: a producer warp bulk-copies tiles of
 *                 consecutive states into a three-stage shared-memory ring for
 *                 consumer warps; 2 direct: every warp takes the next tile and
 *                 streams its columns from global memory itself; 3 single CTA:
 *                 one CTA keeps the model and its values in shared memory and
 *                 runs every iteration of a step call in one launch (sessions of
 *                 one problem with at most 1024 states, 1024 columns and 4096
 *                 transitions that is not a slice; IMDP_EINVAL otherwise); 4 slice:
 *                 one lane per column over a second, interleaved copy of every
 *                 model (its "slice layout": windows of whole states of at most
 *                 256 columns, ordered by length and dealt to slices of 32
 *                 columns, entry t of a slice's 32 columns stored contiguously).
 *                 The layout is built on the device when a session first selects
 *                 this kernel (this waits for `stream`); it stays with the model
 *                 until imdp_model_destroy and takes about 1.06 times the
 *                 model's transition storage. IMDP_ENOMEM when it does not fit.
 *   cta_warps     ring: 16 or 24 warps per CTA (24 only without wide states; rule:
 *                 24 when the tiles hold 16 or more columns on average); direct
 *                 and slice: 8
 *   ctas_per_sm   direct and slice: 3 or 4 (rule 4 for an explicit kernel, else
 *                 as above); ring: 1
 *   tile_entries  tile plan: at most this many transitions per tile, 1..3072
 *                 (rule 3072, 1024 for the direct kernel by rule; a single
 *                 state may exceed a smaller limit; the
 *                 slice kernel has no tile plan and ignores it)
 *   wide_col      a state with a column of this many transitions or more (or
 *                 more than 3072 transitions in all) runs in the block-wide
 *                 kernel (rule 1280; ignored by the slice kernel, whose lanes run
 *                 columns of any length)
 */
typedef struct {
  int32_t kernel;
  int32_t cta_warps;
  int32_t ctas_per_sm;
  int32_t tile_entries;
  int32_t wide_col;
} imdp_launch_config;
/* Use `cfg` from the next step on. A changed tile plan is rebuilt (this waits
 * for `stream`); the session's captured graph is dropped. Problems keep their
 * state, so a configuration may change between steps. IMDP_EINVAL for NULL. */
IMDP_API imdp_status imdp_session_set_launch(imdp_session* s, const imdp_launch_config* cfg, void* stream);
/* The configuration the session's launches use, with every field resolved by
 * the rule where the set configuration left it open. */
IMDP_API imdp_status imdp_session_get_launch(const imdp_session* s, imdp_launch_config* cfg);
/* The session's current tile plan (it follows the launch configuration's
 * tile_entries and wide_col): tiles streamed by the tiled kernels (windows of
 * the slice layout for the slice kernel), wide states and their transitions.
 * Any output may be NULL. */
IMDP_API imdp_status imdp_session_plan(const imdp_session* s, int32_t* n_tiles, int32_t* n_wide,
                                       int64_t* wide_entries);
/*
 * Autotuner. Times candidate launch configurations on this session (each: a
 * reset, then `iters` Bellman iterations, timed with CUDA events on `stream`
 * after one untimed run) and keeps the fastest. The choice is cached in the
 * JSON file `cache_path` (nullable: no cache) under a key describing the
 * session's shape (storage, mean transitions per column, columns per state,
 * states, whether it has wide states); a later call with the same key applies
 * the cached configuration without timing. The session is reset afterwards.
 * `chosen` (nullable) receives the configuration in use; `ms_per_iter`
 * (nullable) its measured time per iteration (0 when taken from the cache).
 */
IMDP_API imdp_status imdp_session_autotune(imdp_session* s, int32_t iters, const char* cache_path, void* stream,
                                           imdp_launch_config* chosen, double* ms_per_iter);

/*
 * Infinite-horizon value iteration on 32-bit storage with 64-bit polishing (no
 * counterpart in the paper, which computes in binary64 throughout; Sec. 3.2).
 * The query `spec` (infinite_time required) first runs on m32 (IMDP_F32) until
 * its residual test passes; the 64-bit model m64 (IMDP_F64, the same IMDP: equal
 * structure, on the same device) then continues from that iterate, with the
 * 32-bit run's threshold hints, until the 64-bit residual test passes (at least
 * one 64-bit sweep). The result therefore meets the same stopping test as
 * imdp_value_iteration on m64, after fewer 64-bit sweeps.
 *   cfg32, cfg64 launch configurations of the two phases (nullable: by rule;
 *                as imdp_session_set_launch)
 *   V_out        double[n_states] (host or device), the polished values
 *   k32_out      int32 (host, nullable): iterations on 32-bit storage
 *   k_out        int32 (host, nullable): all iterations (32-bit + 64-bit)
 *   residual_out, policy_out: as imdp_value_iteration, from the 64-bit phase
 * IMDP_EINVAL for NULL arguments, wrong storage types, different structures,
 * state slices or a finite horizon. Synchronizes `stream`.
 */
IMDP_API imdp_status imdp_value_iteration_polished(imdp_model* m32, imdp_model* m64, const imdp_spec* spec,
                                                   const imdp_launch_config* cfg32, const imdp_launch_config* cfg64,
                                                   double* V_out, int32_t* k32_out, int32_t* k_out,
                                                   double* residual_out, int32_t* policy_out, void* stream);
/*
 * State-sharded value iteration (one model split over several GPUs).
 * Sec. 4 notes that the per-state problems of Eq. 2 are independent within an
 * iteration: a slice that owns states [s0, s1) computes V_k[s0, s1) exactly as
 * the whole model does, given all of V_{k-1}. The caller runs one session per
 * slice, steps every session one iteration at a time, and after each step
 * copies every slice's owned values into all other slices (an all-gather),
 * using imdp_session_values_get / _put on device buffers. An infinite horizon
 * on a slice never stops by itself (its own residual covers its states only):
 * after each step the caller takes imdp_session_residual of every slice, the
 * maximum over the slices (an all-reduce), and stops when it is below the
 * threshold imdp_session_stop_threshold gives, which is the unsharded run's
 * own test (imdp_session_run refuses such a session, IMDP_EINVAL).
 */

/* Contiguous state ranges of about equal work (20 B per transition, 12 B per
 * column, 20 B per state and iteration): bounds int32[n_parts + 1], bounds[0] =
 * 0, bounds[n_parts] = n_states, every range non-empty. stateptr (n_states + 1)
 * and colptr are the whole model's CSC arrays (host). Host-only; needs no
 * device. IMDP_EINVAL unless 1 <= n_parts <= n_states. */
IMDP_API imdp_status imdp_partition_states(int32_t n_states, const int32_t* stateptr, const int32_t* colptr,
                                           int32_t n_parts, int32_t* bounds);

/* Slice of an n_states model that owns states [s0, s1): stateptr has s1 - s0 + 1
 * entries (starting at 0, ending at n_cols) and colptr / rowval / lower / upper
 * hold the columns of those states only, in the layout of imdp_create_csc;
 * rowval indexes the whole state space [0, n_states). Only owned states are
 * updated by a session on the slice; the others hold what imdp_session_values_put
 * writes (initially V_0). Validation and errors as imdp_create_csc. */
IMDP_API imdp_status imdp_create_csc_slice(int32_t n_states, int32_t s0, int32_t s1, int32_t n_cols, int64_t nnz,
                                           const int32_t* stateptr, const int32_t* colptr, const int32_t* rowval,
                                           const double* lower, const double* upper, imdp_dtype dtype, void* stream,
                                           imdp_model** out);

/* Copy V_k[s0, s1) of problem `index` (k = iterations completed; V_0 after a
 * reset) as raw 64-bit words (Q1.63 fixed point, or the affine-mapped value of
 * a reward problem) to / from device memory `dst` / `src` (s1 - s0 words),
 * asynchronously on `stream`. The words move between sessions of identical
 * specifications only. IMDP_EINVAL for a bad index or range or host memory. */
IMDP_API imdp_status imdp_session_values_get(imdp_session* s, int32_t index, int32_t k, int32_t s0, int32_t s1,
                                             uint64_t* dst, void* stream);
IMDP_API imdp_status imdp_session_values_put(imdp_session* s, int32_t index, int32_t k, int32_t s0, int32_t s1,
                                             const uint64_t* src, void* stream);
/* max over states [s0, s1) of |V_k - V_{k-1}| as a raw word (the units of the
 * values words), written to one uint64 of DEVICE memory `dst`, asynchronously on
 * `stream` (Eq. 2's Bellman residual, the quantity the stopping test of an
 * infinite horizon compares). IMDP_EINVAL for k < 1, a bad range or host dst. */
IMDP_API imdp_status imdp_session_residual(imdp_session* s, int32_t index, int32_t k, int32_t s0, int32_t s1,
                                           uint64_t* dst, void* stream);
/* The raw threshold of problem `index`'s stopping test: the run stops after the
 * first iteration whose residual (raw words) is below *eps_raw. IMDP_EINVAL for
 * a finite horizon. */
IMDP_API imdp_status imdp_session_stop_threshold(const imdp_session* s, int32_t index, uint64_t* eps_raw);

/*
 * Checkpoint and resume (not in the paper: value iteration's whole state for one
 * problem is its iterate V_k and k). imdp_session_checkpoint copies problem
 * `index`'s latest iterate (n_states raw 64-bit words as imdp_session_values_get
 * gives them) to `raw_V` (host or device) and its completed iterations to *k.
 * imdp_session_restore writes both into problem `index` of a session built from
 * the same model and specification, which then continues with iteration k + 1
 * (a finite horizon with k = horizon is finished). The problem's threshold hints
 * start empty after a restore, so a resumed run matches an uninterrupted one
 * within the arithmetic's rounding (1e-13 in V), not bit for bit; rows of a
 * time-dependent policy computed before the checkpoint are not part of it. The
 * session may have run before the restore (it need not be fresh): the next
 * imdp_session_run still carries the restored problem to its horizon. A
 * checkpoint does not record that an infinite-horizon problem had already
 * converged (only V_k and k are kept), so such a problem, restored, runs one
 * more iteration before its convergence test stops it again (k + 1). Both
 * calls are ordered on `stream` and synchronize it. IMDP_EINVAL for a bad
 * index, k < 0, k above a finite horizon, or NULL pointers.
 */
IMDP_API imdp_status imdp_session_checkpoint(imdp_session* s, int32_t index, uint64_t* raw_V, int32_t* k,
                                             void* stream);
IMDP_API imdp_status imdp_session_restore(imdp_session* s, int32_t index, const uint64_t* raw_V, int32_t k,
                                          void* stream);

/*
 * Continuous-batching server. Requests (a resident model plus a specification)
 * share the Bellman launches of one slotted batch run by a worker thread: a
 * request is admitted when a slot (up to 1024) and enough of the server's device
 * memory budget are free, joins the running batch between chunks of 8
 * iterations, and retires on its own horizon or convergence test. Each result
 * equals what imdp_value_iteration returns for the same request alone.
 *   hbm_budget   bytes of device memory for per-request state (values, masks,
 *                hints, outputs); allocated once at creation (>= 1 MiB)
 * Thread-safe: submit/poll/wait may be called from any thread. Models must
 * outlive their requests. Policies are not produced by the server.
 */
typedef struct imdp_server imdp_server;
IMDP_API imdp_status imdp_server_create(size_t hbm_budget, imdp_server** out);
/* Launch configuration of the server's Bellman launches (imdp_launch_config;
 * zero fields by rule). Requests admitted afterwards are planned with its tile
 * limits; it may change while requests run (a running request keeps its plan).
 * Thread-safe. IMDP_EINVAL for NULL or a bad configuration. */
IMDP_API imdp_status imdp_server_set_launch(imdp_server* s, const imdp_launch_config* cfg);
/* Where the server's time went since its creation (no counterpart in the paper):
 * device_ms = the device time of its Bellman launches (CUDA events around each
 * chunk), wall_ms = the worker's time while requests were admitted or running
 * (launches, read-back, retirement, admission, table uploads), chunks = chunks of
 * launches, mean_requests = requests in a chunk's launches on average. Any
 * output may be NULL. Thread-safe. */
IMDP_API imdp_status imdp_server_stats(imdp_server* s, double* device_ms, double* wall_ms, int64_t* chunks,
                                       double* mean_requests);
/* Queue a request; returns at once with a ticket. IMDP_ENOMEM if the request
 * alone exceeds the budget, IMDP_EBUSY if the queue is full. */
IMDP_API imdp_status imdp_server_submit(imdp_server* s, imdp_model* m, const imdp_spec* spec, uint64_t* ticket);
/* Result of a finished request (then the ticket is released): V_out double[n]
 * (host or device), k_out iterations, latency_ms from submit to completion.
 * IMDP_EPENDING while it runs, IMDP_ENOTFOUND for an unknown ticket. */
IMDP_API imdp_status imdp_server_poll(imdp_server* s, uint64_t ticket, double* V_out, int32_t* k_out,
                                      double* latency_ms);
/* poll after waiting up to timeout_ms for the request (IMDP_ETIMEOUT if it is still running). */
IMDP_API imdp_status imdp_server_wait(imdp_server* s, uint64_t ticket, double timeout_ms, double* V_out,
                                      int32_t* k_out, double* latency_ms);
IMDP_API void imdp_server_destroy(imdp_server* s);

/*
 * Model files (Sec. 3.1, reading and writing IMDPs): the PRISM explicit format
 * (four files sharing one path stem: .sta states, .lab labels, .tra interval
 * transitions, .pctl the property) and the bmdp-tool format (one file: source,
 * action, destination and the two bounds per line, plus the terminal states).
 * These calls run on the host only and need no CUDA device.
 *
 * bmdp-tool layout (whitespace-separated ASCII, 0-based indices):
 *     n_states
 *     n_actions                (the largest number of actions of a state)
 *     n_terminal
 *     t_1 ... t_n_terminal     (terminal states)
 *     s a s' lower upper       (one line per stored transition, any order)
 * The format stores no horizon and no modes: a read sets spec.property =
 * IMDP_REACH, spec.reach = the terminal states, horizon 0, finite time,
 * pessimistic, maximize, and the caller sets what the query needs.
 *
 * PRISM explicit layout (0-based indices):
 *     .sta  "(vars)" then one line "i:(values)" per state i
 *     .lab  0="init" 1="deadlock" ... (label ids and names) on the first line,
 *           then "s: id id ..." per labelled state
 *     .tra  "n_states n_choices n_transitions" then "s c s' [lower,upper]" per
 *           transition (a plain probability p reads as [p,p]; a trailing action
 *           name is ignored); the choices of a state are numbered 0, 1, ...
 *     .pctl one property: P<strategy><adversary>=? [ F "goal" ], [ F<=K "goal" ],
 *           [ !"avoid" U "goal" ] or [ !"avoid" U<=K "goal" ], with strategy and
 *           adversary each max or min (adversary min = pessimistic); a missing
 *           adversary (Pmax=?, Pmin=?) reads as pessimistic. Without a bound the
 *           property is infinite-time with eps = 1e-6. Reward properties have no
 *           place in these four files and are rejected.
 *
 * A state that has no transition in the file is read as absorbing: one column
 * holding the self-loop [1, 1], whose `action` entry is -1. Columns of a state
 * are ordered by the file's action (choice) index, destinations ascending.
 * Reads check the structure (indices in range, no duplicate transition, counts
 * that match the headers, finite bounds) and return IMDP_EINVAL with
 * "file:line: reason" in imdp_last_error(); feasibility of the intervals is
 * checked when the arrays are passed to imdp_create_csc. A file that cannot be
 * opened or written returns IMDP_EIO. Writers print bounds with 17 significant
 * digits, so a write followed by a read returns the same binary64 values.
 */
typedef struct {
  int32_t n_states;
  int32_t n_cols;
  int64_t nnz;
  int32_t* stateptr; /* int32[n_states + 1] */
  int32_t* colptr;   /* int32[n_cols + 1] */
  int32_t* rowval;   /* int32[nnz], strictly increasing within a column */
  double* lower;     /* double[nnz] */
  double* upper;     /* double[nnz] */
  int32_t* action;   /* int32[n_cols]: the file's action (bmdp-tool) or choice (PRISM) index; -1 for an added self-loop */
  imdp_spec spec;    /* the query the file states; spec.reach and spec.avoid point into this object */
} imdp_file;

/* Read a bmdp-tool file. *out is library-owned: free it with imdp_file_free. */
IMDP_API imdp_status imdp_read_bmdp_tool(const char* path, imdp_file** out);

/* Write a model (the CSC arrays of imdp_create_csc, host pointers) and its
 * terminal states as a bmdp-tool file; the action of column j of state s is
 * j - stateptr[s]. */
IMDP_API imdp_status imdp_write_bmdp_tool(const char* path, int32_t n_states, int32_t n_cols, const int32_t* stateptr,
                                 const int32_t* colptr, const int32_t* rowval, const double* lower,
                                 const double* upper, const int32_t* terminal, int32_t n_terminal);

/* Read the PRISM explicit files path_stem.{sta,lab,tra,pctl}. *out is
 * library-owned: free it with imdp_file_free. */
IMDP_API imdp_status imdp_read_prism(const char* path_stem, imdp_file** out);

/* Write a model (host CSC arrays) and a reachability or reach-avoid
 * specification as PRISM explicit files path_stem.{sta,lab,tra,pctl}. State 0
 * is labelled "init"; the target set is labelled "reach" and the avoid set
 * "avoid". spec->eps is not stored (the format has no place for it). */
IMDP_API imdp_status imdp_write_prism(const char* path_stem, int32_t n_states, int32_t n_cols, const int32_t* stateptr,
                             const int32_t* colptr, const int32_t* rowval, const double* lower,
                             const double* upper, const imdp_spec* spec);

/* Free an imdp_file returned by a read. NULL is ignored. */
IMDP_API void imdp_file_free(imdp_file* f);

#ifdef __cplusplus
}
#endif
#endif /* IMDP_H */
