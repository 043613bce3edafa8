/*
 * paid.h -- C ABI of the GB300 (sm_103a) batched adaptive cubature of
 * Brillouin-zone bubble integrals (PAID hot path).
 *
 * What is computed.  For each integral (kind, q, l, m, T) the library returns
 *
 *   ph: I = (1/(2pi)^2) Int_D f_l(k) f_m(k+q) [nF(e(k+q)) - nF(e(k))] / (e(k) - e(k+q)) d^2k
 *   pp: I = (1/(2pi)^2) Int_D f_l(k) f_m(q-k) [1 - nF(e(k)) - nF(e(q-k))] / (e(k) + e(q-k)) d^2k
 *
 * over D = [-pi, pi]^2, with the analytic limit -nF'(e) at a vanishing
 * denominator -- the momentum integrals of the paper's Eq. chi_ph / chi_pp
 * (Sec. 2) after the Matsubara sum at temperature T.  The dispersion is the
 * t-t' square-lattice one of Sec. 2,
 *   e(k) = -2t (cos kx + cos ky) - 4t' cos kx cos ky - mu,
 * and f_n are the orthonormal lattice form factors of Sec. 2:
 *   f0 = 1, f1 = cx + cy, f2 = cx - cy, f3 = sqrt2 sx, f4 = sqrt2 sy,
 *   f5 = 2 cx cy, f6 = 2 sx sy, f7 = 2 sx cy, f8 = 2 cx sy
 * (cx = cos kx, sx = sin kx, ...).  Two test kinds share the same path:
 * PAID_OVERLAP (kernel = 1, integrand f_l(k) f_m(k+q)/(2pi)^2) and
 * PAID_MONOMIAL (integrand (kx/pi)^l (ky/pi)^m/(2pi)^2, 0 <= l, m <= 30).
 *
 * The flow kinds (options.group_mode only) are the Omega-regulated bubbles of
 * the flow equations, Eqs. chi_ph / chi_pp with G(k) = theta(k0)/(i k0 - e(k)),
 * theta(k0) = k0^2/(k0^2 + Omega^2) (Sec. 2), at zero temperature, their
 * frequency integral (measure dk0/2pi) done analytically and differentiated
 * in Omega; a batch's T field carries Omega > 0.  With symmetric routing
 * (q = the transfer momentum l of Sec. 2) and both form factors at k:
 *   flow ph: I = (1/(2pi)^2) Int f_l(k) f_m(k) Hd(e(k + q/2), e(k - q/2)) d^2k
 *   flow pp: I = -(1/(2pi)^2) Int f_l(k) f_m(k) Hd(e(q/2 + k), -e(q/2 - k)) d^2k
 * where Hd(a, b) = [Hdot(a) - Hdot(b)] / (a - b) is the divided difference of
 * Hdot(e) = e (3|e| + Omega) / (4 (|e| + Omega)^3), the Omega derivative of
 * H(e) = Int dk0/2pi theta^2/(i k0 - e) = -e (2|e| + Omega)/(4 (|e| + Omega)^2).
 *
 * How.  Adaptive cubature (Algorithm 1, with the 4-way split of
 * Algorithm 2): every region carries the nested Clenshaw-Curtis pair
 * Q_N, Q_2N and err = |Q_N - Q_2N| (Sec. 3); the returned value is the sum of
 * Q_2N over the final regions (Listing 5) and the returned error the sum of
 * err.  Unlike the paper's one serial heap per group, each integral keeps its
 * own convergence test E <= max(abs_tol, rel_tol |V|), and each round splits,
 * per unconverged integral, the largest-error set of regions whose error
 * covers the excess over the tolerance (a batched extract-max, Listing 2).
 *
 * Conventions (all entry points):
 *   - Device pointers are CUDA device memory on the context's device; host
 *     pointers are ordinary host memory.  The caller owns every buffer and
 *     must keep it alive until the work on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (0 = legacy default stream).
 *   - Return value: PAID_OK or a negative paid_rc.  Argument errors are
 *     detected on the host before any work is queued.  Per-integral outcomes
 *     are in `status` (paid_status).  paid_last_error() gives a message.
 *   - A context is used by one host thread at a time.
 *   - Output order of a batch: idx = iq * npairs + ip.
 *   - With options.device_loop = 1 (the default) and timing = 0 the integrate
 *     calls are asynchronous on `stream`: they queue the setup, the refinement
 *     loop (one CUDA graph launch) and its finish, and return; their return
 *     code covers argument and launch errors only.  Per-integral outcomes land
 *     in `status` with the values; paid_wait() waits for the call and returns
 *     its outcome (PAID_OK, PAID_ERR_POOL, PAID_ERR_TIMEOUT) and statistics.
 *     paid_integrate_multi_seeded waits once, before the loop, for the size of
 *     its seeded partition.  A call on a context whose previous call is still
 *     pending first waits for that one (they share the loop state and graph).
 *     With device_loop = 0 or timing = 1 the round loop runs from the host and
 *     the calls return when the outputs are complete (they synchronise
 *     `stream`), as do paid_integrate_batch_static and paid_rule_regions.
 *   - The region pool need not hold every integral at once: integrals enter
 *     it as room frees up, and when a round's splits would overflow it the
 *     integrals split in order while the growth fits and the rest wait a
 *     round.  Only a pool that
 *     cannot make progress at all returns PAID_ERR_POOL (status PAID_POOL on
 *     the integrals it could not finish, NaN values for those never started).
 */
#ifndef PAID_H
#define PAID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct paid_ctx paid_ctx;

/* Form-factor sets (Sec. 2): one bond shell (5 functions) or two (9). */
typedef enum { PAID_FF_SHELL1 = 5, PAID_FF_SHELL12 = 9 } paid_ffset;

/* Integrand kinds. */
typedef enum { PAID_PH = 0, PAID_PP = 1, PAID_MONOMIAL = 2, PAID_OVERLAP = 3,
               PAID_FLOW_PH = 4, PAID_FLOW_PP = 5 } paid_kind;

/* Call status. */
typedef enum {
    PAID_OK = 0,
    PAID_ERR_ARG = -1,      /* invalid argument; nothing was queued */
    PAID_ERR_OOM = -2,      /* workspace too small for the integral count */
    PAID_ERR_CUDA = -3,     /* a CUDA call failed; see paid_last_error */
    PAID_ERR_POOL = -4,     /* region pool full; unfinished integrals have status PAID_POOL */
    PAID_ERR_TIMEOUT = -5   /* round cap reached; unfinished integrals have status PAID_ROUNDCAP */
} paid_rc;

/* Per-integral status. */
typedef enum {
    PAID_CONVERGED = 0,     /* E <= max(abs_tol, rel_tol |V|) */
    PAID_BUDGET = 1,        /* region budget (or the deepest level) reached first */
    PAID_NONFINITE = 2,     /* V or E not finite (NaN/Inf input, invalid l or m) */
    PAID_ROUNDCAP = 3,      /* options.max_rounds reached */
    PAID_POOL = 4           /* region pool capacity reached */
} paid_status;

/* Values of options.group_mode. */
typedef enum {
    PAID_GROUP_NONE = 0,      /* one partition per integral, per-integral test */
    PAID_GROUP_PER_PAIR = 1,  /* one partition per (kind, q), every pair meets its own test */
    PAID_GROUP_GLOBAL = 2     /* one partition per (kind, q), one error sum per group
                                 (the global error of Algorithm 2, Sec. 4) */
} paid_group_mode;

/* Options; paid_options_default() fills the defaults named here. */
typedef struct {
    int rule_n;             /* N of the nested CC pair (coarse N, fine 2N intervals): 4 or 6, and
                               with group_mode also 8, 10 or 12. Default 4 */
    int init_level;         /* L0: initial uniform partition of D into 4^L0 regions, 0..8. Default 2 */
    int eval_fp32;          /* 1: integrand on the FP32 pipe.  One partition per integral: FP32
                               integrand, FP64 sums, integrals whose FP32 rounding noise crowds
                               their tolerance re-evaluated in float-float.  group_mode: the
                               kernel F, the rule's row sums and moments (taken in the Fourier
                               basis 1, cos k, sin k, cos 2k, sin 2k of each direction), each
                               region's pair values Q_2N, Q_N and their difference in
                               float-float (unevaluated pairs of FP32 numbers, about 44
                               significant bits after rounding); Q_2N stored in FP64, the error
                               estimate in FP32, all totals in FP64.  Default 0 (all FP64) */
    int max_rounds;         /* cap on refinement rounds of an integral, counted from the round
                               it entered the pool. Default 4096 */
    double cover;           /* the regions split in a round cover (E - cover * tol) of the error. Default 0.5 */
    int64_t pool_capacity;  /* regions in the pool; 0 = the most the workspace holds. Default 0 */
    int timing;             /* 1: time every kernel class with CUDA events on the call's stream
                               (totals in paid_stats); implies device_loop = 0. Default 0 */
    int device_loop;        /* 1: the refinement loop runs on the device as one CUDA graph launch
                               (a conditional WHILE node around one round's kernels) and the
                               integrate calls return without waiting (see paid_wait).  0: the
                               host launches every round and reads its counts back.  Default 1 */
    int group_mode;         /* 1: one shared partition per (kind, q) of a batch serves all of the
                               batch's (l, m) pairs (at most 81; kinds ph, pp, overlap, flow).
                               A region evaluates the kernel F once per node and every pair from
                               81 separable moments; it is split while any pair of the group has
                               not met its own tolerance.  Every integral still meets
                               E <= max(abs_tol, rel_tol |V|) with E its own error sum; the
                               region count reported is the group's.  max_regions bounds the
                               group's regions and pool_capacity counts them (about 2 KB each).
                               2: the same shared partition with the global error of
                               Algorithm 2 (Sec. 4): one error sum and one tolerance per group,
                               done when sum_c E_c <= max(abs_tol, rel_tol sum_c |V_c|) over the
                               group's valid pairs (rel_tol = 0 gives the paper's absolute
                               eps = abs_tol); a region's score is its share of the sum, and
                               every pair of a finished group takes the group's status.
                               Default 0 (one partition per integral) */
    int eval_blocks;        /* group_mode: grid of the region-evaluation kernel (it strides over
                               the eval list); 0 = 152 x 32 blocks.  Default 0 */
    int trace;              /* 1: every integrate call records each unit's final partition as a
                               16 x 16 map (entry c = 16 ix + iy: the level of the coarsest final
                               region meeting level-4 cell (ix, iy); a region of level L < 4
                               counts for all 4^(4-L) cells it covers) into the buffer given to
                               paid_set_trace_buffer (none given: nothing is recorded); a unit is
                               a (kind, q) group in group_mode, else an integral, in the call's
                               global order; cells of units the call never started are NaN.
                               These maps are the training targets of the learned proposal.
                               Default 0 */
} paid_options;

/* Statistics of the last integrate call on a context. */
typedef struct {
    int rounds;                 /* refinement rounds run */
    int64_t region_evals;       /* regions evaluated (each 81 nodes at N = 4) */
    int64_t node_evals;         /* integrand evaluations */
    int64_t peak_pool;          /* largest pool occupancy (regions) */
    int64_t pool_capacity;      /* capacity used */
    int64_t n_integrals;
    int64_t launches;           /* kernels launched by the call */
    int64_t eval_launches;      /* region-evaluation launches */
    double eval_ms;             /* with options.timing: summed device time of ... */
    double reduce_ms;           /* ... region evaluation, reduce + test, */
    double scan_ms;             /* ... slot scan, */
    double split_ms;            /* ... split + compaction (0 without timing) */
    int64_t escalated;          /* eval_fp32: integrals moved to float-float evaluation because
                                   their FP32 rounding-noise term crowded their tolerance */
    int64_t df_regions;         /* eval_fp32: regions evaluated in float-float */
    double df_ms;               /* with options.timing: the float-float kernel's share of eval_ms */
    int64_t throttled_rounds;   /* rounds in which some integrals waited (pool pressure) */
    int64_t graph_launches;     /* device-loop graph launches (1 per call with device_loop) */
} paid_stats;

/* Fill *opt with the defaults.  Returns PAID_OK or PAID_ERR_ARG (opt NULL). */
int paid_options_default(paid_options* opt);

/* Create a context on CUDA device `device` for lattice (t, t', mu) and the
 * form-factor set `ffset` (PAID_FF_SHELL1 or PAID_FF_SHELL12).  `opt` may be
 * NULL for the defaults.  The context owns a small pinned host block and
 * nothing else; all work memory comes from the caller's workspace.
 * Returns PAID_OK and *out, or PAID_ERR_ARG / PAID_ERR_CUDA. */
int paid_create(paid_ctx** out, double t, double tp, double mu, int ffset,
                const paid_options* opt, int device);

/* Release a context (NULL is allowed). */
void paid_destroy(paid_ctx* ctx);

/* Bytes of device workspace needed for `n_units` units of a call -- its
 * integrals, or with options.group_mode its (kind, q) groups (the sum of the
 * batches' nq) -- and a pool of `pool_capacity` regions (pool_capacity >=
 * n_units * 4^init_level).  Returns PAID_OK and *bytes, or PAID_ERR_ARG. */
int paid_workspace_size(paid_ctx* ctx, int64_t n_units, int64_t pool_capacity,
                        size_t* bytes);

/* Largest pool capacity (regions) that `ws_bytes` of workspace holds for
 * `n_units` units.  Returns PAID_OK and *capacity (0 if none fits). */
int paid_pool_capacity(paid_ctx* ctx, int64_t n_units, size_t ws_bytes,
                       int64_t* capacity);

/* One batch of integrals of one kind at one temperature.
 *   q       device, double [nq][2]        transfer momenta (qx, qy)
 *   lm      device, int32  [npairs][2]    form-factor pairs (l, m)
 *   values  device, double [nq*npairs]    sum of Q_2N over the final regions
 *   errors  device, double [nq*npairs]    sum of |Q_N - Q_2N| over them
 *   regions device, int64  [nq*npairs]    final region count
 *   status  device, int32  [nq*npairs]    paid_status
 * rel_tol, abs_tol >= 0; max_regions >= 4^init_level (at most 2^23).
 * workspace: device memory of ws_bytes (>= paid_workspace_size). */
int paid_integrate_batch(paid_ctx* ctx, int kind,
                         int nq, const double* q, int npairs, const int32_t* lm,
                         double T, double rel_tol, double abs_tol, int64_t max_regions,
                         double* values, double* errors, int64_t* regions, int32_t* status,
                         void* workspace, size_t ws_bytes, void* stream);

/* Several batches (kinds and temperatures) drained together in one pool:
 * the argument meanings are those of paid_integrate_batch, per batch.
 *
 * tu_v, tu_out: the truncated-unity right-hand sides of the flow equations
 * (Eqs. matmul-P, matmul-C, matmul-D, Sec. 2) formed in the same call, as each
 * (kind, q) group finishes, from its bubble matrix X[l][m] (the group's values
 * of pair l * nff + m) -- only for the flow kinds with options.group_mode and
 * every pair (l, m), l-major (npairs = nff^2); NULL pointers: no products.
 *   PAID_FLOW_PP: tu_v[0] = V^P, tu_out[0] = dP = V^P X V^P;
 *   PAID_FLOW_PH: tu_v[0] = V^C, tu_v[1] = V^D, tu_out[0] = dC = -V^C X V^C,
 *                 tu_out[1] = dD = 2 V^D X V^D - V^C X V^D - V^D X V^C;
 * all device double [nq][nff][nff], row-major, the outputs not aliasing the
 * inputs.  A batch whose pairs are not in that order gets NaN products; a
 * group the call never started gets NaN products. */
typedef struct {
    int kind;
    double T;
    int nq;
    const double* q;
    int npairs;
    const int32_t* lm;
    double rel_tol;
    double abs_tol;
    int64_t max_regions;
    double* values;
    double* errors;
    int64_t* regions;
    int32_t* status;
    const double* tu_v[2];
    double* tu_out[2];
} paid_batch;

int paid_integrate_multi(paid_ctx* ctx, const paid_batch* batches, int nb,
                         void* workspace, size_t ws_bytes, void* stream);

/* The nested rule of Sec. 3 on given regions, for every pair of one
 * (kind, q): the building block of the shared-partition mode, exposed so that
 * a caller can evaluate a partition of its own.
 *   kind: PAID_PH, PAID_PP or PAID_OVERLAP; T > 0.
 *   q: device double [2]; lm: device int32 [npairs][2], 1 <= npairs <= 81.
 *   regions: device int32 [nreg][3] = (level, ix, iy): the square with lower
 *     corner -pi + 2 pi (ix, iy) / 2^level and side 2 pi / 2^level,
 *     0 <= level <= 29, 0 <= ix, iy < 2^level.  An invalid region gives NaN.
 *   q2N, dq: device double [nreg][npairs], written: Q_2N and Q_N - Q_2N of
 *     pair p on region r, times the region's Jacobian (h/2)^2 / (2 pi)^2, so
 *     that summing q2N over a partition of D gives the integral.
 *   workspace: device, 256-byte aligned, at least paid_workspace_size(ctx, 1,
 *     max(nreg, 16)) bytes.
 * Returns PAID_OK (outputs complete, the stream synchronised), PAID_ERR_ARG,
 * PAID_ERR_OOM (workspace too small) or PAID_ERR_CUDA. */
int paid_rule_regions(paid_ctx* ctx, int kind, double T, const double* q, int npairs,
                      const int32_t* lm, int nreg, const int32_t* regions, double* q2N,
                      double* dq, void* workspace, size_t ws_bytes, void* stream);

/* Diagnostics: the arithmetic of the shared-partition kernel (its own exp
 * after Tang's table-driven method, its own division from the approximate
 * reciprocal and Newton-Raphson steps, and their float-float counterparts
 * of the FP32-pipe path), applied element-wise on device arrays so that tests
 * can hold them to their error bounds.
 *   which = 0: out[i] = exp(-x[i]), x[i] >= 0, FP64 (y unused, may be NULL);
 *   which = 1: out[i] = x[i] / y[i], y[i] normal and non-zero, FP64;
 *   which = 2: out[i] = exp(-x[i]), x[i] >= 0, float-float (x rounded to
 *              float-float first; y unused);
 *   which = 3: out[i] = 2T F(x1, x2) of the temperature bubbles (Sec. 2,
 *              F = [tanh x1 - tanh x2] / (2 (e1 - e2)), x = e/2T) at
 *              x1 = x[i], x2 = y[i], float-float;
 *   which = 4: the same 2T F in FP64;
 *   which = 5: the Omega derivative of the flow kinds' frequency integral,
 *              the divided difference of Hdot at (e1, e2) = (x[i], y[i]) with
 *              Omega = 0.1 (flow ph), float-float;
 *   which = 6: the same in FP64.
 * Returns PAID_OK (stream synchronised), PAID_ERR_ARG or PAID_ERR_CUDA. */
int paid_check_math(paid_ctx* ctx, int which, int64_t n, const double* x, const double* y,
                    double* out, void* stream);

/* The context's current options (after paid_autotune, say). */
int paid_get_options(paid_ctx* ctx, paid_options* out);

/* Autotuner: picks options.rule_n (the nested rule's N; the paper reports N = 6
 * as its best-performing setting, Sec. 5), options.cover (how many regions a
 * round splits), in group_mode options.eval_blocks (the evaluation grid), and
 * options.init_level (the uniform start) for this GPU by timing paid_integrate_multi on `sample` (a few batches the
 * caller chose as representative; their outputs are overwritten), stagewise:
 * rule_n in {4, 6} (group mode: {4, 6, 8, 10, 12}) at cover 1, then cover in
 * {0.5, 0.75, 0.9, 1.0}, then eval_blocks in {608, 1216, 4864, 19456} (group mode),
 * then init_level in {2, 3} (every unit's first batch of regions: 16 or 64),
 * each with the choices made so far.  The fastest candidate that completes
 * becomes the context's setting.
 *   cache_path  NULL, or a JSON Lines file: when it holds an entry for this
 *               device name, eval_fp32 and group_mode the entry is
 *               applied without timing (sample may then be NULL); otherwise
 *               the tuned choice is written there, replacing any older entry
 *               with the same key.
 *   workspace, ws_bytes, stream as for paid_integrate_multi.
 * Returns PAID_OK, PAID_ERR_ARG or PAID_ERR_CUDA (no candidate completed; the
 * options are left unchanged). */
int paid_autotune(paid_ctx* ctx, const paid_batch* sample, int nb, const char* cache_path,
                  void* workspace, size_t ws_bytes, void* stream);

/* Truncated-unity products of the flow equations (Eqs. matmul-P, matmul-C,
 * matmul-D, Sec. 2) for nq transfer momenta:
 *   dP = VP Xpp VP,   dC = -VC Xph VC,   dD = 2 VD Xph VD - VC Xph VD - VD Xph VC
 * All arguments are device arrays of nq row-major nff x nff FP64 matrices
 * (1 <= nff <= 9); Xpp / Xph are the pp / ph bubble matrices in the output
 * order of a batch whose pairs are all (l, m), l-major (idx = iq*nff*nff +
 * l*nff + m).  The outputs must not alias the inputs.  Queued on `stream`
 * (asynchronous; no allocation).  Returns PAID_OK, PAID_ERR_ARG or
 * PAID_ERR_CUDA (launch error). */
int paid_tu_flow_rhs(paid_ctx* ctx, int nq, int nff, const double* VP, const double* VC,
                     const double* VD, const double* Xpp, const double* Xph, double* dP,
                     double* dC, double* dD, void* stream);

/* paid_integrate_batch without a workspace argument, for callers that cannot
 * allocate device memory when they need the integrals: runtimes that fix their
 * device-memory budget at start-up, plug-ins living inside another framework's
 * memory manager, or latency-bound loops that must not allocate (cudaMalloc and
 * cudaFree can synchronise the device).  (The paper has no counterpart; it is
 * a deployment convenience.)
 *   - The region pool is a 64 MiB array built into the library
 *     (PAID_STATIC_SCRATCH_BYTES); every GPU that loads the library keeps it
 *     until the process exits.  The call allocates nothing: no cudaMalloc,
 *     cudaFree, or host heap.  It does need a context, which paid_create makes
 *     (and which allocates a small pinned block once, at creation).
 *   - At most PAID_STATIC_MAX_INTEGRALS = 4096 integrals (nq * npairs) per
 *     call; more returns PAID_ERR_ARG.  A batch whose refinement outgrows the
 *     pool returns PAID_ERR_POOL, with status PAID_POOL on the unfinished
 *     integrals, exactly as paid_integrate_batch does with a small workspace.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) for that device.
 *   - All calls on a device share the one array and each call leaves its
 *     contents behind.  Nothing in it has to start cleared (every part is
 *     written before it is read within a call), but two calls that overlap on
 *     the GPU -- from two host threads or on two streams -- race on it and
 *     corrupt each other: run them one after the other.
 *   - paid_last_error() is not updated by this call (setting the message
 *     could allocate); the return code and paid_error_string() say what
 *     failed.  Other arguments, outputs and statuses are as for
 *     paid_integrate_batch, and the results are the same. */
#define PAID_STATIC_SCRATCH_BYTES (64u << 20)
#define PAID_STATIC_MAX_INTEGRALS 4096
int paid_integrate_batch_static(paid_ctx* ctx, int kind,
                                int nq, const double* q, int npairs, const int32_t* lm,
                                double T, double rel_tol, double abs_tol, int64_t max_regions,
                                double* values, double* errors, int64_t* regions,
                                int32_t* status, void* stream);

/* ---------------------------------------------------------------------------
 * Learned refinement proposal (not in the paper; the workload specification's
 * learned component).  A 16 x 16 map per unit -- (kind, q) group in group_mode,
 * else integral -- of the predicted level of the coarsest final region in each
 * level-4 cell (what options.trace records) decides how deep each cell of the
 * domain starts; it never decides convergence (the |Q_N - Q_2N| sums still
 * do), and a map entry that is too deep only costs evaluations.
 *
 * Map convention: entry c = 16 ix + iy is the level-4 cell (ix, iy) of the
 * region grid.
 * ------------------------------------------------------------------------- */

/* The buffer the integrate calls write their trace maps to when
 * options.trace = 1: device, float [n_units][256], owned by the caller and
 * kept alive until the work on the call's stream has finished.  A call whose
 * unit count exceeds n_units returns PAID_ERR_ARG.  maps = NULL, n_units = 0
 * clears it.  Returns PAID_OK or PAID_ERR_ARG. */
int paid_set_trace_buffer(paid_ctx* ctx, float* maps, int64_t n_units);

/* Rule-error maps of the uniform level-4 grid: evaluate each integral's 256
 * level-4 cells once (FP64, with the context's rule, or N = 6 when the
 * context's N is higher) and write log10(err_c / S), err_c = |Q_N - Q_2N| of
 * cell c as one region, S = sum_c |Q_2N of cell c| (clamped to [-16, 0]), to
 * out (device, float [nq*npairs][256], the batch order of
 * paid_integrate_batch).  Workspace as for paid_integrate_batch with 4^4
 * initial regions per integral.  Returns PAID_OK / ERR_ARG / ERR_OOM / ERR_CUDA. */
int paid_cell_errors(paid_ctx* ctx, int kind, int nq, const double* q, int npairs,
                     const int32_t* lm, double T, float* out, void* workspace, size_t ws_bytes,
                     void* stream);

/* paid_integrate_multi with the initial partition taken from maps:
 *   proposal  device, float [n_units][256] in the global unit order of the
 *             batches (batch 0's units first; units as for options.trace),
 *             or NULL for a uniform level-4 start;
 *   margin    finite: cell c starts at level floor(proposal[c] - margin),
 *             clamped to 2..7 (4^(level-4) regions in the cell from level 4
 *             on; a level-3 block whose four cells all ask for <= 3, and a
 *             level-2 block whose 16 cells all ask for 2, stay one region).
 *             With margin >= the map's error every seed region is an ancestor
 *             of (or equal to) a region of the unseeded run's final partition.
 * A seed above max_regions / 2 regions for a unit falls back to the uniform
 * level-2 start.  Everything else as paid_integrate_multi. */
int paid_integrate_multi_seeded(paid_ctx* ctx, const paid_batch* batches, int nb,
                                const float* proposal, double margin, void* workspace,
                                size_t ws_bytes, void* stream);

/* The network: 32 -> 256 -> 256 -> 256 -> 256 -> 256, GELU after the four
 * hidden layers; BF16 weights and activations, FP32 accumulation (tensor
 * cores), FP32 master parameters in one buffer: for layer l = 0..4,
 * W_l [K_l][256] row-major (K_0 = 32, else 256), then b_l [256]. */
#define PAID_MLP_IN 32
#define PAID_MLP_HIDDEN 256
#define PAID_MLP_OUT 256
#define PAID_MLP_LAYERS 5

/* Number of FP32 parameters (271,616). */
int paid_mlp_param_count(int64_t* n);
/* Workspace bytes for forward / gradient passes over M rows.  The workspace
 * of paid_mlp_forward, paid_mlp_grad and paid_proposal_train must start on a
 * 256-byte boundary (every torch / cudaMalloc allocation does); otherwise
 * PAID_ERR_ARG. */
int paid_mlp_workspace_size(int64_t M, size_t* bytes);
/* Seeded initialisation on the device (uniform +-1/sqrt(K) weights, zero biases). */
int paid_mlp_init(float* params, uint64_t seed, void* stream);
/* Inputs for one batch: x (device, BF16 bits [nq*npairs][32]) =
 * (sin qx, cos qx, sin qy, cos qy, one-hot l [9], one-hot m [9], log10 T, mu, t',
 *  one-hot kind [ph, pp], 0 padding), mu and t' from the context. */
int paid_mlp_features(paid_ctx* ctx, int kind, int nq, const double* q, int npairs,
                      const int32_t* lm, double T, uint16_t* x, void* stream);
/* The same with one row per (kind, q) group (x: [nq][32], the form-factor
 * one-hots zero): the inputs of a group-mode proposal. */
int paid_mlp_group_features(paid_ctx* ctx, int kind, int nq, const double* q, double T,
                            uint16_t* x, void* stream);
/* Forward pass: x (BF16 [M][32], any alignment) -> out (FP32 [M][256],
 * 16-byte aligned, else PAID_ERR_ARG); one launch on the tensor cores for all
 * five layers, 128 rows per CTA. */
int paid_mlp_forward(const float* params, const uint16_t* x, int64_t M, float* out,
                     void* workspace, size_t ws_bytes, void* stream);
/* Mean-squared-error gradient over M rows against target (FP32 [M][256]):
 * grad (FP32, param_count) and loss (FP32 scalar, mean over M x 256) on the device. */
int paid_mlp_grad(const float* params, const uint16_t* x, const float* target, int64_t M,
                  float* grad, float* loss, void* workspace, size_t ws_bytes, void* stream);
/* One AdamW step (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay on the
 * weights only) with moments m, v (FP32, param_count); step counts from 1. */
int paid_mlp_adamw(float* params, const float* grad, float* m, float* v, int step, float lr,
                   float weight_decay, void* stream);

/* Training of the network on the device: `epochs` passes over the M rows
 * (x: BF16 [M][32], target: FP32 [M][256], both device, finite) in minibatches
 * of `batch` rows, each pass in a fresh order drawn from `seed` (splitmix64,
 * Fisher-Yates); per minibatch the mean-squared-error gradient and one AdamW
 * step (paid_mlp_grad, paid_mlp_adamw) with the learning rate decayed from lr
 * to 0 on a cosine over the call's steps.  params, m, v (device, FP32,
 * param_count): master weights and AdamW moments, updated in place.  *step
 * (host): AdamW steps taken so far (0 for a fresh start), advanced.
 * epoch_loss: host float [epochs] (mean minibatch loss per pass), or NULL.
 * workspace: device, >= paid_proposal_train_workspace_size(M, batch) bytes.
 * Synchronises `stream` once per epoch when epoch_loss is given.
 * Returns PAID_OK, PAID_ERR_ARG, PAID_ERR_OOM or PAID_ERR_CUDA. */
int paid_proposal_train_workspace_size(int64_t M, int64_t batch, size_t* bytes);
int paid_proposal_train(float* params, float* m, float* v, const uint16_t* x, const float* target,
                        int64_t M, int epochs, int64_t batch, float lr, float weight_decay,
                        uint64_t seed, int* step, float* epoch_loss, void* workspace,
                        size_t ws_bytes, void* stream);
/* Save the network's FP32 parameters (device, param_count) to a file: the 8
 * bytes "PAIDMLP1", the count as int64, then the values (little-endian IEEE
 * binary32).  Load checks the tag and the count and uploads; a file of another
 * layout returns PAID_ERR_ARG and leaves params unchanged.  Both synchronise
 * `stream`.  Returns PAID_OK, PAID_ERR_ARG (bad path or file) or
 * PAID_ERR_CUDA. */
int paid_proposal_save(const float* params, const char* path, void* stream);
int paid_proposal_load(float* params, const char* path, void* stream);

/* Waits for the last integrate call on ctx (a no-op for a synchronous one)
 * and writes its outcome to *call_rc (may be NULL): PAID_OK, PAID_ERR_POOL
 * (the pool could make no progress; unfinished integrals have status
 * PAID_POOL), PAID_ERR_TIMEOUT (round cap) or PAID_ERR_CUDA.  Returns PAID_OK,
 * or PAID_ERR_CUDA / PAID_ERR_ARG when waiting itself fails. */
int paid_wait(paid_ctx* ctx, int* call_rc);

/* Statistics of the last integrate call (waits for it when it is still
 * pending).  Returns PAID_OK or PAID_ERR_ARG. */
int paid_last_stats(paid_ctx* ctx, paid_stats* out);

/* Static message for a paid_rc. */
const char* paid_error_string(int rc);

/* Message of the last failed call on ctx ("" if none).  Valid until the next call. */
const char* paid_last_error(paid_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PAID_H */
