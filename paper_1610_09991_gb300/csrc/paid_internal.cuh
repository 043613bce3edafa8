// Internal declarations shared by the CUDA translation units of libpaid.
// Device data layout (all structure-of-arrays in the caller's workspace):
//
//   per integral g (global index over all batches of a call)
//     trig[g]   QTrig (cos qx, sin qx, cos qy, sin qy)
//     meta[g]   uint32  kind | l << 3 | m << 8 | valid << 13 | batch << 16
//     seg_base[g], seg_count[g]   uint32: the integral's contiguous pool segment
//   per active slot s (the active list is compacted every round)
//     active[s] uint32 integral index; cnt_new/cnt_eval/thr written by the
//     reduce-test kernel and scanned before the split kernel
//   region pool (ping-pong, capacity C)
//     key[C] uint64  level << 58 | ix << 29 | iy   (dyadic square of Sec. 3's
//                    adaptive scheme, side 2pi / 2^level)
//     val[C] double  Q_2N   err[C] double |Q_N - Q_2N|
//     nse[C] float   bound on the FP32 rounding noise of the region's sums
//                    (0 for regions evaluated in FP64)
//   eval list  uint2[C] (pool position, integral) of regions awaiting evaluation
//   loop state LoopState: the round's counts and the buffer in use, read by
//              every round kernel and advanced by k_control, so that a round
//              needs no host-side arguments (the same launches run from the
//              host loop or inside a CUDA graph's conditional WHILE node)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace paid {

constexpr int kMaxLevel = 29;          // deepest dyadic level (29-bit ix, iy)
constexpr int kMaxRuleN = 12;          // largest supported N of the CC pair
constexpr int kMaxRuleNLow = 6;        // largest N of the per-integral kernels
constexpr int kRuleVariants = 5;       // N = 4, 6 (every kernel), 8, 10, 12 (group kernel)
__host__ __device__ constexpr int rule_variant(int N) { return (N - 4) / 2; }
constexpr int kHistBins = 64;          // error histogram: 4 bins per octave
constexpr int kScanBlock = 1024;       // items per block of the slot scan
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxMonomialDegree = 30;
// FP32 evaluation: per-node rounding error in units of 2^-24 |F| (|f_l|+1)(|f_m|+1)
// (plus |x1| + |x2| for the rounding of the energies), and the multiple of the
// rms noise treated as irreducible by refinement; see paid_eval.cu.
constexpr float kNoiseUlps = 4.0f;
// An FP32 integral moves to float-float evaluation when kNoiseSigmas * sum(nse)
// exceeds kNoiseTol * tol.  Measured against float-float values the FP32 error
// of Q_N - Q_2N is 0.11 nse at the median and 0.59 nse at the 99th percentile,
// so at the threshold the noise left inside the error sum is ~0.2 tol.
constexpr double kNoiseSigmas = 1.0;
constexpr double kNoiseTol = 2.0;
// threshold-bin marker in thr[].x: re-evaluate every region in FP64
constexpr uint32_t kEscalate = 0xfeu;
// Shared-partition (group) mode: most pairs per group, and the pair-vector
// stride of a region in the pool
constexpr int kGroupPairs = 81;
// chunks per group segment in the group reduce (blocks per group)
constexpr int kGroupSplit = 4;

enum Kind : int { PH = 0, PP = 1, MONOMIAL = 2, OVERLAP = 3, FLOW_PH = 4, FLOW_PP = 5 };
__host__ __device__ inline bool is_flow(int kind) { return kind == FLOW_PH || kind == FLOW_PP; }
enum Status : int { CONVERGED = 0, BUDGET = 1, NONFINITE = 2, ROUNDCAP = 3, POOL = 4, RUNNING = -1 };
// force_status of the test kernels: finalize with POOL only if the device
// loop stopped on a pool that could make no progress
constexpr int kFinalizeIfStuck = -2;

__host__ __device__ inline uint64_t make_key(uint32_t L, uint32_t ix, uint32_t iy)
{
    return (uint64_t(L) << 58) | (uint64_t(ix) << 29) | uint64_t(iy);
}
__host__ __device__ inline uint32_t key_level(uint64_t k) { return uint32_t(k >> 58); }
__host__ __device__ inline uint32_t key_ix(uint64_t k) { return uint32_t((k >> 29) & 0x1fffffffu); }
__host__ __device__ inline uint32_t key_iy(uint64_t k) { return uint32_t(k & 0x1fffffffu); }

__host__ __device__ inline uint32_t make_meta(int kind, int l, int m, int valid, int batch)
{
    return uint32_t(kind & 7) | (uint32_t(l & 31) << 3) | (uint32_t(m & 31) << 8) |
           (uint32_t(valid & 1) << 13) | (uint32_t(batch) << 16);
}
// bit 14: the integral is evaluated in FP64 (set at setup for the FP64 path,
// or when its FP32 rounding noise bound exceeds half its tolerance)
constexpr uint32_t kMetaFp64 = 1u << 14;
// bit 15: the integral is evaluated in float-float (set when its FP32 rounding
// noise exceeds a quarter of its tolerance)
constexpr uint32_t kMetaDf32 = 1u << 15;
__host__ __device__ inline int meta_kind(uint32_t mt) { return int(mt & 7u); }
__host__ __device__ inline int meta_l(uint32_t mt) { return int((mt >> 3) & 31u); }
__host__ __device__ inline int meta_m(uint32_t mt) { return int((mt >> 8) & 31u); }
__host__ __device__ inline int meta_valid(uint32_t mt) { return int((mt >> 13) & 1u); }
__host__ __device__ inline int meta_batch(uint32_t mt) { return int(mt >> 16); }

// One batch as the kernels see it.
struct DevBatch {
    int kind, nq, npairs, pad;
    double T, inv2T, inv4T;
    double rel_tol, abs_tol;
    int64_t max_regions;
    int64_t first;             // global index of the batch's first unit (integral, or
                               // in group mode its first (kind, q) group)
    int64_t ifirst;            // global index of the batch's first integral
    const double* q;
    const int32_t* lm;
    double* values;
    double* errors;
    int64_t* regions;
    int32_t* status;
    // flow kinds in group mode: couplings and outputs of the truncated-unity
    // products (pp: V^P -> dP; ph: V^C, V^D -> dC, dD), or null
    const double* tu_v0;
    const double* tu_v1;
    double* tu_out0;
    double* tu_out1;
};

// cos/sin of the transfer momentum of one integral
struct __align__(32) QTrig {
    double cqx, sqx, cqy, sqy;
};

struct Lattice {
    double t, tp, mu;
};

// Totals of one round, written by the slot scan and read by the host.
struct RoundTotals {
    unsigned long long pool;    // regions in the next pool
    unsigned long long eval;    // regions to evaluate next round
    unsigned long long active;  // integrals still refining
    unsigned long long escalated;  // integrals moved from FP32 to float-float evaluation (cumulative)
    unsigned long long df_regions; // regions evaluated in float-float (cumulative)
    unsigned long long roundcap;   // integrals ended by the round cap (cumulative)
    unsigned long long pad[2];
};

// Why the device loop stopped.
enum LoopStop : int { kRunning = 0, kDone = 1, kStuck = 2, kNoRoom = 3, kHardCap = 4 };

// The state of the refinement loop, in device memory.
struct LoopState {
    long long n_active;        // active slots of the coming round
    long long n_eval;          // regions on its eval list
    long long pool;            // regions in its pool
    long long admitted;        // integrals [0, admitted) have entered the pool
    long long n_total;
    long long cap;             // pool capacity (regions per buffer)
    long long wave_g0, wave_g1;    // integrals admitted by the last control step
    unsigned long long wave_pool, wave_eval, wave_act;   // their bases
    long long region_evals;    // statistics
    long long peak_pool;
    long long throttled_rounds;
    int cur;                   // pool buffer of the coming round
    int round;                 // index of the coming round
    int rounds_done;
    int L0;                    // admission start level (< 0: no admission)
    int hard_rounds;           // loop bound: stop after this many rounds
    int stop;                  // LoopStop
    int throttled;             // the current round was throttled
    int pad;
};

// Pointers into the workspace.
struct Work {
    DevBatch* batches;
    int nb;
    int64_t n;                 // integrals
    int64_t cap;               // pool capacity (regions)
    QTrig* trig;
    uint32_t* meta;
    uint32_t* born;            // per integral: the round it entered the pool
    uint32_t* seg_base;
    uint32_t* seg_count;
    uint32_t* active[2];
    uint32_t* cnt_new;         // per slot: regions in the next pool
    uint32_t* cnt_eval;        // per slot: children to evaluate
    uint2* thr;                // per slot: (threshold bin, rank cap in that bin)
    unsigned long long* pre_pool;   // per slot: exclusive prefix within its scan block
    unsigned long long* pre_eval;
    uint32_t* pre_act;
    unsigned long long* blk_pool;   // per scan block: totals, then exclusive offsets
    unsigned long long* blk_eval;
    uint32_t* blk_act;
    RoundTotals* totals;
    LoopState* ls;
    uint64_t* key[2];
    double* val[2];
    double* err[2];
    float* nse[2];
    uint2* evl;
    // group mode (vstride > 0): a unit is one (kind, q) group of a batch and
    // every region carries the Q_2N and |Q_N - Q_2N| of each of the batch's
    // pairs at vval/verr[pos * vstride + pair]; err[pos] holds the region's
    // score for the selection (largest error over the pairs not yet
    // converged, in units of each pair's tolerance)
    double* vval[2];
    float* verr[2];
    uint32_t* vsrc;            // per next-pool slot: the region it copies (~0u: a new child)
    float* tmap;               // with options.trace: per unit the level of the coarsest
                               // region meeting each level-4 cell (256 entries), the
                               // caller's buffer; null otherwise
    // per active slot, temporaries of the group reduce: chunk sums of V and E
    // ([slot][chunk][2][81]), V and E ([slot][2][81]), 1/tol of the pairs not
    // yet converged ([slot][81]), chunk score sum and max ([slot][chunk][2]),
    // status after the test
    double* gpart;
    double* gsum;
    double* gtol;
    double* gsc;
    int* gstate;
    int vstride;
    int nff;
    int kinds;                 // the call's kinds: 1 no flow kind, 2 flow kinds only, 0 mixed
    int gglobal;               // group mode 2: one error sum and one tolerance per group
};

// ---- host-side launch wrappers (defined in the .cu files) -----------------
// Round kernels take their counts and the buffer in use from w.ls; the `hint`
// arguments only size the grids (the exact count, or an upper bound when the
// launch is captured into a graph that runs it for every round).
// paid_eval.cu
cudaError_t init_rule_tables(int device);
// fp32 = 1: the FP32 / FP64 kernel, then the float-float kernel; `mid`, when
// given, is recorded between the two
cudaError_t launch_eval(const Work& w, int64_t hint_eval, int rule_n, int fp32, Lattice lat,
                        cudaStream_t s, cudaEvent_t mid = nullptr);
// group mode: every pair of every region on the eval list; fp32 = 0: FP64,
// 1: the kernel F and the row sums in float-float on the FP32 pipe, moments
// and pair values FP64.  With rule_q2 / rule_d non-null, entry t's Q_2N and
// Q_N - Q_2N (times the region's Jacobian) go to rule_q2 / rule_d[t * npairs +
// pair] instead of the pool.  max_blocks > 0 caps the grid (the kernel is
// grid-stride), else 152 x 32
cudaError_t launch_eval_group(const Work& w, int64_t hint_eval, int rule_n, int fp32, Lattice lat,
                              cudaStream_t s, double* rule_q2 = nullptr, double* rule_d = nullptr,
                              int max_blocks = 0);
// which = 0: the group kernel's exp(-x); 1: its division x / y (diagnostics)
cudaError_t launch_check_math(int which, int64_t n, const double* x, const double* y, double* out,
                              cudaStream_t s);
// paid_tu.cu: flow right-hand sides from the bubbles and couplings, per l
cudaError_t launch_tu_rhs(int nq, int n, const double* VP, const double* VC, const double* VD,
                          const double* Xpp, const double* Xph, double* dP, double* dC,
                          double* dD, cudaStream_t s);
// paid_pool.cu
// Initial loop state: counts of the first round, buffer 0, round 0.
cudaError_t launch_state_init(const Work& w, int64_t n_active, int64_t n_eval, int64_t pool,
                              int64_t admitted, int L0, int hard_rounds, cudaStream_t s);
// Integrals [g0, g1) (g1 < 0: all): descriptors and, for L0 >= 0, their uniform
// level-L0 regions appended at the given bases of pool[buf] / eval list /
// active[buf].  L0 < 0: descriptors only (the partition comes from launch_seed).
cudaError_t launch_setup(const Work& w, int L0, int nff, int fp64, cudaStream_t s, int64_t g0 = 0,
                         int64_t g1 = -1, int buf = 0, unsigned long long pool_base = 0,
                         unsigned long long eval_base = 0, unsigned long long act_base = 0,
                         int round = 0);
// paid_rule_regions: unit 0 = the (kind, q) group, the caller's regions
// (level, ix, iy) on the eval list; invalid regions are flagged in bad[] and
// their outputs set to NaN by launch_rule_flag after the evaluation
cudaError_t launch_rule_setup(const Work& w, int kind, const double* q, const int32_t* regions,
                              int nreg, uint32_t* bad, cudaStream_t s);
cudaError_t launch_rule_flag(const uint32_t* bad, int nreg, int npairs, double* q2, double* dq,
                             cudaStream_t s);
// the admission wave chosen by the last control step (w.ls->wave_*)
cudaError_t launch_setup_wave(const Work& w, int64_t hint_wave, int nff, int fp64, cudaStream_t s);
// pass 0: region counts into cnt_new / cnt_eval (slot = unit); pass 1 (after
// launch_scan): keys, eval list, segments.  proposal: per unit a 16 x 16 map
// of predicted levels of the coarsest final region per level-4 cell, seeded
// at floor(level - margin); null = uniform level 4.
cudaError_t launch_seed(const Work& w, const float* proposal, double margin, int pass,
                        cudaStream_t s);
// with w.tmap: every active unit's current partition as a level map (after
// the round's test, before the split)
cudaError_t launch_trace(const Work& w, int64_t hint_active, cudaStream_t s);
cudaError_t launch_features(int kind, int nq, const double* q, int npairs, const int32_t* lm,
                            double T, double mu, double tp, void* x, cudaStream_t s);
cudaError_t launch_cell_map(const Work& w, float* out, cudaStream_t s);
cudaError_t launch_reduce_test(const Work& w, int64_t hint_active, int max_rounds, double cover,
                               cudaStream_t s);
// group mode: reduce + test + selection, one block per active group
cudaError_t launch_reduce_group(const Work& w, int64_t hint_active, int max_rounds, double cover,
                                cudaStream_t s);
// rescan = 1: only when the last scan's pool total exceeds the capacity (after
// launch_throttle), and then it marks the round as throttled
cudaError_t launch_scan(const Work& w, int64_t hint_active, int rescan, cudaStream_t s);
cudaError_t launch_split(const Work& w, int64_t hint_active, cudaStream_t s);
// group mode, after launch_split: the pair vectors of the regions the split
// kept, into the next pool (hint_pool: bound on the next pool's regions)
cudaError_t launch_copy_vectors(const Work& w, int64_t hint_pool, cudaStream_t s);
// finish every slot still refining with `status` (after a stop)
cudaError_t launch_finalize(const Work& w, int64_t hint_active, int status, cudaStream_t s);
// after the device loop, decided on the device from its stop reason: a pool
// that could make no progress finishes the slots still refining with PAID_POOL;
// integrals never admitted get PAID_POOL or PAID_ROUNDCAP
cudaError_t launch_finish_device(const Work& w, cudaStream_t s);
cudaError_t launch_mark_unadmitted(const Work& w, int64_t g0, int64_t g1, int status, cudaStream_t s);
// after launch_scan, when its pool total exceeds the capacity: integrals past
// cap - pool regions of cumulative growth keep their regions unsplit this round
cudaError_t launch_throttle(const Work& w, int64_t hint_active, cudaStream_t s);
// one thread: statistics, next round's counts, buffer flip, admission wave and
// the stop decision; inside a graph (in_graph = 1) a stop sets the WHILE
// node's condition to 0
cudaError_t launch_control(const Work& w, cudaGraphConditionalHandle h, int in_graph, cudaStream_t s);

}  // namespace paid
