// Region pool management: initial partition, per-unit reduction and
// convergence test, batched selection, 2x2 split and stable compaction, and
// the device-side loop control.  A unit is one integral, or in group mode one
// (kind, q) group whose regions carry every pair's values.
//
// Paper correspondence (Sec. 4, Listings 1-5):
//   k_setup        Listing 1: every integral starts from the uniform level-L0
//                  grid of D; its regions go on the eval list.
//   k_reduce_test  Listing 4 + the master's termination check: per integral,
//                  V = sum Q_2N, E = sum err over its current regions, and
//                  the test E <= max(abs_tol, rel_tol |V|).  Finished
//                  integrals write value/error/regions/status (Listing 5).
//                  For the others it picks the regions to split: a batched
//                  extract-max (Listing 2) that takes the largest-error
//                  regions until their error covers E - cover * tol, using a
//                  64-bin histogram of err on a quarter-octave scale below
//                  the segment's maximum, limited by the region budget.
//   k_scan_*       exclusive prefix sums over the active slots (pool, eval,
//                  active counts) that place every integral's next segment.
//   k_split        Listing 3 (divide into 4) + Listing 4 (insert): marked
//                  regions emit 4 children (level + 1), others are copied;
//                  positions come from a warp ballot / shuffle prefix so the
//                  pool stays sorted by integral and stable within it.
//   k_group_*      group mode: per-pair sums in chunks, the per-pair test, the
//                  region scores (largest error over the unconverged pairs in
//                  units of their tolerances) and the selection on them;
//                  k_copy_vectors moves the kept regions' pair vectors.
//   k_throttle     pool pressure: integrals split in slot order while the
//                  growth fits in the pool, the rest wait a round.
//   k_control      the master's loop control (Listing 5) on the device: next
//                  round's counts, admission of waiting integrals, stop.
// One warp owns one integral in reduce/split; sums use a fixed lane order and
// a xor-butterfly (group mode: fixed chunk and warp order), and the histogram
// sums are integers, so a run is bitwise reproducible.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "paid_internal.cuh"

namespace paid {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}
__device__ __forceinline__ double warp_max(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(kFull, x, o));
    return x;
}
// exclusive warp prefix of a 32-bit count
__device__ __forceinline__ uint32_t warp_excl(uint32_t x, uint32_t& total)
{
    const int lane = threadIdx.x & 31;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    total = __shfl_sync(kFull, inc, 31);
    return inc - x;
}
// quarter-octave log key of a positive double (monotone in the value)
__device__ __forceinline__ int log_key(double x)
{
    return int(uint64_t(__double_as_longlong(x)) >> 50);
}

// ---------------------------------------------------------------------------
// Integral g of the range starting at g0: descriptors, and (write_regions) its
// uniform level-L0 regions at pool[buf][pool_base + (g - g0) n0 ...], on the
// eval list from eval_base and on the active list active[buf] from act_base.
__device__ void setup_one(const Work& w, int64_t g, int64_t g0, int L0, int nff, int fp64, int buf,
                          unsigned long long pool_base, unsigned long long eval_base,
                          unsigned long long act_base, int write_regions, int round)
{
    const int64_t i = g - g0;
    int b = 0;   // batches are sorted by `first`
    {
        int lo = 0, hi = w.nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (w.batches[mid].first <= g) lo = mid; else hi = mid - 1;
        }
        b = lo;
    }
    const DevBatch& B = w.batches[b];
    const int64_t local = g - B.first;
    const bool grp = w.vstride > 0;   // unit = (kind, q) group: every pair of the batch
    const int64_t iq = grp ? local : local / B.npairs, ip = grp ? 0 : local % B.npairs;
    const double qx = B.q[2 * iq], qy = B.q[2 * iq + 1];
    const int l = grp ? 0 : B.lm[2 * ip], m = grp ? 0 : B.lm[2 * ip + 1];
    int valid;
    if (grp)
        valid = 1;   // pairs are checked one by one in the group reduce
    else if (B.kind == MONOMIAL)
        valid = l >= 0 && m >= 0 && l <= kMaxMonomialDegree && m <= kMaxMonomialDegree;
    else
        valid = l >= 0 && m >= 0 && l < nff && m < nff;
    double sx, cx, sy, cy;
    // the flow kinds route the energies symmetrically, k +- q/2: their
    // rotation is by half the transfer momentum
    const double hq = is_flow(B.kind) ? 0.5 : 1.0;
    sincos(hq * qx, &sx, &cx);
    sincos(hq * qy, &sy, &cy);
    w.trig[g] = QTrig{cx, sx, cy, sy};
    w.meta[g] = make_meta(B.kind, valid ? l : 0, valid ? m : 0, valid, b) | (fp64 ? kMetaFp64 : 0u);
    w.born[g] = uint32_t(round);
    if (write_regions) {
        const uint32_t side = 1u << L0, n0 = side * side;
        const unsigned long long base = pool_base + (unsigned long long)(i) * n0;
        const unsigned long long ebase = eval_base + (unsigned long long)(i) * n0;
        w.seg_base[g] = uint32_t(base);
        w.seg_count[g] = n0;
        for (uint32_t r = 0; r < n0; ++r) {
            w.key[buf][base + r] = make_key(uint32_t(L0), r / side, r % side);
            w.evl[ebase + r] = make_uint2(uint32_t(base + r), uint32_t(g));
        }
    }
    w.active[buf][act_base + i] = uint32_t(g);
    if (grp)
        for (int p = 0; p < B.npairs; ++p) B.status[local * B.npairs + p] = RUNNING;
    else
        B.status[local] = RUNNING;
}

__global__ void k_setup(Work w, int64_t g0, int64_t g1, int L0, int nff, int fp64, int buf,
                        unsigned long long pool_base, unsigned long long eval_base,
                        unsigned long long act_base, int write_regions, int round)
{
    const int64_t g = g0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= g1) return;
    setup_one(w, g, g0, L0, nff, fp64, buf, pool_base, eval_base, act_base, write_regions, round);
    if (g == 0) {
        w.totals->escalated = 0ull;
        w.totals->df_regions = 0ull;
        w.totals->roundcap = 0ull;
    }
}

cudaError_t launch_setup(const Work& w, int L0, int nff, int fp64, cudaStream_t s, int64_t g0,
                         int64_t g1, int buf, unsigned long long pool_base,
                         unsigned long long eval_base, unsigned long long act_base, int round)
{
    if (g1 < 0) g1 = w.n;
    if (g1 <= g0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (g1 - g0 + threads - 1) / threads;
    k_setup<<<int(blocks), threads, 0, s>>>(w, g0, g1, L0, nff, fp64, buf, pool_base, eval_base,
                                            act_base, L0 >= 0 ? 1 : 0, round);
    return cudaGetLastError();
}

// The admission wave of the last control step, into the buffer of the coming
// round (grid-stride, so that a fixed grid serves every round of a graph).
__global__ void k_setup_wave(Work w, int nff, int fp64)
{
    const LoopState& L = *w.ls;
    const int64_t g0 = L.wave_g0, g1 = L.wave_g1;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t g = g0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < g1; g += stride)
        setup_one(w, g, g0, L.L0, nff, fp64, L.cur, L.wave_pool, L.wave_eval, L.wave_act, 1,
                  L.round);
}

cudaError_t launch_setup_wave(const Work& w, int64_t hint_wave, int nff, int fp64, cudaStream_t s)
{
    if (hint_wave <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((hint_wave + 255) / 256, 152 * 8);
    k_setup_wave<<<int(blocks), 256, 0, s>>>(w, nff, fp64);
    return cudaGetLastError();
}

// One thread: the loop state of the first round.
__global__ void k_state_init(Work w, int64_t n_active, int64_t n_eval, int64_t pool,
                             int64_t admitted, int L0, int hard_rounds)
{
    LoopState& L = *w.ls;
    L.n_active = n_active;
    L.n_eval = n_eval;
    L.pool = pool;
    L.admitted = admitted;
    L.n_total = w.n;
    L.cap = w.cap;
    L.wave_g0 = L.wave_g1 = 0;
    L.wave_pool = L.wave_eval = L.wave_act = 0ull;
    L.region_evals = 0;
    L.peak_pool = 0;
    L.throttled_rounds = 0;
    L.cur = 0;
    L.round = 0;
    L.rounds_done = 0;
    L.L0 = L0;
    L.hard_rounds = hard_rounds;
    L.stop = kRunning;
    L.throttled = 0;
    L.pad = 0;
}

cudaError_t launch_state_init(const Work& w, int64_t n_active, int64_t n_eval, int64_t pool,
                              int64_t admitted, int L0, int hard_rounds, cudaStream_t s)
{
    k_state_init<<<1, 1, 0, s>>>(w, n_active, n_eval, pool, admitted, L0, hard_rounds);
    return cudaGetLastError();
}

// One thread, after the split: the next round's counts and buffer, the
// statistics, streaming admission (more integrals while the pool is under
// half full) and the stop decision.
__global__ void k_control(Work w, cudaGraphConditionalHandle h, int in_graph)
{
    LoopState& L = *w.ls;
    const RoundTotals t = *w.totals;
    L.region_evals += L.n_eval;
    L.peak_pool = max(L.peak_pool, L.pool);
    L.throttled_rounds += L.throttled;
    L.rounds_done = L.round + 1;
    // throttled to no growth, nothing retired, nothing to evaluate: no progress
    const bool stuck = L.throttled && (long long)t.active == L.n_active && t.eval == 0ull;
    L.throttled = 0;
    // the split wrote the next pool, eval list and active list into cur ^ 1
    L.n_active = (long long)t.active;
    L.n_eval = (long long)t.eval;
    L.pool = (long long)t.pool;
    L.cur ^= 1;
    L.round += 1;
    L.wave_g0 = L.wave_g1 = 0;
    int stop = kRunning;
    if (t.active == 0ull && L.admitted == L.n_total) {
        stop = kDone;
    } else if (stuck) {
        stop = kStuck;
    } else if (t.active == 0ull && L.round > L.hard_rounds) {
        stop = kHardCap;   // the reduce-test ended every active integral at the bound
    } else if (L.admitted < L.n_total && L.L0 >= 0) {
        const long long n0 = 1ll << (2 * L.L0);
        const long long est = max(16 * n0, 4 * (L.pool / max(1ll, L.n_active)));
        long long c = L.cap / 2 > L.pool ? (L.cap / 2 - L.pool) / est : 0;
        if (L.n_active == 0) c = max(c, 1ll);
        c = min(c, L.n_total - L.admitted);
        c = min(c, (L.cap - L.pool) / n0);
        if (c > 0) {
            L.wave_g0 = L.admitted;
            L.wave_g1 = L.admitted + c;
            L.wave_pool = (unsigned long long)L.pool;
            L.wave_eval = (unsigned long long)L.n_eval;
            L.wave_act = (unsigned long long)L.n_active;
            L.admitted += c;
            L.n_active += c;
            L.n_eval += c * n0;
            L.pool += c * n0;
        } else if (L.n_active == 0) {
            stop = kNoRoom;
        }
    }
    L.stop = stop;
    if (in_graph && stop != kRunning) cudaGraphSetConditional(h, 0u);
}

cudaError_t launch_control(const Work& w, cudaGraphConditionalHandle h, int in_graph, cudaStream_t s)
{
    k_control<<<1, 1, 0, s>>>(w, h, in_graph);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// paid_rule_regions: one group (unit 0) and the caller's regions on the eval
// list.  A region with level > kMaxLevel or an index outside 2^level is
// evaluated as the level-0 square and flagged in bad[r].
__global__ void k_rule_setup(Work w, int kind, const double* q, const int32_t* regions, int nreg,
                             uint32_t* bad)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) {
        double sx, cx, sy, cy;
        const double hq = is_flow(kind) ? 0.5 : 1.0;   // flow kinds: k +- q/2
        sincos(hq * q[0], &sx, &cx);
        sincos(hq * q[1], &sy, &cy);
        w.trig[0] = QTrig{cx, sx, cy, sy};
        w.meta[0] = make_meta(kind, 0, 0, 1, 0) | kMetaFp64;
    }
    if (r >= nreg) return;
    const int L = regions[3 * r], ix = regions[3 * r + 1], iy = regions[3 * r + 2];
    const bool ok = L >= 0 && L <= kMaxLevel && ix >= 0 && iy >= 0 &&
                    int64_t(ix) < (int64_t(1) << L) && int64_t(iy) < (int64_t(1) << L);
    w.key[0][r] = ok ? make_key(uint32_t(L), uint32_t(ix), uint32_t(iy)) : make_key(0, 0, 0);
    w.evl[r] = make_uint2(uint32_t(r), 0u);
    bad[r] = ok ? 0u : 1u;
}

__global__ void k_rule_flag(const uint32_t* bad, int nreg, int npairs, double* q2, double* dq)
{
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= int64_t(nreg) * npairs) return;
    if (bad[t / npairs]) { q2[t] = NAN; dq[t] = NAN; }
}

cudaError_t launch_rule_setup(const Work& w, int kind, const double* q, const int32_t* regions,
                              int nreg, uint32_t* bad, cudaStream_t s)
{
    k_rule_setup<<<(nreg + 255) / 256, 256, 0, s>>>(w, kind, q, regions, nreg, bad);
    return cudaGetLastError();
}

cudaError_t launch_rule_flag(const uint32_t* bad, int nreg, int npairs, double* q2, double* dq,
                             cudaStream_t s)
{
    const int64_t n = int64_t(nreg) * npairs;
    if (n <= 0) return cudaSuccess;
    k_rule_flag<<<int((n + 255) / 256), 256, 0, s>>>(bad, nreg, npairs, q2, dq);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Proposal-seeded initial partition.  For unit g (an integral, or in group
// mode a (kind, q) group) the map gives d_c, the predicted level of the
// coarsest final region meeting level-4 cell c (c = 16 ix + iy) -- the map a
// traced run records.  Cell c is seeded at level floor(d_c - margin), that is
// k_c = floor(d_c - margin) - 4 levels below level 4, k_c in [-2, 3]; a
// level-3 block whose four cells all have k <= -1 stays one region, and a
// level-2 block whose 16 cells all have k <= -2 stays one region.  With a
// margin >= the map's error the seed regions are ancestors of (or equal to)
// final regions, so seeding skips the evaluations of coarser regions without
// ever evaluating a region the unseeded run would not.  A non-finite entry
// counts as level 2.  A seed of more than max_regions / 2 regions falls back
// to the uniform level-2 grid.
__device__ __forceinline__ int seed_k(const float* map, int c, float margin)
{
    if (!map) return 0;                          // uniform level-4 start
    const float d = map[c];
    if (!isfinite(d)) return -2;
    return int(fminf(fmaxf(floorf(d - margin) - 4.0f, -2.0f), 3.0f));
}

// regions emitted by level-2 block (bx, by) of integral g; with emit != null
// writes them (keys and eval entries) starting at pool position p
__device__ uint32_t seed_block(const float* map, int bx, int by, float margin,
                              uint64_t* key, uint2* evl, unsigned long long p,
                              unsigned long long e, uint32_t g, bool emit)
{
    int kmax2 = -2;
    for (int u = 0; u < 4; ++u)
        for (int v = 0; v < 4; ++v) kmax2 = max(kmax2, seed_k(map, (4 * bx + u) * 16 + 4 * by + v, margin));
    if (kmax2 <= -2) {
        if (emit) { key[p] = make_key(2, bx, by); evl[e] = make_uint2(uint32_t(p), g); }
        return 1;
    }
    uint32_t cnt = 0;
    for (int a = 0; a < 2; ++a)
        for (int d = 0; d < 2; ++d) {
            const int sx = 2 * bx + a, sy = 2 * by + d;
            int k[4], kmax3 = -2;
            for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v) {
                    k[2 * u + v] = seed_k(map, (2 * sx + u) * 16 + 2 * sy + v, margin);
                    kmax3 = max(kmax3, k[2 * u + v]);
                }
            if (kmax3 <= -1) {
                if (emit) { key[p + cnt] = make_key(3, sx, sy); evl[e + cnt] = make_uint2(uint32_t(p + cnt), g); }
                ++cnt;
                continue;
            }
            for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v) {
                    const int kk = max(k[2 * u + v], 0), side = 1 << kk;
                    const uint32_t ix = uint32_t(2 * sx + u) << kk, iy = uint32_t(2 * sy + v) << kk;
                    for (int x = 0; x < side; ++x)
                        for (int y = 0; y < side; ++y) {
                            if (emit) {
                                key[p + cnt] = make_key(uint32_t(4 + kk), ix + x, iy + y);
                                evl[e + cnt] = make_uint2(uint32_t(p + cnt), g);
                            }
                            ++cnt;
                        }
                }
        }
    return cnt;
}

// one warp per integral; lanes 0..15 own the 16 level-2 blocks
__global__ void __launch_bounds__(256) k_seed(Work w, const float* proposal, float margin, int pass)
{
    const int lane = threadIdx.x & 31;
    const int64_t g = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
    if (g >= w.n) return;
    const DevBatch& B = w.batches[meta_batch(w.meta[g])];
    const float* map = proposal ? proposal + g * 256 : nullptr;
    uint32_t mine = 0;
    if (lane < 16) mine = seed_block(map, lane >> 2, lane & 3, margin, nullptr, nullptr, 0, 0,
                                     uint32_t(g), false);
    uint32_t total = mine;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    const bool fallback = int64_t(total) > B.max_regions / 2;
    if (pass == 0) {
        if (lane == 0) {
            const uint32_t c = fallback ? 16u : total;
            w.cnt_new[g] = c;
            w.cnt_eval[g] = c;
        }
        return;
    }
    const int64_t blk = g / kScanBlock;
    const unsigned long long pbase = w.blk_pool[blk] + w.pre_pool[g];
    const unsigned long long ebase = w.blk_eval[blk] + w.pre_eval[g];
    if (fallback) {
        if (lane < 16) {
            w.key[0][pbase + lane] = make_key(2, lane >> 2, lane & 3);
            w.evl[ebase + lane] = make_uint2(uint32_t(pbase + lane), uint32_t(g));
        }
    } else {
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t off = incl - mine;
        if (lane < 16)
            seed_block(map, lane >> 2, lane & 3, margin, w.key[0], w.evl, pbase + off,
                       ebase + off, uint32_t(g), true);
    }
    if (lane == 0) {
        w.seg_base[g] = uint32_t(pbase);
        w.seg_count[g] = fallback ? 16u : total;
    }
}

// Trace of the current partition: for every active unit the level of the
// coarsest region meeting each level-4 cell (a region of level L < 4 covers
// 4^(4-L) cells), written over the unit's 256 map entries.  Run every round
// after the test, it leaves each unit's final partition in the map: the last
// round a unit is active is the round its outcome is decided.
__global__ void __launch_bounds__(256) k_trace(Work w)
{
    __shared__ int lv[256];
    const LoopState& Ls = *w.ls;
    const int64_t s = blockIdx.x;
    if (s >= Ls.n_active) return;
    const int cur = Ls.cur;
    const uint32_t g = w.active[cur][s];
    const uint32_t base = w.seg_base[g], cnt = w.seg_count[g];
    lv[threadIdx.x] = kMaxLevel + 1;
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
        const uint64_t key = w.key[cur][base + j];
        const int L = int(key_level(key));
        const uint32_t ix = key_ix(key), iy = key_iy(key);
        if (L >= 4) {
            atomicMin(&lv[(ix >> (L - 4)) * 16 + (iy >> (L - 4))], L);
        } else {
            const int side = 1 << (4 - L);
            for (int a = 0; a < side; ++a)
                for (int b = 0; b < side; ++b)
                    atomicMin(&lv[(ix * side + a) * 16 + iy * side + b], L);
        }
    }
    __syncthreads();
    w.tmap[size_t(g) * 256 + threadIdx.x] = float(lv[threadIdx.x]);
}

cudaError_t launch_trace(const Work& w, int64_t hint_active, cudaStream_t s)
{
    if (!w.tmap || hint_active <= 0) return cudaSuccess;
    k_trace<<<int(hint_active), 256, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_seed(const Work& w, const float* proposal, double margin, int pass,
                        cudaStream_t s)
{
    if (w.n <= 0) return cudaSuccess;
    k_seed<<<int((w.n + 7) / 8), 256, 0, s>>>(w, proposal, float(margin), pass);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Proposal inputs (BF16) for one batch, see paid_mlp_features.
__global__ void k_features(int kind, int nq, const double* q, int npairs, const int32_t* lm,
                           double T, double mu, double tp, __nv_bfloat16* x)
{
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= int64_t(nq) * npairs) return;
    const int64_t iq = g / npairs, ip = g % npairs;
    double sx, cx, sy, cy;
    sincos(q[2 * iq], &sx, &cx);
    sincos(q[2 * iq + 1], &sy, &cy);
    // lm null: one row per (kind, q) group, the form-factor one-hots left zero
    const int l = lm ? lm[2 * ip] : -1, m = lm ? lm[2 * ip + 1] : -1;
    float f[32];
    for (int i = 0; i < 32; ++i) f[i] = 0.0f;
    f[0] = float(sx); f[1] = float(cx); f[2] = float(sy); f[3] = float(cy);
    if (l >= 0 && l < 9) f[4 + l] = 1.0f;
    if (m >= 0 && m < 9) f[13 + m] = 1.0f;
    f[22] = float(log10(T));
    f[23] = float(mu);
    f[24] = float(tp);
    f[25] = kind == PH ? 1.0f : 0.0f;
    f[26] = kind == PP ? 1.0f : 0.0f;
    for (int i = 0; i < 32; ++i) x[g * 32 + i] = __float2bfloat16(f[i]);
}

cudaError_t launch_features(int kind, int nq, const double* q, int npairs, const int32_t* lm,
                            double T, double mu, double tp, void* x, cudaStream_t s)
{
    const int64_t n = int64_t(nq) * npairs;
    if (n <= 0) return cudaSuccess;
    k_features<<<int((n + 255) / 256), 256, 0, s>>>(kind, nq, q, npairs, lm, T, mu, tp,
                                                   static_cast<__nv_bfloat16*>(x));
    return cudaGetLastError();
}

// Relative log10 error map of the uniform level-4 grid (one warp per integral).
__global__ void k_cell_map(Work w, float* out)
{
    const int lane = threadIdx.x & 31;
    const int64_t g = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
    if (g >= w.n) return;
    const uint32_t base = w.seg_base[g];
    double sa = 0.0;
    for (int c = lane; c < 256; c += 32) sa += fabs(w.val[0][base + c]);
    sa = warp_sum(sa);
    for (int c = lane; c < 256; c += 32) {
        const double r = sa > 0.0 ? w.err[0][base + c] / sa : 0.0;
        const double t = r > 1e-16 ? log10(r) : -16.0;
        out[g * 256 + c] = float(t > 0.0 ? 0.0 : t);
    }
}

cudaError_t launch_cell_map(const Work& w, float* out, cudaStream_t s)
{
    if (w.n <= 0) return cudaSuccess;
    k_cell_map<<<int((w.n + 7) / 8), 256, 0, s>>>(w, out);
    return cudaGetLastError();
}

// Threshold of the batched extract-max: walking the error histogram from its
// largest bin, the regions whose summed error (in the histogram's integer
// units) first reaches `target` are marked: whole bins below the threshold
// bin, and the first `cap` regions (in pool order) of the threshold bin.
// `allowed` (the region budget) caps the count, whole bins first.
__device__ void select_regions(const Work& w, int64_t s, const unsigned long long* hsum,
                               const uint32_t* hcnt, double target_units, int64_t allowed,
                               int kmax, uint32_t cnt)
{
    const unsigned long long target =
        target_units >= 9.0e18 ? ~0ull : (unsigned long long)fmax(target_units, 0.0);
    unsigned long long cum = 0;
    int64_t marked = 0;
    int tb = kHistBins - 1;
    for (int b = 0; b < kHistBins; ++b) {
        cum += hsum[b];
        marked += hcnt[b];
        if (cum >= target) { tb = b; break; }
    }
    uint32_t cap;
    if (marked > allowed) {           // region budget binds: whole bins while they fit
        int64_t acc = 0;
        int b = 0;
        while (b < tb && acc + hcnt[b] <= allowed) { acc += hcnt[b]; ++b; }
        tb = b;
        cap = uint32_t(allowed - acc);
        marked = allowed;
    } else {
        cap = hcnt[tb];
    }
    w.thr[s] = make_uint2(uint32_t(tb) | (uint32_t(kmax) << 8), cap);
    w.cnt_new[s] = cnt + 3u * uint32_t(marked);
    w.cnt_eval[s] = 4u * uint32_t(marked);
}

// ---------------------------------------------------------------------------
// Per-integral reduction, convergence test and split selection.
// force_status >= 0: finalize every slot that is still refining with that status.
constexpr int kWarpsPerBlock = 8;

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_reduce_test(Work w, int max_rounds, double cover, int force_status)
{
    if (force_status == kFinalizeIfStuck) {   // after the device loop: decided on the device
        if (w.ls->stop != kStuck) return;
        force_status = POOL;
    }
    const int cur = w.ls->cur;
    const int64_t n_active = w.ls->n_active;
    const int round = w.ls->round;
    __shared__ unsigned long long hsum[kWarpsPerBlock][kHistBins];
    __shared__ uint32_t hcnt[kWarpsPerBlock][kHistBins];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t s = int64_t(blockIdx.x) * kWarpsPerBlock + wib;
    if (s >= n_active) return;
    const uint32_t g = w.active[cur][s];
    const uint32_t base = w.seg_base[g], cnt = w.seg_count[g];
    const uint32_t mt = w.meta[g];
    const DevBatch B = w.batches[meta_batch(mt)];
    const double* val = w.val[cur];
    const double* err = w.err[cur];
    const float* nse = w.nse[cur];
    const uint64_t* key = w.key[cur];

    // E = sum |Q_N - Q_2N| over the regions (Sec. 3), exactly as computed:
    // FP32 rounding noise is never subtracted, so it can only delay
    // convergence.  The noise bound sum(nse) (0 for FP64 regions) decides
    // whether an FP32 integral must be re-evaluated at higher precision.
    double sv = 0.0, se = 0.0, sn = 0.0, mx = 0.0;
    for (uint32_t j = lane; j < cnt; j += 32) {
        const double v = val[base + j], e = err[base + j];
        sv += v;
        se += e;
        sn += nse[base + j];
        if (key_level(key[base + j]) < uint32_t(kMaxLevel)) mx = fmax(mx, e);
    }
    const double V = warp_sum(sv), E = warp_sum(se), maxE = warp_max(mx);
    const double noise = kNoiseSigmas * warp_sum(sn);
    const double tol = fmax(B.abs_tol, B.rel_tol * fabs(V));
    const int64_t allowed = (B.max_regions - int64_t(cnt)) / 3;
    const bool fp32 = (mt & (kMetaFp64 | kMetaDf32)) == 0u;

    int st = RUNNING;
    if (force_status >= 0) st = force_status;
    else if (!isfinite(V) || !isfinite(E)) st = NONFINITE;
    else if (E <= tol) st = CONVERGED;
    else if (round - int(w.born[g]) >= max_rounds || round >= w.ls->hard_rounds)
        st = ROUNDCAP;   // rounds since admission, or the loop's own bound
    else if (fp32 && noise > kNoiseTol * tol) {
        // FP32 rounding noise would crowd the tolerance, and refinement does
        // not shrink it: re-evaluate at higher precision
        if (lane == 0) {
            w.thr[s] = make_uint2(kEscalate, 0u);
            w.cnt_new[s] = cnt;
            w.cnt_eval[s] = cnt;
        }
        return;
    }
    else if (allowed <= 0 || !(maxE > 0.0)) st = BUDGET;

    if (st != RUNNING) {
        if (lane == 0) {
            const int64_t local = int64_t(g) - B.first;
            B.values[local] = V;
            B.errors[local] = E;
            B.regions[local] = cnt;
            B.status[local] = st;
            if (st == ROUNDCAP && force_status < 0) atomicAdd(&w.totals->roundcap, 1ull);
            w.cnt_new[s] = 0;
            w.cnt_eval[s] = 0;
        }
        return;
    }

    // histogram of err in quarter octaves below maxE, sums in units of maxE 2^-40
    for (int b = lane; b < kHistBins; b += 32) { hsum[wib][b] = 0ull; hcnt[wib][b] = 0u; }
    __syncwarp();
    const int kmax = log_key(maxE);
    const double unit = ldexp(1.0, 40) / maxE;
    for (uint32_t j = lane; j < cnt; j += 32) {
        const double e = err[base + j];
        if (e > 0.0 && key_level(key[base + j]) < uint32_t(kMaxLevel)) {
            const int bin = min(kHistBins - 1, kmax - log_key(e));
            atomicAdd(&hsum[wib][bin], (unsigned long long)(e * unit));
            atomicAdd(&hcnt[wib][bin], 1u);
        }
    }
    __syncwarp();
    if (lane == 0)
        select_regions(w, s, hsum[wib], hcnt[wib], (E - cover * tol) * unit, allowed, kmax, cnt);
}

cudaError_t launch_reduce_test(const Work& w, int64_t hint_active, int max_rounds, double cover,
                               cudaStream_t s)
{
    if (hint_active <= 0) return cudaSuccess;
    const int64_t blocks = (hint_active + kWarpsPerBlock - 1) / kWarpsPerBlock;
    k_reduce_test<<<int(blocks), kWarpsPerBlock * 32, 0, s>>>(w, max_rounds, cover, -1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared-partition (group) reduce + test + selection for the active groups
// (kind, q) of batches with P pairs.  Per pair c: V_c = sum Q_2N and
// E_c = sum |Q_N - Q_2N| over the group's regions, tol_c = max(abs_tol,
// rel_tol |V_c|).  The group is done when every valid pair has E_c <= tol_c.
// Otherwise each region's score
//   s_r = max over the pairs not yet converged of err_c,r / tol_c
// goes to err[r], and the per-integral selection runs on the scores with unit
// tolerance: the largest scores until their sum covers sum_r s_r - cover, so
// that for every pair the unsplit regions carry at most cover * tol_c of its
// error.  Finished groups write every pair's value, error, region count and
// status (CONVERGED for the pairs that meet their tolerance).
//
// With w.gglobal (group mode 2, the global error of Algorithm 2) the group has
// one error sum and one tolerance: E_g = sum_c E_c over the valid pairs,
// tol_g = max(abs_tol, rel_tol sum_c |V_c|), done when E_g <= tol_g; the
// score of a region is s_r = sum_c err_c,r / tol_g (its share of E_g), so the
// same selection leaves at most cover * tol_g of E_g unsplit, and every pair
// of a finished group takes the group's status.
//
// Four launches, so that a deep group does not keep one block streaming its
// regions alone: each group's segment is cut into kGroupSplit chunks of
// consecutive regions, and
//   k_group_sums    (slot, chunk) blocks: per-pair partial sums of the chunk
//   k_group_test    slot blocks: the chunk sums in chunk order (deterministic),
//                   the test, finished groups' outputs, 1/tol_c of the rest
//   k_group_scores  (slot, chunk) blocks: region scores, the chunk's score sum
//                   and maximum
//   k_group_select  slot blocks: the score histogram and the selection
constexpr int kGroupWarps = 8;

__device__ __forceinline__ void chunk_range(uint32_t cnt, int k, uint32_t& j0, uint32_t& j1)
{
    const uint32_t len = (cnt + kGroupSplit - 1) / kGroupSplit;
    j0 = min(cnt, uint32_t(k) * len);
    j1 = min(cnt, j0 + len);
}

__global__ void __launch_bounds__(kGroupWarps * 32) k_group_sums(Work w)
{
    __shared__ double pv[kGroupWarps][kGroupPairs], pe[kGroupWarps][kGroupPairs];
    const LoopState& Ls = *w.ls;
    const int64_t s = blockIdx.x / kGroupSplit;
    const int k = int(blockIdx.x % kGroupSplit);
    if (s >= Ls.n_active) return;
    const int cur = Ls.cur;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t g = w.active[cur][s];
    const uint32_t base = w.seg_base[g], cnt = w.seg_count[g];
    const int P = w.batches[meta_batch(w.meta[g])].npairs;
    const size_t S = size_t(w.vstride);
    const double* vval = w.vval[cur];
    const float* verr = w.verr[cur];
    uint32_t j0, j1;
    chunk_range(cnt, k, j0, j1);
    // values in FP64; error sums in FP32 per lane (a lane adds about
    // cnt / 64 terms of one sign: relative rounding below 1e-5, far inside
    // what a convergence test or a selection can resolve), then in FP64
    double v[3] = {0.0, 0.0, 0.0};
    float e[3] = {0.0f, 0.0f, 0.0f};
    // unrolled so that several rows' loads are in flight per warp (the sums
    // keep their order)
#pragma unroll 4
    for (uint32_t j = j0 + wid; j < j1; j += kGroupWarps) {
        const size_t r = size_t(base + j) * S;
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3) {
            const int c = lane + 32 * c3;
            if (c < P) { v[c3] += vval[r + c]; e[c3] += verr[r + c]; }
        }
    }
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) {
        const int c = lane + 32 * c3;
        if (c < P) { pv[wid][c] = v[c3]; pe[wid][c] = double(e[c3]); }
    }
    __syncthreads();
    if (tid < P) {
        double V = 0.0, E = 0.0;
        for (int q = 0; q < kGroupWarps; ++q) { V += pv[q][tid]; E += pe[q][tid]; }
        double* out = w.gpart + (size_t(s) * kGroupSplit + k) * 2 * kGroupPairs;
        out[tid] = V;
        out[kGroupPairs + tid] = E;
    }
}

// Outputs of a finished group: per pair value, error, region count, status.
// gconv < 0: each pair's own test decides CONVERGED; otherwise gconv is the
// group's outcome (1 converged, 0 not).
__device__ void group_outputs(const Work& w, const DevBatch& B, uint32_t g, uint32_t cnt, int c,
                              double V, double E, int st, int gconv)
{
    const int l = B.lm[2 * c], m = B.lm[2 * c + 1];
    const bool valid = l >= 0 && m >= 0 && l < w.nff && m < w.nff;
    const bool finite = isfinite(V) && isfinite(E);
    const bool conv = gconv >= 0 ? gconv != 0 : E <= fmax(B.abs_tol, B.rel_tol * fabs(V));
    const int64_t o = (int64_t(g) - B.first) * B.npairs + c;
    B.values[o] = valid ? V : NAN;
    B.errors[o] = valid ? E : NAN;
    B.regions[o] = cnt;
    B.status[o] = !valid || !finite ? NONFINITE : (conv ? CONVERGED : st);
}

// Truncated-unity products of a finished flow group (Eqs. matmul-P/C/D):
// with X its bubble matrix (the group's values, pair l * nff + m at X[l][m]),
//   pp: dP = V^P X V^P;   ph: dC = -V^C X V^C, dD = 2 V^D X V^D - V^C X V^D - V^D X V^C,
// for the group's transfer momentum.  X: the values in shared memory; called by
// every thread of the block (at least nff^2 of them).  Pairs not in l-major
// order give NaN products.
__device__ void group_tu(const Work& w, const DevBatch& B, int64_t iq, const double* X)
{
    __shared__ double A[kGroupPairs], C[kGroupPairs];
    const int n = w.nff, nn = n * n, tid = threadIdx.x;
    const bool ordered = __syncthreads_and(
        tid >= nn || (B.lm[2 * tid] == tid / n && B.lm[2 * tid + 1] == tid % n));
    const size_t o = size_t(iq) * nn;
    const double* V0 = B.tu_v0 + o;
    const double* V1 = B.tu_v1 ? B.tu_v1 + o : nullptr;
    if (tid < nn) {
        // A = X V0, C = X V1: the right factors of every product
        const int a = tid / n, b = tid % n;
        double sa = 0.0, sc = 0.0;
        for (int k = 0; k < n; ++k) {
            sa = fma(X[a * n + k], V0[k * n + b], sa);
            if (V1) sc = fma(X[a * n + k], V1[k * n + b], sc);
        }
        A[tid] = sa;
        C[tid] = sc;
    }
    __syncthreads();
    if (tid < nn) {
        const int a = tid / n, b = tid % n;
        double p = 0.0, d = 0.0;
        if (!V1) {                          // pp: V^P (X V^P)
            for (int k = 0; k < n; ++k) p = fma(V0[a * n + k], A[k * n + b], p);
            B.tu_out0[o + tid] = ordered ? p : NAN;
        } else {                            // ph: V0 = V^C, V1 = V^D
            for (int k = 0; k < n; ++k) {
                p = fma(V0[a * n + k], A[k * n + b], p);           // V^C X V^C
                d = fma(2.0 * V1[a * n + k], C[k * n + b], d);     // 2 V^D X V^D
                d = fma(-V0[a * n + k], C[k * n + b], d);          // - V^C X V^D
                d = fma(-V1[a * n + k], A[k * n + b], d);          // - V^D X V^C
            }
            B.tu_out0[o + tid] = ordered ? -p : NAN;
            B.tu_out1[o + tid] = ordered ? d : NAN;
        }
    }
}

__global__ void __launch_bounds__(128)
k_group_test(Work w, int max_rounds, int force_status)
{
    const LoopState& Ls = *w.ls;
    if (force_status == kFinalizeIfStuck) {   // after the device loop: decided on the device
        if (Ls.stop != kStuck) return;
        force_status = POOL;
    }
    const int64_t s = blockIdx.x;
    if (s >= Ls.n_active) return;
    const int cur = Ls.cur, round = Ls.round;
    const int tid = threadIdx.x;
    const uint32_t g = w.active[cur][s];
    const uint32_t cnt = w.seg_count[g];
    const DevBatch& B = w.batches[meta_batch(w.meta[g])];
    const int P = B.npairs;
    double V = 0.0, E = 0.0;
    bool valid = false, finite = true, conv = true;
    if (tid < P) {
        const double* part = w.gpart + size_t(s) * kGroupSplit * 2 * kGroupPairs;
        for (int k = 0; k < kGroupSplit; ++k) {
            V += part[k * 2 * kGroupPairs + tid];
            E += part[k * 2 * kGroupPairs + kGroupPairs + tid];
        }
        const int l = B.lm[2 * tid], m = B.lm[2 * tid + 1];
        valid = l >= 0 && m >= 0 && l < w.nff && m < w.nff;
        finite = isfinite(V) && isfinite(E);
    }
    double tol = fmax(B.abs_tol, B.rel_tol * fabs(V));
    if (w.gglobal) {
        // one sum in pair order (deterministic), one tolerance for the group
        __shared__ double sE[kGroupPairs], sV[kGroupPairs], sg[2];
        if (tid < P) {
            sE[tid] = valid && finite ? E : 0.0;
            sV[tid] = valid && finite ? fabs(V) : 0.0;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int c = 0; c < P; ++c) { a += sE[c]; b += sV[c]; }
            sg[0] = a;
            sg[1] = fmax(B.abs_tol, B.rel_tol * b);
        }
        __syncthreads();
        tol = sg[1];
        conv = sg[0] <= tol;
    } else {
        conv = E <= tol;
    }
    if (tid < P) {
        w.gtol[size_t(s) * kGroupPairs + tid] =
            (valid && finite && !conv) ? 1.0 / fmax(tol, 1e-300) : 0.0;
        w.gsum[size_t(s) * 2 * kGroupPairs + tid] = V;
        w.gsum[size_t(s) * 2 * kGroupPairs + kGroupPairs + tid] = E;
    }
    const bool any_nonfinite = __syncthreads_or(valid && !finite);
    const bool all_conv = __syncthreads_and(!valid || (finite && conv));
    const int64_t allowed = (B.max_regions - int64_t(cnt)) / 3;
    int st = RUNNING;
    if (force_status >= 0) st = force_status;
    else if (any_nonfinite) st = NONFINITE;
    else if (all_conv) st = CONVERGED;
    else if (round - int(w.born[g]) >= max_rounds || round >= Ls.hard_rounds) st = ROUNDCAP;
    else if (allowed <= 0) st = BUDGET;
    if (tid == 0) w.gstate[s] = st;
    if (st == RUNNING) return;
    if (tid < P) group_outputs(w, B, g, cnt, tid, V, E, st, w.gglobal ? int(conv) : -1);
    if (tid == 0) {
        if (st == ROUNDCAP && force_status < 0) atomicAdd(&w.totals->roundcap, 1ull);
        w.cnt_new[s] = 0;
        w.cnt_eval[s] = 0;
    }
    if (B.tu_out0) {   // the flow step's products, as the group finishes
        __shared__ double X[kGroupPairs];
        if (tid < P) X[tid] = V;
        __syncthreads();
        group_tu(w, B, int64_t(g) - B.first, X);
    }
}

__global__ void __launch_bounds__(kGroupWarps * 32) k_group_scores(Work w)
{
    __shared__ float itol[kGroupPairs];
    __shared__ double ps[kGroupWarps], pm[kGroupWarps];
    const LoopState& Ls = *w.ls;
    const int64_t s = blockIdx.x / kGroupSplit;
    const int k = int(blockIdx.x % kGroupSplit);
    if (s >= Ls.n_active || w.gstate[s] != RUNNING) return;
    const int cur = Ls.cur;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t g = w.active[cur][s];
    const uint32_t base = w.seg_base[g], cnt = w.seg_count[g];
    const int P = w.batches[meta_batch(w.meta[g])].npairs;
    const size_t S = size_t(w.vstride);
    const float* verr = w.verr[cur];
    const uint64_t* key = w.key[cur];
    // scores in FP32 (they only order the regions and size the selection);
    // 1/tol saturates at the FP32 maximum
    if (tid < P) itol[tid] = float(fmin(w.gtol[size_t(s) * kGroupPairs + tid], 3.0e38));
    __syncthreads();
    uint32_t j0, j1;
    chunk_range(cnt, k, j0, j1);
    double ssum = 0.0, smax = 0.0;
#pragma unroll 4
    for (uint32_t j = j0 + wid; j < j1; j += kGroupWarps) {
        const size_t r = size_t(base + j) * S;
        float sc = 0.0f;
        if (w.gglobal) {
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) {
                const int c = lane + 32 * c3;
                if (c < P) sc += verr[r + c] * itol[c];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sc += __shfl_xor_sync(kFull, sc, o);
        } else {
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) {
                const int c = lane + 32 * c3;
                if (c < P) sc = fmaxf(sc, verr[r + c] * itol[c]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sc = fmaxf(sc, __shfl_xor_sync(kFull, sc, o));
        }
        if (lane == 0) {
            const double scd = double(fminf(sc, 1.0e30f));   // finite even for a zero tolerance
            w.err[cur][base + j] = scd;
            ssum += scd;
            if (key_level(key[base + j]) < uint32_t(kMaxLevel)) smax = fmax(smax, scd);
        }
    }
    if (lane == 0) { ps[wid] = ssum; pm[wid] = smax; }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < kGroupWarps; ++q) { a += ps[q]; b = fmax(b, pm[q]); }
        w.gsc[(size_t(s) * kGroupSplit + k) * 2] = a;
        w.gsc[(size_t(s) * kGroupSplit + k) * 2 + 1] = b;
    }
}

__global__ void __launch_bounds__(kGroupWarps * 32) k_group_select(Work w, double cover)
{
    __shared__ unsigned long long hsum[kHistBins];
    __shared__ uint32_t hcnt[kHistBins];
    const LoopState& Ls = *w.ls;
    const int64_t s = blockIdx.x;
    if (s >= Ls.n_active || w.gstate[s] != RUNNING) return;
    const int cur = Ls.cur;
    const int tid = threadIdx.x;
    const uint32_t g = w.active[cur][s];
    const uint32_t base = w.seg_base[g], cnt = w.seg_count[g];
    const DevBatch& B = w.batches[meta_batch(w.meta[g])];
    double Ssum = 0.0, Smax = 0.0;
    for (int k = 0; k < kGroupSplit; ++k) {
        Ssum += w.gsc[(size_t(s) * kGroupSplit + k) * 2];
        Smax = fmax(Smax, w.gsc[(size_t(s) * kGroupSplit + k) * 2 + 1]);
    }
    if (!(Smax > 0.0)) {   // nothing left to split
        if (tid < B.npairs)
            group_outputs(w, B, g, cnt, tid, w.gsum[size_t(s) * 2 * kGroupPairs + tid],
                          w.gsum[size_t(s) * 2 * kGroupPairs + kGroupPairs + tid], BUDGET,
                          w.gglobal ? 0 : -1);
        if (tid == 0) { w.cnt_new[s] = 0; w.cnt_eval[s] = 0; }
        if (B.tu_out0) {
            __shared__ double X[kGroupPairs];
            if (tid < B.npairs) X[tid] = w.gsum[size_t(s) * 2 * kGroupPairs + tid];
            __syncthreads();
            group_tu(w, B, int64_t(g) - B.first, X);
        }
        return;
    }
    for (int b = tid; b < kHistBins; b += blockDim.x) { hsum[b] = 0ull; hcnt[b] = 0u; }
    __syncthreads();
    const uint64_t* key = w.key[cur];
    const int kmax = log_key(Smax);
    const double unit = ldexp(1.0, 40) / Smax;
    for (uint32_t j = tid; j < cnt; j += blockDim.x) {
        const double e = w.err[cur][base + j];
        if (e > 0.0 && key_level(key[base + j]) < uint32_t(kMaxLevel)) {
            const int bin = min(kHistBins - 1, kmax - log_key(e));
            atomicAdd(&hsum[bin], (unsigned long long)(e * unit));
            atomicAdd(&hcnt[bin], 1u);
        }
    }
    __syncthreads();
    if (tid == 0) {
        const int64_t allowed = (B.max_regions - int64_t(cnt)) / 3;
        select_regions(w, s, hsum, hcnt, (Ssum - cover) * unit, allowed, kmax, cnt);
    }
}

cudaError_t launch_reduce_group(const Work& w, int64_t hint_active, int max_rounds, double cover,
                                cudaStream_t s)
{
    if (hint_active <= 0) return cudaSuccess;
    const int nb = int(hint_active);
    k_group_sums<<<nb * kGroupSplit, kGroupWarps * 32, 0, s>>>(w);
    k_group_test<<<nb, 128, 0, s>>>(w, max_rounds, -1);
    k_group_scores<<<nb * kGroupSplit, kGroupWarps * 32, 0, s>>>(w);
    k_group_select<<<nb, kGroupWarps * 32, 0, s>>>(w, cover);
    return cudaGetLastError();
}

// Pool pressure: after the slot scan, an integral keeps its splits only while
// the growth of all slots up to it fits in `room` regions, so the kept slots
// form a prefix and the first integrals always progress; the others keep
// their regions unsplit for this round.  The growth of a slot is 3/4 of its
// eval count (4 children replace each marked region); escalated slots count
// their full eval count there, which only makes the bound conservative.
// With room = capacity - current pool the next pool stays within capacity.
__global__ void k_throttle(Work w)
{
    const LoopState& L = *w.ls;
    if (!((long long)w.totals->pool > L.cap)) return;
    const unsigned long long room = (unsigned long long)(L.cap - L.pool);
    const int64_t n_active = L.n_active;
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= n_active) return;
    const uint32_t nnew = w.cnt_new[s];
    if (nnew == 0 || w.thr[s].x == kEscalate) return;
    const unsigned long long evals =
        w.blk_eval[s / kScanBlock] + w.pre_eval[s] + w.cnt_eval[s];
    if (3ull * evals <= 4ull * room) return;
    w.cnt_new[s] = nnew - w.cnt_eval[s] / 4u * 3u;   // current region count
    w.cnt_eval[s] = 0;
    // threshold bin 0 with rank cap 0 under the same kmax: every region's bin
    // is >= 0 there, so none is marked
    w.thr[s] = make_uint2(w.thr[s].x & ~0xffu, 0u);
}

cudaError_t launch_throttle(const Work& w, int64_t hint_active, cudaStream_t s)
{
    if (hint_active <= 0) return cudaSuccess;
    k_throttle<<<int((hint_active + 255) / 256), 256, 0, s>>>(w);
    return cudaGetLastError();
}

// Integrals [g0, g1) that never entered the pool: status, NaN value and error.
__global__ void k_mark_unadmitted(Work w, int64_t g0, int64_t g1, int status)
{
    const int64_t g = g0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= g1) return;
    int b = 0;
    {
        int lo = 0, hi = w.nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (w.batches[mid].first <= g) lo = mid; else hi = mid - 1;
        }
        b = lo;
    }
    const DevBatch& B = w.batches[b];
    const int64_t local = g - B.first;
    const int width = w.vstride > 0 ? B.npairs : 1;   // outputs of the unit
    for (int p = 0; p < width; ++p) {
        const int64_t o = local * width + p;
        B.values[o] = NAN;
        B.errors[o] = NAN;
        B.regions[o] = 0;
        B.status[o] = status;
        if (B.tu_out0) B.tu_out0[o] = NAN;
        if (B.tu_out1) B.tu_out1[o] = NAN;
    }
}

// After the device loop: the integrals it never admitted, with the status its
// stop reason gives (pool: PAID_POOL, hard round bound: PAID_ROUNDCAP).
__global__ void k_mark_unadmitted_dev(Work w)
{
    const LoopState& L = *w.ls;
    if (L.stop != kStuck && L.stop != kNoRoom && L.stop != kHardCap) return;
    const int64_t g = L.admitted + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= w.n) return;
    const int status = L.stop == kHardCap ? ROUNDCAP : POOL;
    int lo = 0, hi = w.nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (w.batches[mid].first <= g) lo = mid; else hi = mid - 1;
    }
    const DevBatch& B = w.batches[lo];
    const int64_t local = g - B.first;
    const int width = w.vstride > 0 ? B.npairs : 1;
    for (int p = 0; p < width; ++p) {
        const int64_t o = local * width + p;
        B.values[o] = NAN;
        B.errors[o] = NAN;
        B.regions[o] = 0;
        B.status[o] = status;
        if (B.tu_out0) B.tu_out0[o] = NAN;
        if (B.tu_out1) B.tu_out1[o] = NAN;
    }
}

cudaError_t launch_finish_device(const Work& w, cudaStream_t s)
{
    if (w.n <= 0) return cudaSuccess;
    const int64_t n = w.n;
    if (w.vstride > 0) {
        k_group_sums<<<int(n) * kGroupSplit, kGroupWarps * 32, 0, s>>>(w);
        k_group_test<<<int(n), 128, 0, s>>>(w, 0, kFinalizeIfStuck);
    } else {
        const int64_t blocks = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
        k_reduce_test<<<int(blocks), kWarpsPerBlock * 32, 0, s>>>(w, 0, 0.0, kFinalizeIfStuck);
    }
    k_mark_unadmitted_dev<<<int((n + 255) / 256), 256, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_mark_unadmitted(const Work& w, int64_t g0, int64_t g1, int status, cudaStream_t s)
{
    if (g1 <= g0) return cudaSuccess;
    k_mark_unadmitted<<<int((g1 - g0 + 255) / 256), 256, 0, s>>>(w, g0, g1, status);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Work& w, int64_t hint_active, int status, cudaStream_t s)
{
    if (hint_active <= 0) return cudaSuccess;
    if (w.vstride > 0) {
        k_group_sums<<<int(hint_active) * kGroupSplit, kGroupWarps * 32, 0, s>>>(w);
        k_group_test<<<int(hint_active), 128, 0, s>>>(w, 0, status);
    } else {
        const int64_t blocks = (hint_active + kWarpsPerBlock - 1) / kWarpsPerBlock;
        k_reduce_test<<<int(blocks), kWarpsPerBlock * 32, 0, s>>>(w, 0, 0.0, status);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exclusive scan of (cnt_new, cnt_eval, cnt_new > 0) over the active slots.
// rescan = 1 runs only when the last scan's pool total is over capacity.
__device__ __forceinline__ bool over_capacity(const Work& w)
{
    return (long long)w.totals->pool > w.ls->cap;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_blocks(Work w, int rescan)
{
    if (rescan && !over_capacity(w)) return;
    const int64_t n_active = w.ls->n_active;
    if (int64_t(blockIdx.x) * kScanBlock >= n_active) return;
    __shared__ unsigned long long sp[32], se[32];
    __shared__ uint32_t sa[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t s = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
    unsigned long long p = 0, e = 0;
    uint32_t a = 0;
    if (s < n_active) {
        p = w.cnt_new[s];
        e = w.cnt_eval[s];
        a = p > 0 ? 1u : 0u;
    }
    unsigned long long ip = p, ie = e;
    uint32_t ia = a;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long yp = __shfl_up_sync(kFull, ip, o);
        const unsigned long long ye = __shfl_up_sync(kFull, ie, o);
        const uint32_t ya = __shfl_up_sync(kFull, ia, o);
        if (lane >= o) { ip += yp; ie += ye; ia += ya; }
    }
    if (lane == 31) { sp[wid] = ip; se[wid] = ie; sa[wid] = ia; }
    __syncthreads();
    if (wid == 0) {
        unsigned long long xp = sp[lane], xe = se[lane];
        uint32_t xa = sa[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long yp = __shfl_up_sync(kFull, xp, o);
            const unsigned long long ye = __shfl_up_sync(kFull, xe, o);
            const uint32_t ya = __shfl_up_sync(kFull, xa, o);
            if (lane >= o) { xp += yp; xe += ye; xa += ya; }
        }
        sp[lane] = xp; se[lane] = xe; sa[lane] = xa;   // inclusive over warps
    }
    __syncthreads();
    const unsigned long long wp = wid ? sp[wid - 1] : 0ull, we = wid ? se[wid - 1] : 0ull;
    const uint32_t wa = wid ? sa[wid - 1] : 0u;
    if (s < n_active) {
        w.pre_pool[s] = wp + ip - p;
        w.pre_eval[s] = we + ie - e;
        w.pre_act[s] = wa + ia - a;
    }
    if (threadIdx.x == kScanBlock - 1) {
        w.blk_pool[blockIdx.x] = sp[31];
        w.blk_eval[blockIdx.x] = se[31];
        w.blk_act[blockIdx.x] = sa[31];
    }
}

// Single block: exclusive scan of the block totals in place, grand totals out.
__global__ void __launch_bounds__(kScanBlock) k_scan_top(Work w, int rescan)
{
    __shared__ unsigned long long sp[32], se[32];
    __shared__ unsigned long long sa[32];
    __shared__ unsigned long long carry[3];
    __shared__ int go;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        carry[0] = carry[1] = carry[2] = 0ull;
        go = !rescan || over_capacity(w);
        if (rescan && go) w.ls->throttled = 1;
    }
    __syncthreads();
    if (!go) return;
    const int64_t n_active = w.ls->n_active;
    const int nblk = int((n_active + kScanBlock - 1) / kScanBlock);
    for (int c0 = 0; c0 < nblk; c0 += kScanBlock) {
        const int i = c0 + threadIdx.x;
        unsigned long long p = 0, e = 0, a = 0;
        if (i < nblk) { p = w.blk_pool[i]; e = w.blk_eval[i]; a = w.blk_act[i]; }
        unsigned long long ip = p, ie = e, ia = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long yp = __shfl_up_sync(kFull, ip, o);
            const unsigned long long ye = __shfl_up_sync(kFull, ie, o);
            const unsigned long long ya = __shfl_up_sync(kFull, ia, o);
            if (lane >= o) { ip += yp; ie += ye; ia += ya; }
        }
        if (lane == 31) { sp[wid] = ip; se[wid] = ie; sa[wid] = ia; }
        __syncthreads();
        if (wid == 0) {
            unsigned long long xp = sp[lane], xe = se[lane], xa = sa[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long yp = __shfl_up_sync(kFull, xp, o);
                const unsigned long long ye = __shfl_up_sync(kFull, xe, o);
                const unsigned long long ya = __shfl_up_sync(kFull, xa, o);
                if (lane >= o) { xp += yp; xe += ye; xa += ya; }
            }
            sp[lane] = xp; se[lane] = xe; sa[lane] = xa;
        }
        __syncthreads();
        const unsigned long long wp = wid ? sp[wid - 1] : 0ull, we = wid ? se[wid - 1] : 0ull;
        const unsigned long long wa = wid ? sa[wid - 1] : 0ull;
        if (i < nblk) {
            w.blk_pool[i] = carry[0] + wp + ip - p;
            w.blk_eval[i] = carry[1] + we + ie - e;
            w.blk_act[i] = uint32_t(carry[2] + wa + ia - a);
        }
        __syncthreads();
        if (threadIdx.x == 0) { carry[0] += sp[31]; carry[1] += se[31]; carry[2] += sa[31]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        w.totals->pool = carry[0];
        w.totals->eval = carry[1];
        w.totals->active = carry[2];
    }
}

cudaError_t launch_scan(const Work& w, int64_t hint_active, int rescan, cudaStream_t s)
{
    const int64_t nblk = hint_active > 0 ? (hint_active + kScanBlock - 1) / kScanBlock : 0;
    if (nblk > 0) k_scan_blocks<<<int(nblk), kScanBlock, 0, s>>>(w, rescan);
    k_scan_top<<<1, kScanBlock, 0, s>>>(w, rescan);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Split marked regions into 4 children, copy the rest; build the eval list and
// the next active list.  Reads pool[cur], writes pool[cur ^ 1].
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_split(Work w)
{
    const int cur = w.ls->cur;
    const int64_t n_active = w.ls->n_active;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t s = int64_t(blockIdx.x) * kWarpsPerBlock + wib;
    if (s >= n_active) return;
    const uint32_t nnew = w.cnt_new[s];
    if (nnew == 0) return;
    const uint32_t g = w.active[cur][s];
    const int64_t blk = s / kScanBlock;
    const unsigned long long pbase = w.blk_pool[blk] + w.pre_pool[s];
    const unsigned long long ebase = w.blk_eval[blk] + w.pre_eval[s];
    const uint32_t abase = w.blk_act[blk] + w.pre_act[s];
    const uint32_t base = w.seg_base[g], cnt = w.seg_count[g];
    const uint2 th = w.thr[s];
    const int tb = int(th.x & 0xffu), kmax = int(th.x >> 8);
    const uint32_t cap = th.y;
    const int nxt = cur ^ 1;
    const uint64_t* key = w.key[cur];
    const double* val = w.val[cur];
    const double* err = w.err[cur];
    const float* nse = w.nse[cur];
    uint64_t* key_n = w.key[nxt];
    double* val_n = w.val[nxt];
    double* err_n = w.err[nxt];
    float* nse_n = w.nse[nxt];
    const unsigned lt = (1u << lane) - 1u;

    if (th.x == kEscalate) {
        // FP32 noise too large for the tolerance: same regions, re-evaluated in float-float
        for (uint32_t j = lane; j < cnt; j += 32) {
            key_n[pbase + j] = key[base + j];
            w.evl[ebase + j] = make_uint2(uint32_t(pbase + j), g);
        }
        if (lane == 0) {
            w.meta[g] |= kMetaDf32;
            atomicAdd(&w.totals->escalated, 1ull);
            w.seg_base[g] = uint32_t(pbase);
            w.seg_count[g] = nnew;
            w.active[nxt][abase] = g;
        }
        return;
    }

    uint32_t run = 0, erun = 0, tbrun = 0;
    for (uint32_t c0 = 0; c0 < cnt; c0 += 32) {
        const uint32_t j = c0 + lane;
        const bool valid = j < cnt;
        uint64_t k = 0;
        double v = 0.0, e = 0.0;
        float nz = 0.0f;
        int bin = 255;
        if (valid) {
            k = key[base + j];
            v = val[base + j];
            e = err[base + j];
            nz = nse[base + j];
            if (e > 0.0 && key_level(k) < uint32_t(kMaxLevel))
                bin = min(kHistBins - 1, kmax - log_key(e));
        }
        const bool in_tb = bin == tb;
        const unsigned btb = __ballot_sync(kFull, in_tb);
        const uint32_t rank = tbrun + __popc(btb & lt);
        tbrun += __popc(btb);
        const bool mark = valid && (bin < tb || (in_tb && rank < cap));
        const unsigned bm = __ballot_sync(kFull, mark);
        uint32_t tot;
        const uint32_t off = warp_excl(valid ? (mark ? 4u : 1u) : 0u, tot);
        const unsigned long long p = pbase + run + off;
        if (valid && !mark) {
            key_n[p] = k;
            val_n[p] = v;
            err_n[p] = e;
            nse_n[p] = nz;
            if (w.vsrc) w.vsrc[p] = base + j;
        }
        if (mark) {
            const uint32_t L = key_level(k), ix = key_ix(k), iy = key_iy(k);
            const unsigned long long q = ebase + erun + 4u * __popc(bm & lt);
#pragma unroll
            for (uint32_t c = 0; c < 4; ++c) {
                key_n[p + c] = make_key(L + 1, 2 * ix + (c >> 1), 2 * iy + (c & 1));
                w.evl[q + c] = make_uint2(uint32_t(p + c), g);
                if (w.vsrc) w.vsrc[p + c] = 0xffffffffu;
            }
        }
        run += tot;
        erun += 4u * __popc(bm);
    }
    if (lane == 0) {
        w.seg_base[g] = uint32_t(pbase);
        w.seg_count[g] = nnew;
        w.active[nxt][abase] = g;
    }
}

// Group mode: every kept region's pair vectors to its slot in the next pool
// (one thread per (slot, pair) element: coalesced on both sides).
static_assert(kGroupPairs <= 96, "k_copy_vectors: three columns per lane and row");

__global__ void k_copy_vectors(Work w)
{
    // one warp per kept region: its source row once per warp, the row's
    // values and errors in coalesced lane order
    const int cur = w.ls->cur, nxt = cur ^ 1;
    const int S = w.vstride;
    const int64_t pool = int64_t(w.totals->pool);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t p = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; p < pool; p += nwarps) {
        const uint32_t src = w.vsrc[p];
        if (src == 0xffffffffu) continue;
        const double* sv = w.vval[cur] + size_t(src) * S;
        const float* se = w.verr[cur] + size_t(src) * S;
        double* dv = w.vval[nxt] + size_t(p) * S;
        float* de = w.verr[nxt] + size_t(p) * S;
        double a[3];
        float b[3];
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3) {
            const int c = lane + 32 * c3;
            if (c < S) { a[c3] = sv[c]; b[c3] = se[c]; }
        }
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3) {
            const int c = lane + 32 * c3;
            if (c < S) { dv[c] = a[c3]; de[c] = b[c3]; }
        }
    }
}

cudaError_t launch_copy_vectors(const Work& w, int64_t hint_pool, cudaStream_t s)
{
    if (hint_pool <= 0 || w.vstride <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((hint_pool * 32 + 255) / 256, 152 * 16);
    k_copy_vectors<<<int(blocks), 256, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_split(const Work& w, int64_t hint_active, cudaStream_t s)
{
    if (hint_active <= 0) return cudaSuccess;
    const int64_t blocks = (hint_active + kWarpsPerBlock - 1) / kWarpsPerBlock;
    k_split<<<int(blocks), kWarpsPerBlock * 32, 0, s>>>(w);
    return cudaGetLastError();
}

}  // namespace paid
