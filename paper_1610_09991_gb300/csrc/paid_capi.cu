// C ABI of libpaid (declared in include/paid.h) and the refinement loop of
// the paper's Listing 5:
//
//   setup:  uniform level-L0 partition of every integral (Listing 1)
//   round:  evaluate the regions on the eval list (Listing 3)
//           -> per-integral reduce + convergence test + selection (Listings 2, 4)
//           -> prefix scan of the next pool / eval list / active list
//              (+ in-order throttling when the next pool would not fit)
//           -> split the selected regions and compact the pool
//           -> control: next round's counts, admission of waiting
//              integrals, stop decision
//   until no integral is refining (the master's `done`, Listing 5).
//
// Every round kernel reads its counts from the device-side loop state, so
// the round needs no host arguments.  With options.device_loop the rounds run
// inside one CUDA graph: a conditional WHILE node whose body is one round,
// ended by the control kernel; the host waits once.  Otherwise the host
// launches each round and reads the loop state back (per-phase timing).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/paid.h"
#include "paid_internal.cuh"

using namespace paid;

// The instantiated device-loop graph of the last call, reused while the
// workspace layout and the options it was captured with are unchanged.
struct LoopGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* base = nullptr;        // workspace layout it was captured for
    int64_t n = 0, cap = 0;
    int nb = 0, vstride = 0;
    int rule_n = 0, eval_fp32 = 0, max_rounds = 0, eval_blocks = 0;
    const float* tmap = nullptr;       // trace buffer it writes (null: none)
    int kinds = 0;                     // the kernel F variant it launches
    double cover = 0.0;
};

struct paid_ctx {
    int device = 0;
    Lattice lat{};
    int nff = 9;
    paid_options opt{};
    RoundTotals* h_totals = nullptr;   // pinned
    LoopState* h_state = nullptr;      // pinned
    cudaEvent_t ev[7] = {};            // kernel-class timing (options.timing)
    cudaStream_t capture = nullptr;    // stream the device loop is captured on
    LoopGraph loop;
    std::string last_error;
    paid_stats stats{};
    float* trace_buf = nullptr;        // paid_set_trace_buffer
    int64_t trace_units = 0;
    // the outcome of an asynchronous call (device loop): read by paid_wait
    cudaEvent_t done = nullptr;        // recorded after the copy of the final loop state
    bool pending = false;
    int64_t pend_n = 0, pend_cap = 0;
    int last_rc = PAID_OK;
};

namespace {

constexpr int kMaxBatches = 4096;
constexpr int64_t kMaxRegionsPerIntegral = int64_t(1) << 23;
constexpr int64_t kMaxCapacity = int64_t(0xffffffffu);

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t batches, totals, ls, trig, meta, born, seg_base, seg_count, active0, active1, cnt_new, cnt_eval,
        thr, pre_pool, pre_eval, pre_act, blk_pool, blk_eval, blk_act, key0, key1, val0, val1,
        err0, err1, nse0, nse1, evl, vval0, vval1, verr0, verr1, vsrc, gpart, gsum, gtol,
        gsc, gstate, end;
};

// Byte offsets of every workspace array for n integrals and capacity cap.
Layout layout(int64_t n, int64_t cap, bool group)
{
    Layout L{};
    const int64_t nblk = (n + kScanBlock - 1) / kScanBlock + 1;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L.batches = take(sizeof(DevBatch) * kMaxBatches);
    L.totals = take(sizeof(RoundTotals));
    L.ls = take(sizeof(LoopState));
    L.trig = take(sizeof(QTrig) * n);
    L.meta = take(4 * n);
    L.born = take(4 * n);
    L.seg_base = take(4 * n);
    L.seg_count = take(4 * n);
    L.active0 = take(4 * n);
    L.active1 = take(4 * n);
    L.cnt_new = take(4 * n);
    L.cnt_eval = take(4 * n);
    L.thr = take(8 * n);
    L.pre_pool = take(8 * n);
    L.pre_eval = take(8 * n);
    L.pre_act = take(4 * n);
    L.blk_pool = take(8 * nblk);
    L.blk_eval = take(8 * nblk);
    L.blk_act = take(4 * nblk);
    L.key0 = take(8 * cap);
    L.key1 = take(8 * cap);
    L.val0 = take(8 * cap);
    L.val1 = take(8 * cap);
    L.err0 = take(8 * cap);
    L.err1 = take(8 * cap);
    L.nse0 = take(4 * cap);
    L.nse1 = take(4 * cap);
    L.evl = take(8 * cap);
    if (group) {   // pair vectors (shared-partition mode)
        L.vval0 = take(8 * kGroupPairs * cap);
        L.vval1 = take(8 * kGroupPairs * cap);
        L.verr0 = take(4 * kGroupPairs * cap);
        L.verr1 = take(4 * kGroupPairs * cap);
        L.vsrc = take(4 * cap);
        L.gpart = take(8 * size_t(kGroupSplit) * 2 * kGroupPairs * n);
        L.gsum = take(8 * 2 * kGroupPairs * n);
        L.gtol = take(8 * kGroupPairs * n);
        L.gsc = take(8 * size_t(kGroupSplit) * 2 * n);
        L.gstate = take(4 * n);
    }
    L.end = o;
    return L;
}

// Typed pointers into a workspace laid out by layout(n, cap, group).
Work make_work(char* base, const Layout& L, int64_t n, int64_t cap, int nb, bool group, int nff)
{
    Work w{};
    w.batches = reinterpret_cast<DevBatch*>(base + L.batches);
    w.nb = nb;
    w.n = n;
    w.cap = cap;
    w.totals = reinterpret_cast<RoundTotals*>(base + L.totals);
    w.ls = reinterpret_cast<LoopState*>(base + L.ls);
    w.trig = reinterpret_cast<QTrig*>(base + L.trig);
    w.meta = reinterpret_cast<uint32_t*>(base + L.meta);
    w.born = reinterpret_cast<uint32_t*>(base + L.born);
    w.seg_base = reinterpret_cast<uint32_t*>(base + L.seg_base);
    w.seg_count = reinterpret_cast<uint32_t*>(base + L.seg_count);
    w.active[0] = reinterpret_cast<uint32_t*>(base + L.active0);
    w.active[1] = reinterpret_cast<uint32_t*>(base + L.active1);
    w.cnt_new = reinterpret_cast<uint32_t*>(base + L.cnt_new);
    w.cnt_eval = reinterpret_cast<uint32_t*>(base + L.cnt_eval);
    w.thr = reinterpret_cast<uint2*>(base + L.thr);
    w.pre_pool = reinterpret_cast<unsigned long long*>(base + L.pre_pool);
    w.pre_eval = reinterpret_cast<unsigned long long*>(base + L.pre_eval);
    w.pre_act = reinterpret_cast<uint32_t*>(base + L.pre_act);
    w.blk_pool = reinterpret_cast<unsigned long long*>(base + L.blk_pool);
    w.blk_eval = reinterpret_cast<unsigned long long*>(base + L.blk_eval);
    w.blk_act = reinterpret_cast<uint32_t*>(base + L.blk_act);
    w.key[0] = reinterpret_cast<uint64_t*>(base + L.key0);
    w.key[1] = reinterpret_cast<uint64_t*>(base + L.key1);
    w.val[0] = reinterpret_cast<double*>(base + L.val0);
    w.val[1] = reinterpret_cast<double*>(base + L.val1);
    w.err[0] = reinterpret_cast<double*>(base + L.err0);
    w.err[1] = reinterpret_cast<double*>(base + L.err1);
    w.nse[0] = reinterpret_cast<float*>(base + L.nse0);
    w.nse[1] = reinterpret_cast<float*>(base + L.nse1);
    w.evl = reinterpret_cast<uint2*>(base + L.evl);
    if (group) {
        w.vval[0] = reinterpret_cast<double*>(base + L.vval0);
        w.vval[1] = reinterpret_cast<double*>(base + L.vval1);
        w.verr[0] = reinterpret_cast<float*>(base + L.verr0);
        w.verr[1] = reinterpret_cast<float*>(base + L.verr1);
        w.vsrc = reinterpret_cast<uint32_t*>(base + L.vsrc);
        w.gpart = reinterpret_cast<double*>(base + L.gpart);
        w.gsum = reinterpret_cast<double*>(base + L.gsum);
        w.gtol = reinterpret_cast<double*>(base + L.gtol);
        w.gsc = reinterpret_cast<double*>(base + L.gsc);
        w.gstate = reinterpret_cast<int*>(base + L.gstate);
        w.vstride = kGroupPairs;
    }
    w.nff = nff;
    return w;
}

// The largest pool capacity whose layout fits in ws_bytes.
int64_t capacity_for(int64_t n, size_t ws_bytes, bool group)
{
    const size_t fixed = layout(n, 0, group).end;
    // 64 bytes per region (7 arrays of 8 bytes, 2 of 4; group mode: + 2 x 81 x 12
    // for the pair vectors + 4) plus up to 14 * 256 bytes of alignment
    const size_t per = 64 + (group ? 2 * 12 * kGroupPairs + 4 : 0);
    int64_t cap = ws_bytes > fixed + 14 * 256 ? int64_t((ws_bytes - fixed - 14 * 256) / per) : 0;
    cap = std::min(cap, kMaxCapacity);
    while (cap > 0 && layout(n, cap, group).end > ws_bytes) --cap;
    // the estimate above reserves worst-case alignment; take what still fits
    while (cap < kMaxCapacity && layout(n, cap + 1, group).end <= ws_bytes) ++cap;
    return cap;
}

int settle(paid_ctx* ctx, bool no_alloc);

int fail(paid_ctx* ctx, int rc, const std::string& msg)
{
    if (ctx) ctx->last_error = msg;
    return rc;
}

int cuda_fail(paid_ctx* ctx, cudaError_t e, const char* where)
{
    return fail(ctx, PAID_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool is_finite_d(double x) { return std::isfinite(x); }

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) { if (cudaGetDevice(&prev) != cudaSuccess) prev = -1; cudaSetDevice(dev); }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

int check_options(const paid_options& o, std::string& why)
{
    const bool high = o.rule_n == 8 || o.rule_n == 10 || o.rule_n == 12;
    if (o.rule_n != 4 && o.rule_n != 6 && !(high && o.group_mode)) {
        why = "rule_n must be 4 or 6 (or 8, 10, 12 with group_mode)";
        return PAID_ERR_ARG;
    }
    if (o.init_level < 0 || o.init_level > 8) { why = "init_level must be in 0..8"; return PAID_ERR_ARG; }
    if (o.eval_fp32 != 0 && o.eval_fp32 != 1) { why = "eval_fp32 must be 0 or 1"; return PAID_ERR_ARG; }
    if (o.max_rounds < 1) { why = "max_rounds must be >= 1"; return PAID_ERR_ARG; }
    if (!(o.cover >= 0.0 && o.cover <= 1.0)) { why = "cover must be in [0, 1]"; return PAID_ERR_ARG; }
    if (o.pool_capacity < 0) { why = "pool_capacity must be >= 0"; return PAID_ERR_ARG; }
    if (o.timing != 0 && o.timing != 1) { why = "timing must be 0 or 1"; return PAID_ERR_ARG; }
    if (o.device_loop != 0 && o.device_loop != 1) { why = "device_loop must be 0 or 1"; return PAID_ERR_ARG; }
    if (o.group_mode < 0 || o.group_mode > 2) { why = "group_mode must be 0, 1 or 2"; return PAID_ERR_ARG; }
    if (o.eval_blocks < 0) { why = "eval_blocks must be >= 0"; return PAID_ERR_ARG; }
    if (o.trace != 0 && o.trace != 1) { why = "trace must be 0 or 1"; return PAID_ERR_ARG; }
    return PAID_OK;
}

}  // namespace

extern "C" {

int paid_options_default(paid_options* opt)
{
    if (!opt) return PAID_ERR_ARG;
    opt->rule_n = 4;
    opt->init_level = 2;
    opt->eval_fp32 = 0;
    opt->max_rounds = 4096;
    opt->cover = 0.5;
    opt->pool_capacity = 0;
    opt->timing = 0;
    opt->device_loop = 1;
    opt->group_mode = 0;
    opt->eval_blocks = 0;
    opt->trace = 0;
    return PAID_OK;
}

const char* paid_error_string(int rc)
{
    switch (rc) {
    case PAID_OK: return "ok";
    case PAID_ERR_ARG: return "invalid argument";
    case PAID_ERR_OOM: return "workspace too small";
    case PAID_ERR_CUDA: return "CUDA error";
    case PAID_ERR_POOL: return "region pool full";
    case PAID_ERR_TIMEOUT: return "round cap reached";
    default: return "unknown error";
    }
}

const char* paid_last_error(paid_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int paid_create(paid_ctx** out, double t, double tp, double mu, int ffset,
                const paid_options* opt, int device)
{
    if (!out) return PAID_ERR_ARG;
    *out = nullptr;
    if (!is_finite_d(t) || !is_finite_d(tp) || !is_finite_d(mu)) return PAID_ERR_ARG;
    if (ffset != PAID_FF_SHELL1 && ffset != PAID_FF_SHELL12) return PAID_ERR_ARG;
    paid_options o;
    paid_options_default(&o);
    if (opt) o = *opt;
    std::string why;
    if (check_options(o, why) != PAID_OK) return PAID_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return PAID_ERR_CUDA;
    DeviceGuard guard(device);
    if (init_rule_tables(device) != cudaSuccess) return PAID_ERR_CUDA;
    paid_ctx* c = new (std::nothrow) paid_ctx();
    if (!c) return PAID_ERR_OOM;
    c->device = device;
    c->lat = Lattice{t, tp, mu};
    c->nff = ffset;
    c->opt = o;
    if (cudaMallocHost(&c->h_totals, sizeof(RoundTotals)) != cudaSuccess ||
        cudaMallocHost(&c->h_state, sizeof(LoopState)) != cudaSuccess) {
        paid_destroy(c);
        return PAID_ERR_CUDA;
    }
    for (auto& e : c->ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            paid_destroy(c);
            return PAID_ERR_CUDA;
        }
    }
    if (cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess) {
        paid_destroy(c);
        return PAID_ERR_CUDA;
    }
    *out = c;
    return PAID_OK;
}

void paid_destroy(paid_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->loop.exec) cudaGraphExecDestroy(ctx->loop.exec);
    if (ctx->loop.graph) cudaGraphDestroy(ctx->loop.graph);
    if (ctx->capture) cudaStreamDestroy(ctx->capture);
    if (ctx->h_totals) cudaFreeHost(ctx->h_totals);
    if (ctx->h_state) cudaFreeHost(ctx->h_state);
    for (auto e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->done) {
        if (ctx->pending) cudaEventSynchronize(ctx->done);
        cudaEventDestroy(ctx->done);
    }
    delete ctx;
}

int paid_workspace_size(paid_ctx* ctx, int64_t n_integrals, int64_t pool_capacity, size_t* bytes)
{
    if (!ctx || !bytes || n_integrals < 0) return fail(ctx, PAID_ERR_ARG, "bad argument");
    const int64_t n0 = int64_t(1) << (2 * ctx->opt.init_level);
    if (pool_capacity < n_integrals * n0 || pool_capacity > kMaxCapacity)
        return fail(ctx, PAID_ERR_ARG, "pool_capacity must be >= n_integrals * 4^init_level and < 2^32");
    *bytes = layout(n_integrals, pool_capacity, ctx->opt.group_mode != 0).end;
    return PAID_OK;
}

int paid_pool_capacity(paid_ctx* ctx, int64_t n_integrals, size_t ws_bytes, int64_t* capacity)
{
    if (!ctx || !capacity || n_integrals < 0) return fail(ctx, PAID_ERR_ARG, "bad argument");
    *capacity = capacity_for(n_integrals, ws_bytes, ctx->opt.group_mode != 0);
    return PAID_OK;
}

int paid_last_stats(paid_ctx* ctx, paid_stats* out)
{
    if (!ctx || !out) return PAID_ERR_ARG;
    settle(ctx, false);
    *out = ctx->stats;
    return PAID_OK;
}

int paid_wait(paid_ctx* ctx, int* call_rc)
{
    if (!ctx) return PAID_ERR_ARG;
    DeviceGuard guard(ctx->device);
    const int rc = settle(ctx, false);
    if (call_rc) *call_rc = ctx->last_rc;
    return rc;
}

}  // extern "C"

namespace {

// The per-batch argument rules shared by every integrate entry point: null
// when `b` is valid, else a static message (no allocation, so that the
// allocation-free entry point can use it too).  nl0 = 4^init_level.
const char* batch_error(const paid_batch& b, int64_t nl0, bool group)
{
    if (b.kind < PAID_PH || b.kind > PAID_FLOW_PP) return "bad kind";
    const bool flow = b.kind == PAID_FLOW_PH || b.kind == PAID_FLOW_PP;
    if (!group && flow) return "the flow kinds take group_mode = 1 or 2";
    if (flow && !(b.T > 0.0)) return "flow kinds: Omega (the T field) must be > 0";
    if (b.nq < 0 || b.npairs < 0) return "nq, npairs must be >= 0";
    const int64_t nbi = int64_t(b.nq) * b.npairs;
    if (nbi > 0 && (!b.q || !b.lm || !b.values || !b.errors || !b.regions || !b.status))
        return "null buffer";
    if (!(b.rel_tol >= 0.0) || !(b.abs_tol >= 0.0)) return "tolerances must be >= 0";
    if (b.max_regions < nl0 || b.max_regions > kMaxRegionsPerIntegral)
        return "max_regions must be in [4^init_level, 2^23]";
    if (group && b.kind == PAID_MONOMIAL) return "group_mode takes the ph, pp, overlap and flow kinds";
    if (group && b.npairs > kGroupPairs) return "group_mode takes at most 81 pairs per batch";
    const bool tu = b.tu_v[0] || b.tu_v[1] || b.tu_out[0] || b.tu_out[1];
    if (tu) {
        if (!group || !flow) return "truncated-unity products take the flow kinds in group_mode";
        const bool pp = b.kind == PAID_FLOW_PP;
        if (!b.tu_v[0] || !b.tu_out[0] || (pp ? (b.tu_v[1] || b.tu_out[1])
                                              : (!b.tu_v[1] || !b.tu_out[1])))
            return "truncated-unity products: flow pp takes tu_v[0], tu_out[0]; flow ph all four";
    }
    return nullptr;
}

// Validates the batches, sizes the pool, lays out the workspace and uploads
// the batch table.  n0 = regions per integral that the start needs at least.
int prepare(paid_ctx* ctx, const paid_batch* batches, int nb, void* workspace, size_t ws_bytes,
            int64_t n0, cudaStream_t s, Work& w, int64_t& n, int64_t& cap, bool group)
{
    // an earlier asynchronous call on this context completes first: its loop
    // state and the graph are shared with this call
    settle(ctx, false);
    ctx->last_error.clear();
    ctx->stats = paid_stats{};
    if (nb < 0 || nb > kMaxBatches || (nb > 0 && !batches))
        return fail(ctx, PAID_ERR_ARG, "nb must be in 0..4096 with a batch array");
    const paid_options& o = ctx->opt;
    const int64_t nl0 = int64_t(1) << (2 * o.init_level);
    std::vector<DevBatch> hb;
    hb.reserve(nb);
    n = 0;
    int64_t n_int = 0;
    for (int i = 0; i < nb; ++i) {
        const paid_batch& b = batches[i];
        if (const char* why = batch_error(b, nl0, group)) return fail(ctx, PAID_ERR_ARG, why);
        const int64_t nbi = int64_t(b.nq) * b.npairs;
        if (nbi == 0) continue;
        DevBatch d{};
        d.kind = b.kind;
        d.nq = b.nq;
        d.npairs = b.npairs;
        d.T = b.T;
        d.inv2T = 1.0 / (2.0 * b.T);
        d.inv4T = 1.0 / (4.0 * b.T);
        d.rel_tol = b.rel_tol;
        d.abs_tol = b.abs_tol;
        d.max_regions = b.max_regions;
        d.first = n;   // units: integrals, or (group mode) q points
        d.ifirst = n_int;
        d.q = b.q;
        d.lm = b.lm;
        d.values = b.values;
        d.errors = b.errors;
        d.regions = b.regions;
        d.status = b.status;
        d.tu_v0 = b.tu_v[0];
        d.tu_v1 = b.tu_v[1];
        d.tu_out0 = b.tu_out[0];
        d.tu_out1 = b.tu_out[1];
        if (d.tu_out0 && int64_t(b.npairs) != int64_t(ctx->nff) * ctx->nff)
            return fail(ctx, PAID_ERR_ARG, "truncated-unity products need every pair (l, m), "
                                           "npairs = nff^2");
        hb.push_back(d);
        n += group ? int64_t(b.nq) : nbi;
        n_int += nbi;
    }
    ctx->stats.n_integrals = n_int;
    if (n == 0) return PAID_OK;
    if (n > int64_t(0x7fffffff)) return fail(ctx, PAID_ERR_ARG, "too many integrals");
    if (!workspace) return fail(ctx, PAID_ERR_ARG, "null workspace");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
        return fail(ctx, PAID_ERR_ARG, "workspace must be 256-byte aligned");
    cap = capacity_for(n, ws_bytes, group);
    if (o.pool_capacity > 0) cap = std::min(cap, o.pool_capacity);
    if (cap < n * n0) return fail(ctx, PAID_ERR_OOM, "workspace too small for the initial partition");
    const bool trace = o.trace && ctx->trace_buf;
    if (trace && ctx->trace_units < n)
        return fail(ctx, PAID_ERR_ARG, "options.trace: the trace buffer (paid_set_trace_buffer) "
                                       "must hold one map per unit of the call");
    const Layout L = layout(n, cap, group);
    w = make_work(static_cast<char*>(workspace), L, n, cap, int(hb.size()), group, ctx->nff);
    w.gglobal = group && ctx->opt.group_mode == 2;
    bool any_flow = false, any_other = false;
    for (const DevBatch& d : hb) (is_flow(d.kind) ? any_flow : any_other) = true;
    w.kinds = any_flow && any_other ? 0 : (any_flow ? 2 : 1);
    cudaError_t e = cudaMemcpyAsync(w.batches, hb.data(), sizeof(DevBatch) * hb.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch upload");
    if (trace) {
        // NaN in every cell of a unit that never runs (0xffffffff is a NaN)
        w.tmap = ctx->trace_buf;
        if ((e = cudaMemsetAsync(w.tmap, 0xff, sizeof(float) * 256 * size_t(n), s)) != cudaSuccess)
            return cuda_fail(ctx, e, "trace init");
    }
    return PAID_OK;
}

// Kernels of one round: evaluation, reduce + test + selection, scan,
// throttle and rescan (both no-ops while the next pool fits), split, control;
// inside the graph also the admission wave that control chose.  `hint_*`
// size the grids (exact counts in the host loop, bounds in the graph).  `ev`
// (host loop with timing) gets marks between the kernel classes.
cudaError_t launch_round(paid_ctx* ctx, const Work& w, int64_t hint_eval, int64_t hint_active,
                         int64_t hint_pool, cudaGraphConditionalHandle h, int in_graph,
                         cudaStream_t s, cudaEvent_t* ev)
{
    const paid_options& o = ctx->opt;
    auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], s) : cudaSuccess; };
    cudaError_t e;
    const bool group = w.vstride > 0;
    if ((e = mark(0)) != cudaSuccess ||
        (e = group ? launch_eval_group(w, hint_eval, o.rule_n, o.eval_fp32, ctx->lat, s, nullptr,
                                       nullptr, o.eval_blocks)
                   : launch_eval(w, hint_eval, o.rule_n, o.eval_fp32, ctx->lat, s,
                                 ev && o.eval_fp32 ? ev[6] : nullptr)) != cudaSuccess ||
        (e = mark(1)) != cudaSuccess ||
        (e = group ? launch_reduce_group(w, hint_active, o.max_rounds, o.cover, s)
                   : launch_reduce_test(w, hint_active, o.max_rounds, o.cover, s)) != cudaSuccess ||
        (e = launch_trace(w, hint_active, s)) != cudaSuccess ||
        (e = mark(2)) != cudaSuccess ||
        (e = launch_scan(w, hint_active, 0, s)) != cudaSuccess ||
        (e = launch_throttle(w, hint_active, s)) != cudaSuccess ||
        (e = launch_scan(w, hint_active, 1, s)) != cudaSuccess ||
        (e = mark(3)) != cudaSuccess ||
        (e = launch_split(w, hint_active, s)) != cudaSuccess ||
        (e = launch_copy_vectors(w, hint_pool, s)) != cudaSuccess ||
        (e = mark(4)) != cudaSuccess ||
        (e = launch_control(w, h, in_graph, s)) != cudaSuccess)
        return e;
    if (in_graph) e = launch_setup_wave(w, hint_active, ctx->nff, o.eval_fp32 ? 0 : 1, s);
    return e;
}

// kernels one round launches (graph: every node; host loop: those with work)
int64_t round_kernels(const paid_options& o, int64_t n_eval, int64_t n_active, bool in_graph)
{
    const int64_t ev = n_eval > 0 ? (o.eval_fp32 && !o.group_mode ? 2 : 1) : 0;
    const int64_t slots = n_active > 0 ? 1 : 0;
    // eval, reduce (group: 4), scan (2), throttle, rescan (2), split, [vector copy], control,
    // [wave]
    return ev + (o.group_mode ? 4 : 1) * slots + (o.trace ? slots : 0) + (slots + 1) + slots +
           (slots + 1) + slots + (o.group_mode ? slots : 0) + 1 + (in_graph ? 1 : 0);
}

// The device-loop graph for this workspace layout and these options:
// WHILE (condition) { one round }, the condition cleared by k_control.
int loop_graph(paid_ctx* ctx, const Work& w, cudaGraphExec_t* out)
{
    const paid_options& o = ctx->opt;
    LoopGraph& G = ctx->loop;
    if (G.exec && G.base == w.batches && G.n == w.n && G.cap == w.cap && G.nb == w.nb &&
        G.vstride == w.vstride &&
        G.rule_n == o.rule_n && G.eval_fp32 == o.eval_fp32 && G.max_rounds == o.max_rounds &&
        G.eval_blocks == o.eval_blocks && G.tmap == w.tmap && G.kinds == w.kinds &&
        G.cover == o.cover) {
        *out = G.exec;
        return PAID_OK;
    }
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G = LoopGraph{};
    cudaError_t e;
    if (!ctx->capture &&
        (e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(ctx, e, "capture stream");
    cudaGraph_t g = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return cuda_fail(ctx, e, "graph");
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams np{};
    cudaGraphNode_t node;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "graph condition");
    }
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "graph while node");
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(ctx->capture, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "graph capture");
    }
    const cudaError_t el = launch_round(ctx, w, w.cap, w.n, w.cap, h, 1, ctx->capture, nullptr);
    cudaGraph_t captured = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->capture, &captured);
    if (el != cudaSuccess || ec != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, el != cudaSuccess ? el : ec, "graph capture");
    }
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaGraphInstantiate(&exec, g, 0)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "graph instantiate");
    }
    G.graph = g;
    G.exec = exec;
    G.base = w.batches;
    G.n = w.n;
    G.cap = w.cap;
    G.nb = w.nb;
    G.vstride = w.vstride;
    G.rule_n = o.rule_n;
    G.eval_fp32 = o.eval_fp32;
    G.max_rounds = o.max_rounds;
    G.eval_blocks = o.eval_blocks;
    G.tmap = w.tmap;
    G.kinds = w.kinds;
    G.cover = o.cover;
    *out = exec;
    return PAID_OK;
}

// Statistics and return code of a finished loop from its final state.
int loop_outcome(paid_ctx* ctx, const LoopState& L, const RoundTotals& t, int64_t cap,
                 bool no_alloc)
{
    const paid_options& o = ctx->opt;
    paid_stats& st = ctx->stats;
    st.rounds = L.rounds_done;
    st.region_evals = L.region_evals;
    st.peak_pool = L.peak_pool;
    st.throttled_rounds = L.throttled_rounds;
    st.escalated = int64_t(t.escalated);
    st.df_regions = int64_t(t.df_regions);
    st.node_evals = st.region_evals * int64_t(2 * o.rule_n + 1) * (2 * o.rule_n + 1);
    st.pool_capacity = cap;
    if (st.graph_launches) {
        st.launches += int64_t(L.rounds_done) * round_kernels(o, 1, 1, true);
        st.eval_launches += L.rounds_done;
    }
    // (the allocation-free entry point keeps the message alone: no strings)
    auto rfail = [&](int rc, const char* msg) { return no_alloc ? rc : fail(ctx, rc, msg); };
    switch (L.stop) {
    case kDone:
        return t.roundcap > 0 ? rfail(PAID_ERR_TIMEOUT, "round cap reached") : int(PAID_OK);
    case kStuck:
        if (no_alloc) return PAID_ERR_POOL;
        return fail(ctx, PAID_ERR_POOL, "region pool full (capacity " + std::to_string(cap) + ")");
    case kNoRoom:
        return rfail(PAID_ERR_POOL, "region pool too small for one integral's start");
    case kHardCap:
        return rfail(PAID_ERR_TIMEOUT, "round cap reached");
    default:
        return rfail(PAID_ERR_CUDA, "device loop ended without a stop decision");
    }
}

// Completes an asynchronous call still pending on ctx: waits for its final
// loop state, then records its statistics and outcome (ctx->last_rc).
int settle(paid_ctx* ctx, bool no_alloc)
{
    if (!ctx->pending) return PAID_OK;
    ctx->pending = false;
    const cudaError_t e = cudaEventSynchronize(ctx->done);
    if (e != cudaSuccess) {
        ctx->last_rc = no_alloc ? int(PAID_ERR_CUDA) : cuda_fail(ctx, e, "device loop");
        return ctx->last_rc;
    }
    const LoopState L = *ctx->h_state;
    const RoundTotals t = *ctx->h_totals;
    ctx->last_rc = loop_outcome(ctx, L, t, ctx->pend_cap, no_alloc);
    return PAID_OK;
}

// The refinement loop of Listing 5 from a partition already on the eval list.
// Integrals [0, admitted) are in the pool; with L0 >= 0 the rest are admitted
// (uniform level-L0 start) as room frees up.  In a round whose splits would
// overflow the pool, integrals split in slot order while the growth fits and
// the rest wait a round unsplit; only a round that can neither grow nor
// retire anything ends the call with PAID_ERR_POOL.  With the device loop the
// call only queues its work and returns (paid_wait reads the outcome);
// no_alloc = true (the allocation-free entry point) keeps the loop on the
// host, since building a graph allocates, and leaves the error message alone.
int run_loop(paid_ctx* ctx, const Work& w, int64_t admitted, int64_t n_eval, int64_t pool, int L0,
             cudaStream_t s, bool no_alloc = false)
{
    const paid_options& o = ctx->opt;
    const int64_t n = w.n, cap = w.cap;
    const bool timed = o.timing != 0;
    const bool graph = !no_alloc && o.device_loop != 0 && !timed;
    auto cfail = [&](cudaError_t e, const char* where) {
        return no_alloc ? int(PAID_ERR_CUDA) : cuda_fail(ctx, e, where);
    };
    // the loop's own bound: every integral has at most max_rounds rounds from
    // its admission; streaming admission spreads them over more rounds
    const int hard = admitted >= n ? o.max_rounds
                                   : int(std::min<int64_t>(int64_t(o.max_rounds) * 64, 1 << 30));
    paid_stats& st = ctx->stats;
    cudaEvent_t* ev = ctx->ev;
    auto span = [&](int a, int b) {
        float ms = 0.f;
        return cudaEventElapsedTime(&ms, ev[a], ev[b]) == cudaSuccess ? double(ms) : 0.0;
    };
    auto read_state = [&](LoopState& L, RoundTotals& t) -> cudaError_t {
        cudaError_t r = cudaMemcpyAsync(ctx->h_state, w.ls, sizeof(LoopState),
                                        cudaMemcpyDeviceToHost, s);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(ctx->h_totals, w.totals, sizeof(RoundTotals),
                                cudaMemcpyDeviceToHost, s);
        if (r == cudaSuccess) r = cudaStreamSynchronize(s);
        L = *ctx->h_state;
        t = *ctx->h_totals;
        return r;
    };
    cudaError_t e;
    if ((e = launch_state_init(w, admitted, n_eval, pool, admitted, L0, hard, s)) != cudaSuccess)
        return cfail(e, "loop state");
    st.launches += 1;
    LoopState L{};
    RoundTotals t{};
    if (graph) {
        // asynchronous: the loop, the device-decided finish and the copy of the
        // final loop state are queued; paid_wait reads the outcome
        cudaGraphExec_t exec = nullptr;
        const int rc = loop_graph(ctx, w, &exec);
        if (rc != PAID_OK) return rc;
        if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return cfail(e, "graph launch");
        if ((e = launch_finish_device(w, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ctx->h_state, w.ls, sizeof(LoopState), cudaMemcpyDeviceToHost,
                                 s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ctx->h_totals, w.totals, sizeof(RoundTotals),
                                 cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaEventRecord(ctx->done, s)) != cudaSuccess)
            return cfail(e, "device loop");
        st.graph_launches = 1;
        st.launches += w.vstride > 0 ? 3 : 2;
        ctx->pending = true;
        ctx->pend_n = n;
        ctx->pend_cap = cap;
        return PAID_OK;
    }
    L.n_eval = n_eval;
    L.n_active = admitted;
    for (;;) {
        const int64_t ne = L.n_eval, na = L.n_active;
        if ((e = launch_round(ctx, w, ne, na, o.group_mode ? w.cap : 0, 0, 0, s,
                              timed ? ev : nullptr)) != cudaSuccess)
            return cfail(e, "round");
        st.launches += round_kernels(o, ne, na, false);
        st.eval_launches += ne > 0 ? 1 : 0;
        if ((e = read_state(L, t)) != cudaSuccess) return cfail(e, "round sync");
        if (timed) {
            st.eval_ms += span(0, 1);
            if (o.eval_fp32 && !o.group_mode && ne > 0) st.df_ms += span(6, 1);
            st.reduce_ms += span(1, 2);
            st.scan_ms += span(2, 3);
            st.split_ms += span(3, 4);
        }
        if (L.stop != kRunning) break;
        if (L.wave_g1 > L.wave_g0) {
            if ((e = launch_setup_wave(w, L.wave_g1 - L.wave_g0, ctx->nff, o.eval_fp32 ? 0 : 1,
                                       s)) != cudaSuccess)
                return cfail(e, "admit");
            st.launches += 1;
        }
    }
    switch (L.stop) {
    case kStuck:
        if ((e = launch_finalize(w, L.n_active, POOL, s)) != cudaSuccess ||
            (e = launch_mark_unadmitted(w, L.admitted, n, POOL, s)) != cudaSuccess)
            return cfail(e, "finalize");
        st.launches += 2;
        break;
    case kNoRoom:
        if ((e = launch_mark_unadmitted(w, L.admitted, n, POOL, s)) != cudaSuccess)
            return cfail(e, "finalize");
        st.launches += 1;
        break;
    case kHardCap:
        if ((e = launch_mark_unadmitted(w, L.admitted, n, ROUNDCAP, s)) != cudaSuccess)
            return cfail(e, "finalize");
        st.launches += 1;
        break;
    default:
        break;
    }
    if (L.stop != kDone && (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cfail(e, "finalize sync");
    ctx->last_rc = loop_outcome(ctx, L, t, cap, no_alloc);
    return ctx->last_rc;
}

}  // namespace

extern "C" {

int paid_integrate_multi(paid_ctx* ctx, const paid_batch* batches, int nb, void* workspace,
                         size_t ws_bytes, void* stream)
{
    if (!ctx) return PAID_ERR_ARG;
    const paid_options& o = ctx->opt;
    const int64_t n0 = int64_t(1) << (2 * o.init_level);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGuard guard(ctx->device);
    Work w{};
    int64_t n = 0, cap = 0;
    int rc = prepare(ctx, batches, nb, workspace, ws_bytes, 1, s, w, n, cap, o.group_mode != 0);
    if (rc != PAID_OK || n == 0) return rc;
    if (cap < n0) return fail(ctx, PAID_ERR_OOM, "workspace too small for one integral's start");
    // first admission: as many integrals as the pool can take at ~16k regions
    // each (all of them when the pool is large), the rest stream in later
    int64_t a = std::max<int64_t>(1, std::min(n, cap / (2 * std::max<int64_t>(16384, 16 * n0))));
    a = std::min(a, cap / n0);
    cudaError_t e;
    if ((e = launch_setup(w, o.init_level, ctx->nff, o.eval_fp32 ? 0 : 1, s, 0, a)) != cudaSuccess)
        return cuda_fail(ctx, e, "setup");
    ctx->stats.launches = 1;
    return run_loop(ctx, w, a, a * n0, a * n0, o.init_level, s);
}

int paid_integrate_multi_seeded(paid_ctx* ctx, const paid_batch* batches, int nb,
                                const float* proposal, double margin, void* workspace,
                                size_t ws_bytes, void* stream)
{
    if (!ctx) return PAID_ERR_ARG;
    if (!std::isfinite(margin)) return fail(ctx, PAID_ERR_ARG, "margin must be finite");
    const paid_options& o = ctx->opt;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGuard guard(ctx->device);
    Work w{};
    int64_t n = 0, cap = 0;
    const bool group = o.group_mode != 0;
    int rc = prepare(ctx, batches, nb, workspace, ws_bytes, 16, s, w, n, cap, group);
    if (rc != PAID_OK || n == 0) return rc;
    cudaError_t e;
    // the slot scan reads its slot count from the loop state
    if ((e = launch_setup(w, -1, ctx->nff, o.eval_fp32 ? 0 : 1, s)) != cudaSuccess ||
        (e = launch_state_init(w, n, 0, 0, n, -1, o.max_rounds, s)) != cudaSuccess ||
        (e = launch_seed(w, proposal, margin, 0, s)) != cudaSuccess ||
        (e = launch_scan(w, n, 0, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "seed");
    if ((e = cudaMemcpyAsync(ctx->h_totals, w.totals, sizeof(RoundTotals), cudaMemcpyDeviceToHost,
                             s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(ctx, e, "seed totals");
    const RoundTotals t = *ctx->h_totals;
    if (int64_t(t.pool) > cap)
        return fail(ctx, PAID_ERR_OOM, "workspace too small for the seeded partition");
    if ((e = launch_seed(w, proposal, margin, 1, s)) != cudaSuccess) return cuda_fail(ctx, e, "seed");
    ctx->stats.launches = 6;   // setup, state, seed (count), scan (blocks, top), seed (write)
    return run_loop(ctx, w, n, int64_t(t.eval), int64_t(t.pool), -1, s);
}

int paid_set_trace_buffer(paid_ctx* ctx, float* maps, int64_t n_units)
{
    if (!ctx || n_units < 0 || (n_units > 0 && !maps)) return PAID_ERR_ARG;
    ctx->trace_buf = n_units > 0 ? maps : nullptr;
    ctx->trace_units = n_units;
    return PAID_OK;
}

int paid_mlp_group_features(paid_ctx* ctx, int kind, int nq, const double* q, double T,
                            uint16_t* x, void* stream)
{
    if (!ctx || nq < 0) return PAID_ERR_ARG;
    if (nq > 0 && (!q || !x)) return PAID_ERR_ARG;
    DeviceGuard guard(ctx->device);
    return launch_features(kind, nq, q, 1, nullptr, T, ctx->lat.mu, ctx->lat.tp, x,
                           static_cast<cudaStream_t>(stream)) == cudaSuccess ? PAID_OK : PAID_ERR_CUDA;
}

int paid_cell_errors(paid_ctx* ctx, int kind, int nq, const double* q, int npairs,
                     const int32_t* lm, double T, float* out, void* workspace, size_t ws_bytes,
                     void* stream)
{
    if (!ctx) return PAID_ERR_ARG;
    if (int64_t(nq) * npairs > 0 && !out) return fail(ctx, PAID_ERR_ARG, "null output");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGuard guard(ctx->device);
    // One pass over the uniform level-4 grid, no refinement round: no integral
    // is finalised, so values / errors / regions are never written.  The setup
    // kernel marks every integral RUNNING in `status`; that array is aimed at
    // `out`, which k_cell_map then overwrites in full on the same stream.
    paid_batch b{};
    b.kind = kind;
    b.T = T;
    b.nq = nq;
    b.q = q;
    b.npairs = npairs;
    b.lm = lm;
    b.rel_tol = 0.0;
    b.abs_tol = 0.0;
    b.max_regions = 256;
    b.values = reinterpret_cast<double*>(out);
    b.errors = reinterpret_cast<double*>(out);
    b.regions = reinterpret_cast<int64_t*>(out);
    b.status = reinterpret_cast<int32_t*>(out);
    Work w{};
    int64_t n = 0, cap = 0;
    int rc = prepare(ctx, &b, 1, workspace, ws_bytes, 256, s, w, n, cap, false);
    if (rc != PAID_OK || n == 0) return rc;
    cudaError_t e;
    if ((e = launch_setup(w, 4, ctx->nff, 1, s)) != cudaSuccess ||
        (e = launch_state_init(w, n, n * 256, n * 256, n, 4, 1, s)) != cudaSuccess ||
        (e = launch_eval(w, n * 256, std::min(ctx->opt.rule_n, kMaxRuleNLow), 0, ctx->lat, s)) !=
            cudaSuccess ||
        (e = launch_cell_map(w, out, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "cell errors");
    ctx->stats.region_evals = n * 256;
    return PAID_OK;
}

int paid_rule_regions(paid_ctx* ctx, int kind, double T, const double* q, int npairs,
                      const int32_t* lm, int nreg, const int32_t* regions, double* q2N, double* dq,
                      void* workspace, size_t ws_bytes, void* stream)
{
    if (!ctx) return PAID_ERR_ARG;
    ctx->last_error.clear();
    if (kind != PAID_PH && kind != PAID_PP && kind != PAID_OVERLAP && kind != PAID_FLOW_PH &&
        kind != PAID_FLOW_PP)
        return fail(ctx, PAID_ERR_ARG, "kind must be ph, pp, overlap, flow ph or flow pp");
    if (npairs < 1 || npairs > kGroupPairs || nreg < 0)
        return fail(ctx, PAID_ERR_ARG, "npairs must be in 1..81 and nreg >= 0");
    if (!(T > 0.0) || !is_finite_d(T)) return fail(ctx, PAID_ERR_ARG, "T must be > 0");
    if (nreg == 0) return PAID_OK;
    if (!q || !lm || !regions || !q2N || !dq || !workspace)
        return fail(ctx, PAID_ERR_ARG, "null pointer");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
        return fail(ctx, PAID_ERR_ARG, "workspace must be 256-byte aligned");
    const Layout Lw = layout(1, nreg, false);
    if (Lw.end > ws_bytes) return fail(ctx, PAID_ERR_OOM, "workspace too small");
    DeviceGuard guard(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Work w = make_work(static_cast<char*>(workspace), Lw, 1, nreg, 1, false, ctx->nff);
    w.kinds = is_flow(kind) ? 2 : 1;
    DevBatch d{};
    d.kind = kind;
    d.nq = 1;
    d.npairs = npairs;
    d.T = T;
    d.inv2T = 1.0 / (2.0 * T);
    d.inv4T = 1.0 / (4.0 * T);
    d.max_regions = nreg;
    d.q = q;
    d.lm = lm;
    uint32_t* bad = reinterpret_cast<uint32_t*>(w.nse[1]);   // one flag per region
    cudaError_t e;
    if ((e = cudaMemcpyAsync(w.batches, &d, sizeof(DevBatch), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = launch_rule_setup(w, kind, q, regions, nreg, bad, s)) != cudaSuccess ||
        (e = launch_state_init(w, 1, nreg, nreg, 1, 0, 1, s)) != cudaSuccess ||
        (e = launch_eval_group(w, nreg, ctx->opt.rule_n, ctx->opt.eval_fp32, ctx->lat, s, q2N,
                               dq)) != cudaSuccess ||
        (e = launch_rule_flag(bad, nreg, npairs, q2N, dq, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "rule regions");
    // like the integrate calls, return with the outputs complete
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(ctx, e, "rule regions");
    return PAID_OK;
}

int paid_check_math(paid_ctx* ctx, int which, int64_t n, const double* x, const double* y,
                    double* out, void* stream)
{
    if (!ctx || which < 0 || which > 6 || n < 0) return PAID_ERR_ARG;
    if (n > 0 && (!x || !out || (which != 0 && which != 2 && !y))) return PAID_ERR_ARG;
    DeviceGuard guard(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_check_math(which, n, x, y, out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? PAID_OK : cuda_fail(ctx, e, "check math");
}

int paid_get_options(paid_ctx* ctx, paid_options* out)
{
    if (!ctx || !out) return PAID_ERR_ARG;
    *out = ctx->opt;
    return PAID_OK;
}

}  // extern "C"

namespace {

// Autotuner cache: JSON Lines, one object per tuned configuration,
//   {"key": "<device>|eval_fp32=0|group_mode=1", "rule_n": 6, "cover": 1, "eval_blocks": 608,
//    "ms": 9.1}
std::string tune_key(const paid_ctx* ctx)
{
    cudaDeviceProp prop{};
    std::string dev = cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess ? prop.name : "?";
    for (char& c : dev)
        if (c == '"' || c == '\\') c = '_';
    const paid_options& o = ctx->opt;
    return dev + "|eval_fp32=" + std::to_string(o.eval_fp32) + "|group_mode=" +
           std::to_string(o.group_mode);
}

std::vector<std::string> read_lines(const char* path)
{
    std::vector<std::string> lines;
    FILE* f = std::fopen(path, "r");
    if (!f) return lines;
    char buf[1024];
    while (std::fgets(buf, sizeof(buf), f)) {
        std::string l(buf);
        while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
        if (!l.empty()) lines.push_back(l);
    }
    std::fclose(f);
    return lines;
}

bool cached_choice(const char* path, const std::string& key, int& rule_n, double& cover,
                   int& blocks, int& init_level)
{
    const std::string tag = "\"key\": \"" + key + "\"";
    for (const std::string& l : read_lines(path)) {
        if (l.find(tag) == std::string::npos) continue;
        const size_t pr = l.find("\"rule_n\": "), pc = l.find("\"cover\": "),
                     pb = l.find("\"eval_blocks\": ");
        if (pr == std::string::npos || pc == std::string::npos || pb == std::string::npos)
            continue;
        int r = 0, b = 0;
        double c = 0.0;
        if (std::sscanf(l.c_str() + pr + 10, "%d", &r) != 1 ||
            std::sscanf(l.c_str() + pc + 9, "%lf", &c) != 1 ||
            std::sscanf(l.c_str() + pb + 15, "%d", &b) != 1)
            continue;
        if (r < 4 || r > 12 || r % 2 != 0 || !(c >= 0.0 && c <= 1.0) || b < 0) continue;
        // the start level is optional (older entries have none)
        const size_t pl = l.find("\"init_level\": ");
        int lv = init_level;
        if (pl != std::string::npos && (std::sscanf(l.c_str() + pl + 14, "%d", &lv) != 1 ||
                                        lv < 0 || lv > 8))
            continue;
        rule_n = r;
        cover = c;
        blocks = b;
        init_level = lv;
        return true;
    }
    return false;
}

void store_choice(const char* path, const std::string& key, int rule_n, double cover, int blocks,
                  int init_level, double ms)
{
    const std::string tag = "\"key\": \"" + key + "\"";
    std::vector<std::string> keep;
    for (const std::string& l : read_lines(path))
        if (l.find(tag) == std::string::npos) keep.push_back(l);
    char line[512];
    std::snprintf(line, sizeof(line),
                  "{%s, \"rule_n\": %d, \"cover\": %.17g, \"eval_blocks\": %d, "
                  "\"init_level\": %d, \"ms\": %.6g}",
                  tag.c_str(), rule_n, cover, blocks, init_level, ms);
    keep.push_back(line);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const std::string& l : keep) std::fprintf(f, "%s\n", l.c_str());
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

}  // namespace

extern "C" {

int paid_autotune(paid_ctx* ctx, const paid_batch* sample, int nb, const char* cache_path,
                  void* workspace, size_t ws_bytes, void* stream)
{
    if (!ctx) return PAID_ERR_ARG;
    const std::string key = tune_key(ctx);
    int rule_n = ctx->opt.rule_n;
    double cover = ctx->opt.cover;
    int blocks = ctx->opt.eval_blocks;
    int init_level = ctx->opt.init_level;
    if (cache_path && cached_choice(cache_path, key, rule_n, cover, blocks, init_level)) {
        ctx->opt.rule_n = rule_n;
        ctx->opt.cover = cover;
        ctx->opt.eval_blocks = blocks;
        ctx->opt.init_level = init_level;
        return PAID_OK;
    }
    if (nb <= 0 || !sample) return fail(ctx, PAID_ERR_ARG, "autotune needs a sample batch");
    DeviceGuard guard(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const paid_options saved = ctx->opt;
    ctx->opt.timing = 0;
    std::vector<int> rules = {4, 6};
    if (saved.group_mode) rules.insert(rules.end(), {8, 10, 12});
    const double covers[] = {0.5, 0.75, 0.9, 1.0};
    std::vector<int> grids = {0};
    // more blocks than fit at once (each taking one or two chunks of regions)
    // keep the SMs' blocks in different phases of the evaluation; on the flow
    // step 152 x 128 beat 152 x 32 by 2.5 %, and a grid of resident blocks
    // only (152 x 7) lost 10 %
    if (saved.group_mode) grids = {152 * 4, 152 * 8, 152 * 32, 152 * 128};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        ctx->opt = saved;
        return fail(ctx, PAID_ERR_CUDA, "autotune events");
    }
    double best_ms = 1e300, best_cover = saved.cover;
    int best_blocks = saved.eval_blocks, best_rule = saved.rule_n, best_level = saved.init_level;
    bool warm = false;
    // time one candidate; keep it when it is the fastest so far
    auto trial = [&](int rn, double c, int g, int lv) {
        ctx->opt.rule_n = rn;
        ctx->opt.cover = c;
        ctx->opt.eval_blocks = g;
        ctx->opt.init_level = lv;
        if (!warm) {   // first call: graph capture, tables, caches
            if (paid_integrate_multi(ctx, sample, nb, workspace, ws_bytes, stream) == PAID_OK)
                paid_wait(ctx, nullptr);
            warm = true;
        }
        cudaEventRecord(e0, s);
        int rc = paid_integrate_multi(ctx, sample, nb, workspace, ws_bytes, stream);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        int outcome = PAID_OK;
        if (rc == PAID_OK) rc = paid_wait(ctx, &outcome);
        if (rc != PAID_OK || outcome != PAID_OK || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            return;
        if (ms < best_ms) {
            best_ms = ms;
            best_cover = c;
            best_blocks = g;
            best_rule = rn;
            best_level = lv;
        }
    };
    // stagewise: the rule order at cover 1 and the largest grid, then cover,
    // then the grid, then the start level (the first batch of regions of every
    // unit: 16 or 64), each with the choices made so far
    const int lv0 = saved.init_level;
    for (int rn : rules) trial(rn, 1.0, grids.back(), lv0);
    const int rule_pick = best_rule;
    for (double c : covers) trial(rule_pick, c, grids.back(), lv0);
    const double cover_pick = best_cover;
    for (int g : grids) trial(rule_pick, cover_pick, g, lv0);
    const int grid_pick = best_blocks;
    for (int lv : {2, 3})
        if (lv != lv0) trial(rule_pick, cover_pick, grid_pick, lv);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->opt = saved;
    if (best_ms >= 1e300) return fail(ctx, PAID_ERR_CUDA, "autotune: no candidate completed");
    ctx->opt.rule_n = best_rule;
    ctx->opt.cover = best_cover;
    ctx->opt.eval_blocks = best_blocks;
    ctx->opt.init_level = best_level;
    if (cache_path)
        store_choice(cache_path, key, best_rule, best_cover, best_blocks, best_level, best_ms);
    return PAID_OK;
}

int paid_tu_flow_rhs(paid_ctx* ctx, int nq, int nff, const double* VP, const double* VC,
                     const double* VD, const double* Xpp, const double* Xph, double* dP,
                     double* dC, double* dD, void* stream)
{
    if (!ctx || nq < 0 || nff < 1 || nff > 9) return PAID_ERR_ARG;
    if (nq > 0 && (!VP || !VC || !VD || !Xpp || !Xph || !dP || !dC || !dD)) return PAID_ERR_ARG;
    DeviceGuard guard(ctx->device);
    const cudaError_t e = launch_tu_rhs(nq, nff, VP, VC, VD, Xpp, Xph, dP, dC, dD,
                                        static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PAID_OK : cuda_fail(ctx, e, "tu products");
}

int paid_mlp_features(paid_ctx* ctx, int kind, int nq, const double* q, int npairs,
                      const int32_t* lm, double T, uint16_t* x, void* stream)
{
    if (!ctx || nq < 0 || npairs < 0) return PAID_ERR_ARG;
    if (int64_t(nq) * npairs > 0 && (!q || !lm || !x)) return PAID_ERR_ARG;
    DeviceGuard guard(ctx->device);
    return launch_features(kind, nq, q, npairs, lm, T, ctx->lat.mu, ctx->lat.tp, x,
                           static_cast<cudaStream_t>(stream)) == cudaSuccess ? PAID_OK : PAID_ERR_CUDA;
}

int paid_integrate_batch(paid_ctx* ctx, int kind, int nq, const double* q, int npairs,
                         const int32_t* lm, double T, double rel_tol, double abs_tol,
                         int64_t max_regions, double* values, double* errors, int64_t* regions,
                         int32_t* status, void* workspace, size_t ws_bytes, void* stream)
{
    paid_batch b{};
    b.kind = kind;
    b.T = T;
    b.nq = nq;
    b.q = q;
    b.npairs = npairs;
    b.lm = lm;
    b.rel_tol = rel_tol;
    b.abs_tol = abs_tol;
    b.max_regions = max_regions;
    b.values = values;
    b.errors = errors;
    b.regions = regions;
    b.status = status;
    return paid_integrate_multi(ctx, &b, 1, workspace, ws_bytes, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of paid_integrate_batch.
//
// Some callers cannot allocate device memory at the point where they need the
// integrals: host runtimes that hand out a fixed device-memory budget at
// start-up and forbid later allocations, plug-ins that run inside another
// framework's memory manager, or real-time loops where an allocation (and the
// device-wide synchronisation cudaMalloc and cudaFree can imply) is not
// acceptable.  Such callers cannot pass a workspace either, because that
// workspace would itself have to be allocated.  For them the region pool lives
// in the file-scope array below, which is part of the library's device image:
// every GPU that loads the library holds it until the process exits.
//
// Host code must not use the array's name as an address (on the host it is a
// stand-in symbol, not device memory); its device address is looked up once
// per device with cudaGetSymbolAddress and passed to the kernels as their
// workspace.
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB
constexpr int64_t kStaticMaxIntegrals = 4096;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticScratch {
    void* ptr[64] = {};
    bool ready[64] = {};
};
StaticScratch g_static;
std::mutex g_static_mutex;

// Device address of g_static_scratch on `device` (the current device), looked
// up on the first call for that device.
cudaError_t static_scratch(int device, void** out)
{
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static.ready[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static.ptr[device] = p;
        g_static.ready[device] = true;
    }
    *out = g_static.ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int paid_integrate_batch_static(paid_ctx* ctx, int kind, int nq, const double* q,
                                           int npairs, const int32_t* lm, double T,
                                           double rel_tol, double abs_tol, int64_t max_regions,
                                           double* values, double* errors, int64_t* regions,
                                           int32_t* status, void* stream)
{
    if (!ctx) return PAID_ERR_ARG;
    const paid_options& o = ctx->opt;
    const int64_t n0 = int64_t(1) << (2 * o.init_level);
    const bool group = o.group_mode != 0;
    paid_batch b{};
    b.kind = kind;
    b.T = T;
    b.nq = nq;
    b.q = q;
    b.npairs = npairs;
    b.lm = lm;
    b.rel_tol = rel_tol;
    b.abs_tol = abs_tol;
    b.max_regions = max_regions;
    b.values = values;
    b.errors = errors;
    b.regions = regions;
    b.status = status;
    // the same argument rules as paid_integrate_batch
    if (batch_error(b, n0, group)) return PAID_ERR_ARG;
    // an earlier asynchronous call on this context completes first
    if (settle(ctx, true) != PAID_OK) return PAID_ERR_CUDA;
    const int64_t n = int64_t(nq) * npairs;
    if (n > kStaticMaxIntegrals) return PAID_ERR_ARG;
    ctx->stats = paid_stats{};
    ctx->stats.n_integrals = n;
    if (n == 0) return PAID_OK;
    const int64_t units = group ? int64_t(nq) : n;

    DeviceGuard guard(ctx->device);
    void* scratch = nullptr;
    if (static_scratch(ctx->device, &scratch) != cudaSuccess) return PAID_ERR_CUDA;
    int64_t cap = capacity_for(units, kStaticScratchBytes, group);
    if (o.pool_capacity > 0) cap = std::min(cap, o.pool_capacity);
    if (cap < units * n0) return PAID_ERR_OOM;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Layout L = layout(units, cap, group);
    char* base = static_cast<char*>(scratch);
    Work w = make_work(base, L, units, cap, 1, group, ctx->nff);
    w.gglobal = group && o.group_mode == 2;
    w.kinds = is_flow(kind) ? 2 : 1;

    // The scratch keeps whatever the previous call left in it.  Every array
    // is written before it is read within a call; the totals block is cleared
    // all the same so that no count from an earlier call can be seen.
    if (cudaMemsetAsync(w.totals, 0, sizeof(RoundTotals), s) != cudaSuccess) return PAID_ERR_CUDA;
    DevBatch d{};
    d.kind = kind;
    d.nq = nq;
    d.npairs = npairs;
    d.T = T;
    d.inv2T = 1.0 / (2.0 * T);
    d.inv4T = 1.0 / (4.0 * T);
    d.rel_tol = rel_tol;
    d.abs_tol = abs_tol;
    d.max_regions = max_regions;
    d.first = 0;
    d.q = q;
    d.lm = lm;
    d.values = values;
    d.errors = errors;
    d.regions = regions;
    d.status = status;
    if (cudaMemcpyAsync(w.batches, &d, sizeof(DevBatch), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        launch_setup(w, o.init_level, ctx->nff, o.eval_fp32 ? 0 : 1, s) != cudaSuccess)
        return PAID_ERR_CUDA;

    ctx->stats.launches = 1;
    return run_loop(ctx, w, units, units * n0, units * n0, o.init_level, s, true);
}
