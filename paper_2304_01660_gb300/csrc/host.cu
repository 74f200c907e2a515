// Host driver of libpalmad: context and workspace, the MERLIN threshold
// schedule (Algorithm 1), the pass orchestration of DRAG (Algorithms 2-4)
// and the C ABI of include/palmad.h.
//
// A pass evaluates DRAG for a set of lanes (series x length x threshold) in
// one sequence of launches.  Two schedule forms drive the passes:
//  * plain:   every DRAG call of Algorithm 1 is a one-lane pass at exactly
//             the schedule's r;
//  * batched: after the first five lengths (whose r depends on each single
//             previous result), W consecutive lengths run as one pass, each
//             at a speculative r' no larger than the schedule is expected to
//             reach.  A pass at r' yields every window with nnDist >= r'
//             exactly, so for any r >= r' the DRAG result at r is its subset
//             with nnDist >= r, and the greedy top-K at r is the prefix of the
//             top-K at r' with nnDist >= r.  The host then replays Algorithm 1
//             exactly, try by try, and reruns a length (as a one-lane pass at a
//             lower r') only when the schedule needs an r below its r'.
// Both forms return identical results.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <limits>
#include <map>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "palmad.h"
#include "palmad_dev.cuh"

using namespace palmad;

namespace {

constexpr int kDefaultCap = 1024;    // select columns past the strip triangle
constexpr double kPairFlops = 8.0;   // algorithmic FP32 flops of one recurrence-form pair evaluation
constexpr int32_t kLongWindow = 256;  // kpad above which a pass uses direct_below_long
constexpr int kRefineSeg = 1024;      // refine sweep columns per work item (multiple of 256) ...
constexpr int kRefineSegLong = 2048;  // ... and for passes with many columns (lanes x N >= kLongPass)
constexpr int64_t kLongPass = 2000000;
constexpr int kMaxLanes = 4096;      // lanes per pass
constexpr int64_t kPoolBytes = int64_t(1) << 32;  // per-chunk maxima of the refine pool (4 GiB)
constexpr int64_t kSeedBytes = int64_t(1) << 30;  // tensor-core top-row seeds of the refine sweep

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
};

// Counters zeroed per pass.
struct Small {
    int32_t work[8];
    int32_t nref;
    int32_t err;         // a bounded device wait gave up
    int32_t seed_ngroups;
    int32_t pad[5];
    unsigned long long pairs[12];
};

struct Timing {
    int kid;
    cudaEvent_t a, b;
};

// Device buffers of one lane (one length of one series).
struct LaneSet {
    int64_t cap = 0;  // windows
    DBuf<double> mu, var;
    DBuf<float4> win;
    DBuf<uint32_t> bits0, bits;
    DBuf<int32_t> surv, slot_of, scount, didx;
    DBuf<double> dnn;
};

}  // namespace

struct palmad_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int sms = 0;

    DBuf<float> T;                 // staged series (host entry points)
    DBuf<float> heat_stage;        // device heatmap of the host entry points (kept: grown on demand)
    DBuf<int64_t> count_stage;     // per-length range-discord counts of the host entry points
    DBuf<int32_t> hints;           // witness hints of the call's series (one int per point)
    std::vector<LaneSet> sets;
    // pass
    DBuf<Lane> lanes;
    DBuf<LaneState> st;
    DBuf<int32_t> chain;
    DBuf<Small> small;
    DBuf<int64_t> pidx;
    DBuf<double> pnn;
    Lane* h_lanes = nullptr;
    LaneState* h_st = nullptr;
    // finalize's own pinned mirrors: its uploads may still be in flight when
    // the next pass fills h_lanes / h_st (a pass synchronises before the
    // next finalize refills these)
    Lane* h_fin_lanes = nullptr;
    LaneState* h_fin_st = nullptr;
    int h_fin_cap = 0;
    int32_t* h_chain = nullptr;
    Small* h_small = nullptr;
    int64_t* h_pidx = nullptr;
    double* h_pnn = nullptr;
    int h_cap = 0;                 // lanes the pinned mirrors hold
    int64_t h_pick_cap = 0;
    // refine pool
    int32_t pool = 0;
    int32_t pool_kpad = 0, pool_nchunks = 0;
    DBuf<int32_t> slot_lane, slot_win, route, dlist, dlist_alt, dgroups, dead, kcnt, strip_row;
    DBuf<float> topcen, topsum, seeds;
    DBuf<int4> seed_groups;
    bool sets_dirty = false;       // a pass stopped early: slot maps may not be clean
    DBuf<float> acen, asum, cmax;
    DBuf<uint32_t> cmax2;
    DBuf<uint32_t> gmax;
    DBuf<unsigned long long> nn2;
    DBuf<int2> strips;
    DBuf<int32_t> init_flags;

    palmad_stats stats{};
    bool profile = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<Timing> timings;
    // autotuner: tuned options per workload bucket (tune_key)
    std::map<std::array<int64_t, 7>, palmad_options> tuned;
};

namespace {

palmad_status fail(palmad_ctx* c, palmad_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

#define CK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? PALMAD_ERR_OOM : PALMAD_ERR_CUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

#define CKS(expr)                                \
    do {                                         \
        palmad_status s_ = (expr);               \
        if (s_ != PALMAD_OK) return s_;          \
    } while (0)

template <class T>
palmad_status ensure(palmad_ctx* ctx, DBuf<T>& b, size_t n) {
    if (n == 0) n = 1;
    if (b.n >= n) return PALMAD_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    cudaError_t e = cudaMalloc(&b.p, n * sizeof(T));
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(ctx, PALMAD_ERR_OOM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
    }
    b.n = n;
    return PALMAD_OK;
}

template <class T>
void release(DBuf<T>& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
}

void release_set(LaneSet& s) {
    release(s.mu); release(s.var); release(s.win); release(s.bits0); release(s.bits);
    release(s.surv); release(s.slot_of); release(s.scount); release(s.didx); release(s.dnn);
    s.cap = 0;
}

// slot_of stays -1 and scount 0 between refine rounds (each round undoes
// its own entries); a fresh or reset set starts that way.
palmad_status clear_maps(palmad_ctx* ctx, LaneSet& s) {
    CK(cudaMemsetAsync(s.slot_of.p, 0xff, s.slot_of.n * sizeof(int32_t), ctx->stream));
    CK(cudaMemsetAsync(s.scount.p, 0, s.scount.n * sizeof(int32_t), ctx->stream));
    return PALMAD_OK;
}

palmad_status ensure_set(palmad_ctx* ctx, LaneSet& s, int64_t N) {
    if (s.cap >= N) return PALMAD_OK;
    const int64_t P = (N + 31) / 32, S = (N + kRefineH - 1) / kRefineH + 1;
    CKS(ensure(ctx, s.mu, N)); CKS(ensure(ctx, s.var, N)); CKS(ensure(ctx, s.win, N));
    CKS(ensure(ctx, s.bits0, P)); CKS(ensure(ctx, s.bits, P));
    CKS(ensure(ctx, s.surv, N)); CKS(ensure(ctx, s.slot_of, N)); CKS(ensure(ctx, s.scount, S));
    CKS(ensure(ctx, s.didx, N)); CKS(ensure(ctx, s.dnn, N));
    CKS(clear_maps(ctx, s));
    s.cap = N;
    return PALMAD_OK;
}

// ------------------------------------------------------------- profiling

palmad_status tbegin(palmad_ctx* ctx, int kid, Timing& t) {
    t.kid = kid;
    t.a = t.b = nullptr;
    ctx->stats.launches[kid] += 1;
    if (!ctx->profile) return PALMAD_OK;
    for (cudaEvent_t* e : {&t.a, &t.b}) {
        if (!ctx->ev_free.empty()) {
            *e = ctx->ev_free.back();
            ctx->ev_free.pop_back();
        } else {
            CK(cudaEventCreate(e));
        }
    }
    CK(cudaEventRecord(t.a, ctx->stream));
    return PALMAD_OK;
}

palmad_status tend(palmad_ctx* ctx, Timing& t) {
    if (!ctx->profile) return PALMAD_OK;
    CK(cudaEventRecord(t.b, ctx->stream));
    ctx->timings.push_back(t);
    return PALMAD_OK;
}

void tcollect(palmad_ctx* ctx) {
    for (Timing& t : ctx->timings) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) ctx->stats.kernel_ms[t.kid] += ms;
        ctx->ev_free.push_back(t.a);
        ctx->ev_free.push_back(t.b);
    }
    ctx->timings.clear();
}

#define LAUNCH(kid, expr)                                                                     \
    do {                                                                                      \
        Timing t_;                                                                            \
        CKS(tbegin(ctx, kid, t_));                                                            \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) return fail(ctx, PALMAD_ERR_CUDA, std::string(#expr) + ": " + \
                                                                     cudaGetErrorString(e_)); \
        CKS(tend(ctx, t_));                                                                   \
    } while (0)

palmad_status sync(palmad_ctx* ctx) {
    CK(cudaStreamSynchronize(ctx->stream));
    tcollect(ctx);
    return PALMAD_OK;
}

// ------------------------------------------------------------ options

palmad_status read_options(palmad_ctx* ctx, const palmad_options* in, palmad_options& o) {
    palmad_default_options(&o);
    if (!in) return PALMAD_OK;
    if (in->struct_size != int32_t(sizeof(palmad_options)))
        return fail(ctx, PALMAD_ERR_ARG, "palmad_options.struct_size mismatch (call palmad_default_options)");
    o = *in;
    if (!(o.band_rel >= 1e-6 && o.band_rel <= 0.1)) return fail(ctx, PALMAD_ERR_ARG, "band_rel must lie in [1e-6, 0.1]");
    if (o.precision != PALMAD_PREC_FP32 && o.precision != PALMAD_PREC_MIXED)
        return fail(ctx, PALMAD_ERR_ARG, "unknown precision");
    if (o.select_cap < 0) return fail(ctx, PALMAD_ERR_ARG, "select_cap must be >= 0");
    if (o.batch_lengths < 0 || o.batch_lengths > 1024) return fail(ctx, PALMAD_ERR_ARG, "batch_lengths must lie in [0, 1024]");
    if (o.pool_slots < 0) return fail(ctx, PALMAD_ERR_ARG, "pool_slots must be >= 0");
    if (o.direct_below < 0) return fail(ctx, PALMAD_ERR_ARG, "direct_below must be >= 0");
    if (o.tc_seed_min < 0) return fail(ctx, PALMAD_ERR_ARG, "tc_seed_min must be >= 0");
    if (o.seed_rows_max < 0) return fail(ctx, PALMAD_ERR_ARG, "seed_rows_max must be >= 0");
    if (o.refine_seg != 0 && o.refine_seg != kRefineSeg && o.refine_seg != kRefineSegLong)
        return fail(ctx, PALMAD_ERR_ARG, "refine_seg must be 0, 1024 or 2048");
    if (o.knn_k < 0 || o.knn_k > kMaxKnn) return fail(ctx, PALMAD_ERR_ARG, "knn_k must lie in [0, 16]");
    if (o.no_hints != 0 && o.no_hints != 1) return fail(ctx, PALMAD_ERR_ARG, "no_hints must be 0 or 1");
    if (o.spec_scale < 0 || o.spec_scale > 400) return fail(ctx, PALMAD_ERR_ARG, "spec_scale must lie in [0, 400]");
    if (o.autotune != 0 && o.autotune != 1) return fail(ctx, PALMAD_ERR_ARG, "autotune must be 0 or 1");
    if (o.direct_below_long < 0) return fail(ctx, PALMAD_ERR_ARG, "direct_below_long must be >= 0");
    if (o.tc_group != 0 && o.tc_group != 32 && o.tc_group != 64 && o.tc_group != 128 && o.tc_group != 256)
        return fail(ctx, PALMAD_ERR_ARG, "tc_group must be 0, 32, 64, 128 or 256");
    if (o.tc_chunks < 0 || o.tc_chunks > 64) return fail(ctx, PALMAD_ERR_ARG, "tc_chunks must lie in [0, 64]");
    if (o.tc_form < 0 || o.tc_form > 2) return fail(ctx, PALMAD_ERR_ARG, "tc_form must be 0, 1 or 2");
    if (o.refine_rows != 0 && o.refine_rows != kRefineH && o.refine_rows != kRefineHTall)
        return fail(ctx, PALMAD_ERR_ARG, "refine_rows must be 0, 128 or 256");
    return PALMAD_OK;
}

// ======================================================== pass execution

struct PassLane {       // host view of one lane request
    Lane lane;
    LaneState state;    // uploaded before the pass (flags/ab carried for stats_mode 0)
};

struct PassOut {
    std::vector<LaneState> st;
    std::vector<int64_t> idx;   // [nl][K]
    std::vector<double> nn;
};

palmad_status ensure_pass(palmad_ctx* ctx, int nl, int K) {
    CKS(ensure(ctx, ctx->lanes, nl));
    CKS(ensure(ctx, ctx->st, nl));
    CKS(ensure(ctx, ctx->chain, nl));
    CKS(ensure(ctx, ctx->small, 1));
    CKS(ensure(ctx, ctx->pidx, size_t(nl) * K));
    CKS(ensure(ctx, ctx->pnn, size_t(nl) * K));
    if (ctx->h_cap < nl) {
        if (ctx->h_lanes) cudaFreeHost(ctx->h_lanes);
        if (ctx->h_st) cudaFreeHost(ctx->h_st);
        if (ctx->h_chain) cudaFreeHost(ctx->h_chain);
        ctx->h_lanes = nullptr; ctx->h_st = nullptr; ctx->h_chain = nullptr;
        const int cap = std::max(nl, 64);
        if (cudaMallocHost(&ctx->h_lanes, sizeof(Lane) * cap) != cudaSuccess ||
            cudaMallocHost(&ctx->h_st, sizeof(LaneState) * cap) != cudaSuccess ||
            cudaMallocHost(&ctx->h_chain, sizeof(int32_t) * cap) != cudaSuccess) {
            ctx->h_cap = 0;
            return fail(ctx, PALMAD_ERR_OOM, "pinned host allocation failed");
        }
        ctx->h_cap = cap;
    }
    if (ctx->h_pick_cap < int64_t(nl) * K) {
        if (ctx->h_pidx) cudaFreeHost(ctx->h_pidx);
        if (ctx->h_pnn) cudaFreeHost(ctx->h_pnn);
        ctx->h_pidx = nullptr; ctx->h_pnn = nullptr;
        const int64_t cap = std::max<int64_t>(int64_t(nl) * K, 1024);
        if (cudaMallocHost(&ctx->h_pidx, sizeof(int64_t) * cap) != cudaSuccess ||
            cudaMallocHost(&ctx->h_pnn, sizeof(double) * cap) != cudaSuccess) {
            ctx->h_pick_cap = 0;
            return fail(ctx, PALMAD_ERR_OOM, "pinned host allocation failed");
        }
        ctx->h_pick_cap = cap;
    }
    if (!ctx->h_small) {
        if (cudaMallocHost(&ctx->h_small, sizeof(Small)) != cudaSuccess)
            return fail(ctx, PALMAD_ERR_OOM, "pinned host allocation failed");
    }
    return PALMAD_OK;
}

// Refine pool: slots, each with a centred window row and a row of chunk maxima.
palmad_status ensure_pool(palmad_ctx* ctx, int32_t kpad, int32_t nchunks) {
    if (ctx->pool > 0 && kpad <= ctx->pool_kpad && nchunks <= ctx->pool_nchunks) return PALMAD_OK;
    kpad = std::max(kpad, ctx->pool_kpad);
    nchunks = std::max(nchunks, ctx->pool_nchunks);
    const int64_t ncoarse = (int64_t(nchunks) * 32 + kCoarseMin - 1) / kCoarseMin;
    int64_t slots = kPoolBytes / (int64_t(sizeof(float)) * (nchunks + ncoarse + kpad));
    slots = std::min<int64_t>(slots, 1 << 17);
    slots = std::max<int64_t>(64, (slots / 64) * 64);
    CKS(ensure(ctx, ctx->slot_lane, slots)); CKS(ensure(ctx, ctx->slot_win, slots)); CKS(ensure(ctx, ctx->route, slots));
    CKS(ensure(ctx, ctx->dlist, slots)); CKS(ensure(ctx, ctx->dlist_alt, slots));
    CKS(ensure(ctx, ctx->dgroups, slots / 64 + 1));
    CKS(ensure(ctx, ctx->dead, slots)); CKS(ensure(ctx, ctx->kcnt, slots)); CKS(ensure(ctx, ctx->asum, slots)); CKS(ensure(ctx, ctx->gmax, slots));
    CKS(ensure(ctx, ctx->nn2, slots));
    CKS(ensure(ctx, ctx->acen, size_t(slots) * kpad));
    CKS(ensure(ctx, ctx->cmax, size_t(slots) * nchunks));
    CKS(ensure(ctx, ctx->cmax2, size_t(slots) * ncoarse));
    CKS(ensure(ctx, ctx->strips, size_t(slots))); CKS(ensure(ctx, ctx->strip_row, size_t(slots)));
    ctx->pool = int32_t(slots);
    ctx->pool_kpad = kpad;
    ctx->pool_nchunks = nchunks;
    return PALMAD_OK;
}

Pass base_pass(palmad_ctx* ctx, int nl, int K, bool exclusive, const palmad_options& o) {
    Pass p{};
    p.lanes = ctx->lanes.p;
    p.st = ctx->st.p;
    p.nl = nl;
    p.K = K;
    p.exclusive = exclusive ? 1 : 0;
    p.knn = o.knn_k > 1 ? o.knn_k : 1;
    p.seg = kRefineSeg;
    static_assert(kRefineSeg >= kCoarseMin && kRefineSegLong % kRefineSeg == 0, "segments cover the coarse pool");
    p.cap = o.select_cap > 0 ? o.select_cap : kDefaultCap;
    p.slot_lane = ctx->slot_lane.p;
    p.slot_win = ctx->slot_win.p;
    p.route = ctx->route.p;
    p.dlist = ctx->dlist.p;
    p.dlist_alt = ctx->dlist_alt.p;
    p.tc_ns = o.tc_group;
    p.tc_col_lo = 0;
    p.tc_col_hi = int64_t(1) << 40;  // every column
    p.dgroups = ctx->dgroups.p;
    p.acen = ctx->acen.p;
    p.asum = ctx->asum.p;
    p.gmax = ctx->gmax.p;
    p.dead = ctx->dead.p;
    p.kcnt = ctx->kcnt.p;
    p.nn2 = ctx->nn2.p;
    p.cmax = ctx->cmax.p;
    p.cmax2 = ctx->cmax2.p;
    p.strips = ctx->strips.p;
    p.nref = &ctx->small.p->nref;
    p.work = ctx->small.p->work;
    p.err = &ctx->small.p->err;
    p.pairs = ctx->small.p->pairs;
    p.pick_idx = ctx->pidx.p;
    p.pick_nn = ctx->pnn.p;
    return p;
}

// One pass over `req` lanes: statistics, select, compaction, refine rounds
// through the slot pool, gather and top-K.  Fills `out` with every lane's
// state and top-K picks.
// A pass either runs whole DRAG calls (kFull) or one phase of a DRAG call
// whose pair space is split over ranks: kSelect stops after candidate select
// and copies the lane's bitmap to shard_bits_host; kRefine skips select,
// takes the candidates from shard_bits_dev and writes every candidate's
// result over the lane's columns to shard_nn_dev (k_shard_out).
enum PassMode { kFull = 0, kSelect = 1, kRefine = 2 };

struct ShardIO {
    PassMode mode = kFull;
    uint32_t* bits_host = nullptr;      // kSelect: [P] out
    const uint32_t* bits_dev = nullptr; // kRefine: [P] in (device)
    double* nn_dev = nullptr;           // kRefine: [N] out (device)
};

palmad_status run_pass(palmad_ctx* ctx, std::vector<PassLane>& req, int K, bool exclusive, const palmad_options& o,
                       PassOut& out, const ShardIO& io = ShardIO()) {
    const int nl = int(req.size());
    if (nl == 0) return PALMAD_OK;
    if (nl > kMaxLanes) return fail(ctx, PALMAD_ERR_INTERNAL, "too many lanes in a pass");
    CKS(ensure_pass(ctx, nl, K));
    int32_t kpad_max = 32, nchunks_max = 1;
    int64_t nmax = 1, strips = 0;
    int nchains = 0;
    for (int l = 0; l < nl; ++l) {
        Lane& L = req[l].lane;
        L.kpad = ((L.m + 31) / 32) * 32;
        L.nstrips = int32_t(std::max<int64_t>(0, std::min<int64_t>((L.N + kStripH - 1) / kStripH, L.strip_lim) -
                                                  L.strip0));
        L.strip_base = strips;
        const bool sel = L.prune && o.knn_k <= 1;  // select prunes on one pair: nearest neighbour only
        strips += sel ? L.nstrips : 0;
        if (!sel) L.nstrips = 0;
        kpad_max = std::max(kpad_max, L.kpad);
        nchunks_max = std::max<int32_t>(nchunks_max, int32_t((L.N + 31) / 32));
        nmax = std::max(nmax, L.N);
        if (l == 0 || !req[l - 1].lane.chain_next) ctx->h_chain[nchains++] = l;
        ctx->h_lanes[l] = L;
        LaneState s = req[l].state;
        s.nsurv = 0; s.dcount = 0; s.got = 0; s.count_final = 0; s.maxerr = 0; s.ndirect = 0;
        s.seed_rows = 0; s.seed_base = 0; s.seed_eff = 0; s.seed_eps = 0;
        if (L.stats_mode != 0) { s.flags = 0; s.ab[0] = 0; s.ab[1] = 0; }
        ctx->h_st[l] = s;
    }
    CKS(ensure_pool(ctx, kpad_max, nchunks_max));
    ctx->sets_dirty = true;
    Pass p = base_pass(ctx, nl, K, exclusive, o);
    if (io.mode == kRefine) strips = 0;
    p.sel_items = strips;
    p.sharded = io.mode != kFull ? 1 : 0;
    p.shard_nn = io.nn_dev;
    {
        // a pass with few strips (one lane, a rerun) would leave most warps
        // idle while each runs a long piece: shorter pieces spread its scan
        const int64_t slots = int64_t(ctx->sms) * 4 * 4;  // resident select warps
        const int64_t cols = kStripH + 31 + p.cap;
        p.sel_cols = (strips * ((cols + kSelPieceCols - 1) / kSelPieceCols) < 2 * slots) ? kSelPieceColsShort
                                                                                           : kSelPieceCols;
        p.sel_pieces = int32_t((cols + p.sel_cols - 1) / p.sel_cols);
    }
    p.nmax = nmax;
    p.kpad_max = ctx->pool_kpad;
    p.kpad_pass = kpad_max;
    p.nchunks_max = ctx->pool_nchunks;
    p.ncoarse_max = int32_t((int64_t(ctx->pool_nchunks) * 32 + kCoarseMin - 1) / kCoarseMin);
    {
        // long passes: 2048-column segments (fewer items, each first-column
        // seed spread over more columns); short ones keep 1024 for balance
        int64_t cols = 0;
        for (int l = 0; l < nl; ++l) cols += ctx->h_lanes[l].N;
        p.seg = o.refine_seg ? o.refine_seg : (cols >= kLongPass ? kRefineSegLong : kRefineSeg);
    }
    // The tensor-core direct refine records chunk maxima as upper bounds
    // (value + eps_j) and only the survivor maximum as a lower bound; the
    // k-th neighbour re-check needs k columns that reach its threshold, so
    // that variant refines direct strips on the FP32 form, which records
    // the FP32 values themselves.
    p.mixed = (o.precision == PALMAD_PREC_MIXED && p.knn <= 1 && !p.sharded && refine_tc_supported(p)) ? 1 : 0;
    // 256-row refine strips halve the top-row seed work per row: chosen
    // when asked (the autotuner's refine_rows), never with tensor-core seeds
    p.refine_h = (o.refine_rows == kRefineHTall && !(o.precision == PALMAD_PREC_MIXED && o.tc_seed_min > 0))
                     ? kRefineHTall : kRefineH;
    // passes of long windows (kpad > 256) may split their strips differently:
    // the direct form costs 2m flops per survivor-column, the sweep's top-row
    // seed as much per strip-column on top of 8 per row
    p.direct_below = (kpad_max > kLongWindow && o.direct_below_long > 0) ? o.direct_below_long : o.direct_below;
    p.strip_row = ctx->strip_row.p;
    p.seed_ngroups = &ctx->small.p->seed_ngroups;
    p.tc_seeds = 0;
    if (o.precision == PALMAD_PREC_MIXED && o.tc_seed_min > 0 && seed_tc_supported(p)) {
        // seed rows of nmax columns (rounded to the kernel's 1024-column blocks)
        const int64_t stride = (nmax + 1023) / 1024 * 1024;
        int64_t cap = std::min<int64_t>(kSeedBytes / (stride * int64_t(sizeof(float))), ctx->pool);
        if (o.seed_rows_max > 0) cap = std::min<int64_t>(cap, o.seed_rows_max);
        if (cap >= 1) {
            CKS(ensure(ctx, ctx->seeds, size_t(cap * stride)));
            CKS(ensure(ctx, ctx->topcen, size_t(cap) * p.kpad_max));
            CKS(ensure(ctx, ctx->topsum, size_t(cap)));
            CKS(ensure(ctx, ctx->seed_groups, size_t(cap / 32 + nl + 1)));
            p.tc_seeds = 1;
            p.seed_min = o.tc_seed_min;
            p.seeds = ctx->seeds.p;
            p.topcen = ctx->topcen.p;
            p.topsum = ctx->topsum.p;
            p.seed_groups = ctx->seed_groups.p;
            p.seed_stride = stride;
            p.seed_cap = int32_t(cap);
        }
    }

    CK(cudaMemcpyAsync(ctx->lanes.p, ctx->h_lanes, sizeof(Lane) * nl, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->st.p, ctx->h_st, sizeof(LaneState) * nl, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->chain.p, ctx->h_chain, sizeof(int32_t) * nchains, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->small.p, 0, sizeof(Small), ctx->stream));
    LAUNCH(PALMAD_K_STATS, launch_stats(p, ctx->chain.p, nchains, nmax, ctx->sms, ctx->stream));
    if (strips > 0) LAUNCH(PALMAD_K_SELECT, launch_select(p, ctx->sms * 4, ctx->stream));
    if (io.mode == kSelect) {
        const Lane& L0 = ctx->h_lanes[0];
        CK(cudaMemcpyAsync(io.bits_host, L0.bits, sizeof(uint32_t) * size_t((L0.N + 31) / 32), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaMemcpyAsync(ctx->h_small, ctx->small.p, sizeof(Small), cudaMemcpyDeviceToHost, ctx->stream));
        CKS(sync(ctx));
        ctx->sets_dirty = false;
        ctx->stats.select_pairs += int64_t(ctx->h_small->pairs[0]);
        ctx->stats.device_passes += 1;
        return PALMAD_OK;
    }
    if (io.mode == kRefine) {
        // the candidates every shard's select left (ANDed by the caller)
        const Lane& L0 = ctx->h_lanes[0];
        CK(cudaMemcpyAsync(L0.bits, io.bits_dev, sizeof(uint32_t) * size_t((L0.N + 31) / 32),
                           cudaMemcpyDeviceToDevice, ctx->stream));
    }
    LAUNCH(PALMAD_K_COMPACT, launch_compact(p, ctx->stream));
    {
        // witness hints: survivors pruned by a pair near where an earlier
        // length pruned them leave before refine; the survivor list is rebuilt
        bool hinted = false;
        for (int l = 0; l < nl; ++l) hinted |= ctx->h_lanes[l].hint != nullptr && ctx->h_lanes[l].prune && p.knn <= 1;
        if (hinted && hint_supported(p)) {
            LAUNCH(PALMAD_K_HINT, launch_hint(p, ctx->sms, ctx->stream));
            LAUNCH(PALMAD_K_COMPACT, launch_compact(p, ctx->stream));
        }
    }
    CK(cudaMemcpyAsync(ctx->h_st, ctx->st.p, sizeof(LaneState) * nl, cudaMemcpyDeviceToHost, ctx->stream));
    CKS(sync(ctx));
    for (int l = 0; l < nl; ++l) ctx->stats.survivors += ctx->h_st[l].nsurv;
    ctx->stats.device_passes += 1;

    // Refine rounds: lanes' survivors in order, as many as the pool holds.
    const int32_t pool = o.pool_slots > 0 ? std::min(ctx->pool, std::max(64, (o.pool_slots + 63) / 64 * 64)) : ctx->pool;
    std::vector<int32_t> done(nl, 0);
    for (int round = 0;; ++round) {
        // the pinned lane mirror still feeds the previous round's upload
        if (round > 0) CK(cudaStreamSynchronize(ctx->stream));
        int32_t used = 0;
        bool any = false;
        for (int l = 0; l < nl; ++l) {
            Lane& L = ctx->h_lanes[l];
            const int32_t rem = ctx->h_st[l].nsurv - done[l];
            const int32_t room = pool - used;
            const int32_t take = std::max(0, std::min(rem, room));
            L.k_lo = done[l];
            L.k_hi = done[l] + take;
            L.slot_base = used;
            if (take > 0) {
                any = true;
                used += ((take + 63) / 64) * 64;
                done[l] += take;
            }
            if (used >= pool) used = pool;
        }
        if (!any) break;
        p.nslots = used;
        CK(cudaMemcpyAsync(ctx->lanes.p, ctx->h_lanes, sizeof(Lane) * nl, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemsetAsync(&ctx->small.p->work[1], 0, 7 * sizeof(int32_t), ctx->stream));
        CK(cudaMemsetAsync(&ctx->small.p->nref, 0, sizeof(int32_t), ctx->stream));
        LAUNCH(PALMAD_K_PLAN, launch_plan(p, ctx->stream));
        if (p.tc_seeds) LAUNCH(PALMAD_K_SEED_TC, launch_seeds(p, ctx->sms, ctx->stream));
        LAUNCH(PALMAD_K_REFINE_SWEEP, launch_refine_sweep(p, ctx->sms * 4, ctx->stream));
        if (p.mixed) {
            // the tensor-core direct refine in column chunks; between chunks
            // the survivors still alive are re-packed into full groups, so a
            // group no longer runs on while most of its survivors are pruned
            const int chunks = o.tc_chunks > 0 ? o.tc_chunks : 1;
            // survivor-major tiles (windows up to 256) unless asked otherwise
            const bool tcs = o.tc_form != 1 && p.tc_ns == 0 && refine_tcs_supported(p);
            const int64_t span = ((p.nmax + chunks - 1) / chunks + 2047) / 2048 * 2048;
            for (int c = 0; c < chunks && int64_t(c) * span < p.nmax; ++c) {
                p.tc_col_lo = int64_t(c) * span;
                p.tc_col_hi = std::min<int64_t>(p.nmax, p.tc_col_lo + span);
                if (c > 0) {
                    CK(cudaMemsetAsync(&ctx->small.p->work[1], 0, sizeof(int32_t), ctx->stream));
                    CK(cudaMemsetAsync(&ctx->small.p->work[4], 0, sizeof(int32_t), ctx->stream));
                    LAUNCH(PALMAD_K_PLAN, launch_direct_repack(p, ctx->stream));
                    std::swap(p.dlist, p.dlist_alt);
                }
                if (tcs) LAUNCH(PALMAD_K_REFINE_DIRECT, launch_refine_tcs(p, ctx->sms, ctx->stream));
                else LAUNCH(PALMAD_K_REFINE_DIRECT, launch_refine_tc(p, ctx->sms, ctx->stream));
            }
        } else {
            LAUNCH(PALMAD_K_REFINE_DIRECT, launch_refine_direct(p, ctx->sms * 2, ctx->stream));
        }
        LAUNCH(PALMAD_K_RECHECK, launch_recheck(p, ctx->sms * 8, ctx->stream));
        if (io.mode == kRefine) LAUNCH(PALMAD_K_GATHER, launch_shard_out(p, ctx->stream));
        else LAUNCH(PALMAD_K_GATHER, launch_gather(p, ctx->stream));
        LAUNCH(PALMAD_K_PLAN, launch_round_cleanup(p, ctx->stream));
        bool more = false;
        for (int l = 0; l < nl; ++l) more |= done[l] < ctx->h_st[l].nsurv;
        if (!more) break;
    }
    LAUNCH(PALMAD_K_TOPK, launch_topk(p, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_st, ctx->st.p, sizeof(LaneState) * nl, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_pidx, ctx->pidx.p, sizeof(int64_t) * nl * K, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_pnn, ctx->pnn.p, sizeof(double) * nl * K, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_small, ctx->small.p, sizeof(Small), cudaMemcpyDeviceToHost, ctx->stream));
    CKS(sync(ctx));
    ctx->sets_dirty = false;
    out.st.assign(ctx->h_st, ctx->h_st + nl);
    out.idx.assign(ctx->h_pidx, ctx->h_pidx + int64_t(nl) * K);
    out.nn.assign(ctx->h_pnn, ctx->h_pnn + int64_t(nl) * K);
    const Small& sm = *ctx->h_small;
    if (sm.err) return fail(ctx, PALMAD_ERR_TIMEOUT, "tensor-core refine: an MMA did not signal completion");
    ctx->stats.select_pairs += int64_t(sm.pairs[0]);
    ctx->stats.refine_pairs += int64_t(sm.pairs[1]) + int64_t(sm.pairs[4]);
    ctx->stats.direct_pairs += int64_t(sm.pairs[1]);
    ctx->stats.fp64_pairs += int64_t(sm.pairs[2]);
    // algorithmic work: per-lane m is folded with the pass-average m (exact for one length)
    double msum = 0.0;
    for (int l = 0; l < nl; ++l) msum += req[l].lane.m;
    const double mavg = msum / nl;
    // algorithmic work of a pair evaluation: 8 FP32 flops in the recurrence
    // form (the diagonal update, the correlation and the distance of Eq. 6),
    // 2m per direct dot product
    ctx->stats.select_flops += kPairFlops * double(sm.pairs[0]) + 2.0 * mavg * double(sm.pairs[3]);
    ctx->stats.refine_flops += 2.0 * mavg * double(sm.pairs[1]);
    ctx->stats.sweep_flops += kPairFlops * double(sm.pairs[4]) + 2.0 * mavg * double(sm.pairs[5]);
    ctx->stats.refine_strips += int64_t(sm.pairs[9]);
    ctx->stats.sweep_survivors += int64_t(sm.pairs[10]);
    ctx->stats.hint_pairs += int64_t(sm.pairs[7]);
    ctx->stats.hint_kills += int64_t(sm.pairs[8]);
    ctx->stats.seed_pairs += int64_t(sm.pairs[6]);
    ctx->stats.seed_flops += 2.0 * mavg * double(sm.pairs[6]);
    for (int l = 0; l < nl; ++l) {
        const uint32_t e = out.st[l].maxerr;
        if (e) {
            const uint32_t b = (e & 0x80000000u) ? (e & 0x7fffffffu) : ~e;
            float f;
            std::memcpy(&f, &b, 4);
            ctx->stats.max_fp32_rho_err = std::max(ctx->stats.max_fp32_rho_err, double(f));
        }
    }
    return PALMAD_OK;
}

// Heatmap rows and range-discord counts of accepted lanes at their final r
// (asynchronous: results land in device memory).
palmad_status run_finalize(palmad_ctx* ctx, std::vector<PassLane>& req, const palmad_options& o) {
    const int nl = int(req.size());
    if (nl == 0) return PALMAD_OK;
    bool need = false;
    for (auto& q : req) need |= (q.lane.heat != nullptr) || (q.lane.count_out != nullptr);
    if (!need) return PALMAD_OK;
    CKS(ensure_pass(ctx, nl, 1));
    if (ctx->h_fin_cap < nl) {
        if (ctx->h_fin_lanes) cudaFreeHost(ctx->h_fin_lanes);
        if (ctx->h_fin_st) cudaFreeHost(ctx->h_fin_st);
        ctx->h_fin_lanes = nullptr;
        ctx->h_fin_st = nullptr;
        ctx->h_fin_cap = 0;
        const int cap = std::max(nl, 64);
        if (cudaMallocHost(&ctx->h_fin_lanes, sizeof(Lane) * cap) != cudaSuccess ||
            cudaMallocHost(&ctx->h_fin_st, sizeof(LaneState) * cap) != cudaSuccess)
            return fail(ctx, PALMAD_ERR_OOM, "pinned host allocation failed");
        ctx->h_fin_cap = cap;
    }
    for (int l = 0; l < nl; ++l) {
        ctx->h_fin_lanes[l] = req[l].lane;
        ctx->h_fin_st[l] = req[l].state;
        ctx->h_fin_st[l].count_final = 0;
    }
    Pass p = base_pass(ctx, nl, 1, true, o);
    CK(cudaMemcpyAsync(ctx->lanes.p, ctx->h_fin_lanes, sizeof(Lane) * nl, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->st.p, ctx->h_fin_st, sizeof(LaneState) * nl, cudaMemcpyHostToDevice, ctx->stream));
    LAUNCH(PALMAD_K_HEAT, launch_finalize(p, ctx->stream));
    return PALMAD_OK;
}

// ====================================================== MERLIN schedule

// The thresholds MERLIN tries for one length (Sec. 2.2): the first length
// starts at 2 sqrt(minL) and halves; the next four start 1% below the
// previous length's nnDist and lose 1% per failure; later lengths start at
// mean - 2 sd of the last five nnDist values and lose sd per failure
// (0.01 mean when sd is 0).  After 60 halvings, 3000 other failures or at
// r <= 0 the try runs at r = 0 and is the last one.  Each r is the result of
// the same FP64 operations in the same order as any other implementation of
// these rules, so the sequence of r is reproducible bit for bit.
struct Tries {
    int l = 0;       // length index
    int h = 0;       // try number
    double r = 0.0;
    double step = 0.0;

    void start(int li, const std::vector<double>& sched, int32_t minL) {
        l = li;
        h = 0;
        if (l == 0) {
            r = 2.0 * std::sqrt(double(minL));
        } else if (l <= 4) {
            r = 0.99 * sched[l - 1];
        } else {
            double mean = 0.0, var = 0.0;
            for (int q = 1; q <= 5; ++q) mean += sched[l - q];
            mean /= 5.0;
            for (int q = 1; q <= 5; ++q) var += (sched[l - q] - mean) * (sched[l - q] - mean);
            const double sdv = std::sqrt(var / 4.0);
            step = sdv > 0.0 ? sdv : 0.01 * mean;
            r = mean - 2.0 * sdv;
        }
        guard();
    }
    void guard() {
        if (l == 0) {
            if (h >= 60) r = 0.0;
        } else if (h >= 3000 || r <= 0.0) {
            r = 0.0;
        }
    }
    bool last() const { return r <= 0.0; }
    void next() {
        if (l == 0) r = 0.5 * r;
        else if (l <= 4) r = 0.99 * r;
        else r = step > 0.0 ? r - step : 0.0;
        ++h;
        guard();
    }
};

// One series under the schedule.
struct SeriesJob {
    // configuration
    const float* T = nullptr;   // device, 16-byte aligned
    int64_t n = 0;
    int32_t minL = 0, maxL = 0, K = 1;
    bool exclusive = true;
    int W = 1;                  // lanes per window (1: plain form)
    int set0 = 0;               // first LaneSet of this series
    float* heat = nullptr;      // device heatmap base (row l at heat + l*hw) or nullptr
    int64_t hw = 0;
    int64_t* count_dev = nullptr;  // device [L] counts
    int32_t* hint = nullptr;       // device [n] witness hints of the series, or nullptr
    int32_t* init_flag = nullptr;  // device int for the non-finite check
    // resumed run: length index minL - minL_sched of the schedule's own run
    // (loff), and the schedule inputs of the lengths before minL (hist)
    int32_t loff = 0;
    int32_t minL_sched = 0;
    std::vector<double> hist;
    // results
    std::vector<int64_t> idx;
    std::vector<double> nn, r_final;
    std::vector<double> sched;
    std::vector<LaneState> lstate;    // per length: state after its last pass
    // progress
    int32_t L = 0;
    int32_t l = 0;              // next length to decide
    bool done = false;
    int32_t prepared_hi = -1;   // highest length index whose statistics exist
    Tries tr;
    bool tr_started = false;
    enum Phase { kIdle, kPlain, kWindow, kRerun } phase = kIdle;
    // window bookkeeping
    int32_t wl0 = 0, wn = 0;    // window lengths [wl0, wl0+wn)
    std::vector<double> rspec;  // speculative r per window length
    std::vector<LaneState> wst;
    std::vector<std::vector<int64_t>> widx;
    std::vector<std::vector<double>> wnn;
    int32_t rerun_l = -1;       // length awaiting a rerun result
    double rerun_r = 0.0;
    std::vector<double> first_r;  // first try of each length (for the deficit), by schedule index
    std::vector<double> rfin_v;   // final r of each length, by schedule index

    int set_of(int32_t li) const { return set0 + (W > 1 ? (li % W) : 0); }
    int32_t m_of(int32_t li) const { return minL + li; }
};

Lane make_lane(palmad_ctx* ctx, SeriesJob& s, int32_t li, double r, const palmad_options& o) {
    Lane L{};
    LaneSet& S = ctx->sets[s.set_of(li)];
    L.T = s.T;
    L.n = s.n;
    L.m = s.m_of(li);
    L.N = s.n - L.m + 1;
    L.mu = S.mu.p;
    L.var = S.var.p;
    L.win = S.win.p;
    L.bits0 = S.bits0.p;
    L.bits = S.bits.p;
    L.surv = S.surv.p;
    L.slot_of = S.slot_of.p;
    L.scount = S.scount.p;
    L.didx = S.didx.p;
    L.dnn = S.dnn.p;
    L.r = r;
    L.hint = s.hint;
    L.strip0 = 0;
    L.strip_lim = INT64_MAX;
    L.col_lo = 0;
    L.col_hi = L.N;
    // k-th neighbour variant: refine prunes a window at its k-th pair past the
    // threshold; select (one pair decides there) is skipped
    L.prune = r > 0.0 ? 1 : 0;
    L.rho_thr = float(1.0 - r * r / (2.0 * L.m));
    L.band = float(o.band_rel * r * r / L.m);
    // statistics source
    if (li <= s.prepared_hi) {
        L.stats_mode = 0;
    } else if (li == 0) {
        L.stats_mode = 2;  // copy in place after the init kernel
        L.mu_src = S.mu.p;
        L.var_src = S.var.p;
    } else {
        L.stats_mode = 1;
        LaneSet& P = ctx->sets[s.set_of(li - 1)];
        L.mu_src = P.mu.p;
        L.var_src = P.var.p;
    }
    return L;
}

// How far below its first try the schedule ended, recently (largest of the
// last eight decided lengths; l0 and the arrays are schedule indices).
double recent_deficit(const SeriesJob& s, int32_t l0) {
    double d = 0.0;
    for (int32_t q = std::max(5, l0 - 8); q < l0; ++q) d = std::max(d, s.first_r[q] - s.rfin_v[q]);
    return d;
}

// Speculative threshold for the window lengths: below the first try of the
// schedule by about two decrements, 6%, or 1.5x the recent deficit,
// whichever is largest (never below half the recent mean).
double speculative_r(const SeriesJob& s, int32_t l0, double scale) {  // l0: schedule index
    double mean = 0.0, var = 0.0;
    for (int q = 1; q <= 5; ++q) mean += s.sched[l0 - q];
    mean /= 5.0;
    for (int q = 1; q <= 5; ++q) var += (s.sched[l0 - q] - mean) * (s.sched[l0 - q] - mean);
    const double sdv = std::sqrt(var / 4.0);
    const double margin = scale * std::max({2.0 * sdv, 0.06 * mean, 1.5 * recent_deficit(s, l0)});
    return std::max(mean - 2.0 * sdv - margin, 0.5 * mean);
}

void accept_length(SeriesJob& s, int32_t li, double r, const LaneState& st, const int64_t* pidx, const double* pnn,
                   std::vector<PassLane>& fin, palmad_ctx* ctx, const palmad_options& o) {
    (void)ctx;
    int got = 0;
    for (int q = 0; q < s.K; ++q) {
        const bool ok = pidx[q] >= 0 && (r <= 0.0 || pnn[q] >= r);
        s.idx[size_t(li) * s.K + q] = ok ? pidx[q] : -1;
        s.nn[size_t(li) * s.K + q] = ok ? pnn[q] : 0.0;
        got += ok;
    }
    s.sched[li + s.loff] = got > 0 ? s.nn[size_t(li) * s.K + got - 1] : 0.0;
    s.r_final[li] = r;
    s.rfin_v[li + s.loff] = r;
    s.lstate[li] = st;
    PassLane f{};
    f.lane = make_lane(ctx, s, li, r, o);
    f.lane.stats_mode = 0;
    f.lane.heat = s.heat ? s.heat + size_t(li) * s.hw : nullptr;
    f.lane.count_out = s.count_dev ? s.count_dev + li : nullptr;
    f.state = st;
    fin.push_back(f);
}

// Lanes the series wants in the next pass.
void series_request(palmad_ctx* ctx, SeriesJob& s, std::vector<PassLane>& req, std::vector<int>& owner, int sid,
                    const palmad_options& o) {
    if (s.done) return;
    auto push = [&](int32_t li, double r, bool chain_next) {
        PassLane q{};
        q.lane = make_lane(ctx, s, li, r, o);
        q.lane.chain_next = chain_next ? 1 : 0;
        if (q.lane.stats_mode == 0) q.state = s.lstate[li];
        req.push_back(q);
        owner.push_back(sid);
    };
    if (s.phase == SeriesJob::kRerun) {
        push(s.rerun_l, s.rerun_r, false);
        return;
    }
    if (s.W > 1 && s.l + s.loff >= 5) {
        s.wl0 = s.l;
        s.wn = std::min<int32_t>(s.W, s.L - s.l);
        s.rspec.assign(s.wn, speculative_r(s, s.l + s.loff, o.spec_scale > 0 ? 0.01 * o.spec_scale : 1.0));
        for (int w = 0; w < s.wn; ++w) push(s.wl0 + w, s.rspec[w], w + 1 < s.wn);
        s.phase = SeriesJob::kWindow;
        return;
    }
    if (!s.tr_started) {
        s.tr.start(s.l + s.loff, s.sched, s.minL_sched);
        s.tr_started = true;
        s.first_r[s.l + s.loff] = s.tr.r;
    }
    push(s.l, s.tr.r, false);
    s.phase = SeriesJob::kPlain;
}

// Replays Algorithm 1 over the window results; stops when a length needs a
// rerun below its speculative r.
void series_replay(palmad_ctx* ctx, SeriesJob& s, std::vector<PassLane>& fin, const palmad_options& o) {
    const int K = s.K;
    while (s.l < s.wl0 + s.wn) {
        const int w = s.l - s.wl0;
        if (!s.tr_started) {
            s.tr.start(s.l + s.loff, s.sched, s.minL_sched);
            s.tr_started = true;
            s.first_r[s.l + s.loff] = s.tr.r;
        }
        const double rs = s.rspec[w];
        for (;;) {
            const double r = s.tr.r;
            if (!(rs <= 0.0 || r >= rs)) {
                // the schedule needs r below this length's r': rerun it lower,
                // by at least three decrements, 10% or 1.5x the recent deficit
                const double step = s.tr.step > 0.0 ? s.tr.step : 0.01 * r;
                const double drop = (o.spec_scale > 0 ? 0.01 * o.spec_scale : 1.0) *
                                    std::max({3.0 * step, 0.1 * r, 1.5 * recent_deficit(s, s.l + s.loff)});
                s.rerun_l = s.l;
                s.rerun_r = r - drop;
                if (s.rerun_r < 0.05 * r) s.rerun_r = 0.05 * r;  // stay clear of the r = 0 full profile
                if (r <= 0.0) s.rerun_r = 0.0;
                s.phase = SeriesJob::kRerun;
                ctx->stats.reruns += 1;
                return;
            }
            ctx->stats.drag_calls += 1;
            int got = 0;
            for (int q = 0; q < K; ++q)
                if (s.widx[w][q] >= 0 && (r <= 0.0 || s.wnn[w][q] >= r)) ++got;
            if (got == K || s.tr.last()) {
                accept_length(s, s.l, r, s.wst[w], s.widx[w].data(), s.wnn[w].data(), fin, ctx, o);
                break;
            }
            s.tr.next();
        }
        s.l += 1;
        s.tr_started = false;
    }
    s.phase = SeriesJob::kIdle;
    if (s.l >= s.L) s.done = true;
}

// Consumes the results of the series' lanes (in request order).
void series_consume(palmad_ctx* ctx, SeriesJob& s, const PassOut& out, const std::vector<int>& mine,
                    std::vector<PassLane>& fin, const palmad_options& o) {
    const int K = s.K;
    auto pidx = [&](int k) { return out.idx.data() + size_t(mine[k]) * K; };
    auto pnn = [&](int k) { return out.nn.data() + size_t(mine[k]) * K; };
    if (s.phase == SeriesJob::kPlain) {
        const LaneState& st = out.st[mine[0]];
        s.prepared_hi = std::max(s.prepared_hi, s.l);
        s.lstate[s.l] = st;
        ctx->stats.drag_calls += 1;
        if (st.got == K || s.tr.last()) {
            accept_length(s, s.l, s.tr.r, st, pidx(0), pnn(0), fin, ctx, o);
            s.l += 1;
            s.tr_started = false;
            if (s.l >= s.L) s.done = true;
        } else {
            s.tr.next();
        }
        s.phase = SeriesJob::kIdle;
        return;
    }
    if (s.phase == SeriesJob::kWindow) {
        s.wst.resize(s.wn);
        s.widx.resize(s.wn);
        s.wnn.resize(s.wn);
        for (int w = 0; w < s.wn; ++w) {
            s.wst[w] = out.st[mine[w]];
            s.lstate[s.wl0 + w] = s.wst[w];
            s.widx[w].assign(pidx(w), pidx(w) + K);
            s.wnn[w].assign(pnn(w), pnn(w) + K);
        }
        s.prepared_hi = std::max(s.prepared_hi, s.wl0 + s.wn - 1);
    } else if (s.phase == SeriesJob::kRerun) {
        const int w = s.rerun_l - s.wl0;
        s.wst[w] = out.st[mine[0]];
        s.lstate[s.rerun_l] = s.wst[w];
        s.widx[w].assign(pidx(0), pidx(0) + K);
        s.wnn[w].assign(pnn(0), pnn(0) + K);
        s.rspec[w] = s.rerun_r;
        s.rerun_l = -1;
    }
    series_replay(ctx, s, fin, o);
}

// Runs MERLIN over the given series, sharing passes between them.
palmad_status run_jobs(palmad_ctx* ctx, std::vector<SeriesJob>& jobs, const palmad_options& o) {
    // lane buffers
    int nsets = 0;
    for (auto& s : jobs) {
        s.set0 = nsets;
        nsets += std::max(1, s.W);
    }
    if (int(ctx->sets.size()) < nsets) ctx->sets.resize(nsets);
    for (auto& s : jobs) {
        for (int q = 0; q < std::max(1, s.W); ++q) CKS(ensure_set(ctx, ctx->sets[s.set0 + q], s.n - s.minL + 1));
        s.L = s.maxL - s.minL + 1;
        s.idx.assign(size_t(s.L) * s.K, -1);
        s.nn.assign(size_t(s.L) * s.K, 0.0);
        s.r_final.assign(s.L, 0.0);
        if (s.minL_sched == 0) s.minL_sched = s.minL;
        s.sched.assign(s.loff + s.L, 0.0);
        for (size_t q = 0; q < s.hist.size(); ++q) s.sched[s.loff - s.hist.size() + q] = s.hist[q];
        s.lstate.assign(s.L, LaneState{});
        s.first_r.assign(s.loff + s.L, 0.0);
        s.rfin_v.assign(s.loff + s.L, 0.0);
    }
    // witness hints: one int per point of every series, none recorded yet
    if (!o.no_hints) {
        int64_t tot = 0;
        for (auto& s : jobs) tot += s.n;
        CKS(ensure(ctx, ctx->hints, size_t(tot)));
        CK(cudaMemsetAsync(ctx->hints.p, 0xff, sizeof(int32_t) * size_t(tot), ctx->stream));
        tot = 0;
        for (auto& s : jobs) {
            s.hint = ctx->hints.p + tot;
            tot += s.n;
        }
    }
    // initial statistics (Eq. 4 at minL) and the non-finite check
    CKS(ensure(ctx, ctx->init_flags, jobs.size()));
    CK(cudaMemsetAsync(ctx->init_flags.p, 0, sizeof(int32_t) * jobs.size(), ctx->stream));
    for (size_t q = 0; q < jobs.size(); ++q) {
        SeriesJob& s = jobs[q];
        LaneSet& S = ctx->sets[s.set0];
        s.init_flag = ctx->init_flags.p + q;
        LAUNCH(PALMAD_K_STATS, launch_stats_init(s.T, s.n, s.minL, S.mu.p, S.var.p, s.init_flag, ctx->stream));
        if (s.count_dev) CK(cudaMemsetAsync(s.count_dev, 0, sizeof(int64_t) * s.L, ctx->stream));
        if (s.heat) CK(cudaMemsetAsync(s.heat, 0, sizeof(float) * size_t(s.L) * s.hw, ctx->stream));
    }
    std::vector<int32_t> flags(jobs.size());
    CK(cudaMemcpyAsync(flags.data(), ctx->init_flags.p, sizeof(int32_t) * jobs.size(), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CKS(sync(ctx));
    for (size_t q = 0; q < jobs.size(); ++q)
        if (flags[q] & 1) return fail(ctx, PALMAD_ERR_NONFINITE, "T holds a NaN or an infinity");

    std::vector<PassLane> req, fin;
    std::vector<int> owner;
    PassOut out;
    for (;;) {
        req.clear();
        owner.clear();
        for (size_t q = 0; q < jobs.size(); ++q) {
            if (int(req.size()) + std::max(1, jobs[q].W) > kMaxLanes) break;
            series_request(ctx, jobs[q], req, owner, int(q), o);
        }
        if (req.empty()) break;
        const int K = jobs[0].K;
        const bool excl = jobs[0].exclusive;
        CKS(run_pass(ctx, req, K, excl, o, out));
        fin.clear();
        std::vector<std::vector<int>> per(jobs.size());
        for (int k = 0; k < int(owner.size()); ++k) per[owner[k]].push_back(k);
        for (size_t q = 0; q < jobs.size(); ++q)
            if (!per[q].empty()) series_consume(ctx, jobs[q], out, per[q], fin, o);
        CKS(run_finalize(ctx, fin, o));
    }
    for (auto& s : jobs) ctx->stats.lengths += s.L;
    return PALMAD_OK;
}

palmad_status check_args(palmad_ctx* ctx, int64_t n, int32_t minL, int32_t maxL, int32_t topK) {
    if (!ctx) return PALMAD_ERR_ARG;
    if (minL < 3) return fail(ctx, PALMAD_ERR_ARG, "minL must be >= 3");
    if (maxL < minL) return fail(ctx, PALMAD_ERR_ARG, "maxL must be >= minL");
    if (n < 2 * int64_t(maxL)) return fail(ctx, PALMAD_ERR_ARG, "n must be >= 2*maxL");
    if (n > (int64_t(1) << 30)) return fail(ctx, PALMAD_ERR_UNSUPPORTED, "n above 2^30 is not supported");
    if (topK < 1 || topK > kMaxK) return fail(ctx, PALMAD_ERR_ARG, "topK must lie in [1, 1024]");
    return PALMAD_OK;
}

void reset_stats(palmad_ctx* ctx) {
    ctx->stats = palmad_stats{};
    ctx->stats.struct_size = sizeof(palmad_stats);
}

palmad_status begin_call(palmad_ctx* ctx, const palmad_options& o) {
    ctx->err.clear();
    reset_stats(ctx);
    ctx->profile = o.profile != 0;
    CK(cudaSetDevice(ctx->device));
    if (ctx->sets_dirty) {  // an earlier call stopped inside a pass
        for (LaneSet& s : ctx->sets)
            if (s.cap > 0) CKS(clear_maps(ctx, s));
        ctx->sets_dirty = false;
    }
    return PALMAD_OK;
}

// A series on the device that starts on a 16-byte boundary (the sweeps copy
// it with 16-byte asynchronous copies).
palmad_status aligned_series(palmad_ctx* ctx, const float* T_dev, int64_t n, DBuf<float>& stage, const float** out) {
    if (reinterpret_cast<uintptr_t>(T_dev) % 16 == 0) {
        *out = T_dev;
        return PALMAD_OK;
    }
    CKS(ensure(ctx, stage, size_t(n)));
    CK(cudaMemcpyAsync(stage.p, T_dev, size_t(n) * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    *out = stage.p;
    return PALMAD_OK;
}

// Sums the device counts into the stats.
void count_discords(palmad_ctx* ctx, const std::vector<int64_t>& counts) {
    for (int64_t c : counts) ctx->stats.discords += c;
}

// ============================================================= autotuner
//
// The pass configuration -- lengths per pass and the speculation margin of
// the batched form, the select cap, the refine segment and the split
// between the refine forms -- changes how fast a call runs, never what it
// returns.  Which configuration is fastest depends on the data: on short
// series many lengths per pass amortise launches, on long quasi-periodic
// series every speculative margin multiplies the survivors refine must
// scan.  The tuner times candidates on a block of lengths of the caller's
// own series (a fresh schedule started mid-range) by coordinate descent
// and keeps the fastest per workload bucket.

std::array<int64_t, 7> tune_key(int64_t n, int32_t minL, int32_t maxL, int32_t topK, const palmad_options& o) {
    auto lg = [](int64_t v) { int64_t b = 0; while (v > 1) { v >>= 1; ++b; } return b; };
    return {int64_t(o.precision), int64_t(o.knn_k > 1 ? o.knn_k : 1), lg(n), lg(minL), lg(maxL - minL + 1),
            lg(topK), int64_t(o.exclusive_topk != 0)};
}

// A block of lengths [lo, hi] of MERLIN over a device series, resumed from
// the schedule inputs of the lengths before it (hist, lengths since the
// run's first length minL_sched) exactly as the whole run reaches it.
struct Block {
    int32_t lo = 0, hi = 0, minL_sched = 0;
    std::vector<double> hist;
};

// Wall time of one block; sched_out (optional) receives the schedule input
// of every length of the block.
palmad_status time_block(palmad_ctx* ctx, const float* T_dev, int64_t n, const Block& b, int32_t K,
                         const palmad_options& o, double* ms, std::vector<double>* sched_out = nullptr) {
    std::vector<SeriesJob> jobs(1);
    SeriesJob& s = jobs[0];
    s.T = T_dev;
    s.n = n;
    s.minL = b.lo;
    s.maxL = b.hi;
    s.K = K;
    s.exclusive = o.exclusive_topk != 0;
    s.W = std::max(1, o.batch_lengths);
    s.minL_sched = b.minL_sched;
    s.loff = b.lo - b.minL_sched;
    s.hist = b.hist;
    DBuf<int64_t> cnt;
    CKS(ensure(ctx, cnt, size_t(b.hi - b.lo + 1)));
    s.count_dev = cnt.p;
    CK(cudaStreamSynchronize(ctx->stream));
    const auto t0 = std::chrono::steady_clock::now();
    palmad_status st = run_jobs(ctx, jobs, o);
    if (st == PALMAD_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = fail(ctx, PALMAD_ERR_CUDA, std::string("tuning run: ") + cudaGetErrorString(e));
    }
    *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    tcollect(ctx);
    release(cnt);
    if (st == PALMAD_OK && sched_out) {
        sched_out->clear();
        for (int32_t l = 0; l <= b.hi - b.lo; ++l) sched_out->push_back(s.sched[s.loff + l]);
    }
    return st;
}

palmad_status tune(palmad_ctx* ctx, const float* T_dev, int64_t n, int32_t minL, int32_t maxL, int32_t topK,
                   const palmad_options& base, palmad_options* out, palmad_tune_report* rep) {
    const auto t0 = std::chrono::steady_clock::now();
    const int32_t L = maxL - minL + 1;
    palmad_options cur = base;
    cur.autotune = 0;
    cur.profile = 0;
    // Blocks of up to 12 lengths at the start, a third, two thirds and the
    // end of the range.  Each later block resumes from the schedule inputs
    // of its five preceding lengths, found by a short untimed run started at
    // the first of them: a length's picks (and so its schedule input) do not
    // depend on the thresholds tried, so the block then follows the very
    // thresholds the whole run meets there.
    const int32_t B = std::min<int32_t>(L, 12);
    std::vector<Block> blocks;
    for (int q = 0; q < 4; ++q) {
        const int32_t lo = minL + int32_t(int64_t(L - B) * q / 3);
        if (!blocks.empty() && lo <= blocks.back().hi) continue;
        Block b;
        b.lo = lo;
        b.hi = lo + B - 1;
        b.minL_sched = minL;
        if (lo > minL) {
            Block pre;
            pre.lo = std::max(minL, lo - 5);
            pre.hi = lo - 1;
            pre.minL_sched = pre.lo;
            palmad_options po = cur;
            po.batch_lengths = 1;
            double t = 0.0;
            CKS(time_block(ctx, T_dev, n, pre, topK, po, &t, &b.hist));
            b.minL_sched = pre.lo;
        }
        blocks.push_back(b);
    }
    int evals = 0;
    // the summed block time, the best of up to three runs when short
    auto measure = [&](const palmad_options& o, double* ms) -> palmad_status {
        double best = 1e300;
        for (int k = 0; k < 3; ++k) {
            double tot = 0.0;
            for (const Block& b : blocks) {
                double t = 0.0;
                CKS(time_block(ctx, T_dev, n, b, topK, o, &t));
                tot += t;
            }
            best = std::min(best, tot);
            if (tot > 50.0) break;
        }
        ++evals;
        *ms = best;
        return PALMAD_OK;
    };
    double warm = 0.0;
    CKS(time_block(ctx, T_dev, n, blocks[0], topK, cur, &warm));  // first use allocates the buffers
    double best_ms = 0.0;
    CKS(measure(cur, &best_ms));
    const double default_ms = best_ms;
    auto consider = [&](palmad_options o) -> palmad_status {
        double t = 0.0;
        CKS(measure(o, &t));
        if (t < best_ms) {
            best_ms = t;
            cur = o;
        }
        return PALMAD_OK;
    };
    // lengths per pass and the speculation margin
    {
        const palmad_options start = cur;
        for (int32_t W : {1, 2, 4, 16})
            for (int32_t sc : {100, 40}) {
                if (W == 1 && sc != 100) continue;
                palmad_options o = start;
                o.batch_lengths = W;
                o.spec_scale = sc;
                if (o.batch_lengths == std::max(1, start.batch_lengths) && o.spec_scale == (start.spec_scale ? start.spec_scale : 100)) continue;
                CKS(consider(o));
            }
    }
    // select cap
    {
        const palmad_options start = cur;
        for (int32_t cap : {512, 2048, 4096}) {
            palmad_options o = start;
            o.select_cap = cap;
            CKS(consider(o));
        }
    }
    // refine segment
    {
        const palmad_options start = cur;
        for (int32_t seg : {1024, 2048}) {
            palmad_options o = start;
            o.refine_seg = seg;
            CKS(consider(o));
        }
    }
    // column chunks of the tensor-core direct refine (live survivors re-packed
    // between chunks)
    if (cur.precision == PALMAD_PREC_MIXED) {
        const palmad_options start = cur;
        for (int32_t ch : {4, 8}) {
            palmad_options o = start;
            o.tc_chunks = ch;
            CKS(consider(o));
        }
    }
    // rows per refine strip
    {
        const palmad_options start = cur;
        palmad_options o = start;
        o.refine_rows = kRefineHTall;
        CKS(consider(o));
    }
    // strips below this many survivors take the direct form: one threshold
    // for passes of windows up to 256 long, one for longer windows (the two
    // touch disjoint passes, so each is searched on its own)
    {
        const palmad_options start = cur;
        for (int32_t db : {2, 4, 8, 16, 32, 64, 129}) {
            palmad_options o = start;
            o.direct_below = db;
            o.direct_below_long = start.direct_below_long > 0 ? start.direct_below_long : start.direct_below;
            CKS(consider(o));
        }
    }
    if (maxL + 31 > kLongWindow + 32) {
        const palmad_options start = cur;
        for (int32_t db : {4, 8, 16, 32, 64, 129}) {
            palmad_options o = start;
            o.direct_below_long = db;
            CKS(consider(o));
        }
    }
    cur.profile = base.profile;
    cur.autotune = base.autotune;
    *out = cur;
    ctx->tuned[tune_key(n, minL, maxL, topK, base)] = cur;
    if (rep) {
        rep->candidates = evals;
        rep->block_lo = blocks.front().lo;
        rep->block_hi = blocks.back().hi;
        rep->best_ms = best_ms;
        rep->default_ms = default_ms;
        rep->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return PALMAD_OK;
}

// Options of a find call with autotune set: the bucket's tuned options,
// tuning on the call's own series first when the bucket has none.
palmad_status tuned_options(palmad_ctx* ctx, const float* T_dev, int64_t n, int32_t minL, int32_t maxL, int32_t topK,
                            palmad_options& o) {
    if (!o.autotune) return PALMAD_OK;
    auto it = ctx->tuned.find(tune_key(n, minL, maxL, topK, o));
    if (it != ctx->tuned.end()) {
        const int32_t prof = o.profile;
        o = it->second;
        o.profile = prof;
        return PALMAD_OK;
    }
    palmad_tune_report rep{};
    palmad_options t{};
    CKS(tune(ctx, T_dev, n, minL, maxL, topK, o, &t, &rep));
    t.profile = o.profile;
    o = t;
    reset_stats(ctx);
    ctx->stats.tune_ms = rep.tune_ms;
    return PALMAD_OK;
}

}  // namespace

// ======================================================================= C ABI

extern "C" {

palmad_status palmad_default_options(palmad_options* opt) {
    if (!opt) return PALMAD_ERR_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->struct_size = sizeof(palmad_options);
    opt->precision = PALMAD_PREC_FP32;
    opt->exclusive_topk = 1;
    opt->batch_lengths = 0;
    opt->band_rel = 1e-3;
    opt->select_cap = 0;
    opt->reserved_a = 0;
    opt->profile = 0;
    return PALMAD_OK;
}

palmad_status palmad_create(palmad_ctx** out, int device, void* cuda_stream) {
    if (!out) return PALMAD_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return PALMAD_ERR_CUDA;
    }
    if (device < 0 || device >= count) return PALMAD_ERR_ARG;
    palmad_ctx* ctx = new palmad_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        palmad_destroy(ctx);
        return PALMAD_ERR_CUDA;
    }
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            palmad_destroy(ctx);
            return PALMAD_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    ctx->sms = sm_count(device);
    reset_stats(ctx);
    *out = ctx;
    return PALMAD_OK;
}

void palmad_destroy(palmad_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    release(ctx->T); release(ctx->heat_stage); release(ctx->count_stage);
    release(ctx->hints);
    for (LaneSet& s : ctx->sets) release_set(s);
    release(ctx->lanes); release(ctx->st); release(ctx->chain); release(ctx->small);
    release(ctx->pidx); release(ctx->pnn);
    release(ctx->slot_lane); release(ctx->slot_win); release(ctx->route); release(ctx->dlist); release(ctx->dgroups); release(ctx->dead);
    release(ctx->kcnt); release(ctx->dlist_alt);
    release(ctx->acen); release(ctx->asum); release(ctx->cmax); release(ctx->cmax2); release(ctx->gmax); release(ctx->nn2);
    release(ctx->strips); release(ctx->init_flags);
    release(ctx->strip_row); release(ctx->topcen); release(ctx->topsum); release(ctx->seeds); release(ctx->seed_groups);
    if (ctx->h_lanes) cudaFreeHost(ctx->h_lanes);
    if (ctx->h_st) cudaFreeHost(ctx->h_st);
    if (ctx->h_chain) cudaFreeHost(ctx->h_chain);
    if (ctx->h_small) cudaFreeHost(ctx->h_small);
    if (ctx->h_fin_lanes) cudaFreeHost(ctx->h_fin_lanes);
    if (ctx->h_fin_st) cudaFreeHost(ctx->h_fin_st);
    if (ctx->h_pidx) cudaFreeHost(ctx->h_pidx);
    if (ctx->h_pnn) cudaFreeHost(ctx->h_pnn);
    for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
    for (Timing& t : ctx->timings) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* palmad_last_error(const palmad_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

const char* palmad_version(void) { return "palmad-gb300 0.2 (sm_103a)"; }

palmad_status palmad_get_stats(const palmad_ctx* ctx, palmad_stats* out) {
    if (!ctx || !out || out->struct_size != int32_t(sizeof(palmad_stats))) return PALMAD_ERR_ARG;
    *out = ctx->stats;
    return PALMAD_OK;
}

palmad_status palmad_find_discords_device(palmad_ctx* ctx, const float* T_dev, int64_t n, int32_t minL, int32_t maxL,
                                          int32_t topK, const palmad_options* opt, int64_t* out_idx_dev,
                                          double* out_nndist_dev, int64_t* out_count_dev, double* out_r_dev,
                                          float* out_heatmap_dev) {
    CKS(check_args(ctx, n, minL, maxL, topK));
    if (!T_dev || !out_idx_dev || !out_nndist_dev) return fail(ctx, PALMAD_ERR_ARG, "null T or output pointer");
    palmad_options o;
    CKS(read_options(ctx, opt, o));
    CKS(begin_call(ctx, o));
    std::vector<SeriesJob> jobs(1);
    SeriesJob& s = jobs[0];
    CKS(aligned_series(ctx, T_dev, n, ctx->T, &s.T));
    CKS(tuned_options(ctx, s.T, n, minL, maxL, topK, o));
    s.n = n;
    s.minL = minL;
    s.maxL = maxL;
    s.K = topK;
    s.exclusive = o.exclusive_topk != 0;
    s.W = std::max(1, o.batch_lengths);
    const int32_t L = maxL - minL + 1;
    s.heat = out_heatmap_dev;
    s.hw = n - minL + 1;
    DBuf<int64_t> cnt;
    int64_t* count_dev = out_count_dev;
    if (!count_dev) {
        CKS(ensure(ctx, cnt, L));
        count_dev = cnt.p;
    }
    s.count_dev = count_dev;
    palmad_status st = run_jobs(ctx, jobs, o);
    if (st == PALMAD_OK) {
        std::vector<int64_t> counts(L);
        cudaError_t e = cudaMemcpyAsync(out_idx_dev, s.idx.data(), s.idx.size() * sizeof(int64_t),
                                        cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_nndist_dev, s.nn.data(), s.nn.size() * sizeof(double), cudaMemcpyHostToDevice,
                                ctx->stream);
        if (e == cudaSuccess && out_r_dev)
            e = cudaMemcpyAsync(out_r_dev, s.r_final.data(), L * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(counts.data(), count_dev, L * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = fail(ctx, PALMAD_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
        else count_discords(ctx, counts);
        tcollect(ctx);
    }
    release(cnt);
    return st;
}

// One host-pointer series, lengths minL..maxL; a resumed run passes the
// schedule's own first length (minL_sched) and the schedule inputs of the
// lengths just before minL.
static palmad_status find_one(palmad_ctx* ctx, const float* T, int64_t n, int32_t minL, int32_t maxL, int32_t topK,
                              const palmad_options* opt, int64_t* out_idx, double* out_nndist, int64_t* out_count,
                              double* out_r, float* out_heatmap, int32_t minL_sched, const std::vector<double>& hist) {
    palmad_options o;
    CKS(read_options(ctx, opt, o));
    CKS(begin_call(ctx, o));
    const int32_t L = maxL - minL + 1;
    const int64_t hw = n - minL + 1;
    CKS(ensure(ctx, ctx->T, size_t(n)));
    CK(cudaMemcpyAsync(ctx->T.p, T, size_t(n) * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    if (minL_sched == minL) CKS(tuned_options(ctx, ctx->T.p, n, minL, maxL, topK, o));
    // the counts and the heatmap are staged in context buffers kept between
    // calls, so repeated calls do not allocate and free a heatmap that is
    // gigabytes for a long series
    DBuf<int64_t>& cnt = ctx->count_stage;
    DBuf<float>& heat = ctx->heat_stage;
    CKS(ensure(ctx, cnt, L));
    if (out_heatmap) CKS(ensure(ctx, heat, size_t(L) * hw));
    std::vector<SeriesJob> jobs(1);
    SeriesJob& s = jobs[0];
    s.T = ctx->T.p;
    s.n = n;
    s.minL = minL;
    s.maxL = maxL;
    s.K = topK;
    s.exclusive = o.exclusive_topk != 0;
    s.W = std::max(1, o.batch_lengths);
    s.heat = out_heatmap ? heat.p : nullptr;
    s.hw = hw;
    s.count_dev = cnt.p;
    s.minL_sched = minL_sched;
    s.loff = minL - minL_sched;
    s.hist = hist;
    palmad_status st = run_jobs(ctx, jobs, o);
    std::vector<int64_t> counts(L);
    if (st == PALMAD_OK) {
        cudaError_t e = cudaMemcpyAsync(counts.data(), cnt.p, L * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && out_heatmap)
            e = cudaMemcpyAsync(out_heatmap, heat.p, size_t(L) * hw * sizeof(float), cudaMemcpyDeviceToHost,
                                ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = fail(ctx, PALMAD_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
        tcollect(ctx);
    }
    if (st == PALMAD_OK) {
        std::memcpy(out_idx, s.idx.data(), s.idx.size() * sizeof(int64_t));
        std::memcpy(out_nndist, s.nn.data(), s.nn.size() * sizeof(double));
        if (out_count) std::memcpy(out_count, counts.data(), L * sizeof(int64_t));
        if (out_r) std::memcpy(out_r, s.r_final.data(), L * sizeof(double));
        count_discords(ctx, counts);
    }
    return st;
}

palmad_status palmad_find_discords(palmad_ctx* ctx, const float* T, int64_t n, int32_t minL, int32_t maxL,
                                   int32_t topK, const palmad_options* opt, int64_t* out_idx, double* out_nndist,
                                   int64_t* out_count, double* out_r, float* out_heatmap) {
    CKS(check_args(ctx, n, minL, maxL, topK));
    if (!T || !out_idx || !out_nndist) return fail(ctx, PALMAD_ERR_ARG, "null T or output pointer");
    return find_one(ctx, T, n, minL, maxL, topK, opt, out_idx, out_nndist, out_count, out_r, out_heatmap, minL, {});
}

palmad_status palmad_find_discords_resume(palmad_ctx* ctx, const float* T, int64_t n, int32_t minL_sched,
                                          int32_t m0, int32_t maxL, int32_t topK, const palmad_options* opt,
                                          const double* hist, int64_t* out_idx, double* out_nndist,
                                          int64_t* out_count, double* out_r, float* out_heatmap) {
    CKS(check_args(ctx, n, m0, maxL, topK));
    if (minL_sched < 3 || m0 < minL_sched) return fail(ctx, PALMAD_ERR_ARG, "need 3 <= minL_sched <= m0");
    if (!T || !out_idx || !out_nndist) return fail(ctx, PALMAD_ERR_ARG, "null T or output pointer");
    const int32_t nh = std::min(5, m0 - minL_sched);
    if (nh > 0 && !hist) return fail(ctx, PALMAD_ERR_ARG, "null schedule history");
    std::vector<double> h(hist, hist + nh);
    for (double v : h)
        if (!(v >= 0.0) || !std::isfinite(v)) return fail(ctx, PALMAD_ERR_ARG, "schedule history must be finite and >= 0");
    return find_one(ctx, T, n, m0, maxL, topK, opt, out_idx, out_nndist, out_count, out_r, out_heatmap, minL_sched, h);
}

palmad_status palmad_find_discords_batch(palmad_ctx* ctx, int32_t count, const float* const* T, const int64_t* n,
                                         const int32_t* minL, const int32_t* maxL, int32_t topK,
                                         const palmad_options* opt, int64_t* const* out_idx,
                                         double* const* out_nndist, int64_t* const* out_count,
                                         double* const* out_r) {
    if (!ctx) return PALMAD_ERR_ARG;
    if (count < 0 || (count > 0 && (!T || !n || !minL || !maxL || !out_idx || !out_nndist)))
        return fail(ctx, PALMAD_ERR_ARG, "bad batch arrays");
    for (int32_t s = 0; s < count; ++s) {
        CKS(check_args(ctx, n[s], minL[s], maxL[s], topK));
        if (!T[s] || !out_idx[s] || !out_nndist[s]) return fail(ctx, PALMAD_ERR_ARG, "null series or output pointer");
    }
    palmad_options o;
    CKS(read_options(ctx, opt, o));
    CKS(begin_call(ctx, o));
    if (count == 0) return PALMAD_OK;
    // all series in one device buffer, each on a 16-byte boundary
    std::vector<int64_t> off(count);
    int64_t tot = 0;
    for (int32_t s = 0; s < count; ++s) {
        off[s] = tot;
        tot += ((n[s] + 3) / 4) * 4;
    }
    int64_t Ltot = 0;
    for (int32_t s = 0; s < count; ++s) Ltot += maxL[s] - minL[s] + 1;
    CKS(ensure(ctx, ctx->T, size_t(tot)));
    for (int32_t s = 0; s < count; ++s)
        CK(cudaMemcpyAsync(ctx->T.p + off[s], T[s], size_t(n[s]) * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    DBuf<int64_t> cnt;
    CKS(ensure(ctx, cnt, size_t(Ltot)));
    std::vector<SeriesJob> jobs(count);
    int64_t coff = 0;
    for (int32_t s = 0; s < count; ++s) {
        SeriesJob& j = jobs[s];
        j.T = ctx->T.p + off[s];
        j.n = n[s];
        j.minL = minL[s];
        j.maxL = maxL[s];
        j.K = topK;
        j.exclusive = o.exclusive_topk != 0;
        j.W = std::max(1, o.batch_lengths);
        j.count_dev = cnt.p + coff;
        coff += maxL[s] - minL[s] + 1;
    }
    palmad_status st = run_jobs(ctx, jobs, o);
    std::vector<int64_t> counts(size_t(Ltot > 0 ? Ltot : 1));
    if (st == PALMAD_OK) {
        cudaError_t e = cudaMemcpyAsync(counts.data(), cnt.p, Ltot * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = fail(ctx, PALMAD_ERR_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
        tcollect(ctx);
    }
    if (st == PALMAD_OK) {
        coff = 0;
        for (int32_t s = 0; s < count; ++s) {
            const SeriesJob& j = jobs[s];
            const int32_t L = j.maxL - j.minL + 1;
            std::memcpy(out_idx[s], j.idx.data(), j.idx.size() * sizeof(int64_t));
            std::memcpy(out_nndist[s], j.nn.data(), j.nn.size() * sizeof(double));
            if (out_count && out_count[s]) std::memcpy(out_count[s], counts.data() + coff, L * sizeof(int64_t));
            if (out_r && out_r[s]) std::memcpy(out_r[s], j.r_final.data(), L * sizeof(double));
            coff += L;
        }
        count_discords(ctx, counts);
    }
    release(cnt);
    return st;
}

palmad_status palmad_schedule_inputs(const int64_t* idx, const double* nndist, int32_t L, int32_t topK,
                                     double* out) {
    if (L < 0 || topK < 1 || (L > 0 && (!idx || !nndist || !out))) return PALMAD_ERR_ARG;
    for (int32_t l = 0; l < L; ++l) {
        int32_t got = 0;
        while (got < topK && idx[int64_t(l) * topK + got] >= 0) ++got;
        out[l] = got > 0 ? nndist[int64_t(l) * topK + got - 1] : 0.0;
    }
    return PALMAD_OK;
}

palmad_status palmad_autotune(palmad_ctx* ctx, const float* T_dev, int64_t n, int32_t minL, int32_t maxL,
                              int32_t topK, const palmad_options* base, palmad_options* out_opt,
                              palmad_tune_report* report) {
    CKS(check_args(ctx, n, minL, maxL, topK));
    if (!T_dev || !out_opt) return fail(ctx, PALMAD_ERR_ARG, "null T or output pointer");
    if (report && report->struct_size != int32_t(sizeof(palmad_tune_report)))
        return fail(ctx, PALMAD_ERR_ARG, "palmad_tune_report.struct_size mismatch");
    palmad_options o;
    CKS(read_options(ctx, base, o));
    CKS(begin_call(ctx, o));
    const float* T;
    CKS(aligned_series(ctx, T_dev, n, ctx->T, &T));
    palmad_tune_report rep{};
    rep.struct_size = sizeof(palmad_tune_report);
    palmad_options t{};
    CKS(tune(ctx, T, n, minL, maxL, topK, o, &t, &rep));
    reset_stats(ctx);
    ctx->stats.tune_ms = rep.tune_ms;
    *out_opt = t;
    if (report) *report = rep;
    return PALMAD_OK;
}

}  // extern "C"

namespace {

// One lane for a single DRAG call at (m, r) over a host series: uploads T,
// computes the statistics of length m and checks T; the lane covers the
// whole pair space.
palmad_status drag_lane(palmad_ctx* ctx, const float* T, int64_t n, int32_t m, double r, const palmad_options& o,
                        std::vector<PassLane>& req) {
    CKS(ensure(ctx, ctx->T, size_t(n)));
    CK(cudaMemcpyAsync(ctx->T.p, T, size_t(n) * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->sets.empty()) ctx->sets.resize(1);
    LaneSet& S = ctx->sets[0];
    const int64_t N = n - m + 1;
    CKS(ensure_set(ctx, S, N));
    CKS(ensure(ctx, ctx->init_flags, 1));
    CK(cudaMemsetAsync(ctx->init_flags.p, 0, sizeof(int32_t), ctx->stream));
    LAUNCH(PALMAD_K_STATS, launch_stats_init(ctx->T.p, n, m, S.mu.p, S.var.p, ctx->init_flags.p, ctx->stream));
    int32_t flag = 0;
    CK(cudaMemcpyAsync(&flag, ctx->init_flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CKS(sync(ctx));
    if (flag & 1) return fail(ctx, PALMAD_ERR_NONFINITE, "T holds a NaN or an infinity");
    req.assign(1, PassLane{});
    Lane& L = req[0].lane;
    L = Lane{};
    L.T = ctx->T.p;
    L.n = n;
    L.m = m;
    L.N = N;
    L.mu = S.mu.p; L.var = S.var.p; L.win = S.win.p; L.bits0 = S.bits0.p; L.bits = S.bits.p;
    L.surv = S.surv.p; L.slot_of = S.slot_of.p; L.scount = S.scount.p; L.didx = S.didx.p; L.dnn = S.dnn.p;
    L.stats_mode = 2;
    L.mu_src = S.mu.p;
    L.var_src = S.var.p;
    L.r = r;
    L.prune = r > 0.0 ? 1 : 0;
    L.rho_thr = float(1.0 - r * r / (2.0 * m));
    L.band = float(o.band_rel * r * r / m);
    L.strip0 = 0;
    L.strip_lim = INT64_MAX;
    L.col_lo = 0;
    L.col_hi = N;
    req[0].state = LaneState{};
    return PALMAD_OK;
}

palmad_status check_drag_args(palmad_ctx* ctx, const float* T, int64_t n, int32_t m, double r) {
    if (!ctx) return PALMAD_ERR_ARG;
    if (m < 3) return fail(ctx, PALMAD_ERR_ARG, "m must be >= 3");
    if (n < 2 * int64_t(m)) return fail(ctx, PALMAD_ERR_ARG, "n must be >= 2*m");
    if (n > (int64_t(1) << 30)) return fail(ctx, PALMAD_ERR_UNSUPPORTED, "n above 2^30 is not supported");
    if (!T) return fail(ctx, PALMAD_ERR_ARG, "null T");
    if (!std::isfinite(r)) return fail(ctx, PALMAD_ERR_ARG, "r must be finite");
    return PALMAD_OK;
}

}  // namespace

extern "C" {

palmad_status palmad_drag(palmad_ctx* ctx, const float* T, int64_t n, int32_t m, double r, const palmad_options* opt,
                          int64_t* out_idx, double* out_nndist, int64_t cap, int64_t* out_count) {
    CKS(check_drag_args(ctx, T, n, m, r));
    if (!out_count || cap < 0 || (cap > 0 && (!out_idx || !out_nndist)))
        return fail(ctx, PALMAD_ERR_ARG, "bad pointer or cap");
    palmad_options o;
    CKS(read_options(ctx, opt, o));
    CKS(begin_call(ctx, o));
    std::vector<PassLane> req;
    CKS(drag_lane(ctx, T, n, m, r, o, req));
    LaneSet& S = ctx->sets[0];
    PassOut out;
    CKS(run_pass(ctx, req, 1, true, o, out));
    const int64_t cnt = out.st[0].dcount;
    ctx->stats.drag_calls = 1;
    ctx->stats.lengths = 1;
    ctx->stats.discords = cnt;
    const int64_t k = std::min<int64_t>(cap, cnt);
    if (k > 0) {
        std::vector<int32_t> idx(k);
        CK(cudaMemcpyAsync(idx.data(), S.didx.p, k * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(out_nndist, S.dnn.p, k * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CKS(sync(ctx));
        for (int64_t q = 0; q < k; ++q) out_idx[q] = idx[q];
    }
    *out_count = cnt;
    return PALMAD_OK;
}

palmad_status palmad_drag_select_shard(palmad_ctx* ctx, const float* T, int64_t n, int32_t m, double r,
                                       int64_t row_lo, int64_t row_hi, const palmad_options* opt, uint32_t* out_bits) {
    CKS(check_drag_args(ctx, T, n, m, r));
    const int64_t N = n - m + 1;
    if (!out_bits) return fail(ctx, PALMAD_ERR_ARG, "null out_bits");
    if (row_lo < 0 || row_hi < row_lo || row_hi > N) return fail(ctx, PALMAD_ERR_ARG, "need 0 <= row_lo <= row_hi <= N");
    palmad_options o;
    CKS(read_options(ctx, opt, o));
    if (o.knn_k > 1) return fail(ctx, PALMAD_ERR_UNSUPPORTED, "shards run the nearest-neighbour distance only");
    CKS(begin_call(ctx, o));
    std::vector<PassLane> req;
    CKS(drag_lane(ctx, T, n, m, r, o, req));
    Lane& L = req[0].lane;
    L.strip0 = row_lo / kStripH;
    L.strip_lim = (row_hi + kStripH - 1) / kStripH;
    if (row_hi == row_lo) L.strip_lim = L.strip0;
    PassOut out;
    ShardIO io;
    io.mode = kSelect;
    io.bits_host = out_bits;
    CKS(run_pass(ctx, req, 1, true, o, out, io));
    ctx->stats.drag_calls = 1;
    ctx->stats.lengths = 1;
    return PALMAD_OK;
}

palmad_status palmad_drag_refine_shard(palmad_ctx* ctx, const float* T, int64_t n, int32_t m, double r,
                                       const uint32_t* cand_bits, int64_t col_lo, int64_t col_hi,
                                       const palmad_options* opt, double* out_nn) {
    CKS(check_drag_args(ctx, T, n, m, r));
    const int64_t N = n - m + 1;
    if (!cand_bits || !out_nn) return fail(ctx, PALMAD_ERR_ARG, "null cand_bits or out_nn");
    if (col_lo < 0 || col_hi < col_lo || col_hi > N) return fail(ctx, PALMAD_ERR_ARG, "need 0 <= col_lo <= col_hi <= N");
    palmad_options o;
    CKS(read_options(ctx, opt, o));
    if (o.knn_k > 1) return fail(ctx, PALMAD_ERR_UNSUPPORTED, "shards run the nearest-neighbour distance only");
    CKS(begin_call(ctx, o));
    std::vector<PassLane> req;
    CKS(drag_lane(ctx, T, n, m, r, o, req));
    Lane& L = req[0].lane;
    L.col_lo = col_lo;
    L.col_hi = col_hi;
    const int64_t P = (N + 31) / 32;
    DBuf<uint32_t> bits;
    DBuf<double> nn;
    palmad_status st = ensure(ctx, bits, size_t(P));
    if (st == PALMAD_OK) st = ensure(ctx, nn, size_t(N));
    cudaError_t e = cudaSuccess;
    if (st == PALMAD_OK) e = cudaMemcpyAsync(bits.p, cand_bits, sizeof(uint32_t) * size_t(P), cudaMemcpyHostToDevice,
                                             ctx->stream);
    // +inf for every window: windows that are no candidate keep it
    if (st == PALMAD_OK && e == cudaSuccess) {
        std::vector<double> inf(size_t(N), std::numeric_limits<double>::infinity());
        e = cudaMemcpyAsync(nn.p, inf.data(), sizeof(double) * size_t(N), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    if (st == PALMAD_OK && e != cudaSuccess) st = fail(ctx, PALMAD_ERR_CUDA, cudaGetErrorString(e));
    if (st == PALMAD_OK) {
        PassOut out;
        ShardIO io;
        io.mode = kRefine;
        io.bits_dev = bits.p;
        io.nn_dev = nn.p;
        st = run_pass(ctx, req, 1, true, o, out, io);
    }
    if (st == PALMAD_OK) {
        e = cudaMemcpyAsync(out_nn, nn.p, sizeof(double) * size_t(N), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = fail(ctx, PALMAD_ERR_CUDA, cudaGetErrorString(e));
        ctx->stats.drag_calls = 1;
        ctx->stats.lengths = 1;
    }
    release(bits);
    release(nn);
    return st;
}

}  // extern "C"
