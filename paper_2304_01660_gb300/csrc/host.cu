// Host driver of libpalmad: context and workspace, the MERLIN threshold
// schedule (Algorithm 1) and the per-call DRAG orchestration (Algorithms
// 2-4), behind the C ABI of include/palmad.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "palmad.h"
#include "palmad_dev.cuh"

using namespace palmad;

namespace {

constexpr int kSelectH = 256;                    // rows per select strip (32 lanes x 8)
constexpr int kDefaultCap = 512;                 // select columns past the strip triangle
constexpr int kRefineSeg = 512;                  // refine sweep columns per work item (multiple of 256)
constexpr int kMaxTopK = 1024;

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
};

// Small device-side counters, reset per DRAG call (flags persist per length).
struct Small {
    int32_t work[4];          // 0 select, 1 direct refine, 2 sweep refine
    int32_t nsurv;
    int32_t dcount;
    uint32_t maxerr;
    int32_t nref;             // strips swept by refine (this batch)
    int32_t ndirect;          // survivors refined by the direct form (this batch)
    int32_t pad[3];
    unsigned long long pairs[8];  // 0 select, 1 direct refine, 2 fp64, 3 select seeds,
                                  // 4 sweep refine, 5 sweep refine seeds
};
struct Flags {
    int32_t flags;  // |1 non-finite, |2 flat window at the current length
    uint32_t ab[2]; // max |df| inv, max |dg| inv over the windows (float bits)
    int32_t pad;
};

struct Timing {
    int kid;
    cudaEvent_t a, b;
};

}  // namespace

struct palmad_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int sel_grid = 0, ref_grid = 0;

    DBuf<float> T;
    DBuf<double> mu[2], var[2];
    DBuf<float4> win;
    DBuf<uint32_t> bits, bits0;
    DBuf<int32_t> surv, slot_of, strips, direct;
    DBuf<float> acen, asum, cmax;
    DBuf<int32_t> scount;
    DBuf<uint32_t> gmax;
    DBuf<int32_t> dead;
    DBuf<unsigned long long> nn2;
    DBuf<int32_t> didx;
    DBuf<double> dnn;
    DBuf<int64_t> pidx;
    DBuf<double> pnn;
    DBuf<float> heat;
    DBuf<Small> small;
    DBuf<Flags> flags;

    Small* h_small = nullptr;
    Flags* h_flags = nullptr;
    int64_t* h_pidx = nullptr;
    double* h_pnn = nullptr;

    palmad_stats stats{};
    bool profile = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<Timing> timings;
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

// After a stream synchronize: fold recorded launch times into the stats.
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
    if (o.batch_lengths < 0) return fail(ctx, PALMAD_ERR_ARG, "batch_lengths must be >= 0");
    return PALMAD_OK;
}

// ------------------------------------------------------------ workspace

struct Job {
    const float* T;  // device
    int64_t n;
    int32_t minL, maxL, K;
    bool exclusive;
    palmad_options opt;
    int cur = 0;       // mu/var buffer holding the current length
    int32_t m = 0;     // current length
    int32_t refine_cap = 0;
    int32_t kpad_max = 0;
    int32_t nchunks_max = 0;
};

palmad_status reserve(palmad_ctx* ctx, Job& job) {
    const int64_t Nmax = job.n - job.minL + 1;
    const int64_t Pmax = (Nmax + 31) / 32;
    for (int b = 0; b < 2; ++b) {
        CKS(ensure(ctx, ctx->mu[b], Nmax));
        CKS(ensure(ctx, ctx->var[b], Nmax));
    }
    CKS(ensure(ctx, ctx->win, Nmax));
    CKS(ensure(ctx, ctx->bits, Pmax));
    CKS(ensure(ctx, ctx->bits0, Pmax));
    CKS(ensure(ctx, ctx->surv, Nmax));
    CKS(ensure(ctx, ctx->slot_of, Nmax));
    CKS(ensure(ctx, ctx->strips, (Nmax + kSelectH - 1) / kSelectH));
    CKS(ensure(ctx, ctx->didx, Nmax));
    CKS(ensure(ctx, ctx->dnn, Nmax));
    CKS(ensure(ctx, ctx->pidx, kMaxTopK));
    CKS(ensure(ctx, ctx->pnn, kMaxTopK));
    CKS(ensure(ctx, ctx->small, 1));
    CKS(ensure(ctx, ctx->flags, 1));
    job.kpad_max = ((job.maxL + 31) / 32) * 32;
    job.nchunks_max = int32_t((Nmax + 31) / 32);
    // survivors refined per batch: bounded by the per-chunk max table (<= 256 MB)
    int64_t cap = (int64_t(1) << 26) / std::max(1, job.nchunks_max);
    cap = std::min<int64_t>(cap, 16384);
    cap = std::max<int64_t>(64, (cap / 64) * 64);
    job.refine_cap = int32_t(cap);
    CKS(ensure(ctx, ctx->acen, size_t(cap) * job.kpad_max));
    CKS(ensure(ctx, ctx->asum, size_t(cap)));
    CKS(ensure(ctx, ctx->direct, size_t(cap)));
    CKS(ensure(ctx, ctx->cmax, size_t(cap) * job.nchunks_max));
    CKS(ensure(ctx, ctx->scount, (Nmax + kSelectH - 1) / kSelectH + 1));
    CKS(ensure(ctx, ctx->gmax, size_t(cap)));
    CKS(ensure(ctx, ctx->dead, size_t(cap)));
    CKS(ensure(ctx, ctx->nn2, size_t(cap)));
    return PALMAD_OK;
}

// ---------------------------------------------------- statistics per length

// Prepare length m: first length by direct (sliding) Eq. 4, later lengths by
// the Eq. 7-8 recurrence from m-1.
palmad_status prepare_length(palmad_ctx* ctx, Job& job, int32_t m, bool first) {
    CK(cudaMemsetAsync(ctx->flags.p, 0, sizeof(Flags), ctx->stream));
    StatsArgs a{};
    a.T = job.T;
    a.n = job.n;
    a.m = m;
    if (first) {
        LAUNCH(PALMAD_K_STATS, launch_stats_init(job.T, job.n, m, ctx->mu[0].p, ctx->var[0].p, &ctx->flags.p->flags,
                                                 ctx->stream));
        job.cur = 0;
        a.advance = 0;
        a.mu_old = ctx->mu[0].p;
        a.var_old = ctx->var[0].p;
        a.mu = ctx->mu[0].p;
        a.var = ctx->var[0].p;
    } else {
        a.advance = 1;
        a.mu_old = ctx->mu[job.cur].p;
        a.var_old = ctx->var[job.cur].p;
        a.mu = ctx->mu[job.cur ^ 1].p;
        a.var = ctx->var[job.cur ^ 1].p;
        job.cur ^= 1;
    }
    a.win = ctx->win.p;
    a.bits = ctx->bits0.p;
    a.flags = &ctx->flags.p->flags;
    a.ab = ctx->flags.p->ab;
    LAUNCH(PALMAD_K_STATS, launch_stats_step(a, ctx->stream));
    job.m = m;
    if (first) {
        CK(cudaMemcpyAsync(ctx->h_flags, ctx->flags.p, sizeof(Flags), cudaMemcpyDeviceToHost, ctx->stream));
        CKS(sync(ctx));
        if (ctx->h_flags->flags & 1) return fail(ctx, PALMAD_ERR_NONFINITE, "T holds a NaN or an infinity");
    }
    return PALMAD_OK;
}

// ------------------------------------------------------------ one DRAG call

struct DragResult {
    int32_t got = 0;      // top-K picks found
    int32_t count = 0;    // range discords
};

palmad_status drag_call(palmad_ctx* ctx, Job& job, double r, DragResult& out) {
    const int32_t m = job.m;
    const int64_t n = job.n;
    const int64_t N = n - m + 1;
    const int64_t P = (N + 31) / 32;
    const double r2 = r * r;
    const double rho_thr = 1.0 - r2 / (2.0 * m);
    const double band = job.opt.band_rel * r2 / m;
    const int64_t cap = job.opt.select_cap > 0 ? job.opt.select_cap : kDefaultCap;
    Thresh th{};
    th.rho_thr = float(rho_thr);
    th.band = float(band);
    th.prune = r > 0.0 ? 1 : 0;
    th.m = m;
    th.H = kSelectH;
    th.ab = ctx->flags.p->ab;

    CK(cudaMemsetAsync(ctx->small.p, 0, sizeof(Small), ctx->stream));
    CK(cudaMemcpyAsync(ctx->bits.p, ctx->bits0.p, P * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream));

    SweepArgs sa{};
    sa.T = job.T;
    sa.n = n;
    sa.N = N;
    sa.m = m;
    sa.win = ctx->win.p;
    sa.th = th;
    sa.work = &ctx->small.p->work[0];
    sa.pairs = &ctx->small.p->pairs[0];
    sa.seeds = &ctx->small.p->pairs[3];
    sa.bits = ctx->bits.p;
    sa.cap = cap;
    if (r > 0.0) LAUNCH(PALMAD_K_SELECT, launch_select(sa, ctx->sel_grid, ctx->stream));

    CompactArgs ca{ctx->bits.p, N, ctx->surv.p, &ctx->small.p->nsurv};
    LAUNCH(PALMAD_K_COMPACT, launch_compact(ca, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_small, ctx->small.p, sizeof(Small), cudaMemcpyDeviceToHost, ctx->stream));
    CKS(sync(ctx));
    const int32_t nsurv = ctx->h_small->nsurv;
    ctx->stats.survivors += nsurv;
    ctx->stats.device_passes += 1;

    const int32_t kpad = ((m + 31) / 32) * 32;
    const int32_t nchunks = int32_t((N + 31) / 32);
    const int64_t nstrip_all = (N + kSelectH - 1) / kSelectH;
    for (int32_t b0 = 0; b0 < nsurv; b0 += job.refine_cap) {
        const int32_t ns = std::min(job.refine_cap, nsurv - b0);
        const int32_t* surv = ctx->surv.p + b0;
        CK(cudaMemsetAsync(ctx->gmax.p, 0, ns * sizeof(uint32_t), ctx->stream));
        CK(cudaMemsetAsync(ctx->dead.p, 0, ns * sizeof(int32_t), ctx->stream));
        CK(cudaMemsetAsync(ctx->nn2.p, 0x7f, ns * sizeof(unsigned long long), ctx->stream));
        CK(cudaMemsetAsync(ctx->slot_of.p, 0xff, N * sizeof(int32_t), ctx->stream));
        CK(cudaMemsetAsync(&ctx->small.p->work[1], 0, 2 * sizeof(int32_t), ctx->stream));
        CK(cudaMemsetAsync(&ctx->small.p->nref, 0, 2 * sizeof(int32_t), ctx->stream));
        CK(cudaMemsetAsync(ctx->scount.p, 0, nstrip_all * sizeof(int32_t), ctx->stream));
        const int32_t thr = std::max(2, (5 * kSelectH + m + m - 1) / m);
        LAUNCH(PALMAD_K_PLAN, launch_plan(surv, ns, ctx->win.p, kSelectH, thr, ctx->slot_of.p, ctx->scount.p, ctx->strips.p,
                                            &ctx->small.p->nref, ctx->direct.p, &ctx->small.p->ndirect, ctx->stream));
        LAUNCH(PALMAD_K_PLAN,
               launch_refine_prep(job.T, ctx->win.p, surv, ns, m, kpad, ctx->acen.p, ctx->asum.p, ctx->stream));
        SweepArgs wa{};
        wa.T = job.T;
        wa.n = n;
        wa.N = N;
        wa.m = m;
        wa.win = ctx->win.p;
        wa.th = th;
        wa.work = &ctx->small.p->work[2];
        wa.pairs = &ctx->small.p->pairs[4];
        wa.seeds = &ctx->small.p->pairs[5];
        wa.strips = ctx->strips.p;
        wa.nref = &ctx->small.p->nref;
        wa.seg = kRefineSeg;
        wa.slot_of = ctx->slot_of.p;
        wa.dead = ctx->dead.p;
        wa.gmax = ctx->gmax.p;
        wa.cmax = ctx->cmax.p;
        wa.nchunks = nchunks;
        LAUNCH(PALMAD_K_REFINE_SWEEP, launch_refine_sweep(wa, ctx->sel_grid, ctx->stream));
        RefineArgs ra{};
        ra.list = ctx->direct.p;
        ra.nlist = &ctx->small.p->ndirect;
        ra.T = job.T;
        ra.n = n;
        ra.N = N;
        ra.m = m;
        ra.kpad = kpad;
        ra.win = ctx->win.p;
        ra.surv = surv;
        ra.ns = ns;
        ra.acen = ctx->acen.p;
        ra.asum = ctx->asum.p;
        ra.th = th;
        ra.nchunks = nchunks;
        ra.gmax = ctx->gmax.p;
        ra.dead = ctx->dead.p;
        ra.cmax = ctx->cmax.p;
        ra.flags = &ctx->flags.p->flags;
        ra.work = &ctx->small.p->work[1];
        ra.pairs = &ctx->small.p->pairs[1];
        LAUNCH(PALMAD_K_REFINE_DIRECT, launch_refine(ra, ctx->ref_grid, ctx->stream));
        RecheckArgs rc{};
        rc.T = job.T;
        rc.n = n;
        rc.N = N;
        rc.m = m;
        rc.kpad = kpad;
        rc.win = ctx->win.p;
        rc.mu = ctx->mu[job.cur].p;
        rc.var = ctx->var[job.cur].p;
        rc.surv = surv;
        rc.ns = ns;
        rc.acen = ctx->acen.p;
        rc.gmax = ctx->gmax.p;
        rc.dead = ctx->dead.p;
        rc.cmax = ctx->cmax.p;
        rc.nchunks = nchunks;
        rc.th = th;
        rc.nn2 = ctx->nn2.p;
        rc.flags = &ctx->flags.p->flags;
        rc.pairs = &ctx->small.p->pairs[2];
        rc.maxerr = &ctx->small.p->maxerr;
        LAUNCH(PALMAD_K_RECHECK, launch_recheck(rc, ctx->stream));
        GatherArgs ga{surv, ns, ctx->dead.p, ctx->nn2.p, r, ctx->didx.p, ctx->dnn.p, &ctx->small.p->dcount};
        LAUNCH(PALMAD_K_GATHER, launch_gather(ga, ctx->stream));
    }
    TopkArgs ta{ctx->didx.p, ctx->dnn.p, &ctx->small.p->dcount, job.K, m, job.exclusive ? 1 : 0, ctx->pidx.p,
                ctx->pnn.p};
    LAUNCH(PALMAD_K_TOPK, launch_topk(ta, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_small, ctx->small.p, sizeof(Small), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_pidx, ctx->pidx.p, job.K * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_pnn, ctx->pnn.p, job.K * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CKS(sync(ctx));
    const Small& sm = *ctx->h_small;
    ctx->stats.select_pairs += int64_t(sm.pairs[0]);
    ctx->stats.refine_pairs += int64_t(sm.pairs[1]);
    ctx->stats.refine_pairs += int64_t(sm.pairs[4]);
    ctx->stats.select_flops += 5.0 * double(sm.pairs[0]) + 2.0 * m * double(sm.pairs[3]);
    ctx->stats.refine_flops += 2.0 * m * double(sm.pairs[1]);
    ctx->stats.sweep_flops += 5.0 * double(sm.pairs[4]) + 2.0 * m * double(sm.pairs[5]);
    ctx->stats.fp64_pairs += int64_t(sm.pairs[2]);
    {
        uint32_t e = sm.maxerr;
        if (e) {
            uint32_t bbits = (e & 0x80000000u) ? (e & 0x7fffffffu) : ~e;
            float f;
            std::memcpy(&f, &bbits, 4);
            ctx->stats.max_fp32_rho_err = std::max(ctx->stats.max_fp32_rho_err, double(f));
        }
    }
    out.count = sm.dcount;
    out.got = 0;
    while (out.got < job.K && ctx->h_pidx[out.got] >= 0) ++out.got;
    return PALMAD_OK;
}

// ------------------------------------------------------------- MERLIN

struct LengthOut {
    std::vector<int64_t> idx;
    std::vector<double> nn;
    std::vector<int64_t> count;
    std::vector<double> r;
};

// One schedule step: DRAG at r, then the success test of reading R6.
palmad_status try_r(palmad_ctx* ctx, Job& job, double r, DragResult& res, bool& ok) {
    CKS(drag_call(ctx, job, r, res));
    ctx->stats.drag_calls += 1;
    ok = res.got == job.K;
    return PALMAD_OK;
}

palmad_status merlin(palmad_ctx* ctx, Job& job, LengthOut& out, float* heat_dev) {
    const int32_t L = job.maxL - job.minL + 1;
    const int64_t W = job.n - job.minL + 1;
    out.idx.assign(size_t(L) * job.K, -1);
    out.nn.assign(size_t(L) * job.K, 0.0);
    out.count.assign(L, 0);
    out.r.assign(L, 0.0);
    std::vector<double> sched(L, 0.0);
    if (heat_dev) CK(cudaMemsetAsync(heat_dev, 0, size_t(L) * W * sizeof(float), ctx->stream));
    for (int32_t l = 0; l < L; ++l) {
        const int32_t m = job.minL + l;
        CKS(prepare_length(ctx, job, m, l == 0));
        DragResult res;
        bool ok = false;
        double r;
        if (l == 0) {
            r = 2.0 * std::sqrt(double(job.minL));
            for (int h = 0;; ++h) {
                if (h >= 60) r = 0.0;
                CKS(try_r(ctx, job, r, res, ok));
                if (ok || r <= 0.0) break;
                r = 0.5 * r;
            }
        } else if (l <= 4) {
            r = 0.99 * sched[l - 1];
            for (int h = 0;; ++h) {
                if (h >= 3000 || r <= 0.0) r = 0.0;
                CKS(try_r(ctx, job, r, res, ok));
                if (ok || r <= 0.0) break;
                r = 0.99 * r;
            }
        } else {
            double mean = 0.0, var = 0.0;
            for (int q = 1; q <= 5; ++q) mean += sched[l - q];
            mean /= 5.0;
            for (int q = 1; q <= 5; ++q) var += (sched[l - q] - mean) * (sched[l - q] - mean);
            const double sdv = std::sqrt(var / 4.0);
            const double step = sdv > 0.0 ? sdv : 0.01 * mean;
            r = mean - 2.0 * sdv;
            for (int h = 0;; ++h) {
                if (h >= 3000 || r <= 0.0) r = 0.0;
                CKS(try_r(ctx, job, r, res, ok));
                if (ok || r <= 0.0) break;
                r = step > 0.0 ? r - step : 0.0;
            }
        }
        for (int q = 0; q < res.got; ++q) {
            out.idx[size_t(l) * job.K + q] = ctx->h_pidx[q];
            out.nn[size_t(l) * job.K + q] = ctx->h_pnn[q];
        }
        sched[l] = res.got > 0 ? ctx->h_pnn[res.got - 1] : 0.0;
        out.count[l] = res.count;
        out.r[l] = r;
        ctx->stats.discords += res.count;
        if (heat_dev && res.count > 0) {
            HeatArgs ha{ctx->didx.p, ctx->dnn.p, &ctx->small.p->dcount, m, heat_dev + size_t(l) * W};
            LAUNCH(PALMAD_K_HEAT, launch_heat(ha, ctx->stream));
        }
    }
    ctx->stats.lengths += L;
    return PALMAD_OK;
}

palmad_status check_args(palmad_ctx* ctx, int64_t n, int32_t minL, int32_t maxL, int32_t topK) {
    if (!ctx) return PALMAD_ERR_ARG;
    if (minL < 3) return fail(ctx, PALMAD_ERR_ARG, "minL must be >= 3");
    if (maxL < minL) return fail(ctx, PALMAD_ERR_ARG, "maxL must be >= minL");
    if (n < 2 * int64_t(maxL)) return fail(ctx, PALMAD_ERR_ARG, "n must be >= 2*maxL");
    if (n > (int64_t(1) << 30)) return fail(ctx, PALMAD_ERR_UNSUPPORTED, "n above 2^30 is not supported");
    if (topK < 1 || topK > kMaxTopK) return fail(ctx, PALMAD_ERR_ARG, "topK must lie in [1, 1024]");
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
    opt->use_graph = 0;
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
    auto bail = [&](palmad_status st) {
        palmad_destroy(ctx);
        return st;
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(PALMAD_ERR_CUDA);
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(PALMAD_ERR_CUDA);
        ctx->own_stream = true;
    }
    if (cudaMallocHost(&ctx->h_small, sizeof(Small)) != cudaSuccess) return bail(PALMAD_ERR_OOM);
    if (cudaMallocHost(&ctx->h_flags, sizeof(Flags)) != cudaSuccess) return bail(PALMAD_ERR_OOM);
    if (cudaMallocHost(&ctx->h_pidx, kMaxTopK * sizeof(int64_t)) != cudaSuccess) return bail(PALMAD_ERR_OOM);
    if (cudaMallocHost(&ctx->h_pnn, kMaxTopK * sizeof(double)) != cudaSuccess) return bail(PALMAD_ERR_OOM);
    ctx->sel_grid = sweep_grid(device);
    ctx->ref_grid = refine_grid(device);
    reset_stats(ctx);
    *out = ctx;
    return PALMAD_OK;
}

void palmad_destroy(palmad_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    release(ctx->T);
    for (int b = 0; b < 2; ++b) {
        release(ctx->mu[b]);
        release(ctx->var[b]);
    }
    release(ctx->win);
    release(ctx->bits);
    release(ctx->bits0);
    release(ctx->surv);
    release(ctx->slot_of);
    release(ctx->strips);
    release(ctx->direct);
    release(ctx->acen);
    release(ctx->asum);
    release(ctx->cmax);
    release(ctx->scount);
    release(ctx->gmax);
    release(ctx->dead);
    release(ctx->nn2);
    release(ctx->didx);
    release(ctx->dnn);
    release(ctx->pidx);
    release(ctx->pnn);
    release(ctx->heat);
    release(ctx->small);
    release(ctx->flags);
    if (ctx->h_small) cudaFreeHost(ctx->h_small);
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
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

const char* palmad_version(void) { return "palmad-gb300 0.1 (sm_103a)"; }

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
    // The sweeps copy the series with 16-byte asynchronous copies: stage a
    // series that does not start on a 16-byte boundary.
    if (reinterpret_cast<uintptr_t>(T_dev) % 16 != 0) {
        CKS(ensure(ctx, ctx->T, size_t(n)));
        CK(cudaMemcpyAsync(ctx->T.p, T_dev, size_t(n) * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
        T_dev = ctx->T.p;
    }
    Job job{};
    job.T = T_dev;
    job.n = n;
    job.minL = minL;
    job.maxL = maxL;
    job.K = topK;
    job.exclusive = o.exclusive_topk != 0;
    job.opt = o;
    CKS(reserve(ctx, job));
    LengthOut lo;
    CKS(merlin(ctx, job, lo, out_heatmap_dev));
    const int32_t L = maxL - minL + 1;
    CK(cudaMemcpyAsync(out_idx_dev, lo.idx.data(), lo.idx.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(out_nndist_dev, lo.nn.data(), lo.nn.size() * sizeof(double), cudaMemcpyHostToDevice,
                       ctx->stream));
    if (out_count_dev)
        CK(cudaMemcpyAsync(out_count_dev, lo.count.data(), L * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    if (out_r_dev) CK(cudaMemcpyAsync(out_r_dev, lo.r.data(), L * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CKS(sync(ctx));
    return PALMAD_OK;
}

palmad_status palmad_find_discords(palmad_ctx* ctx, const float* T, int64_t n, int32_t minL, int32_t maxL,
                                   int32_t topK, const palmad_options* opt, int64_t* out_idx, double* out_nndist,
                                   int64_t* out_count, double* out_r, float* out_heatmap) {
    CKS(check_args(ctx, n, minL, maxL, topK));
    if (!T || !out_idx || !out_nndist) return fail(ctx, PALMAD_ERR_ARG, "null T or output pointer");
    palmad_options o;
    CKS(read_options(ctx, opt, o));
    CKS(begin_call(ctx, o));
    CKS(ensure(ctx, ctx->T, size_t(n)));
    CK(cudaMemcpyAsync(ctx->T.p, T, size_t(n) * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    Job job{};
    job.T = ctx->T.p;
    job.n = n;
    job.minL = minL;
    job.maxL = maxL;
    job.K = topK;
    job.exclusive = o.exclusive_topk != 0;
    job.opt = o;
    CKS(reserve(ctx, job));
    const int32_t L = maxL - minL + 1;
    const int64_t W = n - minL + 1;
    float* heat_dev = nullptr;
    if (out_heatmap) {
        CKS(ensure(ctx, ctx->heat, size_t(L) * W));
        heat_dev = ctx->heat.p;
    }
    LengthOut lo;
    CKS(merlin(ctx, job, lo, heat_dev));
    if (heat_dev) {
        CK(cudaMemcpyAsync(out_heatmap, heat_dev, size_t(L) * W * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        CKS(sync(ctx));
    }
    std::memcpy(out_idx, lo.idx.data(), lo.idx.size() * sizeof(int64_t));
    std::memcpy(out_nndist, lo.nn.data(), lo.nn.size() * sizeof(double));
    if (out_count) std::memcpy(out_count, lo.count.data(), L * sizeof(int64_t));
    if (out_r) std::memcpy(out_r, lo.r.data(), L * sizeof(double));
    return PALMAD_OK;
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
    palmad_stats total{};
    total.struct_size = sizeof(palmad_stats);
    for (int32_t s = 0; s < count; ++s) {
        const int32_t L = maxL[s] - minL[s] + 1;
        std::vector<int64_t> idx(size_t(L) * topK), cnt(L);
        std::vector<double> nn(size_t(L) * topK), rr(L);
        CKS(palmad_find_discords(ctx, T[s], n[s], minL[s], maxL[s], topK, opt, idx.data(), nn.data(), cnt.data(),
                                 rr.data(), nullptr));
        std::memcpy(out_idx[s], idx.data(), idx.size() * sizeof(int64_t));
        std::memcpy(out_nndist[s], nn.data(), nn.size() * sizeof(double));
        if (out_count && out_count[s]) std::memcpy(out_count[s], cnt.data(), L * sizeof(int64_t));
        if (out_r && out_r[s]) std::memcpy(out_r[s], rr.data(), L * sizeof(double));
        const palmad_stats& st = ctx->stats;
        total.lengths += st.lengths;
        total.drag_calls += st.drag_calls;
        total.device_passes += st.device_passes;
        total.select_pairs += st.select_pairs;
        total.refine_pairs += st.refine_pairs;
        total.fp64_pairs += st.fp64_pairs;
        total.survivors += st.survivors;
        total.discords += st.discords;
        total.max_fp32_rho_err = std::max(total.max_fp32_rho_err, st.max_fp32_rho_err);
        total.select_flops += st.select_flops;
        total.refine_flops += st.refine_flops;
        total.sweep_flops += st.sweep_flops;
        for (int k = 0; k < PALMAD_K_COUNT; ++k) {
            total.launches[k] += st.launches[k];
            total.kernel_ms[k] += st.kernel_ms[k];
        }
    }
    ctx->stats = total;
    return PALMAD_OK;
}

palmad_status palmad_drag(palmad_ctx* ctx, const float* T, int64_t n, int32_t m, double r, const palmad_options* opt,
                          int64_t* out_idx, double* out_nndist, int64_t cap, int64_t* out_count) {
    if (!ctx) return PALMAD_ERR_ARG;
    if (m < 3) return fail(ctx, PALMAD_ERR_ARG, "m must be >= 3");
    if (n < 2 * int64_t(m)) return fail(ctx, PALMAD_ERR_ARG, "n must be >= 2*m");
    if (!T || !out_count || cap < 0 || (cap > 0 && (!out_idx || !out_nndist)))
        return fail(ctx, PALMAD_ERR_ARG, "bad pointer or cap");
    if (!std::isfinite(r)) return fail(ctx, PALMAD_ERR_ARG, "r must be finite");
    palmad_options o;
    CKS(read_options(ctx, opt, o));
    CKS(begin_call(ctx, o));
    CKS(ensure(ctx, ctx->T, size_t(n)));
    CK(cudaMemcpyAsync(ctx->T.p, T, size_t(n) * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    Job job{};
    job.T = ctx->T.p;
    job.n = n;
    job.minL = m;
    job.maxL = m;
    job.K = 1;
    job.exclusive = true;
    job.opt = o;
    CKS(reserve(ctx, job));
    CKS(prepare_length(ctx, job, m, true));
    DragResult res;
    CKS(drag_call(ctx, job, r, res));
    ctx->stats.drag_calls += 1;
    ctx->stats.lengths = 1;
    ctx->stats.discords = res.count;
    const int64_t k = std::min<int64_t>(cap, res.count);
    if (k > 0) {
        std::vector<int32_t> idx(k);
        CK(cudaMemcpyAsync(idx.data(), ctx->didx.p, k * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(out_nndist, ctx->dnn.p, k * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CKS(sync(ctx));
        for (int64_t q = 0; q < k; ++q) out_idx[q] = idx[q];
    }
    *out_count = res.count;
    return PALMAD_OK;
}

}  // extern "C"
