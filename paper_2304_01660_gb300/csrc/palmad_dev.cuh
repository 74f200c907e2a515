// Internal declarations shared by the CUDA translation units of libpalmad.
//
// Notation follows the paper: T is the series (Eq. 1), m the window length,
// N = n - m + 1 the number of windows (Sec. 2.1), mu / sigma the window mean
// and population deviation (Eq. 4).  Distances use Eq. 6 in its centred
// form: with cov(i, j) = sum_k (t[i+k] - mu_i)(t[j+k] - mu_j),
//     rho = cov / (m sigma_i sigma_j),   ED^2_norm = 2m (1 - rho).
// Every kernel works on rho; d < r  <=>  rho > 1 - r^2 / (2m).
//
// Work is organised in passes.  A pass holds one or more lanes; a lane is one
// DRAG evaluation (Algorithm 2): one series, one length m, one threshold r.
// Every kernel of a pass processes all its lanes, so many lengths (and many
// series) share each launch.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace palmad {

constexpr int kWarp = 32;
constexpr float kInf = __builtin_huge_valf();
constexpr int kStripH = 128;   // rows per strip of the select sweep (32 lanes x 4)
constexpr int kRefineH = 128;  // rows per strip of the refine sweep (32 lanes x 4) ...
constexpr int kRefineHTall = 256;  // ... or, chosen per pass, 32 lanes x 8 (fewer top-row seeds per row)
constexpr int kCoarseMin = 1024;  // smallest coarse block of the chunk maxima (the pool is sized for it)
constexpr int kSelPieceCols = 512;       // columns per select work item (a strip's scan is cut into pieces)
constexpr int kSelPieceColsShort = 256;  // the same for passes with too few strips to fill the GPU
constexpr int kMaxK = 1024;    // largest top-K
constexpr int kDGroup = 256;   // direct-form survivors per group (packed per lane; the direct kernels split them)
constexpr int kMaxKnn = 16;    // largest k of the k-th neighbour variant

// Per-window data the FP32 kernels read, one 16-byte record per window:
//   x = df_i = (t[i+m-1] - t[i-1]) / 2          (Eq. 9 diagonal update)
//   y = dg_i = (t[i+m-1] - mu_i) + (t[i-1] - mu_{i-1})
//   z = inv_i = 1 / (sqrt(m) sigma_i), 0 for a flat window
//   w = mu_i (FP32)
// so that cov(i, j) = cov(i-1, j-1) + df_i dg_j + df_j dg_i.
using WinRec = float4;

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// Order-preserving float <-> uint32 map (for atomicMax on floats of any sign).
__device__ __forceinline__ uint32_t enc_f32(float x) {
    uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float dec_f32(uint32_t e) {
    uint32_t b = (e & 0x80000000u) ? (e & 0x7fffffffu) : ~e;
    return __uint_as_float(b);
}

// One DRAG evaluation.  Written by the host before the pass.
struct Lane {
    const float* T;        // series, 16-byte aligned
    int64_t n;
    int64_t N;             // windows at this length
    int32_t m;
    int32_t kpad;          // m rounded up to 32
    // statistics (Eq. 4, Eq. 7-8): 0 keep, 1 advance from src (m-1), 2 copy src
    int32_t stats_mode;
    int32_t chain_next;    // 1 when the next lane advances from this one
    const double* mu_src;
    const double* var_src;
    double* mu;
    double* var;
    WinRec* win;
    uint32_t* bits0;       // initial candidate bitmap (windows with a non-self match)
    uint32_t* bits;        // working candidate bitmap
    int32_t* surv;         // survivors of select, ascending
    int32_t* slot_of;      // window -> pool slot of this round, -1 otherwise
    int32_t* scount;       // per refine strip: survivors this round (+ flat flag in bit 30)
    int32_t* didx;         // range discords found (ascending), with
    double* dnn;           //   their FP64 nearest-neighbour distances
    float* heat;           // heatmap row or nullptr
    int64_t* count_out;    // where finalize adds the range-discord count, or nullptr
    // threshold
    double r;
    float rho_thr;         // 1 - r^2 / (2m)
    float band;            // band_rel * r^2 / m
    int32_t prune;         // 0 when r <= 0
    int32_t nstrips;       // select strips
    int64_t strip_base;    // prefix of nstrips over the lanes
    // refine round: survivors [k_lo, k_hi) occupy pool slots from slot_base
    int32_t k_lo, k_hi;
    int32_t slot_base;
    int32_t pad;
    // per window of the series (shared by every lane of the series): a
    // column near a pair that pruned the window at some length, -1 if none
    // (nullptr: hints off)
    int32_t* hint;
    // a shard of the pair space (one series split over ranks): select runs
    // the strips from strip0 on (nstrips of them), refine compares
    // survivors with the columns [col_lo, col_hi) only; whole lane
    // otherwise (strip0 = 0, col_lo = 0, col_hi >= N)
    int64_t strip0, strip_lim;  // select strips [strip0, min(all strips, strip_lim))
    int64_t col_lo, col_hi;
};

// Per-lane device-written state.
struct LaneState {
    int32_t flags;         // |1 non-finite, |2 flat window present
    uint32_t ab[2];        // max |df| inv, max |dg| inv (float bits), see eps_bound
    int32_t nsurv;         // survivors of select
    int32_t dcount;        // range discords gathered
    int32_t got;           // top-K picks
    int32_t count_final;   // range discords at the final r (finalize)
    uint32_t maxerr;       // enc_f32 of the largest |rho_fp32 - rho_fp64| seen
    int32_t ndirect;       // survivors of this refine round routed to the direct form
    int32_t seed_rows;     // refine strips of this round asking for tensor-core seeds
    int32_t seed_base;     // their first row in the seed buffer
    int32_t seed_eff;      // rows granted (seed_rows clipped to the buffer)
    uint32_t seed_eps;     // float bits: error bound of the tensor-core seeds (rho units)
};

// Everything a pass kernel needs, passed by value.
struct Pass {
    const Lane* lanes;
    LaneState* st;
    int32_t nl;
    int32_t K;
    int32_t exclusive;
    int32_t seg;           // refine sweep columns per work item (multiple of 256)
    int64_t cap;           // select columns per strip past its triangle
    int64_t sel_items;     // total select strips
    int32_t sel_pieces;    // column pieces per select strip
    int32_t sel_cols;      // columns per select piece (multiple of 32)
    int32_t knn;           // k-th neighbour distance (1: nearest neighbour)
    int32_t direct_below;  // > 0: strips with fewer survivors take the direct form
    int64_t nmax;          // largest N over the lanes
    // refine pool (this round)
    int32_t nslots;        // slots in use this round (64-aligned per lane)
    int32_t kpad_max;
    int32_t nchunks_max;   // 32-column chunks of the largest lane
    int32_t mixed;         // 1: direct refine on the tensor cores (k_refine_tc)
    int32_t kpad_pass;     // largest kpad of this pass's lanes (kpad_max is the pool's stride)
    int32_t refine_h;      // rows per refine strip this pass: kRefineH or kRefineHTall
    int32_t* slot_lane;    // [slots] lane of each slot
    int32_t* slot_win;     // [slots] window of each slot, -1 for padding
    int32_t* route;        // [slots] 0 sweep, 1 direct, -1 none
    int32_t* dlist;        // [slots] direct-form slots of each lane, packed from its slot_base
    int32_t* dgroups;      // [slots/64] first dlist entry of every kDGroup-entry group holding direct slots
    float* acen;           // [slots][kpad_max] centred survivor windows
    float* asum;           // [slots]
    uint32_t* gmax;        // [slots] enc_f32 of the maximum rho
    int32_t* dead;         // [slots]
    int32_t* kcnt;         // [slots] k-th neighbour variant: pairs past the pruning threshold so far
    unsigned long long* nn2;  // [slots] FP64 bits of the smallest d^2
    float* cmax;           // [slots][nchunks_max] maximum rho per 32-column chunk
    uint32_t* cmax2;       // [slots][ncoarse_max] enc_f32 of the maximum per coarse block (seg columns:
                           //   a refine segment is one coarse block; 1024 or 2048)
    int32_t ncoarse_max;
    int32_t pad6;
    int2* strips;          // (lane, strip) swept by refine
    int32_t* nref;
    // tensor-core top-row seeds of refine strips (mixed precision)
    int32_t tc_seeds;      // 1: strips with >= seed_min survivors take seeds from `seeds`
    int32_t seed_min;
    int32_t* strip_row;    // [slots] per refine strip: its lane-local seed row, -1 for none
    float* topcen;         // [seed_cap][kpad_max] centred top-row windows
    float* topsum;         // [seed_cap]
    float* seeds;          // [seed_cap][seed_stride] cov(top row, j)
    int64_t seed_stride;
    int32_t seed_cap;      // rows in the seed buffer
    int32_t pad4;
    int4* seed_groups;     // (lane, first row, rows, -) per group of <= 32 rows of one lane
    int32_t* seed_ngroups;
    int32_t sharded;       // 1: a lane restricts its columns (k_prep clears every coarse maximum)
    int32_t tc_ns;         // survivors per tensor-core MMA (0: 64, or 32 for windows above 512)
    int32_t* dlist_alt;    // [slots] second packed direct list (alive survivors re-packed between column chunks)
    int64_t tc_col_lo, tc_col_hi;  // the tensor-core direct refine's columns this launch (multiples of 2048)
    double* shard_nn;      // [N of lane 0] per-candidate result of a refine shard, or nullptr
    int32_t* err;          // set to 1 by a kernel whose bounded wait gave up
    int32_t* work;         // [8] work counters, zeroed per launch group
    unsigned long long* pairs;  // [12] 0 select, 1 direct refine, 2 fp64, 3 select seeds,
                                //      4 sweep refine, 5 sweep seeds, 6 tensor-core seeds,
                                //      7 hint pairs, 8 survivors removed by hints,
                                //      9 swept refine strips, 10 survivors in them
    int64_t* pick_idx;     // [nl][K]
    double* pick_nn;       // [nl][K]
};

// FP32 error bound on rho and the pruning threshold of a lane, from the
// per-length window maxima the statistics kernel records:
//   a = |df_i| inv_i,  b = |dg_i| inv_i.
// A row of a strip sweep is at most H-1 recurrence steps away from a
// directly computed dot product (H the tallest strip, 256 rows); each step adds at most
// 2u + 3u (a_i b_j + a_j b_i) to rho, and a direct dot product of m terms at
// most ~2mu (1 + 14 a) (centring offsets within 8 columns), u = 2^-24.  The
// bound doubles that sum.
__device__ __forceinline__ float eps_bound(int32_t m, const LaneState& s) {
    const float u = 5.9604644775390625e-08f;
    const float amax = __uint_as_float(__ldcg(&s.ab[0]));
    const float bmax = __uint_as_float(__ldcg(&s.ab[1]));
    const float rec = float(kRefineHTall - 1) * (2.f + 6.f * amax * bmax);
    const float dir = 2.f * float(m + 4) * (1.f + 14.f * amax);
    // top-row seeds from the tensor cores carry their own bound (0 otherwise)
    return 2.f * u * (rec + dir + 32.f) + __uint_as_float(__ldcg(&s.seed_eps));
}
__device__ __forceinline__ float rho_prune_of(const Lane& L, const LaneState& s) {
    return L.prune ? L.rho_thr + fmaxf(eps_bound(L.m, s), L.band) : kInf;
}

// Lane of a global item index given the per-lane prefix `base` (ascending)
// staged in shared memory: largest l with base[l] <= item.
__device__ __forceinline__ int lane_of(const int64_t* base, int nl, int64_t item) {
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Launchers (each returns the launch's cudaError_t).
cudaError_t launch_stats_init(const float* T, int64_t n, int32_t m, double* mu, double* var, int32_t* flags,
                              cudaStream_t s);
cudaError_t launch_stats(const Pass& p, const int32_t* chain_first, int32_t nchains, int64_t nmax, int sms,
                         cudaStream_t s);
cudaError_t launch_select(const Pass& p, int grid, cudaStream_t s);
cudaError_t launch_compact(const Pass& p, cudaStream_t s);
bool hint_supported(const Pass& p);
cudaError_t launch_hint(const Pass& p, int sms, cudaStream_t s);
cudaError_t launch_plan(const Pass& p, cudaStream_t s);
cudaError_t launch_refine_sweep(const Pass& p, int grid, cudaStream_t s);
cudaError_t launch_refine_direct(const Pass& p, int grid, cudaStream_t s);
bool refine_tc_supported(const Pass& p);
bool seed_tc_supported(const Pass& p);
cudaError_t launch_seeds(const Pass& p, int sms, cudaStream_t s);
cudaError_t launch_refine_tc(const Pass& p, int sms, cudaStream_t s);
bool refine_tcs_supported(const Pass& p);
cudaError_t launch_refine_tcs(const Pass& p, int sms, cudaStream_t s);
cudaError_t launch_direct_repack(const Pass& p, cudaStream_t s);
cudaError_t launch_recheck(const Pass& p, int grid, cudaStream_t s);
cudaError_t launch_round_cleanup(const Pass& p, cudaStream_t s);
cudaError_t launch_shard_out(const Pass& p, cudaStream_t s);
cudaError_t launch_gather(const Pass& p, cudaStream_t s);
cudaError_t launch_topk(const Pass& p, cudaStream_t s);
cudaError_t launch_finalize(const Pass& p, cudaStream_t s);
int sm_count(int device);

}  // namespace palmad
