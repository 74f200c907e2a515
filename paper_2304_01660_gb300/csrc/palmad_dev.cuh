// Internal declarations shared by the CUDA translation units of libpalmad.
//
// Notation follows the paper: T is the series (Eq. 1), m the window length,
// N = n - m + 1 the number of windows (Sec. 2.1), mu / sigma the window mean
// and population deviation (Eq. 4).  Distances use Eq. 6 in its centred
// form: with cov(i, j) = sum_k (t[i+k] - mu_i)(t[j+k] - mu_j),
//     rho = cov / (m sigma_i sigma_j),   ED^2_norm = 2m (1 - rho).
// Every kernel works on rho; d < r  <=>  rho > 1 - r^2 / (2m).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace palmad {

constexpr int kWarp = 32;
constexpr float kInf = __builtin_huge_valf();

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

// FP32 error bound on rho and the pruning threshold, evaluated on the device
// from per-length window maxima the statistics kernel records:
//   a = |df_i| inv_i,  b = |dg_i| inv_i   (ab[0], ab[1]: float bits, >= 0).
// A row of a strip sweep is at most H-1 recurrence steps away from a
// directly computed dot product; each step adds at most
// 2u + 3u (a_i b_j + a_j b_i) to rho, and a direct dot product of m terms at
// most ~2mu (1 + 14 a) (centring offsets within 8 columns), u = 2^-24.  The
// bound below doubles that sum.
struct Thresh {
    float rho_thr;   // 1 - r^2 / (2m): d < r  <=>  rho > rho_thr
    float band;      // band_rel * r^2 / m: the |d - r| < band_rel r floor in rho units
    int32_t prune;   // 0 when r <= 0 (nothing is ever pruned)
    int32_t m;
    int32_t H;       // strip height of the sweeps
    const uint32_t* ab;
};

__device__ __forceinline__ float eps_bound(const Thresh& t) {
    const float u = 5.9604644775390625e-08f;
    const float amax = __uint_as_float(__ldcg(&t.ab[0]));
    const float bmax = __uint_as_float(__ldcg(&t.ab[1]));
    const float rec = float(t.H - 1) * (2.f + 6.f * amax * bmax);
    const float dir = 2.f * float(t.m + 4) * (1.f + 14.f * amax);
    return 2.f * u * (rec + dir + 32.f);
}
__device__ __forceinline__ float rho_prune_of(const Thresh& t) {
    return t.prune ? t.rho_thr + fmaxf(eps_bound(t), t.band) : kInf;
}

struct StatsArgs {
    const float* T;
    int64_t n;
    int32_t m;           // length being prepared
    int32_t advance;     // 1: Eq. 7-8 from (mu_old, var_old) at m-1; 0: copy
    const double* mu_old;
    const double* var_old;
    double* mu;          // [N] FP64 mean at m
    double* var;         // [N] FP64 variance at m
    WinRec* win;         // [N]
    uint32_t* bits;      // [ceil(N/32)] candidate bitmap, initialised here
    int32_t* flags;      // [0] |= 1 non-finite, |= 2 flat window present
    uint32_t* ab;        // [2] max a, max b (float bits) -- see Thresh
};

// Strip sweeps (select and the recurrence form of refine).
struct SweepArgs {
    const float* T;
    int64_t n;
    int64_t N;
    int32_t m;
    const WinRec* win;
    Thresh th;           // a pair prunes iff rho_fp32 > rho_prune_of(th)
    int32_t* work;       // work counter (zeroed before launch)
    unsigned long long* pairs;  // evaluated pairs
    unsigned long long* seeds;  // direct dot products computed (top-row / first-column)
    // select
    uint32_t* bits;      // candidate bitmap
    int64_t cap;         // columns scanned per strip beyond its triangle
    // refine
    const int32_t* strips;  // strips (of 32*D rows) to sweep
    const int32_t* nref;    // number of strips (device)
    int32_t seg;         // columns per work item (multiple of 256)
    const int32_t* slot_of; // window -> survivor slot of this batch, -1 otherwise
    int32_t* dead;       // [slots]
    uint32_t* gmax;      // [slots] enc_f32 of the maximum rho
    float* cmax;         // [slots][nchunks] maximum rho per 32-column chunk
    int32_t nchunks;
};

struct CompactArgs {
    const uint32_t* bits;
    int64_t N;
    int32_t* surv;       // out: ascending survivor indices
    int32_t* nsurv;      // out: count
};

struct RefineArgs {
    const int32_t* list;   // survivor slots handled by the direct form
    const int32_t* nlist;  // their number (device)
    const float* T;
    int64_t n;
    int64_t N;
    int32_t m;
    int32_t kpad;        // m rounded up to the K chunk
    const WinRec* win;
    const int32_t* surv; // survivor indices of this batch
    int32_t ns;          // survivors in this batch
    const float* acen;   // [ns][kpad] centred survivor windows (FP32)
    const float* asum;   // [ns] sum of acen row
    Thresh th;           // mark dead iff rho_fp32 > rho_prune_of(th)
    int32_t nchunks;     // 32-column chunks
    uint32_t* gmax;      // [ns] enc_f32 of max rho
    int32_t* dead;       // [ns]
    float* cmax;         // [ns][nchunks] maximum rho per 32-column chunk
    const int32_t* flags;
    int32_t* work;
    unsigned long long* pairs;
};

struct RecheckArgs {
    const float* T;
    int64_t n;
    int64_t N;
    int32_t m;
    int32_t kpad;
    const WinRec* win;
    const double* mu;
    const double* var;
    const int32_t* surv;
    int32_t ns;
    const float* acen;
    const uint32_t* gmax;
    const int32_t* dead;
    const float* cmax;
    int32_t nchunks;
    Thresh th;           // columns with rho_fp32 >= max - 2 eps_bound(th) are re-checked
    unsigned long long* nn2;   // [ns] FP64 bits of min d^2 (atomicMin)
    const int32_t* flags;
    unsigned long long* pairs;
    unsigned int* maxerr;      // enc of max |rho_fp32 - rho_fp64|
};

struct GatherArgs {
    const int32_t* surv;
    int32_t ns;
    const int32_t* dead;
    const unsigned long long* nn2;
    double r;
    int32_t* out_idx;    // discord list (appended)
    double* out_nn;
    int32_t* count;      // running count (device)
};

struct TopkArgs {
    const int32_t* idx;
    const double* nn;
    const int32_t* count;
    int32_t K;
    int32_t m;
    int32_t exclusive;
    int64_t* pick_idx;   // [K]
    double* pick_nn;     // [K]
};

struct HeatArgs {
    const int32_t* idx;
    const double* nn;
    const int32_t* count;
    int32_t m;
    float* row;
};

// Launchers (each returns the launch's cudaError_t).
cudaError_t launch_stats_init(const float* T, int64_t n, int32_t m, double* mu, double* var,
                              int32_t* flags, cudaStream_t s);
cudaError_t launch_stats_step(const StatsArgs& a, cudaStream_t s);
cudaError_t launch_select(const SweepArgs& a, int grid, cudaStream_t s);
cudaError_t launch_refine_sweep(const SweepArgs& a, int grid, cudaStream_t s);
int sweep_grid(int device);
cudaError_t launch_plan(const int32_t* surv, int32_t ns, const WinRec* win, int32_t H, int32_t thr, int32_t* slot_of,
                        int32_t* scount, int32_t* strips, int32_t* nstrips, int32_t* direct, int32_t* ndirect,
                        cudaStream_t s);
cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s);
cudaError_t launch_refine_prep(const float* T, const WinRec* win, const int32_t* surv, int32_t ns, int32_t m,
                               int32_t kpad, float* acen, float* asum, cudaStream_t s);
cudaError_t launch_refine(const RefineArgs& a, int grid, cudaStream_t s);
int refine_grid(int device);
cudaError_t launch_recheck(const RecheckArgs& a, cudaStream_t s);
cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s);
cudaError_t launch_topk(const TopkArgs& a, cudaStream_t s);
cudaError_t launch_heat(const HeatArgs& a, cudaStream_t s);

}  // namespace palmad
