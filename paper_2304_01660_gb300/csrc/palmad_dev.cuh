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
};

struct SelectArgs {
    const float* T;
    int64_t n;
    int64_t N;
    int32_t m;
    const WinRec* win;
    uint32_t* bits;
    float rho_prune;     // prune pair iff rho_fp32 > rho_prune
    int64_t cap;         // columns scanned per strip beyond its triangle
    int32_t* work;       // work counter (zeroed before launch)
    unsigned long long* pairs;  // evaluated valid pairs
};

struct CompactArgs {
    const uint32_t* bits;
    int64_t N;
    int32_t* surv;       // out: ascending survivor indices
    int32_t* nsurv;      // out: count
};

struct RefineArgs {
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
    float rho_prune;     // mark dead iff rho_fp32 > rho_prune
    int32_t ntiles;      // column tiles of 256
    uint32_t* gmax;      // [ns] enc_f32 of max rho
    int32_t* dead;       // [ns]
    float* tilemax;      // [ns][ntiles]
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
    const float* tilemax;
    int32_t ntiles;
    float eps2;          // 2 * FP32 rho error bound
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
cudaError_t launch_select(const SelectArgs& a, int grid, cudaStream_t s);
int select_grid(int device);
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
