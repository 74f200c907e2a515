// Window statistics: mean and deviation of every length-m window (Eq. 4),
// carried from m to m+1 by the recurrences of Eq. 7-8 (Sec. 3.1.1), plus the
// per-window FP32 records the pair kernels read and the candidate bitmaps.
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr int kRun = 16;                              // windows per thread in the init pass
constexpr double kFlatRel = 2.384185791015625e-07;    // 2^-22: flat window threshold
constexpr double kNearFlatRel = 3.814697265625e-06;   // 2^-18: recompute two-pass below this

// Initial statistics at the first length (Eq. 4).  Each thread slides over
// kRun consecutive windows with sums shifted by the run's first value; a
// window whose deviation comes out near the flat threshold is recomputed
// two-pass so that the flat decision is exact.
__global__ void k_stats_init(const float* __restrict__ T, int64_t n, int32_t m, double* __restrict__ mu,
                             double* __restrict__ var, int32_t* __restrict__ flags) {
    const int64_t N = n - m + 1;
    const int64_t i0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * kRun;
    if (i0 >= N) return;
    const double tref = T[i0];
    double S = 0.0, SS = 0.0;
    bool bad = false;
    for (int k = 0; k < m; ++k) {
        const float x = T[i0 + k];
        bad |= !isfinite(x);
        const double d = double(x) - tref;
        S += d;
        SS += d * d;
    }
    const double inv_m = 1.0 / double(m);
    const int64_t i1 = min(i0 + kRun, N);
    for (int64_t i = i0; i < i1; ++i) {
        if (i > i0) {
            const float xa = T[i + m - 1], xr = T[i - 1];
            bad |= !isfinite(xa);
            const double da = double(xa) - tref, dr = double(xr) - tref;
            S += da - dr;
            SS += da * da - dr * dr;
        }
        const double mean_s = S * inv_m;
        double v = fmax(SS * inv_m - mean_s * mean_s, 0.0);
        double mean = tref + mean_s;
        if (v <= (kNearFlatRel * mean) * (kNearFlatRel * mean)) {
            double s2 = 0.0;
            for (int k = 0; k < m; ++k) s2 += double(T[i + k]);
            mean = s2 * inv_m;
            double q = 0.0;
            for (int k = 0; k < m; ++k) {
                const double d = double(T[i + k]) - mean;
                q += d * d;
            }
            v = q * inv_m;
        }
        mu[i] = mean;
        var[i] = v;
    }
    if (bad) atomicOr(flags, 1);
}

// New (mu, var) of window i at length m from its values at m-1 (Eq. 7-8);
// inv_m = 1/m.
__device__ __forceinline__ void advance_one(double mu_o, double var_o, float t_new, int32_t m, double inv_m,
                                            double& mu_n, double& var_n) {
    const double mm1 = double(m - 1);
    const double d = mu_o - double(t_new);
    mu_n = (mm1 * mu_o + double(t_new)) * inv_m;
    var_n = mm1 * inv_m * (var_o + d * d * inv_m);
}

// Statistics of every lane of a pass.  blockIdx.y selects a chain of lanes
// (consecutive lengths of one series); a thread owns a fixed set of window
// indices i and walks the chain, so lane l+1 advances (Eq. 7-8) from the
// values lane l just wrote at the same i.  Per lane it writes the FP64
// mean / variance, the FP32 window records, the candidate bitmaps and the
// maxima behind the FP32 error bound.
__global__ void k_stats(const Pass p, const int32_t* __restrict__ chain_first) {
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int l = chain_first[blockIdx.y];; ++l) {
        const Lane& L = p.lanes[l];
        LaneState& S = p.st[l];
        const int64_t N = L.N;
        const int32_t m = L.m;
        const int64_t P = (N + 31) / 32;
        const float* T = L.T;
        if (L.stats_mode != 0) {
            bool any_flat = false;
            float amax = 0.f, bmax = 0.f;
            const double inv_m = 1.0 / double(m);
            for (int64_t i = tid; i < N; i += stride) {
                double mu_i, var_i;
                const float t_add = T[i + m - 1];
                if (L.stats_mode == 1) advance_one(L.mu_src[i], L.var_src[i], t_add, m, inv_m, mu_i, var_i);
                else { mu_i = L.mu_src[i]; var_i = L.var_src[i]; }
                L.mu[i] = mu_i;
                L.var[i] = var_i;
                // sigma <= 2^-22 |mu|, compared squared (a variance the recurrence
                // left slightly negative counts as flat)
                const double fl = kFlatRel * mu_i;
                const bool flat = var_i <= fl * fl;
                any_flat |= flat;
                float df = 0.f, dg = 0.f;
                if (i >= 1) {
                    // mu_{i-1} = mu_i - (t[i+m-1] - t[i-1]) / m for windows of one length
                    const double diff = double(t_add) - double(T[i - 1]);
                    const double mu_p = mu_i - diff * inv_m;
                    df = float(0.5 * diff);
                    dg = float((double(t_add) - mu_i) + (double(T[i - 1]) - mu_p));
                }
                const float inv = flat ? 0.f : rsqrtf(float(double(m) * var_i));
                L.win[i] = make_float4(df, dg, inv, float(mu_i));
                amax = fmaxf(amax, fabsf(df) * inv);
                bmax = fmaxf(bmax, fabsf(dg) * inv);
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
            }
            if ((threadIdx.x & 31) == 0) {
                atomicMax(&S.ab[0], __float_as_uint(amax));
                atomicMax(&S.ab[1], __float_as_uint(bmax));
            }
            if (any_flat) atomicOr(&S.flags, 2);
            // Candidate bitmap: a window starts alive iff it has a non-self match.
            for (int64_t w = tid; w < P; w += stride) {
                uint32_t word = 0;
                for (int b = 0; b < 32; ++b) {
                    const int64_t i = w * 32 + b;
                    if (i < N && (i + m <= N - 1 || i - m >= 0)) word |= 1u << b;
                }
                L.bits0[w] = word;
                L.bits[w] = word;
            }
        } else {
            for (int64_t w = tid; w < P; w += stride) L.bits[w] = L.bits0[w];
        }
        if (!L.chain_next) break;
    }
}

}  // namespace

cudaError_t launch_stats_init(const float* T, int64_t n, int32_t m, double* mu, double* var, int32_t* flags,
                              cudaStream_t s) {
    const int64_t N = n - m + 1;
    const int64_t threads = (N + kRun - 1) / kRun;
    const int block = 128;
    const int grid = int((threads + block - 1) / block);
    k_stats_init<<<grid, block, 0, s>>>(T, n, m, mu, var, flags);
    return cudaGetLastError();
}

cudaError_t launch_stats(const Pass& p, const int32_t* chain_first, int32_t nchains, int64_t nmax, int sms,
                         cudaStream_t s) {
    if (nchains <= 0) return cudaSuccess;
    const int block = 256;
    int64_t gx = (nmax + block - 1) / block;
    if (gx > int64_t(sms) * 8) gx = int64_t(sms) * 8;  // 8 CTAs per SM cover every chain
    k_stats<<<dim3(unsigned(gx), unsigned(nchains)), block, 0, s>>>(p, chain_first);
    return cudaGetLastError();
}

int sm_count(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms;
}

}  // namespace palmad
