// palmad_discord_interest: the most interesting discords across lengths
// (Eq. 11, Sec. 5).  The interest of index i is the largest discord-heatmap
// value over the lengths (Eq. 10: nnDist^2 / (2m) at the range discords of
// length m, 0 elsewhere) and its length the smallest m reaching it; the
// top-K interesting discords are taken greedily by (interest desc, index
// asc) among indices of positive interest, optionally with windows that do
// not overlap an earlier pick.
//
//  k_interest_max   one thread per index, a column maximum down the L rows
//                   of the heatmap (coalesced: consecutive threads read
//                   consecutive columns of a row); bound by the heatmap read,
//                   L x W x 4 bytes of HBM.
//  k_interest_topk  one CTA: K rounds of a block-wide arg-max over the
//                   eligible indices.
#include "palmad.h"
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void k_interest_max(const float* __restrict__ heat, int32_t L, int64_t W, int32_t minL,
                               float* __restrict__ score, int32_t* __restrict__ best_m) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < W; i += int64_t(gridDim.x) * blockDim.x) {
        float best = heat[i];
        int32_t at = 0;
        int32_t l = 1;
        for (; l + 4 <= L; l += 4) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcs(heat + int64_t(l + u) * W + i);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (v[u] > best) { best = v[u]; at = l + u; }
        }
        for (; l < L; ++l) {
            const float v = __ldcs(heat + int64_t(l) * W + i);
            if (v > best) { best = v; at = l; }
        }
        score[i] = best;
        best_m[i] = minL + at;
    }
}

__device__ __forceinline__ bool better(float s, int64_t i, float bs, int64_t bi) {
    return s > bs || (s == bs && i < bi);
}

__global__ void __launch_bounds__(1024) k_interest_topk(const float* __restrict__ score, const int32_t* __restrict__ best_m,
                                                        int64_t W, int32_t K, int32_t exclusive, int64_t* out_idx,
                                                        int32_t* out_m, float* out_score) {
    __shared__ int64_t pick_i[kMaxK];
    __shared__ int32_t pick_m[kMaxK];
    __shared__ float ws[32];
    __shared__ int64_t wi[32];
    __shared__ int done_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int got = 0;
    for (; got < K; ++got) {
        float bs = 0.f;
        int64_t bi = -1;
        for (int64_t i = tid; i < W; i += blockDim.x) {
            const float s = score[i];
            if (!(s > 0.f) || (bi >= 0 && !better(s, i, bs, bi))) continue;
            bool ok = true;
            const int32_t mi = best_m[i];
            for (int g = 0; g < got && ok; ++g) {
                if (pick_i[g] == i) ok = false;
                else if (exclusive && i < pick_i[g] + pick_m[g] && pick_i[g] < i + mi) ok = false;
            }
            if (ok) { bs = s; bi = i; }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const float os = __shfl_xor_sync(kFull, bs, o);
            const int64_t oi = __shfl_xor_sync(kFull, bi, o);
            if (oi >= 0 && (bi < 0 || better(os, oi, bs, bi))) { bs = os; bi = oi; }
        }
        if (lane == 0) { ws[wid] = bs; wi[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            float s = 0.f;
            int64_t i = -1;
            for (int q = 0; q < int(blockDim.x >> 5); ++q)
                if (wi[q] >= 0 && (i < 0 || better(ws[q], wi[q], s, i))) { s = ws[q]; i = wi[q]; }
            done_s = i < 0;
            if (i >= 0) {
                pick_i[got] = i;
                pick_m[got] = best_m[i];
                out_idx[got] = i;
                out_m[got] = best_m[i];
                out_score[got] = s;
            }
        }
        __syncthreads();
        if (done_s) break;
    }
    for (int g = got + tid; g < K; g += blockDim.x) {
        out_idx[g] = -1;
        out_m[g] = 0;
        out_score[g] = 0.f;
    }
}

}  // namespace

}  // namespace palmad

extern "C" palmad_status palmad_discord_interest(const float* heat_dev, int32_t L, int64_t W, int32_t minL, int32_t K,
                                                 int32_t exclusive, float* score_dev, int32_t* best_m_dev,
                                                 int64_t* out_idx_dev, int32_t* out_m_dev, float* out_score_dev,
                                                 void* cuda_stream) {
    using namespace palmad;
    if (!heat_dev || !score_dev || !best_m_dev || !out_idx_dev || !out_m_dev || !out_score_dev || L < 1 || W < 1 ||
        minL < 1 || K < 1 || K > kMaxK)
        return PALMAD_ERR_ARG;
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return PALMAD_ERR_CUDA;
    }
    const int64_t blocks = min64((W + 255) / 256, int64_t(sms) * 8);
    k_interest_max<<<unsigned(blocks), 256, 0, s>>>(heat_dev, L, W, minL, score_dev, best_m_dev);
    k_interest_topk<<<1, 1024, 0, s>>>(score_dev, best_m_dev, W, K, exclusive ? 1 : 0, out_idx_dev, out_m_dev,
                                       out_score_dev);
    if (cudaGetLastError() != cudaSuccess) return PALMAD_ERR_CUDA;
    return PALMAD_OK;
}
