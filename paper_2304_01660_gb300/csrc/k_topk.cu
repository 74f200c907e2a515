// Per-length results (Sec. 2.2 and Sec. 5):
//  k_gather  range discords of this DRAG call: live survivors whose FP64
//            nearest-neighbour distance is >= r (Sec. 2.1), appended in
//            ascending index order to the discord list.
//  k_topk    greedy top-K over the list: largest distance first (ties to
//            the lower index), optionally keeping picks >= m apart; one CTA,
//            warp-shuffle argmax per round.
//  k_heat    heatmap row of Eq. 10: nnDist^2 / (2m) at every discord.
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

__global__ void __launch_bounds__(1024) k_gather(const GatherArgs a) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t base_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) base_s = *a.count;
    const int64_t per = (int64_t(a.ns) + blockDim.x - 1) / blockDim.x;
    const int64_t s0 = tid * per, s1 = min64(a.ns, s0 + per);
    auto is_discord = [&](int64_t s) -> bool {
        if (a.dead[s]) return false;
        const unsigned long long b = a.nn2[s];
        if (b >= kInfBits) return false;
        return a.r <= 0.0 || sqrt(__longlong_as_double(static_cast<long long>(b))) >= a.r;
    };
    int32_t cnt = 0;
    for (int64_t s = s0; s < s1; ++s) cnt += is_discord(s);
    int32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int32_t v = warp_tot[lane];
        int32_t s = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += u;
        }
        warp_tot[lane] = s - v;
        if (lane == 31) *a.count = base_s + s;
    }
    __syncthreads();
    int32_t off = base_s + warp_tot[wid] + incl - cnt;
    for (int64_t s = s0; s < s1; ++s) {
        if (!is_discord(s)) continue;
        a.out_idx[off] = a.surv[s];
        a.out_nn[off] = sqrt(__longlong_as_double(static_cast<long long>(a.nn2[s])));
        ++off;
    }
}

// (nn, idx) ordering: larger nn first, then smaller idx.
__device__ __forceinline__ bool better(double nn, int32_t idx, double bnn, int32_t bidx) {
    return nn > bnn || (nn == bnn && idx < bidx);
}

__global__ void __launch_bounds__(1024) k_topk(const TopkArgs a) {
    __shared__ int32_t picks[1024];
    __shared__ double wbest_nn[32];
    __shared__ int32_t wbest_idx[32];
    __shared__ int32_t wbest_pos[32];
    __shared__ int done_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t count = *a.count;
    int got = 0;
    for (int round = 0; round < a.K; ++round) {
        double bnn = -1.0;
        int32_t bidx = 0x7fffffff, bpos = -1;
        for (int32_t p = tid; p < count; p += blockDim.x) {
            const int32_t idx = a.idx[p];
            const double nn = a.nn[p];
            if (!better(nn, idx, bnn, bidx)) continue;
            bool ok = true;
            for (int q = 0; q < got && ok; ++q) {
                const int32_t d = idx - picks[q];
                ok = a.exclusive ? (d >= a.m || d <= -a.m) : (d != 0);
            }
            if (ok) { bnn = nn; bidx = idx; bpos = p; }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const double onn = __shfl_xor_sync(kFull, bnn, o);
            const int32_t oidx = __shfl_xor_sync(kFull, bidx, o);
            const int32_t opos = __shfl_xor_sync(kFull, bpos, o);
            if (opos >= 0 && (bpos < 0 || better(onn, oidx, bnn, bidx))) { bnn = onn; bidx = oidx; bpos = opos; }
        }
        if (lane == 0) { wbest_nn[wid] = bnn; wbest_idx[wid] = bidx; wbest_pos[wid] = bpos; }
        __syncthreads();
        if (tid == 0) {
            double nn = -1.0;
            int32_t idx = 0x7fffffff, pos = -1;
            for (int q = 0; q < int(blockDim.x / 32); ++q)
                if (wbest_pos[q] >= 0 && (pos < 0 || better(wbest_nn[q], wbest_idx[q], nn, idx))) {
                    nn = wbest_nn[q]; idx = wbest_idx[q]; pos = wbest_pos[q];
                }
            done_s = pos < 0;
            if (pos >= 0) {
                picks[got] = idx;
                a.pick_idx[got] = idx;
                a.pick_nn[got] = nn;
            }
        }
        __syncthreads();
        if (done_s) break;
        ++got;
    }
    for (int q = got + tid; q < a.K; q += blockDim.x) {
        a.pick_idx[q] = -1;
        a.pick_nn[q] = 0.0;
    }
}

__global__ void k_heat(const HeatArgs a) {
    const int32_t count = *a.count;
    const double inv2m = 1.0 / (2.0 * a.m);
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < count; p += gridDim.x * blockDim.x) {
        const double nn = a.nn[p];
        a.row[a.idx[p]] = float(nn * nn * inv2m);
    }
}

}  // namespace

cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s) {
    if (a.ns <= 0) return cudaSuccess;
    k_gather<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_topk(const TopkArgs& a, cudaStream_t s) {
    k_topk<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_heat(const HeatArgs& a, cudaStream_t s) {
    k_heat<<<152, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace palmad
