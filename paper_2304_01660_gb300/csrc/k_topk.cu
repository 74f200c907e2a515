// Per-lane results (Sec. 2.2 and Sec. 5):
//  k_round_cleanup undoes a refine round's window -> slot map and per-strip
//                 survivor counts.
//  k_gather       range discords of the lane: live survivors whose FP64
//                 nearest-neighbour distance is >= r (Sec. 2.1), appended in
//                 ascending index order to the lane's discord list.
//  k_topk         greedy top-K over the lane's list: largest distance first
//                 (ties to the lower index), optionally keeping picks >= m
//                 apart; one CTA per lane, warp-shuffle argmax per round.
//  k_finalize     at the final r of each lane: the number of range
//                 discords and the heatmap row of Eq. 10 (nnDist^2 / (2m)).
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

// Undo the round's window -> slot map and per-strip counts (both stay -1 /
// 0 between rounds, so only the entries a round wrote need clearing).
__global__ void k_round_cleanup(const Pass p) {
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < p.nslots; g += gridDim.x * blockDim.x) {
        const int l = p.slot_lane[g];
        const Lane& L = p.lanes[l];
        if (g == L.slot_base) {
            p.st[l].ndirect = 0;
            p.st[l].seed_rows = 0;
        }
        const int32_t w = p.slot_win[g];
        if (w < 0) continue;
        L.slot_of[w] = -1;
        L.scount[w / p.refine_h] = 0;
    }
}

// Result of a refine shard for the round's candidates: -1 for a candidate
// that some pair of the shard's columns pruned (d < r), else its FP64
// nearest-neighbour distance over those columns (+inf when none is a
// non-self match).  One lane per pass.
__global__ void k_shard_out(const Pass p) {
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < p.nslots; g += gridDim.x * blockDim.x) {
        const int32_t w = p.slot_win[g];
        if (w < 0) continue;
        const unsigned long long b = p.nn2[g];
        p.shard_nn[w] = p.dead[g] ? -1.0 : (b >= kInfBits ? __longlong_as_double(static_cast<long long>(kInfBits))
                                                          : sqrt(__longlong_as_double(static_cast<long long>(b))));
    }
}

__global__ void __launch_bounds__(1024) k_gather(const Pass p) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t base_s;
    const int l = blockIdx.x;
    const Lane& L = p.lanes[l];
    LaneState& S = p.st[l];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t ns = L.k_hi - L.k_lo;
    if (tid == 0) base_s = S.dcount;
    const int64_t per = (int64_t(ns) + blockDim.x - 1) / blockDim.x;
    const int64_t s0 = tid * per, s1 = min64(ns, s0 + per);
    auto is_discord = [&](int64_t s) -> bool {
        const int64_t g = L.slot_base + s;
        if (p.dead[g]) return false;
        const unsigned long long b = p.nn2[g];
        if (b >= kInfBits) return false;
        return L.r <= 0.0 || sqrt(__longlong_as_double(static_cast<long long>(b))) >= L.r;
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
        if (lane == 31) S.dcount = base_s + s;
    }
    __syncthreads();
    int32_t off = base_s + warp_tot[wid] + incl - cnt;
    for (int64_t s = s0; s < s1; ++s) {
        if (!is_discord(s)) continue;
        const int64_t g = L.slot_base + s;
        L.didx[off] = p.slot_win[g];
        L.dnn[off] = sqrt(__longlong_as_double(static_cast<long long>(p.nn2[g])));
        ++off;
    }
}

// (nn, idx) ordering: larger nn first, then smaller idx.
__device__ __forceinline__ bool better(double nn, int32_t idx, double bnn, int32_t bidx) {
    return nn > bnn || (nn == bnn && idx < bidx);
}

__global__ void __launch_bounds__(1024) k_topk(const Pass p) {
    __shared__ int32_t picks[kMaxK];
    __shared__ double wbest_nn[32];
    __shared__ int32_t wbest_idx[32];
    __shared__ int32_t wbest_pos[32];
    __shared__ int done_s;
    const int l = blockIdx.x;
    const Lane& L = p.lanes[l];
    LaneState& S = p.st[l];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t count = S.dcount;
    const int32_t m = L.m;
    int64_t* pidx = p.pick_idx + int64_t(l) * p.K;
    double* pnn = p.pick_nn + int64_t(l) * p.K;
    int got = 0;
    for (int round = 0; round < p.K; ++round) {
        double bnn = -1.0;
        int32_t bidx = 0x7fffffff, bpos = -1;
        for (int32_t q = tid; q < count; q += blockDim.x) {
            const int32_t idx = L.didx[q];
            const double nn = L.dnn[q];
            if (!better(nn, idx, bnn, bidx)) continue;
            bool ok = true;
            for (int r = 0; r < got && ok; ++r) {
                const int32_t d = idx - picks[r];
                ok = p.exclusive ? (d >= m || d <= -m) : (d != 0);
            }
            if (ok) { bnn = nn; bidx = idx; bpos = q; }
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
                pidx[got] = idx;
                pnn[got] = nn;
            }
        }
        __syncthreads();
        if (done_s) break;
        ++got;
    }
    for (int q = got + tid; q < p.K; q += blockDim.x) {
        pidx[q] = -1;
        pnn[q] = 0.0;
    }
    if (tid == 0) S.got = got;
}

__global__ void k_finalize(const Pass p) {
    const int l = blockIdx.y;
    const Lane& L = p.lanes[l];
    LaneState& S = p.st[l];
    const int32_t count = S.dcount;
    const double inv2m = 1.0 / (2.0 * L.m);
    int32_t c = 0;
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
        const double nn = L.dnn[q];
        if (L.r > 0.0 && nn < L.r) continue;
        ++c;
        if (L.heat) L.heat[L.didx[q]] = float(nn * nn * inv2m);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) {
        atomicAdd(&S.count_final, c);
        if (L.count_out) atomicAdd(reinterpret_cast<unsigned long long*>(L.count_out), (unsigned long long)c);
    }
}

}  // namespace

cudaError_t launch_round_cleanup(const Pass& p, cudaStream_t s) {
    if (p.nslots <= 0) return cudaSuccess;
    const int grid = int(min64((int64_t(p.nslots) + 255) / 256, 1024));
    k_round_cleanup<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_shard_out(const Pass& p, cudaStream_t s) {
    if (p.nslots <= 0) return cudaSuccess;
    k_shard_out<<<int(min64((int64_t(p.nslots) + 255) / 256, 1024)), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_gather(const Pass& p, cudaStream_t s) {
    k_gather<<<p.nl, 1024, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_topk(const Pass& p, cudaStream_t s) {
    k_topk<<<p.nl, 1024, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Pass& p, cudaStream_t s) {
    k_finalize<<<dim3(8, unsigned(p.nl)), 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace palmad
