// Witness hints carried across lengths (between DRAG phase 1 and phase 2).
//
// A window that is not a range discord at some length has a non-self match
// closer than r (Sec. 2.1).  When the window grows by one sample, that match
// usually stays close: both windows gain one aligned sample.  The sweeps
// therefore record, per window of a series, a column near the pair that
// pruned it (select: the chunk where a row died, or the strip whose rows
// cleared a column's bit; refine: the chunk where a survivor died).  At the
// next lengths, k_hint tests every survivor of select against the 128
// columns around its recorded column before refine starts: a pair whose FP32
// rho clears the pruning threshold with the error bound of the sweeps
// removes the survivor from the candidate bitmap, and compaction runs again.
//
// A hint only decides which pairs are tried first; the pruning test is the
// sweeps' own sound test, so the range discords, their distances and every
// later decision are the same with or without hints.  Refine otherwise
// finds such a witness only after scanning every column nearer the
// survivor, which on quasi-periodic series can be most of the series.
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kHintWarps = 4;
constexpr int kHintCols = 128;   // columns tried per survivor (4 per lane)
constexpr int kHintMaxKpad = 2048;

__host__ __device__ __forceinline__ size_t hint_warp_floats(int kp) { return size_t(kp) + size_t(kp) + kHintCols + 8; }

// grid.y: lane of the pass; each warp takes survivors of that lane in turn.
__global__ void __launch_bounds__(kHintWarps * 32) k_hint(const Pass p) {
    extern __shared__ __align__(16) float smem[];
    const int l = blockIdx.y;
    const Lane& L = p.lanes[l];
    if (!L.prune || !L.hint || p.knn > 1) return;  // one pair decides nothing in the k-th neighbour variant
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int kps = p.kpad_pass;
    float* a = smem + hint_warp_floats(kps) * wid;  // [kps]               centred survivor window
    float* s = a + kps;                             // [kps + kHintCols + 8] series slice
    const LaneState& S = p.st[l];
    const int32_t nsurv = S.nsurv;
    const int32_t m = L.m;
    const int64_t N = L.N, n = L.n;
    const int kp = L.kpad;
    const float* T = L.T;
    const WinRec* win = L.win;
    const float rho_prune = rho_prune_of(L, S);
    unsigned long long pairs = 0, kills = 0;
    for (int32_t k = blockIdx.x * kHintWarps + wid; k < nsurv; k += gridDim.x * kHintWarps) {
        const int32_t i = L.surv[k];
        const int32_t h = __ldcg(&L.hint[i]);
        if (h < 0) continue;
        const float4 ri = win[i];
        if (ri.z == 0.f) continue;  // flat survivor: refine decides it
        // columns [j0, j0 + 128), clipped to the windows
        int64_t j0 = int64_t(h) - kHintCols / 2;
        j0 = max64(0, min64(j0, N - kHintCols));
        float part = 0.f;
        for (int q = lane; q < kp; q += 32) {
            const float v = q < m ? T[i + q] - ri.w : 0.f;
            a[q] = v;
            part += v;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
        const float suma = part;
        for (int q = lane; q < kp + kHintCols + 8; q += 32) {
            const int64_t t = j0 + q;
            s[q] = t < n ? T[t] : 0.f;
        }
        __syncwarp();
        // lane: columns j0 + 4 lane + c (c < 4), offset by the mean of its
        // first column (centring offsets within 3 columns, as eps_bound allows)
        const int64_t jl = j0 + 4 * lane;
        const float b0 = win[min64(jl, N - 1)].w;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const float* sp = s + 4 * lane;
        for (int q = 0; q < kp; q += 4) {
            const float4 av = *reinterpret_cast<const float4*>(a + q);
            const float4 u0 = *reinterpret_cast<const float4*>(sp + q);
            const float4 u1 = *reinterpret_cast<const float4*>(sp + q + 4);
            const float y[7] = {u0.x - b0, u0.y - b0, u0.z - b0, u0.w - b0, u1.x - b0, u1.y - b0, u1.z - b0};
            const float x[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] = fmaf(x[t], y[t + c], acc[c]);
        }
        bool hit = false;
        int np = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = jl + c;
            const int64_t dj = j - i;
            if (j >= N || (dj < m && dj > -int64_t(m))) continue;
            const float4 rj = win[j];
            if (rj.z == 0.f) continue;
            const float rho = (acc[c] - (rj.w - b0) * suma) * ri.z * rj.z;
            hit |= rho > rho_prune;
            ++np;
        }
        pairs += np;
        if (__any_sync(kFull, hit)) {
            if (lane == 0) {
                atomicAnd(&L.bits[i >> 5], ~(1u << (i & 31)));
                ++kills;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
    if (lane == 0) {
        if (pairs) atomicAdd(p.pairs + 7, pairs);
        if (kills) atomicAdd(p.pairs + 8, kills);
    }
}

}  // namespace

bool hint_supported(const Pass& p) { return p.kpad_pass <= kHintMaxKpad; }

cudaError_t launch_hint(const Pass& p, int sms, cudaStream_t s) {
    if (!hint_supported(p)) return cudaSuccess;
    const int kps = p.kpad_pass;
    const size_t sm = sizeof(float) * hint_warp_floats(kps) * kHintWarps;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_hint, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
    }
    // about 8 CTAs per SM over the pass, at least one per lane
    const int gx = max(1, min(1024, (sms * 8 + p.nl - 1) / p.nl));
    k_hint<<<dim3(gx, p.nl), kHintWarps * 32, sm, s>>>(p);
    return cudaGetLastError();
}

}  // namespace palmad
