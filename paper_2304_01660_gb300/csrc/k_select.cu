// Candidate select (DRAG phase 1; Algorithm 3, Sec. 3.2).
//
// A warp owns a strip of H = 32*D consecutive windows (rows i) and scans the
// windows to their right (columns j >= i + m), 32 columns per chunk, exactly
// the paper's segment-scans-right scheme, re-cut for a GB300 warp:
//   * lane l holds rows i0 + l*D .. i0 + l*D + D-1 in registers; one step
//     advances every row by one column with the diagonal recurrence of Eq. 9
//     (cov(i,j) = cov(i-1,j-1) + df_i dg_j + df_j dg_i), the value of the
//     row above arriving from the previous lane by one shuffle;
//   * the strip's top row has no row above: its dot products ("QTrow") are
//     computed per chunk by a transposed register-blocked pass over the
//     staged series, then reduce-scattered so lane l holds column c0 + l;
//   * a pair with rho > rho_prune (i.e. d < r beyond the FP32 error band)
//     clears the row's and the column's candidate bits (Cand and Neighbor of
//     Algorithm 3 are one bitmap here, since refine ANDs them anyway);
//   * the warp leaves the strip once every row is dead (Algorithm 3 lines
//     14-15) or after `cap` columns past its triangle; rows still alive go
//     to refine, which is exact.
// Pruning is sound: a pair is only used when its FP32 rho exceeds the exact
// threshold by more than the error bound, so no range discord is dropped.
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerCta = 4;

struct WarpSmem {
    float* ahat;    // [kp]      centred top-row window, zero padded
    float* tw;      // [kp + 32] series for this chunk, minus offset b0
    float4* colrec; // [32]      column records of this chunk
    float* seed;    // [32]      top-row dot products of this chunk
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sum over lanes of acc[c] lands in lane c (reduce-scatter, 31 shuffles).
__device__ __forceinline__ float reduce_scatter32(float (&acc)[32], int lane) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < o; ++k) {
            const float send = upper ? acc[k] : acc[k + o];
            const float keep = upper ? acc[k + o] : acc[k];
            acc[k] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    return acc[0];
}

template <int D>
__global__ void __launch_bounds__(kWarpsPerCta * 32) k_select(const SelectArgs a) {
    constexpr int H = 32 * D;
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t m = a.m;
    const int kp = ((m + 127) / 128) * 128;  // padded window length (multiple of 128)
    const int s4 = kp / 32;                  // k-slice per lane (multiple of 4)
    const size_t per_warp = size_t(kp) + kp + 32 + 4 * 32 + 32;
    float* base = smem + per_warp * wid;
    WarpSmem sm{base, base + kp, reinterpret_cast<float4*>(base + 2 * kp + 32), base + 2 * kp + 32 + 128};

    const int64_t N = a.N;
    const int64_t nstrips = (N + H - 1) / H;
    unsigned long long pairs = 0;

    for (;;) {
        int64_t s = 0;
        if (lane == 0) s = atomicAdd(a.work, 1);
        s = __shfl_sync(kFull, s, 0);
        if (s >= nstrips) break;
        const int64_t i0 = s * H;

        // Rows of this lane.
        float df_r[D], dg_r[D], thr_r[D], cov[D], rmax[D];
        const int64_t r0 = i0 + int64_t(lane) * D;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int64_t i = r0 + d;
            float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < N) rec = a.win[i];
            df_r[d] = rec.x;
            dg_r[d] = rec.y;
            thr_r[d] = (i >= N) ? kInf
                       : (rec.z > 0.f ? a.rho_prune / rec.z : (a.rho_prune < 0.f ? -kInf : kInf));
            cov[d] = 0.f;
            rmax[d] = -kInf;
        }
        const int64_t wrd = r0 >> 5;
        const int sh = int(r0 & 31);
        const uint32_t dmask = (D == 32) ? kFull : ((1u << D) - 1u);
        uint32_t alive = (r0 < N) ? ((__ldcg(&a.bits[wrd]) >> sh) & dmask) : 0u;
        if (!__any_sync(kFull, alive)) continue;

        const int64_t jstart = i0 + m;
        if (jstart >= N) continue;  // no window to the right: left to column marks / refine
        const int64_t jend = min(N, i0 + H - 1 + m + a.cap);

        // Centred top-row window and its sum (FP32; the sum absorbs the
        // rounding of mu so the seed correction below is exact to rounding).
        const float mu_top = a.win[i0].w;
        float part = 0.f;
        for (int k = lane; k < kp; k += 32) {
            const float v = (k < m) ? (a.T[i0 + k] - mu_top) : 0.f;
            sm.ahat[k] = v;
            part += v;
        }
        const float suma = warp_sum(part);
        __syncwarp();

        for (int64_t c0 = jstart & ~int64_t(31); c0 < jend; c0 += 32) {
            // Stage the series for this chunk's seeds.
            const float b0 = a.win[c0].w;
            for (int x = lane; x < kp + 32; x += 32) {
                const int64_t t = c0 + x;
                sm.tw[x] = (t < a.n) ? (a.T[t] - b0) : 0.f;
            }
            __syncwarp();
            // Transposed partial dot products: lane covers k in [lane*s4, lane*s4+s4).
            float acc[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0.f;
            const int kl = lane * s4;
            for (int q = 0; q < s4; q += 4) {
                const float4 av = *reinterpret_cast<const float4*>(sm.ahat + kl + q);
                const float a4[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
                for (int cb = 0; cb < 4; ++cb) {
                    const float* tp = sm.tw + kl + q + cb * 8;
                    const float4 t0 = *reinterpret_cast<const float4*>(tp);
                    const float4 t1 = *reinterpret_cast<const float4*>(tp + 4);
                    const float4 t2 = *reinterpret_cast<const float4*>(tp + 8);
                    const float tv[12] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x, t2.y, t2.z, t2.w};
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
#pragma unroll
                        for (int cc = 0; cc < 8; ++cc) acc[cb * 8 + cc] = fmaf(a4[qq], tv[qq + cc], acc[cb * 8 + cc]);
                }
            }
            const float dot = reduce_scatter32(acc, lane);
            {
                const int64_t j = c0 + lane;
                float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
                float sd = 0.f;
                if (j < N) {
                    rec = a.win[j];
                    sd = dot - (rec.w - b0) * suma;
                }
                sm.colrec[lane] = rec;
                sm.seed[lane] = sd;
            }
            __syncwarp();

            const int steps = int(min64(32, jend - c0));
            const bool masked = (c0 - jstart) < int64_t(H - 1);
            uint32_t colmask = 0;
            if (masked) {
                for (int st = 0; st < steps; ++st) {
                    const float4 cr = sm.colrec[st];
                    const float sd = sm.seed[st];
                    const float up = __shfl_up_sync(kFull, cov[D - 1], 1);
#pragma unroll
                    for (int d = D - 1; d >= 1; --d) cov[d] = fmaf(df_r[d], cr.y, fmaf(cr.x, dg_r[d], cov[d - 1]));
                    cov[0] = (lane == 0) ? sd : fmaf(df_r[0], cr.y, fmaf(cr.x, dg_r[0], up));
                    const int64_t lim = c0 + st - jstart - int64_t(lane) * D;  // row d valid iff d <= lim
                    bool pred = false;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        float x = cov[d] * cr.z;
                        x = (int64_t(d) <= lim) ? x : -kInf;
                        rmax[d] = fmaxf(rmax[d], x);
                        pred |= x > thr_r[d];
                    }
                    if (pred) colmask |= 1u << st;
                }
            } else {
                for (int st = 0; st < steps; ++st) {
                    const float4 cr = sm.colrec[st];
                    const float sd = sm.seed[st];
                    const float up = __shfl_up_sync(kFull, cov[D - 1], 1);
#pragma unroll
                    for (int d = D - 1; d >= 1; --d) cov[d] = fmaf(df_r[d], cr.y, fmaf(cr.x, dg_r[d], cov[d - 1]));
                    cov[0] = (lane == 0) ? sd : fmaf(df_r[0], cr.y, fmaf(cr.x, dg_r[0], up));
                    bool pred = false;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        const float x = cov[d] * cr.z;
                        rmax[d] = fmaxf(rmax[d], x);
                        pred |= x > thr_r[d];
                    }
                    if (pred) colmask |= 1u << st;
                }
            }
            // Valid pairs of this chunk (rows < N with i <= j - m).
            if (lane == 0) {
                const int64_t rows = min64(H, N - i0);
                for (int st = 0; st < steps; ++st) {
                    const int64_t v = min64(rows, c0 + st - jstart + 1);
                    if (v > 0) pairs += uint64_t(v);
                }
            }
            // Neighbour (column) marks of this chunk.
            const uint32_t cw = __reduce_or_sync(kFull, colmask);
            if (lane == 0 && cw) atomicAnd(&a.bits[c0 >> 5], ~cw);
            // Row deaths.
            uint32_t newdead = 0;
#pragma unroll
            for (int d = 0; d < D; ++d)
                if (((alive >> d) & 1u) && rmax[d] > thr_r[d]) newdead |= 1u << d;
            if (newdead) {
                alive &= ~newdead;
                atomicAnd(&a.bits[wrd], ~(newdead << sh));
            }
            if (r0 < N) alive &= (__ldcg(&a.bits[wrd]) >> sh) & dmask;  // rows killed by other strips' column marks
            if (!__any_sync(kFull, alive)) break;
            __syncwarp();
        }
    }
    if (lane == 0 && pairs) atomicAdd(a.pairs, pairs);
}

template <int D>
size_t select_smem(int32_t m) {
    const int kp = ((m + 127) / 128) * 128;
    return sizeof(float) * (size_t(kp) + kp + 32 + 4 * 32 + 32) * kWarpsPerCta;
}

}  // namespace

int select_grid(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms * 4;
}

cudaError_t launch_select(const SelectArgs& a, int grid, cudaStream_t s) {
    constexpr int D = 8;
    const size_t sm = select_smem<D>(a.m);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_select<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
    }
    k_select<D><<<grid, kWarpsPerCta * 32, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace palmad
