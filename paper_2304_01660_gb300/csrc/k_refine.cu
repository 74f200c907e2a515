// Refinement (DRAG phase 2; Algorithm 4, Sec. 3.3).
//
//  k_compact      Cand AND Neighbor (Algorithm 4 lines 1-2; already one
//                 bitmap here) -> ascending survivor list, warp-ballot /
//                 popcount prefix in one CTA.
//  k_plan_*       split a batch of survivors: strips (32*D consecutive
//                 windows) holding at least `thr` survivors, none flat, go to
//                 the recurrence sweep (k_sweep.cu); the others to the direct
//                 form below.  Also map window -> survivor slot.
//  k_refine_prep  centred FP32 window of every survivor and its sum.
//  k_refine       direct FP32 form for scattered survivors: a register-tiled
//                 product of the survivors' windows with the Hankel matrix of
//                 the series (64 survivors x 256 columns per CTA tile, 8x8 per
//                 thread, one new series value per k step thanks to the
//                 Hankel structure).  Per tile it records the survivor's
//                 maximum rho; a pair with rho > rho_prune (d < r beyond the
//                 error band) marks the survivor dead -- the early abandon of
//                 Algorithm 4 -- and later tiles of dead survivors are
//                 skipped.
//  k_recheck      exact finish: for every live survivor, every column whose
//                 FP32 rho lies within 2 eps of its FP32 maximum (a set that
//                 provably holds the true nearest neighbour) is recomputed in
//                 FP64 (Eq. 4-5 directly), and the minimum FP64 d^2 kept.
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kFlatRel = 2.384185791015625e-07;  // 2^-22

// ------------------------------------------------------------- compaction

__global__ void __launch_bounds__(1024) k_compact(const CompactArgs a) {
    __shared__ int32_t warp_tot[32];
    const int64_t P = (a.N + 31) / 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t per = (P + blockDim.x - 1) / blockDim.x;
    const int64_t w0 = tid * per, w1 = min(P, w0 + per);
    int32_t cnt = 0;
    for (int64_t w = w0; w < w1; ++w) cnt += __popc(a.bits[w]);
    // block exclusive scan of cnt
    int32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int32_t v = (lane < int(blockDim.x / 32)) ? warp_tot[lane] : 0;
        int32_t s = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += u;
        }
        warp_tot[lane] = s - v;  // exclusive warp offsets
        if (lane == 31) *a.nsurv = s;
    }
    __syncthreads();
    int32_t off = warp_tot[wid] + incl - cnt;
    for (int64_t w = w0; w < w1; ++w) {
        uint32_t b = a.bits[w];
        while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            a.surv[off++] = int32_t(w * 32 + bit);
        }
    }
}

// --------------------------------------------------------------- plan

// Per survivor: its slot, and the survivor count / flat flag of its strip.
__global__ void k_plan_count(const int32_t* __restrict__ surv, int32_t ns, const WinRec* __restrict__ win, int32_t H,
                             int32_t* __restrict__ slot_of, int32_t* __restrict__ scount) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < ns; k += gridDim.x * blockDim.x) {
        const int32_t w = surv[k];
        slot_of[w] = k;
        const int32_t st = w / H;
        // count in the low bits, flat flag in bit 30
        atomicAdd(&scount[st], 1);
        if (win[w].z == 0.f) atomicOr(&scount[st], 1 << 30);
    }
}

// The first survivor of every strip routes the strip: to the sweep when it
// holds >= thr survivors and no flat window, else its survivors to the
// direct form.
__global__ void k_plan_split(const int32_t* __restrict__ surv, int32_t ns, int32_t H, int32_t thr,
                             const int32_t* __restrict__ scount, int32_t* __restrict__ strips,
                             int32_t* __restrict__ nstrips, int32_t* __restrict__ direct,
                             int32_t* __restrict__ ndirect) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < ns; k += gridDim.x * blockDim.x) {
        const int32_t st = surv[k] / H;
        if (k > 0 && surv[k - 1] / H == st) continue;
        const int32_t c = scount[st];
        const int32_t len = c & ((1 << 30) - 1);
        if (len >= thr && !(c >> 30)) {
            strips[atomicAdd(nstrips, 1)] = st;
        } else {
            const int32_t b = atomicAdd(ndirect, len);
            for (int32_t q = 0; q < len; ++q) direct[b + q] = k + q;
        }
    }
}

// --------------------------------------------------------------- prep

__global__ void k_refine_prep(const float* __restrict__ T, const WinRec* __restrict__ win,
                              const int32_t* __restrict__ surv, int32_t ns, int32_t m, int32_t kpad,
                              float* __restrict__ acen, float* __restrict__ asum) {
    const int lane = threadIdx.x & 31;
    const int64_t slot = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (slot >= ns) return;
    const int32_t c = surv[slot];
    const float mu = win[c].w;
    float part = 0.f;
    float* row = acen + slot * int64_t(kpad);
    for (int k = lane; k < kpad; k += 32) {
        const float v = (k < m) ? (T[c + k] - mu) : 0.f;
        row[k] = v;
        part += v;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
    if (lane == 0) asum[slot] = part;
}

// -------------------------------------------------------- FP32 refine pass

constexpr int kRS = 64;    // survivors per CTA tile
constexpr int kRC = 256;   // columns per CTA tile
constexpr int kKC = 32;    // k chunk staged per iteration

__global__ void __launch_bounds__(256) k_refine(const RefineArgs a) {
    __shared__ __align__(16) float As[kRS][kKC];
    __shared__ __align__(16) float Bs[kRC + kKC + 16];
    __shared__ int64_t item_s;
    __shared__ int alive_s;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int32_t nl = *a.nlist;
    const int64_t ngroups = (nl + kRS - 1) / kRS;
    const int32_t ntiles = int32_t((a.N + kRC - 1) / kRC);
    const int64_t nitems = ngroups * ntiles;
    const bool has_flat = (a.flags[0] & 2) != 0;
    const float rho_prune = rho_prune_of(a.th);
    unsigned long long pairs = 0;

    for (;;) {
        if (tid == 0) item_s = atomicAdd(a.work, 1);
        if (tid == 0) alive_s = 0;
        __syncthreads();
        const int64_t item = item_s;
        if (item >= nitems) break;
        const int64_t g = item / ntiles;
        const int32_t t = int32_t(item % ntiles);
        const int64_t sbase = g * kRS;
        if (tid < kRS) {
            const int64_t e = sbase + tid;
            if (e < nl && !__ldcg(&a.dead[a.list[e]])) atomicOr(&alive_s, 1);
        }
        __syncthreads();
        if (!alive_s) { __syncthreads(); continue; }

        const int64_t j0 = int64_t(t) * kRC;
        const int64_t jc = j0 + 8 * lane;  // this thread's first column
        const float b0 = a.win[min(jc, a.N - 1)].w;
        float acc[8][8];
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[s][c] = 0.f;

        for (int k0 = 0; k0 < a.kpad; k0 += kKC) {
            // stage survivors' window slice and the series slice
            for (int e = tid; e < kRS * kKC / 4; e += 256) {
                const int s = e / (kKC / 4), q = (e % (kKC / 4)) * 4;
                const int64_t le = sbase + s;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (le < nl) v = *reinterpret_cast<const float4*>(a.acen + int64_t(a.list[le]) * a.kpad + k0 + q);
                *reinterpret_cast<float4*>(&As[s][q]) = v;
            }
            for (int x = tid; x < kRC + kKC + 16; x += 256) {
                const int64_t idx = j0 + k0 + x;
                Bs[x] = (idx < a.n) ? a.T[idx] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kKC; kk += 8) {
                float b[16];
                const float* bp = Bs + 8 * lane + kk;
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    const float4 v = *reinterpret_cast<const float4*>(bp + q);
                    b[q] = v.x - b0; b[q + 1] = v.y - b0; b[q + 2] = v.z - b0; b[q + 3] = v.w - b0;
                }
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const float4 a0 = *reinterpret_cast<const float4*>(&As[8 * w + s][kk]);
                    const float4 a1 = *reinterpret_cast<const float4*>(&As[8 * w + s][kk + 4]);
                    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                    for (int q = 0; q < 8; ++q)
#pragma unroll
                        for (int c = 0; c < 8; ++c) acc[s][c] = fmaf(av[q], b[q + c], acc[s][c]);
                }
            }
            __syncthreads();
        }

        // epilogue: rho per pair, tile max per survivor
        float invj[8], muj[8];
        bool colok[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t j = jc + c;
            colok[c] = j < a.N;
            const float4 r = colok[c] ? a.win[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            invj[c] = r.z;
            muj[c] = r.w;
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int64_t le = sbase + 8 * w + s;
            const bool sok = le < nl;
            const int64_t sl = sok ? a.list[le] : 0;
            const int32_t ci = sok ? a.surv[sl] : 0;
            const float invc = sok ? a.win[ci].z : 0.f;
            const float sa = sok ? a.asum[sl] : 0.f;
            float mx = -kInf;
            int np = 0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int64_t j = jc + c;
                const int64_t dj = j - ci;
                const bool ok = sok && colok[c] && (dj >= a.m || dj <= -a.m);
                float rho = (acc[s][c] - (muj[c] - b0) * sa) * invc * invj[c];
                if (has_flat && (invc == 0.f || invj[c] == 0.f)) rho = (invc == 0.f && invj[c] == 0.f) ? 1.f : 0.f;
                mx = ok ? fmaxf(mx, rho) : mx;
                np += ok;
            }
            pairs += np;
            // 32-column chunk maxima (4 lanes), then the tile maximum
            mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, 1));
            mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, 2));
            if ((lane & 3) == 0 && sok && jc < a.N) a.cmax[sl * a.nchunks + (jc >> 5)] = mx;
#pragma unroll
            for (int o = 4; o <= 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
            if (lane == 0 && sok) {
                if (mx > -kInf) atomicMax(&a.gmax[sl], enc_f32(mx));
                if (mx > rho_prune) a.dead[sl] = 1;
            }
        }
    }
    if (pairs) atomicAdd(a.pairs, pairs);
}

// -------------------------------------------------------- FP64 re-check

__device__ __forceinline__ bool is_flat64(double mu, double sd) { return sd <= kFlatRel * fabs(mu); }

__global__ void __launch_bounds__(256) k_recheck(const RecheckArgs a) {
    __shared__ int32_t flagged[256];
    __shared__ int nflag;
    const int64_t slot = blockIdx.x;
    if (slot >= a.ns || a.dead[slot]) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int32_t c = a.surv[slot];
    const float gm = dec_f32(a.gmax[slot]);
    const float thr = gm - 2.f * eps_bound(a.th);
    const bool has_flat = (a.flags[0] & 2) != 0;
    const float invc = a.win[c].z;
    const double muc = a.mu[c], sdc = sqrt(a.var[c]);
    const bool flatc = is_flat64(muc, sdc);
    const float* arow = a.acen + slot * int64_t(a.kpad);
    const float* cm = a.cmax + slot * int64_t(a.nchunks);
    unsigned long long fp64 = 0;
    for (int32_t cb = 0; cb < a.nchunks; cb += 256) {
        if (threadIdx.x == 0) nflag = 0;
        __syncthreads();
        const int32_t q = cb + threadIdx.x;
        if (q < a.nchunks && cm[q] >= thr) flagged[atomicAdd(&nflag, 1)] = q;
        __syncthreads();
        const int nf = nflag;
        for (int f = wid; f < nf; f += 8) {
            const int64_t j = int64_t(flagged[f]) * 32 + lane;
            if (j >= a.N || (j - c < a.m && c - j < a.m)) continue;
            const float4 rj = a.win[j];
            float acc = 0.f;
            for (int k = 0; k < a.m; ++k) acc = fmaf(arow[k], a.T[j + k] - rj.w, acc);
            float rho32 = acc * invc * rj.z;
            if (has_flat && (invc == 0.f || rj.z == 0.f)) rho32 = (invc == 0.f && rj.z == 0.f) ? 1.f : 0.f;
            if (rho32 < thr) continue;
            const double muj = a.mu[j], sdj = sqrt(a.var[j]);
            const bool flatj = is_flat64(muj, sdj);
            double d2;
            if (flatc && flatj) d2 = 0.0;
            else if (flatc || flatj) d2 = 2.0 * a.m;
            else {
                d2 = 0.0;
                const double ic = 1.0 / sdc, ij = 1.0 / sdj;
                for (int k = 0; k < a.m; ++k) {
                    const double x = (double(a.T[c + k]) - muc) * ic - (double(a.T[j + k]) - muj) * ij;
                    d2 = fma(x, x, d2);
                }
            }
            atomicMin(&a.nn2[slot], static_cast<unsigned long long>(__double_as_longlong(d2)));
            const float err = fabsf(rho32 - float(1.0 - d2 / (2.0 * a.m)));
            atomicMax(a.maxerr, enc_f32(err));
            ++fp64;
        }
        __syncthreads();
    }
    if (fp64) atomicAdd(a.pairs, fp64);
}

}  // namespace

cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s) {
    k_compact<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_plan(const int32_t* surv, int32_t ns, const WinRec* win, int32_t H, int32_t thr, int32_t* slot_of,
                        int32_t* scount, int32_t* strips, int32_t* nstrips, int32_t* direct, int32_t* ndirect,
                        cudaStream_t s) {
    if (ns <= 0) return cudaSuccess;
    const int block = 256;
    const int grid = int(min64((int64_t(ns) + block - 1) / block, 1024));
    k_plan_count<<<grid, block, 0, s>>>(surv, ns, win, H, slot_of, scount);
    k_plan_split<<<grid, block, 0, s>>>(surv, ns, H, thr, scount, strips, nstrips, direct, ndirect);
    return cudaGetLastError();
}

cudaError_t launch_refine_prep(const float* T, const WinRec* win, const int32_t* surv, int32_t ns, int32_t m,
                               int32_t kpad, float* acen, float* asum, cudaStream_t s) {
    if (ns <= 0) return cudaSuccess;
    const int block = 256;
    const int grid = int((int64_t(ns) * 32 + block - 1) / block);
    k_refine_prep<<<grid, block, 0, s>>>(T, win, surv, ns, m, kpad, acen, asum);
    return cudaGetLastError();
}

int refine_grid(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms * 2;
}

cudaError_t launch_refine(const RefineArgs& a, int grid, cudaStream_t s) {
    if (a.ns <= 0) return cudaSuccess;
    k_refine<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_recheck(const RecheckArgs& a, cudaStream_t s) {
    if (a.ns <= 0) return cudaSuccess;
    k_recheck<<<a.ns, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace palmad
