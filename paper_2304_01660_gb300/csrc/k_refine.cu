// Refinement (DRAG phase 2; Algorithm 4, Sec. 3.3), for every lane of a pass.
//
//  k_compact      Cand AND Neighbor (Algorithm 4, its first step; already one
//                 bitmap here) -> ascending survivor list; one CTA per lane,
//                 popcount prefix over the bitmap words.
//  k_plan_count   survivors of this refine round -> pool slots (64-aligned
//                 per lane), window -> slot map, survivors per strip.
//  k_plan_split   routes every strip: >= thr survivors and none flat -> the
//                 recurrence sweep (k_sweep.cu), else its survivors -> the
//                 direct form below.
//  k_prep         centred FP32 window of every slot and its sum.
//  k_refine       direct FP32 form for scattered survivors (packed per lane,
//                 64 per group): a register-tiled
//                 product of 64 survivors' windows with the Hankel matrix of
//                 the series (256 columns per CTA tile, 8x8 per thread, one new
//                 series value per k step thanks to the Hankel structure).
//                 It records the maximum rho per 32-column chunk; a pair with
//                 rho > rho_prune (d < r beyond the error band) marks the
//                 survivor dead (the early abandon of Algorithm 4), and later
//                 tiles of dead survivors are skipped.
//  k_recheck      exact finish: for every live survivor, every column whose
//                 FP32 rho lies within 2 eps of its FP32 maximum (a set that
//                 provably holds the true nearest neighbour) is recomputed in
//                 FP64 (Eq. 4-5 directly), and the minimum FP64 d^2 kept.
//                 In the k-th neighbour variant the threshold comes from the
//                 k-th largest coarse maximum and the k-th smallest d^2 is
//                 kept.
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kFlatRel = 2.384185791015625e-07;  // 2^-22
constexpr int kMaxLanesSmem = 4096;

// ------------------------------------------------------------- compaction

__global__ void __launch_bounds__(1024) k_compact(const Pass p) {
    __shared__ int32_t warp_tot[32];
    const Lane& L = p.lanes[blockIdx.x];
    const int64_t P = (L.N + 31) / 32;
    const uint32_t* bits = L.bits;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t per = (P + blockDim.x - 1) / blockDim.x;
    const int64_t w0 = tid * per, w1 = min64(P, w0 + per);
    int32_t cnt = 0;
    for (int64_t w = w0; w < w1; ++w) cnt += __popc(bits[w]);
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
        if (lane == 31) p.st[blockIdx.x].nsurv = s;
    }
    __syncthreads();
    int32_t off = warp_tot[wid] + incl - cnt;
    for (int64_t w = w0; w < w1; ++w) {
        uint32_t b = bits[w];
        while (b) {
            const int bit = __ffs(b) - 1;
            b &= b - 1;
            L.surv[off++] = int32_t(w * 32 + bit);
        }
    }
}

// ------------------------------------------------------------------ plan

__device__ __forceinline__ void stage_slot_bases(const Pass& p, int64_t* sb) {
    for (int l = threadIdx.x; l < p.nl; l += blockDim.x) sb[l] = p.lanes[l].slot_base;
    __syncthreads();
}

__global__ void k_plan_count(const Pass p) {
    __shared__ int64_t sb[kMaxLanesSmem];
    stage_slot_bases(p, sb);
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < p.nslots; g += gridDim.x * blockDim.x) {
        const int l = lane_of(sb, p.nl, g);
        const Lane& L = p.lanes[l];
        const int32_t k = L.k_lo + (g - L.slot_base);
        p.slot_lane[g] = l;
        p.dead[g] = 0;
        p.kcnt[g] = 0;
        p.gmax[g] = 0u;
        p.nn2[g] = 0x7ff0000000000000ull;
        if (k >= L.k_hi) {
            p.slot_win[g] = -1;
            p.route[g] = -1;
            continue;
        }
        const int32_t w = L.surv[k];
        p.slot_win[g] = w;
        L.slot_of[w] = g;
        const int32_t st = w / p.refine_h;
        atomicAdd(&L.scount[st], 1);                              // survivors of the strip
        if (L.win[w].z == 0.f) atomicOr(&L.scount[st], 1 << 30);  // a flat window among them
    }
}

__global__ void k_plan_split(const Pass p) {
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < p.nslots; g += gridDim.x * blockDim.x) {
        const int32_t w = p.slot_win[g];
        if (w < 0) continue;
        const int l = p.slot_lane[g];
        const Lane& L = p.lanes[l];
        const int32_t k = L.k_lo + (g - L.slot_base);
        const int32_t st = w / p.refine_h;
        if (k > L.k_lo && L.surv[k - 1] / p.refine_h == st) continue;  // not the first of its strip
        const int32_t c = L.scount[st];
        const int32_t len = c & ((1 << 30) - 1);
        // sweep when cheaper than the direct form: FP32 direct costs 2m flops per
        // survivor-column against ~5 per row-column of the sweep.  The
        // tensor-core direct form takes only lone survivors: measured on the
        // sine, random-walk and multi-series workloads, any larger share ran
        // slower than the sweep, whose strips stop at the first 32-column
        // chunk where every row is pruned
        const int32_t thr = p.direct_below > 0 ? p.direct_below
                           : (p.mixed ? 2 : max(2, (5 * p.refine_h + 2 * L.m - 1) / L.m));
        const int sweep = (len >= thr && !(c >> 30)) ? 1 : 0;
        if (sweep) {
            atomicAdd(p.pairs + 9, 1ull);
            atomicAdd(p.pairs + 10, static_cast<unsigned long long>(len));
            const int32_t e = atomicAdd(p.nref, 1);
            p.strips[e] = make_int2(l, st);
            if (p.tc_seeds) p.strip_row[e] = len >= p.seed_min ? atomicAdd(&p.st[l].seed_rows, 1) : -1;
        } else {
            const int32_t b = atomicAdd(&p.st[l].ndirect, len);  // packed from the lane's slot_base
            for (int32_t q = 0; q < len; ++q) p.dlist[L.slot_base + b + q] = g + q;
        }
        for (int32_t q = 0; q < len; ++q) p.route[g + q] = sweep ? 0 : 1;
    }
}

// Groups of kDGroup packed direct slots, listed so the direct refine visits
// only groups that hold work (count in work[4]).
__global__ void k_plan_groups(const Pass p) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= p.nl) return;
    const int32_t nd = p.st[l].ndirect;
    if (nd <= 0) return;
    const int32_t ng = (nd + kDGroup - 1) / kDGroup;
    const int32_t at = atomicAdd(p.work + 4, ng);
    const int32_t base = p.lanes[l].slot_base;
    for (int32_t k = 0; k < ng; ++k) p.dgroups[at + k] = base + kDGroup * k;
}

// Between the column chunks of the tensor-core direct refine: the lane's
// direct survivors still alive, re-packed in order from dlist into dlist_alt
// (one CTA per lane, prefix sum over the entries); ndirect becomes their
// number, so the next chunk's groups hold live survivors only.
__global__ void __launch_bounds__(1024) k_direct_compact(const Pass p) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t total_s;
    const int l = blockIdx.x;
    const int32_t nd = p.st[l].ndirect;
    const int32_t base = p.lanes[l].slot_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t per = (nd + int32_t(blockDim.x) - 1) / int32_t(blockDim.x);
    const int32_t q0 = min(nd, tid * per), q1 = min(nd, q0 + per);
    int32_t cnt = 0;
    for (int32_t q = q0; q < q1; ++q) cnt += __ldcg(&p.dead[p.dlist[base + q]]) ? 0 : 1;
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
        int32_t t = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t - v;
        if (lane == 31) total_s = t;
    }
    __syncthreads();
    int32_t off = warp_tot[wid] + incl - cnt;
    for (int32_t q = q0; q < q1; ++q) {
        const int32_t g = p.dlist[base + q];
        if (!__ldcg(&p.dead[g])) p.dlist_alt[base + off++] = g;
    }
    __syncthreads();  // every thread has read ndirect before it changes
    if (tid == 0) p.st[l].ndirect = total_s;
}

// --------------------------------------------------------------- prep

__global__ void k_prep(const Pass p) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t g = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; g < p.nslots; g += nw) {
        const int32_t w = p.slot_win[g];
        if (w < 0) continue;
        const Lane& L = p.lanes[p.slot_lane[g]];
        const float mu = L.win[w].w;
        float part = 0.f;
        float* row = p.acen + g * int64_t(p.kpad_max);
        for (int k = lane; k < p.kpad_max; k += 32) {
            const float v = (k < L.m) ? (L.T[w + k] - mu) : 0.f;
            row[k] = v;
            part += v;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
        if (lane == 0) p.asum[g] = part;
        if (p.route[g] == 1 || p.sharded)  // raised with atomicMax / written per segment; enc_f32 order: 0 is lowest
            for (int k = lane; k < p.ncoarse_max; k += 32) p.cmax2[g * p.ncoarse_max + k] = 0u;
    }
}

// -------------------------------------------------------- direct refine

constexpr int kRS = 64;    // survivors per CTA tile
constexpr int kRC = 256;   // columns per CTA tile
constexpr int kKC = 32;    // k chunk staged per iteration

__global__ void __launch_bounds__(256) k_refine(const Pass p) {
    __shared__ __align__(16) float As[kRS][kKC];
    __shared__ __align__(16) float Bs[kRC + kKC + 16];
    __shared__ int64_t item_s;
    __shared__ int alive_s;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t ngroups = *reinterpret_cast<volatile int32_t*>(p.work + 4);
    const int64_t ntiles = (p.nmax + kRC - 1) / kRC;
    constexpr int64_t kSub = kDGroup / kRS;  // 64-survivor tiles per group
    const int64_t nitems = ngroups * kSub * ntiles;
    unsigned long long pairs = 0;

    for (;;) {
        if (tid == 0) {
            item_s = atomicAdd(p.work + 1, 1);
            alive_s = 0;
        }
        __syncthreads();
        const int64_t item = item_s;
        if (item >= nitems) break;
        const int64_t gsub = item / ntiles;
        const int64_t g0 = p.dgroups[gsub / kSub];     // a slot of the group's lane
        const int64_t gbase = g0 + (gsub % kSub) * kRS;
        const int32_t t = int32_t(item % ntiles);
        const int l = p.slot_lane[g0];
        const Lane& L = p.lanes[l];
        const int64_t N = L.N;
        const int64_t j0 = int64_t(t) * kRC;
        // entries [gbase, gbase+64) of the lane's packed direct list
        const int32_t nd = p.st[l].ndirect - int32_t(gbase - L.slot_base);
        if (tid < kRS && tid < nd && j0 < N && j0 < L.col_hi && j0 + kRC > L.col_lo) {
            if (!__ldcg(&p.dead[p.dlist[gbase + tid]])) atomicOr(&alive_s, 1);
        }
        __syncthreads();
        if (!alive_s) {
            __syncthreads();
            continue;
        }
        const float* T = L.T;
        const int64_t n = L.n;
        const int32_t m = L.m;
        const WinRec* win = L.win;
        const bool has_flat = (p.st[l].flags & 2) != 0;
        const float rho_prune = rho_prune_of(L, p.st[l]);
        const int64_t jc = j0 + 8 * lane;  // this thread's first column
        const float b0 = win[min64(jc, N - 1)].w;
        float acc[8][8];
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[s][c] = 0.f;

        for (int k0 = 0; k0 < L.kpad; k0 += kKC) {
            for (int e = tid; e < kRS * kKC / 4; e += 256) {
                const int s = e / (kKC / 4), q = (e % (kKC / 4)) * 4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (s < nd) v = *reinterpret_cast<const float4*>(p.acen + int64_t(p.dlist[gbase + s]) * p.kpad_max + k0 + q);
                *reinterpret_cast<float4*>(&As[s][q]) = v;
            }
            for (int x = tid; x < kRC + kKC + 16; x += 256) {
                const int64_t idx = j0 + k0 + x;
                Bs[x] = (idx < n) ? T[idx] : 0.f;
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

        // epilogue: rho per pair, chunk and tile maxima per survivor
        float invj[8], muj[8];
        bool colok[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t j = jc + c;
            colok[c] = j < N && j >= L.col_lo && j < L.col_hi;
            const float4 r = colok[c] ? win[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            invj[c] = r.z;
            muj[c] = r.w;
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int e = 8 * w + s;
            const bool sok = e < nd;
            const int64_t g = sok ? p.dlist[gbase + e] : 0;
            const int32_t ci = sok ? p.slot_win[g] : 0;
            const float invc = sok ? win[ci].z : 0.f;
            const float sa = sok ? p.asum[g] : 0.f;
            float mx = -kInf;
            int np = 0, nk = 0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int64_t dj = jc + c - ci;
                const bool ok = sok && colok[c] && (dj >= m || dj <= -int64_t(m));
                float rho = (acc[s][c] - (muj[c] - b0) * sa) * invc * invj[c];
                if (has_flat && (invc == 0.f || invj[c] == 0.f)) rho = (invc == 0.f && invj[c] == 0.f) ? 1.f : 0.f;
                mx = ok ? fmaxf(mx, rho) : mx;
                np += ok;
                nk += (ok && rho > rho_prune) ? 1 : 0;
            }
            pairs += np;
            if (p.knn > 1) {  // pairs of the tile past the threshold, over the 32 lanes
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) nk += __shfl_xor_sync(kFull, nk, o);
            }
            mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, 1));
            mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, 2));
            if ((lane & 3) == 0 && sok && jc < N) p.cmax[g * p.nchunks_max + (jc >> 5)] = mx;
#pragma unroll
            for (int o = 4; o <= 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
            if (lane == 0 && sok) {
                if (mx > -kInf) {
                    atomicMax(&p.gmax[g], enc_f32(mx));
                    atomicMax(&p.cmax2[g * p.ncoarse_max + (j0 / p.seg)], enc_f32(mx));  // tile inside one block
                }
                const bool die = p.knn > 1 ? (nk > 0 && atomicAdd(&p.kcnt[g], nk) + nk >= p.knn) : mx > rho_prune;
                if (die) {
                    p.dead[g] = 1;
                    if (L.hint) L.hint[ci] = int32_t(j0 + kRC / 2);  // witness hint: this tile
                }
            }
        }
    }
    if (pairs) atomicAdd(p.pairs + 1, pairs);
}

// -------------------------------------------------------- FP64 re-check

// sigma <= 2^-22 |mu|, compared squared, exactly as the statistics kernel
// decides it (a variance left slightly negative counts as flat)
__device__ __forceinline__ bool is_flat_var(double mu, double var) {
    const double fl = kFlatRel * mu;
    return var <= fl * fl;
}

// One warp per live survivor slot (persistent, no block barriers).  The
// warp scans the survivor's coarse maxima, then the chunk maxima of the
// coarse blocks that can hold its nearest neighbour, recomputes the FP32 rho
// of each flagged 32-column chunk (a lane per column), and evaluates every
// column within 2 eps of the FP32 maximum in FP64 with the m terms split
// over the lanes; the survivor's z-normalised FP64 window is staged once in
// the warp's shared memory.
constexpr double kInfD = __builtin_huge_val();
constexpr int kRecheckWarps = 8;
constexpr int kRecheckWin = 512;    // survivor windows up to this length use shared memory

// k-th largest of n encoded (order-preserving) coarse maxima, by at most k
// rounds of a warp maximum below the previous one; 0 (below every encoded
// float) when fewer than k values exist.
__device__ uint32_t kth_largest_enc(const uint32_t* __restrict__ c2, int32_t n, int32_t k, int lane) {
    unsigned long long cur = 0x100000000ull;  // exclusive upper bound of this round
    for (int t = 0; t < k; ++t) {
        uint32_t mx = 0;
        bool any = false;
        for (int32_t q = lane; q < n; q += 32) {
            const uint32_t v = c2[q];
            if (v < cur) {
                mx = v > mx ? v : mx;
                any = true;
            }
        }
        mx = __reduce_max_sync(kFull, mx);
        if (!__any_sync(kFull, any)) return 0u;
        uint32_t cnt = 0;
        for (int32_t q = lane; q < n; q += 32) cnt += c2[q] >= mx ? 1u : 0u;
        cnt = __reduce_add_sync(kFull, cnt);
        if (cnt >= uint32_t(k)) return mx;
        cur = mx;
    }
    return 0u;
}

// KNN: the k-th neighbour variant (p.knn = k > 1).  The row's threshold is
// the k-th largest coarse maximum minus 2 eps: at least k columns reach that
// maximum in FP32, so the k-th largest FP64 rho is at least it minus eps, and
// every column among the k nearest in FP64 is at least it minus 2 eps in
// FP32.  When fewer than k coarse blocks hold a non-self column the row is
// re-checked over every non-self column.  The k smallest FP64 distances are
// kept sorted in registers (identical in every lane of the warp) and the k-th
// becomes the survivor's distance; with fewer than k it stays infinite, so
// the window is not a discord.
template <bool KNN>
__global__ void __launch_bounds__(kRecheckWarps * 32) k_recheck(const Pass p) {
    __shared__ double zc_all[kRecheckWarps][kRecheckWin];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* zc = zc_all[wid];
    unsigned long long fp64 = 0;
    for (;;) {
        int64_t g = 0;
        if (lane == 0) g = atomicAdd(p.work + 3, 1);
        g = __shfl_sync(kFull, g, 0);
        if (g >= p.nslots) break;
        const int32_t c = p.slot_win[g];
        if (c < 0 || __ldcg(&p.dead[g])) continue;
        const int l = p.slot_lane[g];
        const Lane& L = p.lanes[l];
        LaneState& S = p.st[l];
        const int32_t m = L.m;
        const int64_t N = L.N;
        const float* T = L.T;
        const WinRec* win = L.win;
        const uint32_t* c2 = p.cmax2 + g * int64_t(p.ncoarse_max);
        const int32_t ncoarse = int32_t((N + p.seg - 1) / p.seg);
        float thr;
        if (KNN) {
            const uint32_t ek = kth_largest_enc(c2, ncoarse, p.knn, lane);
            thr = ek >= enc_f32(-3.402823466e38f) ? dec_f32(ek) - 2.f * eps_bound(m, S) : -kInf;
        } else {
            const float gm = dec_f32(__ldcg(&p.gmax[g]));
            thr = gm - 2.f * eps_bound(m, S);
        }
        const uint32_t thr_enc = enc_f32(thr);
        double best[KNN ? kMaxKnn : 1];
#pragma unroll
        for (int t = 0; t < (KNN ? kMaxKnn : 1); ++t) best[t] = kInfD;
        const bool has_flat = (S.flags & 2) != 0;
        const float invc = win[c].z;
        const double muc = L.mu[c], varc = L.var[c];
        const bool flatc = is_flat_var(muc, varc);
        const double ic = flatc ? 0.0 : 1.0 / sqrt(varc);
        const bool zc_smem = m <= kRecheckWin;
        if (zc_smem)
            for (int k = lane; k < m; k += 32) zc[k] = __dmul_rn(double(T[c + k]) - muc, ic);
        __syncwarp();
        const float* arow = p.acen + g * int64_t(p.kpad_max);
        const float* cm = p.cmax + g * int64_t(p.nchunks_max);
        const int32_t nchunks = int32_t((N + 31) / 32);
        const int32_t cpb = p.seg / 32;  // chunks per coarse block
        for (int32_t cb = 0; cb < ncoarse; cb += 32) {
            const int32_t q2l = cb + lane;
            uint32_t bq2 = __ballot_sync(kFull, q2l < ncoarse && c2[q2l] >= thr_enc);
            while (bq2) {
                const int32_t q2 = cb + __ffs(bq2) - 1;
                bq2 &= bq2 - 1;
                // chunks of the coarse block above the threshold, 32 at a time
                for (int32_t qb = q2 * cpb; qb < (q2 + 1) * cpb; qb += 32) {
                const int32_t q = qb + lane;
                uint32_t bq = __ballot_sync(kFull, q < (q2 + 1) * cpb && q < nchunks && cm[q] >= thr);
                while (bq) {
                    const int32_t qq = qb + __ffs(bq) - 1;
                    bq &= bq - 1;
                    // FP32 rho of the chunk's columns, one per lane
                    const int64_t j = int64_t(qq) * 32 + lane;
                    float rho32 = -kInf;
                    const bool valid = j < N && (j - c >= m || c - j >= m) && j >= L.col_lo && j < L.col_hi;
                    if (valid) {
                        const float4 rj = win[j];
                        float acc = 0.f;
                        for (int k = 0; k < m; ++k) acc = fmaf(arow[k], T[j + k] - rj.w, acc);
                        rho32 = acc * invc * rj.z;
                        if (has_flat && (invc == 0.f || rj.z == 0.f)) rho32 = (invc == 0.f && rj.z == 0.f) ? 1.f : 0.f;
                    }
                    uint32_t bc = __ballot_sync(kFull, valid && rho32 >= thr);
                    while (bc) {
                        const int cl = __ffs(bc) - 1;
                        bc &= bc - 1;
                        const int64_t jc = int64_t(qq) * 32 + cl;
                        const float rc32 = __shfl_sync(kFull, rho32, cl);
                        const double muj = L.mu[jc], varj = L.var[jc];
                        const bool flatj = is_flat_var(muj, varj);
                        double d2 = 0.0;
                        if (flatc && flatj) d2 = 0.0;
                        else if (flatc || flatj) d2 = 2.0 * m;
                        else {
                            const double ij = 1.0 / sqrt(varj);
                            // each z value rounded on its own (no FMA contraction), so
                            // d(c, j) and d(j, c) are bit-identical and ties break by index
                            for (int k = lane; k < m; k += 32) {
                                const double zck = zc_smem ? zc[k] : __dmul_rn(double(T[c + k]) - muc, ic);
                                const double zjk = __dmul_rn(double(T[jc + k]) - muj, ij);
                                const double x = zck - zjk;
                                d2 = fma(x, x, d2);
                            }
#pragma unroll
                            for (int o = 16; o >= 1; o >>= 1) d2 += __shfl_xor_sync(kFull, d2, o);
                        }
                        if (KNN) {
                            // sorted insertion into the k smallest (uniform over the warp)
                            double v = d2;
#pragma unroll
                            for (int t = 0; t < (KNN ? kMaxKnn : 1); ++t)
                                if (t < p.knn && v < best[t]) {
                                    const double w = best[t];
                                    best[t] = v;
                                    v = w;
                                }
                        }
                        if (lane == 0) {
                            if (!KNN)
                                atomicMin(&p.nn2[g], static_cast<unsigned long long>(__double_as_longlong(d2)));
                            atomicMax(&S.maxerr, enc_f32(fabsf(rc32 - float(1.0 - d2 / (2.0 * m)))));
                            ++fp64;
                        }
                    }
                }
                }
            }
        }
        if (KNN && lane == 0) {
            // the k-th smallest (infinite when fewer than k non-self columns)
            double kth = best[0];
#pragma unroll
            for (int t = 0; t < (KNN ? kMaxKnn : 1); ++t)
                if (t == p.knn - 1) kth = best[t];
            p.nn2[g] = static_cast<unsigned long long>(__double_as_longlong(kth));
        }
        __syncwarp();
    }
    if (lane == 0 && fp64) atomicAdd(p.pairs + 2, fp64);
}

}  // namespace

cudaError_t launch_compact(const Pass& p, cudaStream_t s) {
    k_compact<<<p.nl, 1024, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_plan(const Pass& p, cudaStream_t s) {
    if (p.nslots <= 0) return cudaSuccess;
    if (p.nl > kMaxLanesSmem) return cudaErrorInvalidValue;
    const int block = 256;
    const int grid = int(min64((int64_t(p.nslots) + block - 1) / block, 1024));
    k_plan_count<<<grid, block, 0, s>>>(p);
    k_plan_split<<<grid, block, 0, s>>>(p);
    k_plan_groups<<<(p.nl + block - 1) / block, block, 0, s>>>(p);
    const int pgrid = int(min64((int64_t(p.nslots) * 32 + block - 1) / block, 4096));
    k_prep<<<pgrid, block, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_direct_repack(const Pass& p, cudaStream_t s) {
    if (p.nslots <= 0) return cudaSuccess;
    k_direct_compact<<<p.nl, 1024, 0, s>>>(p);
    k_plan_groups<<<(p.nl + 255) / 256, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_refine_direct(const Pass& p, int grid, cudaStream_t s) {
    if (p.nslots <= 0) return cudaSuccess;
    k_refine<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_recheck(const Pass& p, int grid, cudaStream_t s) {
    if (p.nslots <= 0) return cudaSuccess;
    if (p.knn > 1) k_recheck<true><<<grid, kRecheckWarps * 32, 0, s>>>(p);
    else k_recheck<false><<<grid, kRecheckWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace palmad
