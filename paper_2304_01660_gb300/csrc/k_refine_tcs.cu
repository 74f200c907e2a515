// Direct refine on the tensor cores, survivor-major (PALMAD_PREC_MIXED; DRAG
// phase 2, Algorithm 4, for survivors the plan routes to the direct form;
// windows up to 256 points).
//
// The same contraction as k_refine_tc.cu, with the roles of the operands
// swapped: 128 survivors g of one lane are the MMA's M side (the TMEM lanes)
// and 256 consecutive columns j its N side,
//     D[g][j] = sum_k a_g[k] (t[j+k] - b0),    a_g = centred FP32 window of g,
// as tcgen05.mma kind::f16, M = 128, N = 256, FP32 accumulation in TMEM, each
// FP32 operand split into two BF16 terms and three MMAs per K step (hi*hi +
// hi*lo + lo*hi).  The Hankel operand (N = 256 columns x K, K-major, no
// swizzle) is again 8 shifted copies of the series slice, so that core matrix
// (J, Kg) starts at 128 (J + Kg) bytes.  Compared with the column-major
// kernel one MMA carries four times the work (the issuing thread was the
// limit there), and each epilogue thread owns one survivor, so the maximum
// over a 32-column chunk is a chain of in-thread FMNMX instead of a warp
// reduction per survivor.
//
// The CTA (one per SM, all 512 TMEM columns) is warp-specialised:
//   warp 0       one lane issues the MMAs of a tile into one of two TMEM
//                accumulators (256 columns each) and commits them;
//   warps 1-7    producers: for every tile, the column factors
//                1/(sqrt(m) sigma_j), the chunk error bounds and the split
//                Hankel copies of the series slice into a ring slot (up to
//                6 slots);
//   warps 8-15   epilogue: warp w reads TMEM lane quarter w % 4 and column
//                half (w - 8) / 4 of the finished accumulator, releases it,
//                and reduces 32-column chunks.
// Seven producer warps keep the ring ahead of the MMAs (with three, the MMA
// warp waited on them for about a quarter of its time).
// Ring slots and accumulators are handed over with mbarriers (full / empty
// per slot, a second release per slot for the column factors and chunk
// bounds the epilogue reads, full / empty per accumulator).  The survivor
// operand is staged by every thread at the start of a work item (128
// survivors x up to 8192 columns).  Every wait is bounded; a thread whose wait gives up raises a
// shared abort flag, every role leaves its tile loop, and the CTA reports the
// error through p.err.
//
// Numerics follow k_refine_tc.cu: the same split, the same number of
// accumulating MMAs (3 kpad / 16), b0 the FP32 mean of the tile's middle
// column.  The epilogue takes rho(g, j) = D[g][j] / (sqrt(m) sigma_j) /
// (sqrt(m) sigma_g), without the centring correction (mu_j - b0) sum_k a_g[k]
// of the column-major kernel: a_g is centred, so its FP32 sum is a few
// roundings of the window, and the bound takes the dropped term instead,
//     eps_j = eps_j(column-major) + |mu_j - b0| / (sqrt(m) sigma_j) * S,
//     S = max over the item's survivors of |sum_k a_g[k]| / (sqrt(m) sigma_g),
// so a column needs one FP32 record (1 / (sqrt(m) sigma_j)) and one multiply
// per survivor.  1/sigma_j is applied per column and 1/sigma_g after the
// chunk maximum (both positive, so the maximum commutes), and the lane's
// FP32 bound covers those roundings as it covers the column-major
// epilogue's.  A survivor is pruned only when rho - eps exceeds the lane's
// pruning threshold; chunk maxima hold upper bounds and the survivor maximum
// a lower bound for the FP64 re-check.
#include "tc_util.cuh"

namespace palmad {

namespace {

using namespace tc;

constexpr int kSM = 128;          // survivors per MMA (M, TMEM lanes)
constexpr int kSN = 256;          // columns per tile (N)
constexpr int kSProd = 7;                     // producer warps (warps 1 .. kSProd)
constexpr int kSEpi0 = kSProd + 1;            // first of the 8 epilogue warps
constexpr int kSThreads = 32 * (kSEpi0 + 8);  // MMA warp, producers, epilogue
static_assert(kSEpi0 % 4 == 0, "epilogue warp w reads TMEM lane quarter w % 4");
constexpr int kSKpadMax = 256;    // the survivor operand of longer windows does not fit
constexpr int kSTilesItem = 32;   // tiles per work item (8192 columns)
constexpr int kSMaxStages = 6;

struct TcsLayout {
    int kp, stages;
    size_t a_bytes;     // one split of the survivor operand
    size_t h_bytes;     // one split of a tile's Hankel copies
    size_t slot_bytes;  // bh, bl, column factors 1 / (sqrt(m) sigma_j), chunk bounds
    size_t off_ah, off_al, off_ring, off_bar, total;
};

__host__ __device__ inline TcsLayout tcs_layout(int kp, int stages) {
    TcsLayout t{};
    t.kp = kp;
    t.stages = stages;
    t.a_bytes = size_t(kSM) * kp * 2;
    t.h_bytes = size_t(kSN / 8 + kp / 8) * 128;
    t.slot_bytes = 2 * t.h_bytes + size_t(kSN) * 4 + 64;
    t.slot_bytes = (t.slot_bytes + 127) / 128 * 128;
    t.off_ah = 0;
    t.off_al = t.a_bytes;
    t.off_ring = 2 * t.a_bytes;
    t.off_bar = t.off_ring + size_t(stages) * t.slot_bytes;
    // barriers: full, empty, cfree per stage; accfull, accempty per
    // accumulator; then the item, the TMEM slot, the abort and alive flags,
    // the item's survivor slots and the partial maxima of S
    t.total = t.off_bar + size_t(3 * stages + 4) * 8 + 32 + size_t(kSM) * 4 + 16;
    return t;
}

__host__ __device__ inline int tcs_stages(int kp) {
    int s = kSMaxStages;
    while (s > 2 && tcs_layout(kp, s).total > size_t(227 * 1024)) --s;
    return s;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(smem_u32(b)) : "memory");
}

// max(a, b, c) in one instruction (three-input max.f32).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// One lane of the warp polls (bounded), the warp learns the outcome; a
// timeout raises the CTA's abort flag.  Returns false when the wait gave up
// or another role has aborted.
__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        ok = *abort_flag ? 0 : (mbar_wait(b, parity) ? 1 : 0);
        if (!ok) *abort_flag = 1;
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    return ok != 0;
}


__global__ void __launch_bounds__(kSThreads, 1) k_refine_tcs(const Pass p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int S = tcs_stages(p.kpad_pass);
    const TcsLayout lay = tcs_layout(p.kpad_pass, S);
    unsigned char* ah = smem + lay.off_ah;
    unsigned char* al = smem + lay.off_al;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + lay.off_bar);  // [S] producers -> MMA, epilogue
    uint64_t* empty = full + S;          // [S] MMAs of the slot done -> producers
    uint64_t* cfree = full + 2 * S;      // [S] epilogue done with the slot's column records -> producers
    uint64_t* accfull = full + 3 * S;    // [2] MMAs of the accumulator done -> epilogue
    uint64_t* accempty = accfull + 2;    // [2] epilogue has read the accumulator -> MMA
    int64_t* s_item = reinterpret_cast<int64_t*>(accempty + 2);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_item + 1);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
    volatile int* s_alive = s_abort + 1;
    int32_t* s_slot = const_cast<int32_t*>(reinterpret_cast<volatile int32_t*>(s_alive + 1));  // [kSM]
    float* s_smax = reinterpret_cast<float*>(s_slot + kSM);  // [4] S of the first four epilogue warps' survivors

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], kSProd);
            mbar_init(&empty[s], 1);
            mbar_init(&cfree[s], 8);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], 8);
        }
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"(2 * kSN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *s_tmem;

    const int64_t ngroups = *reinterpret_cast<volatile int32_t*>(p.work + 4);
    const int64_t nhalf = kDGroup / kSM;  // MMA groups per direct group
    const int64_t iw = int64_t(kSN) * kSTilesItem;
    const int64_t clo = p.tc_col_lo, chi = min64(p.tc_col_hi, p.nmax);
    const int64_t nblk = chi > clo ? (chi - clo + iw - 1) / iw : 0;
    const int64_t nitems = ngroups * nhalf * nblk;
    uint32_t gt = 0;  // tiles this CTA has run: the phase of every ring slot and accumulator
    unsigned long long pairs = 0;

    for (;;) {
        if (tid == 0) {
            *s_item = atomicAdd(p.work + 1, 1);
            *s_alive = 0;
        }
        __syncthreads();
        const int64_t item = *s_item;
        if (item >= nitems) break;
        const int64_t hg = item / nblk, blk = item % nblk;
        const int32_t g64 = p.dgroups[hg / nhalf];
        const int64_t gbase = g64 + (hg % nhalf) * kSM;
        const int l = p.slot_lane[g64];
        const Lane& L = p.lanes[l];
        const LaneState& St = p.st[l];
        const int32_t m = L.m, kpad = L.kpad;
        const int32_t nd = int32_t(min64(kSM, int64_t(St.ndirect) - (gbase - L.slot_base)));
        const int64_t jstart = clo + blk * iw;
        const int64_t jend = min64(min64(jstart + iw, chi), L.N);
        if (nd <= 0 || jstart >= jend) {
            __syncthreads();
            continue;
        }
        // survivor records: epilogue thread (warp w, lane) owns survivor 32 (w % 4) + lane
        int32_t g = -1, zs = 0;
        float inv_s = 0.f, suma = 0.f;
        bool mine = false;
        if (warp >= kSEpi0) {
            const int s = 32 * (warp & 3) + lane;
            if (s < nd) {
                g = p.dlist[gbase + s];
                const int32_t w = p.slot_win[g];
                inv_s = L.win[w].z;
                suma = p.asum[g];
                zs = w - m + 1;  // columns zs .. zs + 2m - 2 overlap the survivor
                mine = !__ldcg(&p.dead[g]);
                if (mine) *s_alive = 1;
                if (warp < kSEpi0 + 4) s_slot[s] = g;
            } else if (warp < kSEpi0 + 4) {
                s_slot[s] = -1;
            }
            if (warp < kSEpi0 + 4) {
                // S of the item: the largest |sum_k a_g[k]| / (sqrt(m) sigma_g)
                const float sg = warp_max(g >= 0 ? fabsf(suma) * inv_s : 0.f);
                if (lane == 0) s_smax[warp - kSEpi0] = sg;
            }
        }
        __syncthreads();
        if (!*s_alive) {
            __syncthreads();
            continue;
        }
        // survivor operand (every thread): core matrix (G, Kg) at 128 (G kpad/8 + Kg),
        // row r at +16 r; entry e is row 8G + (e & 7) of core matrix e >> 3
        {
            const int kg8 = kpad / 8;
            for (int e = tid; e < kSM * kg8; e += kSThreads) {
                const int cm = e >> 3, kg = cm % kg8;
                const int s = 8 * (cm / kg8) + (e & 7);
                float x[8];
                const int32_t gs = s_slot[s];
                if (gs >= 0) {
                    const float4* src = reinterpret_cast<const float4*>(p.acen + int64_t(gs) * p.kpad_max + 8 * kg);
                    const float4 u0 = __ldg(src), u1 = __ldg(src + 1);
                    x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
                    x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
                } else {
#pragma unroll
                    for (int c = 0; c < 8; ++c) x[c] = 0.f;
                }
                uint4 hi, lo;
                split8(x, hi, lo);
                *reinterpret_cast<uint4*>(ah + size_t(16) * e) = hi;
                *reinterpret_cast<uint4*>(al + size_t(16) * e) = lo;
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        const int ntiles = int((jend - jstart + kSN - 1) / kSN);

        if (warp == 0) {
            // ---- MMA issue: one lane, tile after tile
            const uint32_t idesc = instr_desc(kSM, kSN);
            const uint32_t a_h = smem_u32(ah), a_l = smem_u32(al);
            const uint32_t sbo_a = 16u * uint32_t(kpad);
            for (int t = 0; t < ntiles; ++t) {
                const uint32_t u = gt + uint32_t(t);
                const int sl = int(u % uint32_t(S));
                const uint32_t ph = (u / uint32_t(S)) & 1u;
                const int b = int(u & 1u);
                const uint32_t pa = (u >> 1) & 1u;
                if (!warp_wait(&full[sl], ph, s_abort)) break;
                if (!warp_wait(&accempty[b], pa ^ 1u, s_abort)) break;
                fence_after();
                if (lane == 0) {
                    const uint32_t b_h = smem_u32(smem + lay.off_ring + size_t(sl) * lay.slot_bytes);
                    const uint32_t b_l = b_h + uint32_t(lay.h_bytes);
                    const uint32_t d = tmem + uint32_t(b * kSN);
                    // a K step of 16 advances every operand by 256 bytes (16 in
                    // the start-address field; addresses stay below 2^18)
                    uint64_t dah = mat_desc(a_h, 128, sbo_a), dal = mat_desc(a_l, 128, sbo_a);
                    uint64_t dbh = mat_desc(b_h, 128, 128), dbl = mat_desc(b_l, 128, 128);
                    for (int k = 0; k < kpad / 16; ++k) {
                        mma_bf16(d, dah, dbh, idesc, k > 0);
                        mma_bf16(d, dah, dbl, idesc, 1);
                        mma_bf16(d, dal, dbh, idesc, 1);
                        dah += 16; dal += 16; dbh += 16; dbl += 16;
                    }
                    mma_commit(&empty[sl]);
                    mma_commit(&accfull[b]);
                }
                __syncwarp();
            }
        } else if (warp <= kSProd) {
            // ---- producers: column records, chunk bounds and Hankel copies of each tile
            const int pw = warp - 1, ptid = tid - 32;
            const float sqrt_m = sqrtf(float(m));
            const float cmul = 1.01f * (3.02f * 1.52587890625e-05f + 5.9604644775390625e-08f +
                                        float(3 * kpad / 16 + 1) * 1.1920928955078125e-07f);
            const float* T = L.T;
            const int64_t n = L.n;
            const float smax = 1.01f * fmaxf(fmaxf(s_smax[0], s_smax[1]), fmaxf(s_smax[2], s_smax[3]));
            for (int t = 0; t < ntiles; ++t) {
                const uint32_t u = gt + uint32_t(t);
                const int sl = int(u % uint32_t(S));
                const uint32_t ph = (u / uint32_t(S)) & 1u;
                if (!warp_wait(&empty[sl], ph ^ 1u, s_abort)) break;
                if (!warp_wait(&cfree[sl], ph ^ 1u, s_abort)) break;
                unsigned char* slot = smem + lay.off_ring + size_t(sl) * lay.slot_bytes;
                unsigned char* bh = slot;
                unsigned char* bl = slot + lay.h_bytes;
                float* cinv = reinterpret_cast<float*>(slot + 2 * lay.h_bytes);
                float* ceps = cinv + kSN;
                const int64_t j0 = jstart + int64_t(t) * kSN;
                const float b0 = L.win[min64(j0 + kSN / 2, L.N - 1)].w;
                // columns 32 c + lane of the tile: 1 / (sqrt(m) sigma_j) and the
                // largest eps_j of each 32-column chunk
                for (int c = pw; c < kSN / 32; c += kSProd) {
                    const int64_t j = j0 + 32 * c + lane;
                    float inv = 0.f, eps = 0.f;
                    if (j < jend) {
                        const float4 w = __ldg(L.win + j);
                        inv = w.z;
                        const float dmu = w.w - b0;
                        const float tt = dmu * inv * sqrt_m;
                        eps = inv > 0.f ? 2.f * cmul * sqrtf(fmaf(tt, tt, 1.f)) * 1.000001f + 2.384185791015625e-07f +
                                              fabsf(dmu * inv) * 1.01f * smax
                                        : 0.f;
                    }
                    cinv[32 * c + lane] = inv;
                    const float em = warp_max(eps);
                    if (lane == 0) ceps[c] = em;
                }
                // Hankel copies: chunk q, copy r holds x[8q + r .. 8q + r + 8),
                // x = t[j0 + .] - b0; entry e = 8q + r reads t[j0 + e + c], so a
                // warp's loads of one c are 32 consecutive floats
                const int ne = 8 * (kSN / 8 + kpad / 8);
                for (int e = ptid; e < ne; e += 32 * kSProd) {
                    const int q = e >> 3, r = e & 7;
                    float x[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int64_t i = j0 + e + c;
                        x[c] = (i < n ? __ldg(T + i) : 0.f) - b0;
                    }
                    uint4 hi, lo;
                    split8(x, hi, lo);
                    *reinterpret_cast<uint4*>(bh + 128 * q + 16 * r) = hi;
                    *reinterpret_cast<uint4*>(bl + 128 * q + 16 * r) = lo;
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[sl]);
            }
        } else {
            // ---- epilogue: survivor 32 (warp % 4) + lane, column half (warp - kSEpi0) / 4
            const int q4 = warp & 3, hf = (warp - kSEpi0) >> 2;
            const float rp = rho_prune_of(L, St);
            const uint32_t excl = uint32_t(2 * m - 1);
            const int64_t zlo = zs, zhi = int64_t(zs) + 2 * m - 2;
            uint32_t c2run = 0u;  // enc_f32 maximum of the current coarse block (0: none)
            int64_t cb_cur = -1;
            float lorun = -kInf;
            for (int t = 0; t < ntiles; ++t) {
                const uint32_t u = gt + uint32_t(t);
                const int sl = int(u % uint32_t(S));
                const uint32_t ph = (u / uint32_t(S)) & 1u;
                const int b = int(u & 1u);
                const uint32_t pa = (u >> 1) & 1u;
                if (!warp_wait(&accfull[b], pa, s_abort)) break;
                // the slot's phase cannot move on before this warp releases it:
                // the wait returns at once and orders the producers' records
                if (!warp_wait(&full[sl], ph, s_abort)) break;
                fence_after();
                const unsigned char* slot = smem + lay.off_ring + size_t(sl) * lay.slot_bytes;
                const float* cinv = reinterpret_cast<const float*>(slot + 2 * lay.h_bytes);
                const float* ceps = cinv + kSN;
                const int64_t j0 = jstart + int64_t(t) * kSN;
                const int64_t cb = j0 / p.seg;  // a tile lies in one coarse block
                if (cb != cb_cur) {
                    if (mine && c2run) atomicMax(&p.cmax2[int64_t(g) * p.ncoarse_max + cb_cur], c2run);
                    c2run = 0u;
                    cb_cur = cb;
                }
                if (warp == kSEpi0 && lane == 0) pairs += uint64_t(nd) * uint64_t(min64(kSN, jend - j0));
#pragma unroll 1
                for (int c4 = 0; c4 < 4; ++c4) {
                    float v[32];
                    __syncwarp();  // tcgen05.ld is warp-aligned: reconverge after the divergent tail
                    tmem_ld32(tmem + (uint32_t(32 * q4) << 16) + uint32_t(b * kSN + 128 * hf + 32 * c4), v);
                    if (c4 == 3) {
                        // the accumulator is in registers: hand it back to the MMA warp
                        fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&accempty[b]);
                    }
                    const int cl = 128 * hf + 32 * c4;  // first column of the chunk in the tile
                    const int64_t cj = j0 + cl;
                    const float4* i4 = reinterpret_cast<const float4*>(cinv + cl);
                    float mx = -kInf;
                    if (cj + 31 < jend && (cj > zhi || cj + 31 < zlo)) {
                        // no column of the chunk is excluded or past the last window
#pragma unroll
                        for (int c = 0; c < 32; c += 4) {
                            const float4 iv = i4[c >> 2];
                            mx = fmax3(mx, v[c] * iv.x, v[c + 1] * iv.y);
                            mx = fmax3(mx, v[c + 2] * iv.z, v[c + 3] * iv.w);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; c += 4) {
                            const float4 iv = i4[c >> 2];
                            const float x[4] = {v[c] * iv.x, v[c + 1] * iv.y, v[c + 2] * iv.z, v[c + 3] * iv.w};
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int64_t j = cj + c + q;
                                const bool ok = j < jend && uint32_t(int32_t(j) - zs) >= excl;
                                mx = ok ? fmaxf(mx, x[q]) : mx;
                            }
                        }
                    }
                    // 1 / sigma_g >= 0 commutes with the maximum (a flat survivor: rho = 0)
                    const float keep = inv_s > 0.f ? mx * inv_s : (mx > -kInf ? 0.f : -kInf);
                    if (mine && cj < jend) {
                        // chunk upper bound, survivor lower bound, prune on the lower bound
                        const float e = ceps[cl >> 5];
                        p.cmax[int64_t(g) * p.nchunks_max + (cj >> 5)] = keep + e;
                        c2run = max(c2run, enc_f32(keep + e));
                        const float lo = keep - e;
                        lorun = fmaxf(lorun, lo);
                        if (lo > rp) {
                            p.dead[g] = 1;
                            if (L.hint) L.hint[zs + m - 1] = int32_t(cj) + 16;  // witness hint
                            mine = false;  // later maxima of a pruned survivor are not read
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&cfree[sl]);
            }
            if (mine) {
                if (c2run) atomicMax(&p.cmax2[int64_t(g) * p.ncoarse_max + cb_cur], c2run);
                if (lorun > -kInf) atomicMax(&p.gmax[g], enc_f32(lorun));
            }
        }
        gt += uint32_t(ntiles);
        fence_before();
        const bool abort = __syncthreads_or(*s_abort) != 0;  // uniform: every thread leaves together
        fence_after();
        if (abort) {
            // a wait gave up (an MMA or a role never signalled): report it and stop this CTA
            if (tid == 0) atomicExch(p.err, 1);
            break;
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kSN) : "memory");
    if (warp == kSEpi0 && lane == 0 && pairs) atomicAdd(p.pairs + 1, pairs);
}

}  // namespace

bool refine_tcs_supported(const Pass& p) {
    return p.kpad_pass <= kSKpadMax && p.nmax < (int64_t(1) << 31) - 2 * kSN * kSTilesItem &&
           tcs_layout(p.kpad_pass, 2).total <= size_t(227 * 1024);
}

cudaError_t launch_refine_tcs(const Pass& p, int sms, cudaStream_t s) {
    if (p.nslots <= 0) return cudaSuccess;
    if (!refine_tcs_supported(p)) return cudaErrorInvalidValue;
    const TcsLayout lay = tcs_layout(p.kpad_pass, tcs_stages(p.kpad_pass));
    // one CTA per SM: it holds all 512 TMEM columns (more than half of shared
    // memory keeps a second CTA off the SM)
    const size_t smem = lay.total > size_t(116 * 1024) ? lay.total : size_t(116 * 1024);
    cudaError_t e = cudaFuncSetAttribute(k_refine_tcs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_refine_tcs<<<sms, kSThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace palmad
