// Direct refine on the tensor cores (PALMAD_PREC_MIXED; DRAG phase 2,
// Algorithm 4, for survivors the plan routes to the direct form).
//
// For a group of NS survivors g of one lane and a tile of 128 consecutive
// columns j, the dot products
//     D[j][g] = sum_k (t[j+k] - b0) * a_g[k],    a_g = centred FP32 window of g,
// form a dense contraction whose column operand is a Hankel matrix of the
// series.  It runs as tcgen05.mma kind::f16 with FP32 accumulation in TMEM:
//   * every FP32 operand is split into two BF16 terms (hi = bf16(v),
//     lo = bf16(v - hi)); three MMAs (hi*hi + hi*lo + lo*hi) give each
//     product to about 2^-15 of |a_k| |x_k|;
//   * the Hankel operand (M = 128 columns x K, K-major, no swizzle) is not
//     materialised: 8 shifted copies of the series slice, interleaved in
//     16-byte rows, make core matrix (J, Kg) start at 128 (J + Kg) bytes, so
//     one shared-memory descriptor with both strides 128 B walks it;
//   * the survivor operand (N = NS rows x K) is staged once per work item in
//     the canonical K-major layout and reused by every tile of the item.
// b0 (the FP32 mean of the tile's middle column) is subtracted from the
// series slice before the split; the centred covariance is
//     cov(g, j) = D[j][g] - (mu_j - b0) * sum_k a_g[k].
// Two TMEM accumulators alternate, so the epilogue of one tile overlaps the
// MMAs of the next.
//
// Error bound (per column j, in rho units): each split product is within
// 3.02 * 2^-16 |a_k| |x_k| (+ 2^-24 for the FP32 subtraction), and every MMA
// adds at most one FP32 rounding (2^-23) of the magnitudes summed so far.
// Sum_k |a_k| |x_k| <= |a| |x_j| and |x_j|^2 = m (sigma_j^2 + (mu_j - b0)^2),
// so relative to m sigma_g sigma_j the bound is
//     eps_j = 2 * C(kpad) * sqrt(1 + ((mu_j - b0) / sigma_j)^2) + 2^-22,
// doubled for safety, on top of the lane's FP32 bound (centring and the
// epilogue arithmetic).  The epilogue keeps the FP32 paths' contract: a
// survivor is pruned only when rho - eps_j exceeds the lane's pruning
// threshold, the chunk maxima hold upper bounds and the survivor maximum a
// lower bound, so the FP64 re-check sees every column that can hold the
// nearest neighbour.
#include "tc_util.cuh"

namespace palmad {

namespace {

using namespace tc;

constexpr int kTcM = 128;       // columns per MMA tile (TMEM lanes)
constexpr int kTcTiles = 8;     // tiles per work item (1024 columns) ...
constexpr int kTcTilesLong = 16;  // ... or a whole 2048-column refine segment when shared memory allows
constexpr int kTcThreads = 256;  // two warpgroups; each reads every TMEM lane quarter

struct TcLayout {
    int kp;          // kpad_max (multiple of 32)
    int ns;          // survivors per MMA
    int tiles;       // tiles per work item
    size_t b_bytes;  // one split of the survivor operand
    size_t a_bytes;  // one split of one Hankel buffer
    size_t off_bh, off_bl, off_ah, off_al, off_t, off_c, off_misc, total;
};

// Series floats staged per work item: its columns plus the window tail.
__host__ __device__ constexpr int tc_span(int kp, int tiles) { return tiles * kTcM + kp + 16; }

__host__ __device__ inline TcLayout tc_layout(int kp, int ns, int tiles) {
    TcLayout t{};
    t.kp = kp;
    t.ns = ns;
    t.tiles = tiles;
    t.b_bytes = size_t(ns) * kp * 2;
    t.a_bytes = size_t(kTcM / 8 + kp / 8) * 128;
    t.off_bh = 0;
    t.off_bl = t.b_bytes;
    t.off_ah = 2 * t.b_bytes;                // [2] buffers
    t.off_al = t.off_ah + 2 * t.a_bytes;     // [2] buffers
    t.off_t = t.off_al + 2 * t.a_bytes;      // series slice (FP32)
    t.off_c = t.off_t + size_t(tc_span(kp, tiles)) * 4;  // column records (inv, mu)
    t.off_misc = t.off_c + size_t(tiles * kTcM) * 8;
    // misc: survivor records (float4), slots, lower-bound maxima, coarse
    // maxima; mbar[2]; tmem slot; flag
    t.total = t.off_misc + size_t(ns) * (16 + 4 + 4 + 8) + 64;
    return t;
}

// a tile lies inside one coarse block (p.seg is a multiple of 1024), and a
// work item of 1024 columns, or of 2048 when the segment (coarse block) is
// 2048 columns, touches one block
static_assert(kCoarseMin % kTcM == 0 && kTcM * kTcTiles <= kCoarseMin, "tiles and items inside coarse blocks");

// Tiles per work item: a whole 2048-column segment when the pass uses such
// segments and the layout fits in shared memory (the survivor operand, staged
// once per item, is then reused by twice as many tiles), else 1024 columns.
__host__ __device__ inline int tc_tiles(const Pass& p, int ns) {
    return (p.seg >= kTcTilesLong * kTcM && tc_layout(p.kpad_pass, ns, kTcTilesLong).total <= size_t(227 * 1024))
               ? kTcTilesLong : kTcTiles;
}

template <int NS>
__global__ void __launch_bounds__(kTcThreads, 1) k_refine_tc(const Pass p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tiles_item = tc_tiles(p, NS);
    const TcLayout lay = tc_layout(p.kpad_pass, NS, tiles_item);
    unsigned char* bh = smem + lay.off_bh;
    unsigned char* bl = smem + lay.off_bl;
    float* s_T = reinterpret_cast<float*>(smem + lay.off_t);
    float2* s_C = reinterpret_cast<float2*>(smem + lay.off_c);
    float4* s_rec = reinterpret_cast<float4*>(smem + lay.off_misc);  // inv, sum of a, exclusion start bits, -
    int32_t* s_slot = reinterpret_cast<int32_t*>(s_rec + NS);
    uint32_t* s_lo = reinterpret_cast<uint32_t*>(s_slot + NS);
    uint32_t* s_c2 = s_lo + NS;  // [2][NS] coarse-block maxima of the item (enc_f32)
    uint64_t* mbar = reinterpret_cast<uint64_t*>(s_c2 + 2 * NS);  // 8-byte aligned: off_misc and NS*32 are
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(mbar + 2);
    int* s_flag = reinterpret_cast<int*>(s_tmem + 1);           // a survivor of the item is alive

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t idesc = instr_desc(kTcM, NS);
    const int64_t ngroups = *reinterpret_cast<volatile int32_t*>(p.work + 4);
    const int64_t nhalf = kDGroup / NS;  // MMA groups per direct group
    // the launch's column chunk [tc_col_lo, tc_col_hi), in work-item blocks
    const int64_t iw = int64_t(kTcM) * tiles_item;
    const int64_t blk0 = p.tc_col_lo / iw;
    const int64_t nblk = max64(0, min64((p.tc_col_hi + iw - 1) / iw, (p.nmax + iw - 1) / iw) - blk0);
    const int64_t nitems = ngroups * nhalf * nblk;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(s_tmem)), "r"(2 * NS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *s_tmem;
    uint32_t phase = 0u;   // bit b: parity of the next completion of mbar[b]
    bool tmo = false;      // this thread's bounded wait gave up
    unsigned long long pairs = 0;

    for (;;) {
        __shared__ int64_t item_s;
        if (tid == 0) item_s = atomicAdd(p.work + 1, 1);
        __syncthreads();
        const int64_t item = item_s;
        if (item >= nitems) break;
        const int64_t hg = item / nblk;
        const int64_t blk = item % nblk;
        const int32_t g64 = p.dgroups[hg / nhalf];
        const int64_t gbase = g64 + (hg % nhalf) * NS;
        const int l = p.slot_lane[g64];
        const Lane& L = p.lanes[l];
        const LaneState& S = p.st[l];
        const int64_t N = L.N, n = L.n;
        const int32_t m = L.m, kpad = L.kpad;
        const int32_t nd = min64(NS, int64_t(S.ndirect) - (gbase - L.slot_base));
        const int64_t jstart = (blk0 + blk) * iw;
        if (nd <= 0 || jstart >= N) {
            __syncthreads();
            continue;
        }
        // survivors of the group and whether any is alive
        if (tid == 0) s_flag[0] = 0;
        __syncthreads();
        if (tid < NS) {
            int32_t g = -1, w = 0;
            float inv = 0.f, suma = 0.f;
            if (tid < nd) {
                g = p.dlist[gbase + tid];
                w = p.slot_win[g];
                inv = L.win[w].z;
                suma = p.asum[g];
                if (!__ldcg(&p.dead[g])) s_flag[0] = 1;
            }
            s_slot[tid] = g;
            // columns w-m+1 .. w+m-1 overlap the survivor (no non-self match)
            s_rec[tid] = make_float4(inv, suma, __int_as_float(w - m + 1), 0.f);
            s_lo[tid] = 0u;  // enc_f32 order: 0 is below every float
            s_c2[tid] = 0u;
            s_c2[NS + tid] = 0u;
        }
        __syncthreads();
        if (!s_flag[0]) {
            __syncthreads();
            continue;
        }
        const int ntiles = int(min64(tiles_item, (N - jstart + kTcM - 1) / kTcM));
        // series slice t[jstart, jstart + span) and column records (inv, mu) of
        // the item's columns, loaded with many loads in flight
        {
            const int span4 = (ntiles * kTcM + kpad + 8 + 3) / 4;
#pragma unroll 4
            for (int e = tid; e < span4; e += kTcThreads) {
                const int64_t i = jstart + 4 * int64_t(e);
                float4 v;
                if (i + 3 < n) {
                    v = __ldg(reinterpret_cast<const float4*>(L.T + i));  // T and jstart are 16-byte aligned
                } else {
                    v.x = i < n ? L.T[i] : 0.f;
                    v.y = i + 1 < n ? L.T[i + 1] : 0.f;
                    v.z = i + 2 < n ? L.T[i + 2] : 0.f;
                    v.w = 0.f;
                }
                reinterpret_cast<float4*>(s_T)[e] = v;
            }
#pragma unroll 4
            for (int e = tid; e < ntiles * kTcM; e += kTcThreads) {
                const int64_t j = jstart + e;
                const float4 w = j < N ? __ldg(L.win + j) : make_float4(0.f, 0.f, 0.f, 0.f);
                s_C[e] = make_float2(w.z, w.w);
            }
        }
        // survivor operand: core matrix (G, Kg) at 128 (G kpad/8 + Kg), row r at
        // +16 r; entry e covers row s = 8G + (e & 7) of core matrix e >> 3, so a
        // warp's 16-byte stores are contiguous (byte offset 16 e)
        const int kg8 = kpad / 8;
#pragma unroll 4
        for (int e = tid; e < NS * kg8; e += kTcThreads) {
            const int cm = e >> 3, kg = cm % kg8;
            const int s = 8 * (cm / kg8) + (e & 7);
            float x[8];
            if (s < nd) {
                const float4* src = reinterpret_cast<const float4*>(p.acen + int64_t(s_slot[s]) * p.kpad_max + 8 * kg);
                const float4 u0 = __ldg(src), u1 = __ldg(src + 1);
                x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
                x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) x[c] = 0.f;
            }
            uint4 hi, lo;
            split8(x, hi, lo);
            *reinterpret_cast<uint4*>(bh + size_t(16) * e) = hi;
            *reinterpret_cast<uint4*>(bl + size_t(16) * e) = lo;
        }
        __syncthreads();
        const float sqrt_m = sqrtf(float(m));
        const float cmul = 1.01f * (3.02f * 1.52587890625e-05f + 5.9604644775390625e-08f +
                                    float(3 * kpad / 16 + 1) * 1.1920928955078125e-07f);
        const float rp = rho_prune_of(L, S);
        const int nloc = int(min64(int64_t(ntiles) * kTcM, N - jstart));  // valid staged columns

        // Epilogue of tile t (accumulator t & 1).
        auto epilogue = [&](int t) {
            const int b = t & 1;
            // one lane per warp polls the barrier (256 spinning threads would
            // flood shared memory while the MMAs run), then the warp syncs
            int done = 1;
            if (lane == 0) done = mbar_wait(&mbar[b], (phase >> b) & 1u) ? 1 : 0;
            done = __shfl_sync(0xffffffffu, done, 0);
            __syncwarp();
            if (!done) tmo = true;
            phase ^= 1u << b;
            fence_after();
            const int64_t j0 = jstart + int64_t(t) * kTcM;
            const float b0 = s_C[min(t * kTcM + kTcM / 2, nloc - 1)].y;
            const int wq = warp & 3, hs = warp >> 2;  // TMEM lane quarter, survivor half
            const int jl = t * kTcM + 32 * wq + lane;
            const bool jok = jl < nloc;
            const float2 cw = jok ? s_C[jl] : make_float2(0.f, 0.f);
            const int32_t j32 = int32_t(jstart) + jl;
            const float dmu = cw.y - b0;
            const float tt = dmu * cw.x * sqrt_m;
            const float eps = cw.x > 0.f ? 2.f * cmul * sqrtf(fmaf(tt, tt, 1.f)) * 1.000001f + 2.384185791015625e-07f
                                         : 0.f;
            const float epsmax = warp_max(eps);
            const int32_t chunk = int32_t((j0 >> 5) + wq);
            const bool chunk_ok = t * kTcM + 32 * wq < nloc;  // chunks past the lane's last column are not stored
            const uint32_t excl = uint32_t(2 * m - 1);
            // survivor sub-blocks hs, hs + 2, ... (32 survivors each)
            for (int h = hs; h < NS / 32 && 32 * h < nd; h += 2) {
                float v[32];
                tmem_ld32(tmem + (uint32_t(32 * wq) << 16) + uint32_t(b * NS + 32 * h), v);
                float keep = -kInf;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int s = 32 * h + c;
                    if (s >= nd) break;
                    const float4 rec = s_rec[s];
                    const bool ok = jok && uint32_t(j32 - __float_as_int(rec.z)) >= excl;
                    const float rho = fmaf(-dmu, rec.y, v[c]) * rec.x * cw.x;
                    const float rmax = warp_max(ok ? rho : -kInf);
                    if (lane == c) keep = rmax;
                }
                const int s = 32 * h + lane;
                if (s < nd && chunk_ok && !tmo) {
                    // chunk upper bound, survivor lower bound, prune on the lower bound
                    const int32_t g = s_slot[s];
                    const float lo = keep - epsmax;
                    p.cmax[int64_t(g) * p.nchunks_max + chunk] = keep + epsmax;
                    atomicMax(&s_c2[s], enc_f32(keep + epsmax));
                    if (lo > -kInf) atomicMax(&s_lo[s], enc_f32(lo));
                    if (lo > rp) {
                        p.dead[g] = 1;
                        if (L.hint) L.hint[__float_as_int(s_rec[s].z) + m - 1] = int32_t(j0) + 32 * wq + 16;  // witness hint
                    }
                }
            }
            fence_before();
        };

        bool abort = false;
        for (int t = 0; t < ntiles; ++t) {
            const int b = t & 1;
            const int64_t j0 = jstart + int64_t(t) * kTcM;
            const float b0 = s_C[min(t * kTcM + kTcM / 2, nloc - 1)].y;
            unsigned char* ah = smem + lay.off_ah + b * lay.a_bytes;
            unsigned char* al = smem + lay.off_al + b * lay.a_bytes;
            // Hankel copies: chunk q, copy r holds x[8q + r .. 8q + r + 8), x = t[j0 + .] - b0
            const int nq = kTcM / 8 + kpad / 8;
            const float* tl = s_T + t * kTcM;
            for (int e = tid; e < nq * 8; e += kTcThreads) {
                const int q = e >> 3, r = e & 7;
                float x[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) x[c] = tl[8 * q + r + c] - b0;
                uint4 hi, lo;
                split8(x, hi, lo);
                *reinterpret_cast<uint4*>(ah + 128 * q + 16 * r) = hi;
                *reinterpret_cast<uint4*>(al + 128 * q + 16 * r) = lo;
            }
            fence_async_smem();
            fence_before();
            abort = __syncthreads_or(tmo) != 0;  // uniform: every thread leaves together
            fence_after();
            if (abort) break;
            if (tid == 0) {
                const uint32_t d = tmem + uint32_t(b * NS);
                const uint32_t a_h = smem_u32(ah), a_l = smem_u32(al), b_h = smem_u32(bh), b_l = smem_u32(bl);
                const uint32_t sbo_b = 16u * uint32_t(kpad);
                // a K step of 16 advances every operand by 256 bytes: 16 in the
                // descriptors' start-address field (addresses stay below 2^18)
                uint64_t dah = mat_desc(a_h, 128, 128), dal = mat_desc(a_l, 128, 128);
                uint64_t dbh = mat_desc(b_h, 128, sbo_b), dbl = mat_desc(b_l, 128, sbo_b);
                for (int k = 0; k < kpad / 16; ++k) {
                    mma_bf16(d, dah, dbh, idesc, k > 0);
                    mma_bf16(d, dah, dbl, idesc, 1);
                    mma_bf16(d, dal, dbh, idesc, 1);
                    dah += 16; dal += 16; dbh += 16; dbl += 16;
                }
                mma_commit(&mbar[b]);
            }
            pairs += uint64_t(nd) * uint64_t(min64(kTcM, N - j0));
            if (t > 0) epilogue(t - 1);
        }
        if (!abort) epilogue(ntiles - 1);
        abort = __syncthreads_or(tmo) != 0;
        if (abort) {
            // an MMA never signalled completion: report it and stop this CTA
            if (tid == 0) atomicExch(p.err, 1);
            break;
        }
        if (tid < nd) {
            if (s_lo[tid]) atomicMax(&p.gmax[s_slot[tid]], s_lo[tid]);
            // the coarse block holding the item (rows zeroed by the plan;
            // with 2048-column blocks two items share one)
            atomicMax(&p.cmax2[int64_t(s_slot[tid]) * p.ncoarse_max + jstart / p.seg], s_c2[tid]);
        }
        __syncthreads();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * NS) : "memory");
    if (tid == 0 && pairs) atomicAdd(p.pairs + 1, pairs);
}

}  // namespace

bool refine_tc_supported(const Pass& p) { return p.kpad_pass <= 1024 && p.nmax < (int64_t(1) << 31) - 4096; }

cudaError_t launch_refine_tc(const Pass& p, int sms, cudaStream_t s) {
    if (p.nslots <= 0) return cudaSuccess;
    // survivors per MMA (the MMA's N): 64, or 32 for windows above 512 (shared
    // memory); 128 or 256 when asked (palmad_options.tc_group): each
    // tcgen05.mma then carries more work for the one issuing thread, but a
    // group runs until its last survivor is pruned
    int ns = p.tc_ns > 0 ? p.tc_ns : (p.kpad_pass <= 512 ? 64 : 32);
    while (ns > 32 && tc_layout(p.kpad_pass, ns, kTcTiles).total > size_t(227 * 1024)) ns /= 2;  // what fits
    const TcLayout lay = tc_layout(p.kpad_pass, ns, tc_tiles(p, ns));
    // at least 76 KB per CTA: at most 2 CTAs (2 x 128 TMEM columns) per SM;
    // NS = 128 and 256 take half or all of TMEM and run one CTA per SM
    const size_t smem = lay.total > 78 * 1024 ? lay.total : size_t(78 * 1024);
    if (smem > size_t(227 * 1024)) return cudaErrorInvalidValue;
    auto go = [&](auto kern, int ctas) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        kern<<<sms * ctas, kTcThreads, smem, s>>>(p);
        return cudaGetLastError();
    };
    if (ns == 256) return go(k_refine_tc<256>, 1);
    if (ns == 128) return go(k_refine_tc<128>, 1);
    if (ns == 64) return go(k_refine_tc<64>, 2);
    return go(k_refine_tc<32>, 2);
}

}  // namespace palmad
