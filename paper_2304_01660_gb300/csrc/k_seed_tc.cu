// Top-row seeds of the refine sweep on the tensor cores (mixed precision;
// DRAG phase 2, Algorithm 4, recurrence form).
//
// A refine strip of the sweep needs, for every column j it visits, the dot
// product of its top row with column j (the value that enters the diagonal
// recurrence of Eq. 9 from above).  On CUDA cores that costs m FMAs per
// column per strip, about a third of the sweep's instructions.  Here the
// seeds of every strip that holds at least `seed_min` survivors are computed
// ahead of the sweep as one dense contraction per lane:
//     seeds[row][j] = sum_k (t[j+k] - b0) * a_row[k] - (mu_j - b0) * sum_k a_row[k],
// with a_row the strip's centred top window (FP32, as the sweep computes
// it), M = 128 columns x N = 32 strips per tcgen05.mma, K = kpad.
//
// The products carry three BF16 terms per operand (hi + mid + lo holds the
// full FP32 significand) and six MMAs per K step keep every product of
// combined order <= 2 (hi*hi, hi*mid, mid*hi, hi*lo, mid*mid, lo*hi).  Per
// product the dropped terms and the split residues stay within
// 5.01 * 2^-24 |a_k| |x_k|; every MMA adds at most one FP32 rounding
// (2^-23) of the magnitudes accumulated.  With |x_j|^2 = m (sigma_j^2 +
// (mu_j - b0)^2), the seed of column j is within
//     eps_j = 2 * C(kpad) * sqrt(1 + ((mu_j - b0) / sigma_j)^2) + 2^-22
// of the exact value, in rho units.  The largest eps_j of a lane goes into
// LaneState::seed_eps, which eps_bound adds to the lane's FP32 bound, so the
// sweep's pruning stays sound and its FP64 re-check complete.
//
// Kernels: k_seed_plan (one CTA: rows per lane, seed groups), k_seed_prep
// (centred top windows), k_seed_tc (the contraction).
//
// Off by default (palmad_options.tc_seed_min = 0).  The contraction is
// skinny: a lane has a few dozen dense strips against 10^5 or more columns,
// so every MMA is small (N = 32) and this kernel makes ~0.1 T seeds/s.  It
// also seeds every column, while most strips that hold no discord are
// pruned after a few segments.  On the sine, random-walk and multi-series
// workloads the sweep time it saved was at most what it cost.
#include "tc_util.cuh"

namespace palmad {

namespace {

using namespace tc;

constexpr int kSM = 128;        // columns per MMA tile
constexpr int kSTiles = 8;      // tiles per work item
constexpr int kSN = 32;         // strips per MMA (N)
constexpr int kSThreads = 128;

// Rows of the seed buffer per lane (exclusive scan over the lanes), and the
// list of groups of <= 32 rows of one lane.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_seed_plan(const Pass p) {
    __shared__ int32_t scan_r[1024], scan_g[1024];
    __shared__ int32_t base_r, base_g;
    const int tid = threadIdx.x;
    if (tid == 0) {
        base_r = 0;
        base_g = 0;
    }
    __syncthreads();
    for (int l0 = 0; l0 < p.nl; l0 += 1024) {
        const int l = l0 + tid;
        const int32_t cnt = l < p.nl ? p.st[l].seed_rows : 0;
        // rows granted: the buffer holds seed_cap rows; groups of 32
        scan_r[tid] = cnt;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int32_t v = tid >= o ? scan_r[tid - o] : 0;
            __syncthreads();
            scan_r[tid] += v;
            __syncthreads();
        }
        const int32_t base = base_r + scan_r[tid] - cnt;
        const int32_t eff = max(0, min(cnt, p.seed_cap - base));
        const int32_t ng = (eff + kSN - 1) / kSN;
        scan_g[tid] = ng;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int32_t v = tid >= o ? scan_g[tid - o] : 0;
            __syncthreads();
            scan_g[tid] += v;
            __syncthreads();
        }
        const int32_t gb = base_g + scan_g[tid] - ng;
        if (l < p.nl) {
            p.st[l].seed_base = base;
            p.st[l].seed_eff = eff;
            for (int32_t k = 0; k < ng; ++k) p.seed_groups[gb + k] = make_int4(l, base + kSN * k, min(kSN, eff - kSN * k), 0);
        }
        __syncthreads();
        if (tid == 1023) {
            base_r += scan_r[1023];
            base_g += scan_g[1023];
        }
        __syncthreads();
    }
    if (tid == 0) *p.seed_ngroups = base_g;
}

// Centred FP32 top window of every seeded strip (one warp per strip), the
// same values the sweep would compute for itself.
__global__ void k_seed_prep(const Pass p) {
    const int lane = threadIdx.x & 31;
    const int64_t nref = *p.nref;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t e = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; e < nref; e += nw) {
        const int32_t loc = p.strip_row[e];
        const int2 sl = p.strips[e];
        const LaneState& S = p.st[sl.x];
        if (loc < 0 || loc >= S.seed_eff) continue;
        const Lane& L = p.lanes[sl.x];
        const int64_t row = int64_t(S.seed_base) + loc;
        const int64_t i0 = int64_t(sl.y) * p.refine_h;
        const float mu = L.win[i0].w;
        float part = 0.f;
        float* dst = p.topcen + row * p.kpad_max;
        for (int k = lane; k < p.kpad_max; k += 32) {
            const float v = k < L.m ? L.T[i0 + k] - mu : 0.f;
            dst[k] = v;
            part += v;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) p.topsum[row] = part;
    }
}

struct SeedLayout {
    size_t b_bytes, a_bytes;  // one split of the strip operand / of one Hankel buffer
    size_t off_b, off_a, off_t, off_c, off_misc, total;
};

__host__ __device__ constexpr int seed_span(int kp) { return kSTiles * kSM + kp + 16; }

__host__ __device__ inline SeedLayout seed_layout(int kp) {
    SeedLayout t{};
    t.b_bytes = size_t(kSN) * kp * 2;
    t.a_bytes = size_t(kSM / 8 + kp / 8) * 128;
    t.off_b = 0;                                     // [3] splits
    t.off_a = 3 * t.b_bytes;                         // [2] buffers x [3] splits
    t.off_t = t.off_a + 6 * t.a_bytes;               // series slice
    t.off_c = t.off_t + size_t(seed_span(kp)) * 4;  // column records (inv, mu)
    t.off_misc = t.off_c + size_t(kSTiles * kSM) * 8;
    t.total = t.off_misc + kSN * 4 + 64;             // strip sums, mbar[2], tmem slot
    return t;
}

__global__ void __launch_bounds__(kSThreads, 1) k_seed_tc(const Pass p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const SeedLayout lay = seed_layout(p.kpad_pass);
    float* s_T = reinterpret_cast<float*>(smem + lay.off_t);
    float2* s_C = reinterpret_cast<float2*>(smem + lay.off_c);
    float* s_sum = reinterpret_cast<float*>(smem + lay.off_misc);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(s_sum + kSN);  // off_misc and kSN*4 are multiples of 8
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(mbar + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t idesc = instr_desc(kSM, kSN);
    const int64_t ngroups = *reinterpret_cast<volatile int32_t*>(p.seed_ngroups);
    const int64_t nblk = (p.nmax + kSM * kSTiles - 1) / (kSM * kSTiles);
    const int64_t nitems = ngroups * nblk;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
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
    uint32_t phase = 0u;
    bool tmo = false;
    unsigned long long seeds = 0;

    for (;;) {
        __shared__ int64_t item_s;
        if (tid == 0) item_s = atomicAdd(p.work + 6, 1);
        __syncthreads();
        const int64_t item = item_s;
        if (item >= nitems) break;
        const int4 grp = p.seed_groups[item / nblk];
        const int64_t jstart = (item % nblk) * int64_t(kSM * kSTiles);
        const int l = grp.x;
        const int64_t row0 = grp.y;
        const int cnt = grp.z;
        const Lane& L = p.lanes[l];
        LaneState& S = p.st[l];
        const int64_t N = L.N, n = L.n;
        const int32_t m = L.m, kpad = L.kpad;
        if (jstart >= N) {
            __syncthreads();
            continue;
        }
        const int ntiles = int(min64(kSTiles, (N - jstart + kSM - 1) / kSM));
        const int nloc = int(min64(int64_t(ntiles) * kSM, N - jstart));
        {
            const int span4 = (ntiles * kSM + kpad + 8 + 3) / 4;
#pragma unroll 4
            for (int e = tid; e < span4; e += kSThreads) {
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
            for (int e = tid; e < ntiles * kSM; e += kSThreads) {
                const int64_t j = jstart + e;
                const float4 w = j < N ? __ldg(L.win + j) : make_float4(0.f, 0.f, 0.f, 0.f);
                s_C[e] = make_float2(w.z, w.w);
            }
            if (tid < kSN) s_sum[tid] = tid < cnt ? p.topsum[row0 + tid] : 0.f;
        }
        // strip operand, three splits; entry e is row 8G + (e & 7) of core matrix e >> 3
        const int kg8 = kpad / 8;
#pragma unroll 2
        for (int e = tid; e < kSN * kg8; e += kSThreads) {
            const int cm = e >> 3, kg = cm % kg8;
            const int s = 8 * (cm / kg8) + (e & 7);
            float x[8];
            if (s < cnt) {
                const float4* src = reinterpret_cast<const float4*>(p.topcen + (row0 + s) * p.kpad_max + 8 * kg);
                const float4 u0 = __ldg(src), u1 = __ldg(src + 1);
                x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
                x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) x[c] = 0.f;
            }
            uint4 h, md, lo;
            split8x3(x, h, md, lo);
            *reinterpret_cast<uint4*>(smem + lay.off_b + size_t(16) * e) = h;
            *reinterpret_cast<uint4*>(smem + lay.off_b + lay.b_bytes + size_t(16) * e) = md;
            *reinterpret_cast<uint4*>(smem + lay.off_b + 2 * lay.b_bytes + size_t(16) * e) = lo;
        }
        __syncthreads();
        const float sqrt_m = sqrtf(float(m));
        const float cmul = 1.01f * (5.01f * 5.9604644775390625e-08f + float(6 * kpad / 16 + 1) * 1.1920928955078125e-07f);

        auto epilogue = [&](int t) {
            const int b = t & 1;
            if (!mbar_wait(&mbar[b], (phase >> b) & 1u)) tmo = true;
            phase ^= 1u << b;
            fence_after();
            const float b0 = s_C[min(t * kSM + kSM / 2, nloc - 1)].y;
            const int jl = t * kSM + 32 * warp + lane;
            const bool jok = jl < nloc;
            const float2 cw = jok ? s_C[jl] : make_float2(0.f, 0.f);
            const float dmu = cw.y - b0;
            const float tt = dmu * cw.x * sqrt_m;
            const float eps = cw.x > 0.f ? 2.f * cmul * sqrtf(fmaf(tt, tt, 1.f)) * 1.000001f + 2.384185791015625e-07f
                                         : 0.f;
            float v[32];
            tmem_ld32(tmem + (uint32_t(32 * warp) << 16) + uint32_t(b * kSN), v);
            if (jok && !tmo) {
                float* dst = p.seeds + row0 * p.seed_stride + jstart + jl;
#pragma unroll
                for (int s = 0; s < kSN; ++s)
                    if (s < cnt) dst[int64_t(s) * p.seed_stride] = fmaf(-dmu, s_sum[s], v[s]);
            }
            const float em = warp_max(eps);
            if (lane == 0 && em > 0.f) atomicMax(&S.seed_eps, __float_as_uint(em));  // non-negative floats order as uints
            fence_before();
        };

        bool abort = false;
        for (int t = 0; t < ntiles; ++t) {
            const int b = t & 1;
            const float b0 = s_C[min(t * kSM + kSM / 2, nloc - 1)].y;
            unsigned char* a0 = smem + lay.off_a + size_t(3 * b) * lay.a_bytes;
            // Hankel copies, three splits: chunk q, copy r holds x[8q + r .. 8q + r + 8)
            const int nq = kSM / 8 + kpad / 8;
            const float* tl = s_T + t * kSM;
            for (int e = tid; e < nq * 8; e += kSThreads) {
                const int q = e >> 3, r = e & 7;
                float x[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) x[c] = tl[8 * q + r + c] - b0;
                uint4 h, md, lo;
                split8x3(x, h, md, lo);
                *reinterpret_cast<uint4*>(a0 + 128 * q + 16 * r) = h;
                *reinterpret_cast<uint4*>(a0 + lay.a_bytes + 128 * q + 16 * r) = md;
                *reinterpret_cast<uint4*>(a0 + 2 * lay.a_bytes + 128 * q + 16 * r) = lo;
            }
            fence_async_smem();
            fence_before();
            abort = __syncthreads_or(tmo) != 0;
            fence_after();
            if (abort) break;
            if (tid == 0) {
                const uint32_t d = tmem + uint32_t(b * kSN);
                const uint32_t ax = smem_u32(a0), bx = smem_u32(smem + lay.off_b);
                const uint32_t ab = uint32_t(lay.a_bytes), bb = uint32_t(lay.b_bytes);
                const uint32_t sbo_b = 16u * uint32_t(kpad);
                // (x term, a term) pairs of combined order <= 2: (0,0) (1,0) (0,1) (2,0) (1,1) (0,2)
                const int xi[6] = {0, 1, 0, 2, 1, 0}, ai[6] = {0, 0, 1, 0, 1, 2};
                for (int k = 0; k < kpad / 16; ++k)
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        mma_bf16(d, mat_desc(ax + xi[q] * ab + 256 * k, 128, 128),
                                 mat_desc(bx + ai[q] * bb + 256 * k, 128, sbo_b), idesc, (k | q) != 0);
                mma_commit(&mbar[b]);
            }
            seeds += uint64_t(cnt) * uint64_t(min64(kSM, N - jstart - int64_t(t) * kSM));
            if (t > 0) epilogue(t - 1);
        }
        if (!abort) epilogue(ntiles - 1);
        abort = __syncthreads_or(tmo) != 0;
        if (abort) {
            if (tid == 0) atomicExch(p.err, 1);
            break;
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kSN) : "memory");
    if (tid == 0 && seeds) atomicAdd(p.pairs + 6, seeds);
}

}  // namespace

bool seed_tc_supported(const Pass& p) { return p.kpad_pass <= 512 && p.nmax < (int64_t(1) << 31) - 4096; }

cudaError_t launch_seeds(const Pass& p, int sms, cudaStream_t s) {
    if (p.nl > 0) k_seed_plan<<<1, 1024, 0, s>>>(p);
    k_seed_prep<<<sms * 2, 256, 0, s>>>(p);
    const SeedLayout lay = seed_layout(p.kpad_pass);
    // at least 60 KB per CTA: at most 3 CTAs (3 x 64 TMEM columns) per SM
    const size_t smem = lay.total > 60 * 1024 ? lay.total : size_t(60 * 1024);
    cudaError_t e = cudaFuncSetAttribute(k_seed_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_seed_tc<<<sms * 2, kSThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace palmad
