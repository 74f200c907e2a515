// Strip sweeps: candidate select (DRAG phase 1; Algorithm 3, Sec. 3.2) and
// the recurrence form of refine (DRAG phase 2; Algorithm 4, Sec. 3.3).
//
// A warp owns a strip of H = 32*D consecutive windows (rows i; D = 4, so
// 128 rows, in both sweeps) and steps across a range of windows (columns j),
// 32 columns per chunk:
//   * lane l holds rows i0 + l*D .. i0 + l*D + D-1 in registers; one step
//     advances every row by one column with the diagonal recurrence of Eq. 9
//     (cov(i,j) = cov(i-1,j-1) + df_i dg_j + df_j dg_i); the value of the row
//     above arrives from the previous lane by one shuffle;
//   * the strip's top row has no row above: its dot products ("QTrow" of
//     Algorithm 3) are computed per chunk by a register-blocked pass over
//     the staged series (4 groups of 8 columns, each lane one eighth of the
//     window in interleaved blocks of 4), then reduce-scattered within each
//     group;
//   * select scans to the right (j >= i + m) from the strip's triangle, as
//     the paper's segment-scans-right; a pair with rho > rho_prune (d < r
//     beyond the FP32 error band) clears the row's and the column's
//     candidate bit (Cand and Neighbor of Algorithm 3 are one bitmap here,
//     since refine ANDs them anyway); the warp leaves the strip once every
//     row is dead (the early exit of Algorithm 3) or after `cap` columns;
//   * refine sweeps a 1024-column segment of every strip that holds enough
//     survivors (both sides of the exclusion zone |i - j| < m, which is
//     masked), starting from directly computed first-column dot products;
//     per survivor it records the maximum rho of every 32-column chunk, and
//     a pair with rho > rho_prune marks the survivor dead (the early abandon
//     of Algorithm 4).
// Pruning is sound: a pair is used only when its FP32 rho exceeds the exact
// threshold by more than the error bound, so no range discord is dropped.
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerCta = 4;

struct WarpSmem {
    float* ahat;    // [kp]         centred top-row window, zero padded
    float* tw;      // [2][kp + 32] series slices of this and the next chunk
    float4* colrec; // [2][32]      column records of this and the next chunk
    float* seed;    // [32]         top-row dot products of this chunk
    float* tcseed;  // [2][32]      tensor-core top-row seeds of this and the next chunk
};

__device__ __forceinline__ size_t warp_smem_floats(int kp) { return size_t(kp) + 2 * (kp + 32) + 2 * 128 + 32 + 64; }

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc, int src_bytes) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Fields of the lane a work item belongs to.
struct LaneView {
    const float* T;
    int64_t n, N;
    int32_t m;
    const WinRec* win;
};

// Start the asynchronous copy of chunk c0's series slice and column records
// into buffer b (zero fill past the ends of T and of the windows).  T and
// win are 16-byte aligned and c0 is a multiple of 32.  With tensor-core
// seeds (tcs: the strip's seed row) the chunk's seeds replace the slice.
__device__ __forceinline__ void issue_chunk(const LaneView& a, const WarpSmem& sm, int kps, int b, int64_t c0,
                                            int kp, int lane, const float* tcs) {
    const int64_t j = c0 + lane;
    if (tcs) {
        cp_async4(sm.tcseed + b * 32 + lane, j < a.N ? static_cast<const void*>(tcs + j) : static_cast<const void*>(tcs),
                  j < a.N ? 4 : 0);
    } else {
        float* tw = sm.tw + b * (kps + 32);
        for (int x = lane * 4; x < kp + 32; x += 128) {
            const int64_t t = c0 + x;
            const int64_t rem = a.n - t;
            const int bytes = rem >= 4 ? 16 : (rem > 0 ? int(rem) * 4 : 0);
            cp_async16(tw + x, bytes > 0 ? static_cast<const void*>(a.T + t) : static_cast<const void*>(a.T), bytes);
        }
    }
    cp_async16(sm.colrec + b * 32 + lane, j < a.N ? static_cast<const void*>(a.win + j) : static_cast<const void*>(a.win),
               j < a.N ? 16 : 0);
    cp_async_commit();
}

// max(a, b, c) in one instruction (three-input max.f32, sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Reduce-scatter over the 8 lanes of a column group (lanes g, g+4, ..., g+28):
// the group's sum of acc[c] lands in the lane whose k-slice index
// ks = lane >> 2 equals c (3 shuffle stages).
__device__ __forceinline__ float reduce_scatter8(float (&acc)[8], int lane) {
#pragma unroll
    for (int o = 16, w = 4; o >= 4; o >>= 1, w >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < w; ++k) {
            const float send = upper ? acc[k] : acc[k + w];
            const float keep = upper ? acc[k + w] : acc[k];
            acc[k] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    return acc[0];
}

// Top-row dot products cov(top, c0 + c) of one chunk's 32 columns from the
// staged buffer b (series slice minus the offset b0 = mu of column c0).
// Lane = ks*4 + g: column group g (columns 8g .. 8g+7) and k-slice ks, the
// blocks k = 32t + 4ks .. 32t + 4ks + 3 (t = 0 .. kp/32 - 1).  Interleaving
// the slices in blocks of 4 puts the 8 lanes of every quarter-warp on 8
// distinct 16-byte bank groups for both the series and the window loads, so
// the 128-bit shared loads run without bank conflicts.  Each lane
// accumulates its 8 columns over its slice, then the group's 8 lanes
// reduce-scatter so that lane (g, ks) holds column 8g + ks.
__device__ __forceinline__ void chunk_seeds(const LaneView& a, const WarpSmem& sm, int kps, int b, int64_t c0,
                                            float suma, int kp, int lane) {
    float* tw = sm.tw + b * (kps + 32);
    const float4* cr = sm.colrec + b * 32;
    const float b0 = cr[0].w;
    for (int x = lane; x < kp + 32; x += 32) tw[x] -= b0;
    __syncwarp();
    const int g = lane & 3, ks = lane >> 2;
    float acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.f;
    const float* ap = sm.ahat + 4 * ks;
    const float* tp = tw + 8 * g + 4 * ks;
    for (int q = 0; q < kp; q += 32) {
        const float4 av = *reinterpret_cast<const float4*>(ap + q);
        const float4 t0 = *reinterpret_cast<const float4*>(tp + q);
        const float4 t1 = *reinterpret_cast<const float4*>(tp + q + 4);
        const float4 t2 = *reinterpret_cast<const float4*>(tp + q + 8);
        const float a4[4] = {av.x, av.y, av.z, av.w};
        const float tv[12] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w, t2.x, t2.y, t2.z, t2.w};
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = fmaf(a4[qq], tv[qq + c], acc[c]);
    }
    const float dot = reduce_scatter8(acc, lane);
    const int col = g * 8 + ks;
    const int64_t j = c0 + col;
    sm.seed[col] = (j < a.N) ? dot - (cr[col].w - b0) * suma : 0.f;
    __syncwarp();
}

// cov(r0 + d, ja) for d < D: direct dot products of this lane's rows with
// column ja (centred column window x, rows offset by b0 = mu of row r0).
template <int D>
__device__ __forceinline__ void first_col_seeds(const LaneView& a, int64_t r0, int64_t ja, float (&cov)[D]) {
    const int32_t m = a.m;
    const float mux = a.win[ja].w;
    const float b0 = (r0 < a.N) ? a.win[r0].w : 0.f;
    float acc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) acc[d] = 0.f;
    float sx = 0.f;
    for (int k = 0; k < m; k += 8) {
        float x[8], y[D + 8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t t = ja + k + q;
            x[q] = (k + q < m && t < a.n) ? (a.T[t] - mux) : 0.f;
            sx += x[q];
        }
#pragma unroll
        for (int q = 0; q < D + 8; ++q) {
            const int64_t t = r0 + k + q;
            y[q] = (t < a.n) ? (a.T[t] - b0) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int d = 0; d < D; ++d) acc[d] = fmaf(x[q], y[d + q], acc[d]);
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int64_t i = r0 + d;
        const float mui = (i < a.N) ? a.win[i].w : 0.f;
        cov[d] = acc[d] - (mui - b0) * sx;
    }
}

// KNN (refine only): the k-th neighbour variant; a survivor dies once k of
// its pairs clear the pruning threshold (counted per slot over every work
// item), instead of at its first such pair.
template <int D, bool REFINE, bool KNN = false>
__global__ void __launch_bounds__(kWarpsPerCta * 32, D <= 4 ? 4 : 3) k_sweep(const Pass p) {
    constexpr int H = 32 * D;
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int kps = ((p.kpad_max + 127) / 128) * 128;  // smem stride (largest lane)
    float* base = smem + warp_smem_floats(kps) * wid;
    const WarpSmem sm{base, base + kps, reinterpret_cast<float4*>(base + kps + 2 * (kps + 32)),
                      base + kps + 2 * (kps + 32) + 256, base + kps + 2 * (kps + 32) + 256 + 32};
    int64_t* strip_base = reinterpret_cast<int64_t*>(smem + warp_smem_floats(kps) * kWarpsPerCta);
    if (!REFINE) {
        for (int l = threadIdx.x; l < p.nl; l += blockDim.x) strip_base[l] = p.lanes[l].strip_base;
        __syncthreads();
    }
    const int64_t nseg = REFINE ? (p.nmax + p.seg - 1) / p.seg : 1;
    const int64_t nref = REFINE ? int64_t(*p.nref) : 0;
    // refine items: rank k (0, +1, -1, +2, -2, ... segments away from the
    // strip's own segment) major, strip minor -- the segments nearest every
    // strip run first, so survivors pruned there skip the far ones
    // select items: column piece major, strip minor -- every strip's first
    // piece (its triangle and what follows) runs before any second piece, so
    // a later piece usually finds its rows already dead and is skipped, and
    // no single strip's scan holds the launch open
    const int64_t nitems = REFINE ? nref * 2 * nseg : p.sel_items * int64_t(p.sel_pieces);
    unsigned long long pairs = 0, seeds = 0;

    for (;;) {
        int64_t item = 0;
        if (lane == 0) item = atomicAdd(p.work + (REFINE ? 2 : 0), 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= nitems) break;
        int l;
        int64_t s;
        int64_t kq = 0, piece = 0;
        if (REFINE) {
            const int2 e = p.strips[item % nref];
            l = e.x;
            s = e.y;
            kq = item / nref;
        } else {
            piece = item / p.sel_items;
            const int64_t si = item % p.sel_items;
            l = lane_of(strip_base, p.nl, si);
            s = si - strip_base[l] + p.lanes[l].strip0;
        }
        const Lane& Lg = p.lanes[l];
        const LaneView a{Lg.T, Lg.n, Lg.N, Lg.m, Lg.win};
        const int32_t m = a.m;
        const int64_t N = a.N;
        const int kp = ((m + 31) / 32) * 32;  // top-row seed loop: 32 values of k per step
        const float rho_prune = rho_prune_of(Lg, p.st[l]);
        // [ja, jb): columns of this item; jt: first column right of the
        // exclusion zone of the top row (select's triangle starts there)
        int64_t ja, jb, jt = 0;
        if (REFINE) {
            const int64_t q0 = (s * H + H / 2) / p.seg;
            const int64_t d = (kq + 1) / 2;
            const int64_t q = (kq & 1) ? q0 + d : q0 - d;
            ja = q * p.seg;
            if (q < 0 || ja >= N) continue;
            jb = min64(N, ja + p.seg);
            // a refine shard compares with its own columns only
            ja = max64(ja, Lg.col_lo);
            jb = min64(jb, Lg.col_hi);
            if (ja >= jb) continue;
        } else {
            jt = s * H + m;
            if (jt >= N) continue;  // no window to the right: column marks / refine decide these rows
            const int64_t pc = (jt & ~int64_t(31)) + piece * int64_t(p.sel_cols);
            ja = piece == 0 ? jt : pc;
            jb = min64(min64(N, s * H + H - 1 + m + p.cap), pc + p.sel_cols);
            if (ja >= jb) continue;
        }
        // rows start from directly computed dot products at column ja
        // (refine, and select pieces after the first)
        const bool seeded = REFINE || piece > 0;
        // tensor-core seed row of a refine strip, if it has one
        const float* tcs = nullptr;
        if (REFINE && p.tc_seeds) {
            const int32_t loc = p.strip_row[item % nref];
            const LaneState& S = p.st[l];
            if (loc >= 0 && loc < S.seed_eff) tcs = p.seeds + (int64_t(S.seed_base) + loc) * p.seed_stride;
        }
        uint32_t* bits = Lg.bits;
        const int32_t* slot_of = Lg.slot_of;
        const int64_t i0 = s * H;
        const int64_t r0 = i0 + int64_t(lane) * D;

        // Rows of this lane.
        float df_r[D], dg_r[D], inv_r[D], thr_r[D], cov[D], rmax[D];
        int32_t slot[D];
        int32_t kc[D];  // KNN: pairs of this chunk past the threshold, per row
#pragma unroll
        for (int d = 0; d < D; ++d) kc[d] = 0;
        uint32_t alive = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int64_t i = r0 + d;
            float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < N) rec = a.win[i];
            df_r[d] = rec.x;
            dg_r[d] = rec.y;
            inv_r[d] = rec.z;
            thr_r[d] = (i >= N) ? kInf : (rec.z > 0.f ? rho_prune / rec.z : (rho_prune < 0.f ? -kInf : kInf));
            cov[d] = 0.f;
            rmax[d] = -kInf;
            slot[d] = -1;
            if (REFINE && i < N) {
                slot[d] = slot_of[i];
                if (slot[d] >= 0 && !__ldcg(&p.dead[slot[d]])) alive |= 1u << d;
            }
        }
        const int64_t wrd = r0 >> 5;
        const int sh = int(r0 & 31);
        const uint32_t dmask = (D == 32) ? kFull : ((1u << D) - 1u);
        if (!REFINE) alive = (r0 < N) ? ((__ldcg(&bits[wrd]) >> sh) & dmask) : 0u;
        if (!__any_sync(kFull, alive)) continue;

        const int64_t cfirst = ja & ~int64_t(31);
        issue_chunk(a, sm, kps, 0, cfirst, kp, lane, tcs);

        // Centred top-row window and its sum (FP32; the sum absorbs the
        // rounding of mu so the seed correction is exact to rounding).
        float suma = 0.f;
        if (!tcs) {
            const float mu_top = a.win[i0].w;
            float part = 0.f;
            for (int k = lane; k < kp; k += 32) {
                const float v = (k < m) ? (a.T[i0 + k] - mu_top) : 0.f;
                sm.ahat[k] = v;
                part += v;
            }
            suma = warp_sum(part);
        }
        __syncwarp();

        float tmax[D];
#pragma unroll
        for (int d = 0; d < D; ++d) tmax[d] = -kInf;
        if (seeded) {
            first_col_seeds<D>(a, r0, ja, cov);
            seeds += H;
        }
        const int64_t rows = min64(H, N - i0);

        int buf = 0;
        for (int64_t c0 = cfirst; c0 < jb; c0 += 32, buf ^= 1) {
            cp_async_wait_all();
            __syncwarp();
            if (c0 + 32 < jb) issue_chunk(a, sm, kps, buf ^ 1, c0 + 32, kp, lane, tcs);
            // state other warps may have changed, read early and used at the chunk end
            uint32_t gbits = 0, gdead = 0;
            if (!REFINE && r0 < N) gbits = __ldcg(&bits[wrd]);
            if (REFINE) {
#pragma unroll
                for (int d = 0; d < D; ++d)
                    if (((alive >> d) & 1u) && __ldcg(&p.dead[slot[d]])) gdead |= 1u << d;
            }
            const float* seedv = tcs ? sm.tcseed + buf * 32 : sm.seed;
            if (!tcs) chunk_seeds(a, sm, kps, buf, c0, suma, kp, lane);
            const float4* crb = sm.colrec + buf * 32;
            const int steps = int(min64(32, jb - c0));
            const int st0 = int(max64(0, ja - c0));
            bool masked;
            if (REFINE) masked = !(c0 >= i0 + H - 1 + m || c0 + 31 <= i0 - m);
            else masked = (c0 - jt) < int64_t(H - 1);
            uint32_t colmask = 0;
            // One column: every row advances along its diagonal (Eq. 9), and
            // x[d] = cov * inv_j is rho up to the row factor.
            auto advance = [&](int st, bool first_col, float (&x)[D]) {
                const float4 cr = crb[st];
                const float sd = seedv[st];
                const float up = __shfl_up_sync(kFull, cov[D - 1], 1);
                if (!first_col) {
#pragma unroll
                    for (int d = D - 1; d >= 1; --d) cov[d] = fmaf(df_r[d], cr.y, fmaf(cr.x, dg_r[d], cov[d - 1]));
                    cov[0] = (lane == 0) ? sd : fmaf(df_r[0], cr.y, fmaf(cr.x, dg_r[0], up));
                }
#pragma unroll
                for (int d = 0; d < D; ++d) x[d] = cov[d] * cr.z;
            };
            // One column step: x feeds the row maxima and, in select, the
            // column mark (pairs inside the exclusion zone masked out).
            auto step = [&](int st, bool first_col, bool mask) {
                float x[D];
                advance(st, first_col, x);
                bool pred = false;
                const int64_t lim = c0 + st - r0;  // j - i for d = 0
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    if (mask) {
                        const int64_t dj = lim - d;  // j - i
                        const bool ok = REFINE ? (dj >= m || dj <= -int64_t(m)) : (dj >= m);
                        x[d] = ok ? x[d] : -kInf;
                    }
                    rmax[d] = fmaxf(rmax[d], x[d]);
                    if (!REFINE) pred |= x[d] > thr_r[d];
                    if (KNN) kc[d] += x[d] > thr_r[d] ? 1 : 0;
                }
                if (!REFINE && pred) colmask |= 1u << st;
            };
            if (!masked && st0 == 0 && steps == 32 && !(seeded && c0 == ja)) {
                // full unmasked chunk, unrolled so loads and FMAs of
                // consecutive steps interleave; two columns per iteration
                // enter the row maxima through one three-input max
#pragma unroll
                for (int st = 0; st < 32; st += 2) {
                    float x0[D], x1[D];
                    advance(st, false, x0);
                    advance(st + 1, false, x1);
                    bool p0 = false, p1 = false;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        rmax[d] = fmax3(rmax[d], x0[d], x1[d]);
                        if (KNN) kc[d] += (x0[d] > thr_r[d] ? 1 : 0) + (x1[d] > thr_r[d] ? 1 : 0);
                        if (!REFINE) {
                            p0 |= x0[d] > thr_r[d];
                            p1 |= x1[d] > thr_r[d];
                        }
                    }
                    if (!REFINE) colmask |= (p0 ? 1u << st : 0u) | (p1 ? 2u << st : 0u);
                }
            } else {
                for (int st = st0; st < steps; ++st) step(st, seeded && c0 + st == ja, masked);
            }
            if (lane == 0) {
                if (!tcs) seeds += 32;
                if (REFINE) pairs += uint64_t(rows) * uint64_t(steps - st0);
                else
                    for (int st = st0; st < steps; ++st) {
                        const int64_t v = min64(rows, c0 + st - jt + 1);
                        if (v > 0) pairs += uint64_t(v);
                    }
            }
            if (!REFINE) {
                // Neighbour (column) marks, row deaths, rows killed elsewhere.
                // Columns and rows pruned here record where (witness hints for
                // the next lengths: the strip's middle row, the chunk's middle
                // column).
                const uint32_t cw = __reduce_or_sync(kFull, colmask);
                if (cw) {
                    uint32_t was = 0;
                    if (lane == 0) was = atomicAnd(&bits[c0 >> 5], ~cw);
                    if (Lg.hint) {
                        was = __shfl_sync(kFull, was, 0);
                        if (((cw & was) >> lane) & 1u) Lg.hint[c0 + lane] = int32_t(i0 + H / 2);
                    }
                }
                uint32_t newdead = 0;
#pragma unroll
                for (int d = 0; d < D; ++d)
                    if (((alive >> d) & 1u) && rmax[d] > thr_r[d]) newdead |= 1u << d;
                if (newdead) {
                    alive &= ~newdead;
                    atomicAnd(&bits[wrd], ~(newdead << sh));
                    if (Lg.hint)
#pragma unroll
                        for (int d = 0; d < D; ++d)
                            if ((newdead >> d) & 1u) Lg.hint[r0 + d] = int32_t(c0 + 16);
                }
                if (r0 < N) alive &= (gbits >> sh) & dmask;
                if (!__any_sync(kFull, alive)) break;
            } else {
                // Per-survivor chunk maximum and deaths.
                const int32_t t = int32_t(c0 >> 5);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    if (slot[d] >= 0) {
                        const float rho = rmax[d] > -kInf ? rmax[d] * inv_r[d] : -kInf;
                        p.cmax[int64_t(slot[d]) * p.nchunks_max + t] = rho;
                        tmax[d] = fmaxf(tmax[d], rho);
                        const bool die = KNN ? (kc[d] > 0 && atomicAdd(&p.kcnt[slot[d]], kc[d]) + kc[d] >= p.knn)
                                             : rmax[d] > thr_r[d];
                        if (die) {
                            p.dead[slot[d]] = 1;
                            alive &= ~(1u << d);
                            if (Lg.hint) Lg.hint[r0 + d] = int32_t(c0 + 16);
                        }
                    }
                    rmax[d] = -kInf;
                    if (KNN) kc[d] = 0;
                }
                alive &= ~gdead;
                if (!__any_sync(kFull, alive)) break;
            }
            __syncwarp();
        }
        cp_async_wait_all();  // no copy may land in a buffer the next item reuses
        __syncwarp();
        if (REFINE) {
            // the segment is one coarse block: its maximum is this row's tmax
            const int64_t qb = ja / p.seg;
#pragma unroll
            for (int d = 0; d < D; ++d)
                if (slot[d] >= 0) {
                    p.cmax2[int64_t(slot[d]) * p.ncoarse_max + qb] = enc_f32(tmax[d]);
                    if (tmax[d] > -kInf) atomicMax(&p.gmax[slot[d]], enc_f32(tmax[d]));
                }
        }
    }
    if (lane == 0 && pairs) atomicAdd(p.pairs + (REFINE ? 4 : 0), pairs);
    if (lane == 0 && seeds) atomicAdd(p.pairs + (REFINE ? 5 : 3), seeds);
}

size_t sweep_smem(const Pass& p) {
    const size_t kp = ((p.kpad_max + 127) / 128) * 128;
    return sizeof(float) * (kp + 2 * (kp + 32) + 2 * 128 + 32 + 64) * kWarpsPerCta + sizeof(int64_t) * size_t(p.nl);
}

template <bool REFINE, int D, bool KNN = false>
cudaError_t launch_sweep_impl(const Pass& p, int grid, cudaStream_t s) {
    const size_t sm = sweep_smem(p);
    if (sm > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k_sweep<D, REFINE, KNN>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
    }
    k_sweep<D, REFINE, KNN><<<grid, kWarpsPerCta * 32, sm, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_select(const Pass& p, int grid, cudaStream_t s) {
    return launch_sweep_impl<false, kStripH / 32>(p, grid, s);
}

cudaError_t launch_refine_sweep(const Pass& p, int grid, cudaStream_t s) {
    if (p.knn > 1) return launch_sweep_impl<true, kRefineH / 32, true>(p, grid, s);  // 128-row strips
    if (p.refine_h == kRefineHTall) return launch_sweep_impl<true, kRefineHTall / 32>(p, grid * 3 / 4, s);
    return launch_sweep_impl<true, kRefineH / 32>(p, grid, s);
}

}  // namespace palmad
