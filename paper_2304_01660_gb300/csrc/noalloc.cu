// palmad_topk_profile_noalloc: greedy top-K range discords of a given
// nearest-neighbour profile, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another
// component owns the whole device memory through its own allocator, or a
// latency-critical path that must not pay cudaMalloc's implicit device
// synchronisation.  This entry point allocates nothing.  The caller passes
// the profile and the output arrays; the one intermediate buffer -- the
// compacted list of range discords the top-K rounds scan -- lives in the
// file-scope array g_scratch below, whose size caps the profile length at
// PALMAD_NOALLOC_MAX_WINDOWS windows (3 MiB per device; the array stays
// resident on every GPU that loads the library until the process exits).
//
// Host code cannot use g_scratch's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and caches it; make that first call before any
// stream capture.  Every call on a device shares the one array and leaves
// its contents behind: nothing in it needs to start at zero (the kernel
// writes every entry it reads), but two calls whose kernels overlap on the
// GPU (different streams, no ordering between them) race on it.
#include <mutex>

#include "palmad.h"
#include "palmad_dev.cuh"

namespace palmad {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int64_t kMaxWindows = PALMAD_NOALLOC_MAX_WINDOWS;
constexpr int kMaxDevices = 64;

// [0, 8*max): FP64 distances of the compacted list; then its int32 indices.
__device__ __align__(256) unsigned char g_scratch[kMaxWindows * (sizeof(double) + sizeof(int32_t))];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

__device__ __forceinline__ bool better(double nn, int32_t idx, double bnn, int32_t bidx) {
    return nn > bnn || (nn == bnn && idx < bidx);
}

// One CTA: compaction of the range discords (finite distance >= r; every
// finite entry when r <= 0) into the scratch list in ascending index order,
// then greedy top-K (largest distance first, ties to the lower index,
// optionally >= m apart) over the list.
__global__ void __launch_bounds__(1024) k_topk_profile(const double* __restrict__ prof, int64_t N, int32_t m,
                                                        double r, int32_t K, int32_t exclusive, double* snn,
                                                        int32_t* sidx, int64_t* out_idx, double* out_nn,
                                                        int64_t* out_count) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t total_s;
    __shared__ int32_t picks[kMaxK];
    __shared__ double wbest_nn[32];
    __shared__ int32_t wbest_idx[32];
    __shared__ int32_t wbest_pos[32];
    __shared__ int done_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    auto keep = [&](int64_t i) -> bool {
        const double v = prof[i];
        return isfinite(v) && (r <= 0.0 || v >= r);
    };
    const int64_t per = (N + blockDim.x - 1) / blockDim.x;
    const int64_t i0 = tid * per, i1 = min64(N, i0 + per);
    int32_t cnt = 0;
    for (int64_t i = i0; i < i1; ++i) cnt += keep(i);
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
        if (lane == 31) total_s = s;
    }
    __syncthreads();
    int32_t off = warp_tot[wid] + incl - cnt;
    for (int64_t i = i0; i < i1; ++i) {
        if (!keep(i)) continue;
        sidx[off] = int32_t(i);
        snn[off] = prof[i];
        ++off;
    }
    __syncthreads();
    const int32_t count = total_s;
    int got = 0;
    for (int round = 0; round < K; ++round) {
        double bnn = -1.0;
        int32_t bidx = 0x7fffffff, bpos = -1;
        for (int32_t q = tid; q < count; q += blockDim.x) {
            const int32_t idx = sidx[q];
            const double nn = snn[q];
            if (!better(nn, idx, bnn, bidx)) continue;
            bool ok = true;
            for (int p = 0; p < got && ok; ++p) {
                const int32_t d = idx - picks[p];
                ok = exclusive ? (d >= m || d <= -m) : (d != 0);
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
                out_idx[got] = idx;
                out_nn[got] = nn;
            }
        }
        __syncthreads();
        if (done_s) break;
        ++got;
    }
    for (int q = got + tid; q < K; q += blockDim.x) {
        out_idx[q] = -1;
        out_nn[q] = 0.0;
    }
    if (tid == 0 && out_count) *out_count = count;
}

// Device address of g_scratch on the current device (looked up once).
palmad_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PALMAD_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return PALMAD_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PALMAD_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PALMAD_OK;
}

}  // namespace

}  // namespace palmad

extern "C" palmad_status palmad_topk_profile_noalloc(const double* nn_dev, int64_t N, int32_t m, double r,
                                                     int32_t K, int32_t exclusive, int64_t* out_idx_dev,
                                                     double* out_nn_dev, int64_t* out_count_dev,
                                                     void* cuda_stream) {
    using namespace palmad;
    if (!nn_dev || !out_idx_dev || !out_nn_dev || N < 1 || m < 1 || K < 1 || K > kMaxK || !(r == r))
        return PALMAD_ERR_ARG;
    if (N > kMaxWindows) return PALMAD_ERR_TOO_LARGE;
    void* base = nullptr;
    const palmad_status st = scratch_address(&base);
    if (st != PALMAD_OK) return st;
    double* snn = static_cast<double*>(base);
    int32_t* sidx = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(base) + kMaxWindows * sizeof(double));
    k_topk_profile<<<1, 1024, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        nn_dev, N, m, r, K, exclusive ? 1 : 0, snn, sidx, out_idx_dev, out_nn_dev, out_count_dev);
    if (cudaGetLastError() != cudaSuccess) return PALMAD_ERR_CUDA;
    return PALMAD_OK;
}
