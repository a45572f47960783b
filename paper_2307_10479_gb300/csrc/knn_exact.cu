// Exact k nearest neighbours (paper Eq. 1) by exhaustive search, in two kernels per chunk of
// queries:
//   1. a tiled distance kernel writes the float32 squared distances D[q][i] = sum_d (q_d - x_id)^2
//      for a chunk of queries against every base row;
//   2. a selection kernel (one block per query) finds the k-th smallest key (d2 bits, id) by an
//      8-bit-digit radix select over the 64-bit key -- exact, ties ordered by id -- gathers the
//      keys not above it and sorts them.
// Squared distances of non-negative floats order like their bit patterns, so the select works
// on the raw bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "deg_internal.h"

namespace deg {
namespace {

constexpr int kTile = 64, kKc = 32;

__global__ void __launch_bounds__(256) dist_tile_kernel(const float* __restrict__ Q, int64_t nq,
                                                        const float* __restrict__ X, int64_t n, int dim,
                                                        float* __restrict__ out) {
    __shared__ float qs[kKc][kTile + 4];
    __shared__ float xs[kKc][kTile + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t q0 = (int64_t)blockIdx.y * kTile, x0 = (int64_t)blockIdx.x * kTile;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < dim; k0 += kKc) {
        for (int t = threadIdx.x; t < kTile * kKc; t += 256) {
            const int r = t / kKc, c = t % kKc;
            const bool kc = k0 + c < dim;
            qs[c][r] = (kc && q0 + r < nq) ? Q[(q0 + r) * dim + k0 + c] : 0.f;
            xs[c][r] = (kc && x0 + r < n) ? X[(x0 + r) * dim + k0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < kKc; ++c) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = qs[c][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = xs[c][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float t = a[i] - b[j];
                    acc[i][j] = fmaf(t, t, acc[i][j]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t q = q0 + ty + 16 * i;
        if (q >= nq) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t x = x0 + tx + 16 * j;
            if (x < n) out[q * n + x] = acc[i][j];
        }
    }
}

constexpr int kSelThreads = 1024;

__global__ void __launch_bounds__(kSelThreads) select_topk_kernel(const float* __restrict__ D, int64_t n, int k,
                                                                 int32_t* ids, float* dists) {
    __shared__ uint32_t hist[256];
    __shared__ unsigned long long keys[1024];              // k <= 1024
    __shared__ uint64_t prefix_s;
    __shared__ uint32_t rank_s;
    __shared__ int count_s;
    const float* d = D + (int64_t)blockIdx.x * n;
    if (threadIdx.x == 0) {
        prefix_s = 0;
        rank_s = (uint32_t)(k - 1);
        count_s = 0;
    }
    for (int pass = 0; pass < 8; ++pass) {
        for (int i = threadIdx.x; i < 256; i += kSelThreads) hist[i] = 0;
        __syncthreads();
        const int shift = 56 - 8 * pass;
        const uint64_t want = prefix_s;
        const uint64_t hmask = pass == 0 ? 0ull : (~0ull << (shift + 8));
        for (int64_t i = threadIdx.x; i < n; i += kSelThreads) {
            const uint64_t key = ((uint64_t)__float_as_uint(d[i]) << 32) | (uint32_t)i;
            if ((key & hmask) == (want & hmask)) atomicAdd(&hist[(key >> shift) & 0xffu], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t acc = 0, r = rank_s;
            int dg = 0;
            for (; dg < 256; ++dg) {
                if (acc + hist[dg] > r) break;
                acc += hist[dg];
            }
            rank_s = r - acc;
            prefix_s = want | ((uint64_t)dg << shift);
        }
        __syncthreads();
    }
    const uint64_t kth = prefix_s;          // the k-th smallest key itself
    for (int64_t i = threadIdx.x; i < n; i += kSelThreads) {
        const uint64_t key = ((uint64_t)__float_as_uint(d[i]) << 32) | (uint32_t)i;
        if (key <= kth) {
            const int p = atomicAdd(&count_s, 1);
            if (p < 1024) keys[p] = key;
        }
    }
    __syncthreads();
    int P = 1;
    while (P < k) P <<= 1;
    for (int i = k + threadIdx.x; i < P; i += kSelThreads) keys[i] = ~0ull;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += kSelThreads) {
                const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = keys[lo], b = keys[hi];
                if ((a > b) == up) { keys[lo] = b; keys[hi] = a; }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < k; i += kSelThreads) {
        ids[(int64_t)blockIdx.x * k + i] = (int32_t)(uint32_t)keys[i];
        dists[(int64_t)blockIdx.x * k + i] = sqrtf(__uint_as_float((uint32_t)(keys[i] >> 32)));
    }
}

// Queries per launch of dist_tile_kernel: its grid.y (one block row per kTile queries) is at most
// 65,535.
constexpr int64_t kMaxChunkQueries = 65535ll * kTile;

}  // namespace

int launch_knn_simt(const float* base, int64_t n, const float* queries, int64_t nq, int32_t dim, int32_t k,
                    int32_t* ids, float* dists, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (k > n) return *why = "k larger than n", (int)cudaErrorInvalidValue;
    // grid.y = ceil(chunk / kTile) must stay within 65,535
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>({nq, (int64_t)(2ll << 30) / (4 * n), kMaxChunkQueries}));
    float* D = nullptr;
    // A plain allocation, released before returning (the call is a one-off: ground truth).
    cudaError_t e = cudaMalloc(&D, sizeof(float) * chunk * n);
    if (e != cudaSuccess) return *why = std::string("distance buffer: ") + cudaGetErrorString(e), (int)e;
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t qc = std::min(chunk, nq - q0);
        const dim3 grid((unsigned)((n + kTile - 1) / kTile), (unsigned)((qc + kTile - 1) / kTile));
        dist_tile_kernel<<<grid, 256, 0, st>>>(queries + q0 * dim, qc, base, n, dim, D);
        select_topk_kernel<<<(unsigned)qc, kSelThreads, 0, st>>>(D, n, k, ids + q0 * k, dists + q0 * k);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(D);
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

}  // namespace deg

// ---- knn_exact_noalloc: the same two kernels on a fixed, statically allocated scratch --------
// For callers that cannot allocate device memory during the call. The distance buffer is a
// file-scope __device__ array (32 MiB), so every GPU that loads the library holds it until the
// process exits. Host code cannot use the array's name as a device address: the first call on a
// device looks the address up with cudaGetSymbolAddress (that device current) and caches it with
// the id of the CUDA context it belongs to. A later call in another context of that device (after
// cudaDeviceReset, say, which unloads the module and frees the array) looks it up again instead
// of handing the kernels a freed address.
#include <cuda.h>

#include <mutex>

namespace deg {
namespace {

constexpr int64_t kNoAllocScratchFloats = 8ll << 20;                 // 32 MiB of float32 distances
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoAllocSlot {
    unsigned long long ctx = 0;                                      // id of the context the address is in
    float* ptr = nullptr;
};
NoAllocSlot g_noalloc_slot[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

}  // namespace

// Id of the calling thread's current context (driver entry points found through the runtime, so
// the library does not link the driver library); 0 when there is none.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q1{}, q2{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void**>(&get_current), 12000,
                                             cudaEnableDefault, &q1) != cudaSuccess || q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void**>(&get_id), 12000, cudaEnableDefault,
                                             &q2) != cudaSuccess || q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

int64_t knn_noalloc_capacity() { return kNoAllocScratchFloats; }

int launch_knn_exact_noalloc(const float* base, int64_t n, const float* queries, int64_t nq, int32_t dim,
                             int32_t k, int32_t* ids, float* dists, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (n > kNoAllocScratchFloats)
        return *why = "n exceeds the static scratch (at most 8388608 base rows)", (int)cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    if (dev < 0 || dev >= kMaxDevices) return *why = "device index above 63", (int)cudaErrorInvalidValue;
    float* D = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        NoAllocSlot& slot = g_noalloc_slot[dev];
        const unsigned long long ctx = current_context_id();
        if (!slot.ptr || ctx == 0 || ctx != slot.ctx) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return *why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e), (int)e;
            slot.ptr = static_cast<float*>(p);
            slot.ctx = current_context_id();                 // the lookup made the device's context current
        }
        D = slot.ptr;
    }
    // Every distance a chunk reads is written first by the same chunk: nothing needs clearing.
    // grid.y = ceil(chunk / kTile) stays within 65,535.
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>({nq, kNoAllocScratchFloats / n, kMaxChunkQueries}));
    for (int64_t q0 = 0; q0 < nq; q0 += chunk) {
        const int64_t qc = std::min(chunk, nq - q0);
        const dim3 grid((unsigned)((n + kTile - 1) / kTile), (unsigned)((qc + kTile - 1) / kTile));
        dist_tile_kernel<<<grid, 256, 0, st>>>(queries + q0 * dim, qc, base, n, dim, D);
        select_topk_kernel<<<(unsigned)qc, kSelThreads, 0, st>>>(D, n, k, ids + q0 * k, dists + q0 * k);
        if ((e = cudaGetLastError()) != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    }
    return 0;
}

}  // namespace deg
