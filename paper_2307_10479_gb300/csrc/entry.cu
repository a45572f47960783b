// Fixed entry vertex of the search: the graph's median vertex, which Sec. 5.4 names as the seed.
// Reading: per coordinate take the lower median -- the element of rank floor((n-1)/2) in
// ascending order -- and return the row nearest to that vector (float32 squared distance,
// tie -> lower id). The median is found exactly by an 8-bit-digit radix select on the
// order-preserving integer image of each float, four passes over the rows.
#include <cuda_runtime.h>

#include <string>

#include "deg_internal.h"

namespace deg {
namespace {

__device__ __forceinline__ uint32_t order_key(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_order_key(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

constexpr int kRowsPerBlock = 4096;

// Histogram of digit `pass` (most significant first) of column blockIdx.x, counting only the
// elements whose higher digits equal the prefix selected so far.
__global__ void median_hist_kernel(const float* x, int64_t n, int32_t dim_pad, int pass,
                                   const uint32_t* prefix, uint32_t* hist) {
    __shared__ uint32_t h[256];
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int shift = 24 - 8 * pass;
    const uint32_t want = prefix[j];
    const uint32_t hmask = pass == 0 ? 0u : (0xffffffffu << (shift + 8));
    const int64_t lo = (int64_t)blockIdx.y * kRowsPerBlock;
    const int64_t hi = lo + kRowsPerBlock < n ? lo + kRowsPerBlock : n;
    for (int64_t r = lo + threadIdx.x; r < hi; r += blockDim.x) {
        const uint32_t k = order_key(x[r * dim_pad + j]);
        if ((k & hmask) == (want & hmask)) atomicAdd(&h[(k >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[(int64_t)j * 256 + i], h[i]);
}

// Choose the digit holding the wanted rank; clear the histogram for the next pass.
__global__ void median_select_kernel(int32_t dim, int pass, uint32_t* prefix, uint32_t* rank, uint32_t* hist) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= dim) return;
    uint32_t* h = hist + (int64_t)j * 256;
    uint32_t r = rank[j], acc = 0;
    int d = 0;
    for (; d < 256; ++d) {
        if (acc + h[d] > r) break;
        acc += h[d];
    }
    rank[j] = r - acc;
    prefix[j] |= (uint32_t)d << (24 - 8 * pass);
    for (int i = 0; i < 256; ++i) h[i] = 0;
}

__global__ void median_init_kernel(int32_t dim, uint32_t target, uint32_t* prefix, uint32_t* rank) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < dim) {
        prefix[j] = 0;
        rank[j] = target;
    }
}

// Nearest row to the median vector: one warp per row, packed (d2 bits, id) atomic minimum.
__global__ void nearest_kernel(const float* x, int64_t n, int32_t dim, int32_t dim_pad, const uint32_t* prefix,
                               unsigned long long* best) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nw) {
        float a = 0.f;
        for (int i = lane; i < dim; i += 32) {
            const float t = x[r * dim_pad + i] - from_order_key(prefix[i]);
            a = fmaf(t, t, a);
        }
#pragma unroll
        for (int m = 16; m; m >>= 1) a += __shfl_xor_sync(0xffffffffu, a, m);
        if (lane == 0) atomicMin(best, ((unsigned long long)__float_as_uint(a) << 32) | (uint32_t)r);
    }
}

}  // namespace

int compute_entry_vertex(DeviceIndex& ix, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    uint32_t *prefix = nullptr, *rank = nullptr, *hist = nullptr;
    unsigned long long* best = nullptr;
    const int dim = ix.dim;
    if ((e = cudaMalloc(&prefix, 4 * dim)) != cudaSuccess || (e = cudaMalloc(&rank, 4 * dim)) != cudaSuccess ||
        (e = cudaMalloc(&hist, 4ll * 256 * dim)) != cudaSuccess || (e = cudaMalloc(&best, 8)) != cudaSuccess) {
        cudaFree(prefix); cudaFree(rank); cudaFree(hist); cudaFree(best);
        *why = cudaGetErrorString(e);
        return (int)e;
    }
    const int tb = 128, jb = (dim + tb - 1) / tb;
    if ((e = cudaMemsetAsync(hist, 0, 4ll * 256 * dim, st)) != cudaSuccess || (e = cudaMemsetAsync(best, 0xff, 8, st)) != cudaSuccess) {
        cudaFree(prefix); cudaFree(rank); cudaFree(hist); cudaFree(best);
        *why = cudaGetErrorString(e);
        return (int)e;
    }
    median_init_kernel<<<jb, tb, 0, st>>>(dim, (uint32_t)((ix.n - 1) / 2), prefix, rank);
    const dim3 hg(dim, (unsigned)((ix.n + kRowsPerBlock - 1) / kRowsPerBlock));
    for (int pass = 0; pass < 4; ++pass) {
        median_hist_kernel<<<hg, 256, 0, st>>>(ix.x32, ix.n, ix.dim_pad, pass, prefix, hist);
        median_select_kernel<<<jb, tb, 0, st>>>(dim, pass, prefix, rank, hist);
    }
    nearest_kernel<<<1024, 256, 0, st>>>(ix.x32, ix.n, dim, ix.dim_pad, prefix, best);
    unsigned long long h = ~0ull;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, best, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(prefix); cudaFree(rank); cudaFree(hist); cudaFree(best);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return (int)e;
    }
    ix.entry = (int32_t)(uint32_t)(h & 0xffffffffull);
    return 0;
}

}  // namespace deg
