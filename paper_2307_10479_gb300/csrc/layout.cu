// Locality layout of an uploaded index (not part of the paper's method; a device-memory layout).
//
// Vertices get new internal ids so that vectors near each other in space get nearby ids: P
// pivot rows (every (n/P)-th vertex) are chosen, every vertex is labelled with its nearest
// pivot (float32 L2, ties -> lower pivot index), and vertices are ordered by (label, original
// id) with a deterministic counting sort. Rows and the adjacency are then stored in that order.
// A query's visited bitmap words, its rows and its adjacency rows then cluster in a few address
// ranges, which keeps them in L2. The adjacency stays indexed by caller id and holds, for every
// neighbour, its internal id (to read its row and mark it visited) beside its caller id (the id in
// the search keys, so distance ties are broken by caller id exactly as Alg. 1 over the caller's
// numbering breaks them). The layout is invisible to callers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>
#include <string>

#include "deg_internal.h"

namespace deg {
namespace {

constexpr int kTile = 64, kKc = 32, kChunk = 1024;

// labels[v] = argmin_p |r_v - x_{pivot p}|^2 (ties -> lower p) for rows r_v = rows[v * rstride..]
// and pivot rows x[pivots[p] * dim_pad..]; d2[v] = that minimum (if d2 is given). 64 rows x 64
// pivots per tile.
__global__ void __launch_bounds__(256) nearest_pivot_kernel(const float* __restrict__ rows, int64_t rstride,
                                                            const float* __restrict__ x, int64_t n, int32_t dim,
                                                            int32_t dim_pad, const int32_t* __restrict__ pivots,
                                                            int32_t np, int32_t* __restrict__ labels,
                                                            float* __restrict__ d2) {
    __shared__ float xs[kKc][kTile + 4];
    __shared__ float ps[kKc][kTile + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * kTile;
    unsigned long long best[4] = {~0ull, ~0ull, ~0ull, ~0ull};
    for (int p0 = 0; p0 < np; p0 += kTile) {
        float acc[4][4] = {};
        for (int k0 = 0; k0 < dim; k0 += kKc) {
            for (int t = threadIdx.x; t < kTile * kKc; t += 256) {
                const int r = t / kKc, c = t % kKc;
                const bool kc = k0 + c < dim;
                xs[c][r] = (kc && r0 + r < n) ? rows[(r0 + r) * rstride + k0 + c] : 0.f;
                ps[c][r] = (kc && p0 + r < np) ? x[(int64_t)pivots[p0 + r] * dim_pad + k0 + c] : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int c = 0; c < kKc; ++c) {
                float a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = xs[c][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = ps[c][tx + 16 * j];
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
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = p0 + tx + 16 * j;
                if (p < np) best[i] = min(best[i], ((unsigned long long)__float_as_uint(acc[i][j]) << 32) | (uint32_t)p);
            }
    }
    // reduce over the 16 threads sharing a row (same ty, lanes differ in tx)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned long long v = best[i];
#pragma unroll
        for (int m = 8; m; m >>= 1) {
            const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
            const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
            v = min(v, ((unsigned long long)hi << 32) | lo);
        }
        const int64_t r = r0 + ty + 16 * i;
        if (tx == 0 && r < n) {
            labels[r] = (int32_t)(uint32_t)v;
            if (d2) d2[r] = __uint_as_float((uint32_t)(v >> 32));
        }
    }
}

// Per chunk of kChunk vertices: how many carry each label.
__global__ void chunk_hist_kernel(const int32_t* labels, int64_t n, int32_t np, int32_t* chunk_hist) {
    extern __shared__ int32_t h[];
    for (int i = threadIdx.x; i < np; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t lo = (int64_t)blockIdx.x * kChunk, hi = lo + kChunk < n ? lo + kChunk : n;
    for (int64_t v = lo + threadIdx.x; v < hi; v += blockDim.x) atomicAdd(h + labels[v], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += blockDim.x) chunk_hist[(int64_t)blockIdx.x * np + i] = h[i];
}

// For each label: totals, and the running count before each chunk (in place).
__global__ void label_scan_kernel(int32_t* chunk_hist, int64_t nchunks, int32_t np, int32_t* totals) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= np) return;
    int32_t run = 0;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int32_t t = chunk_hist[c * np + l];
        chunk_hist[c * np + l] = run;
        run += t;
    }
    totals[l] = run;
}

// Exclusive scan of the label totals (one block).
__global__ void offsets_kernel(const int32_t* totals, int32_t np, int32_t* offsets) {
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int l = 0; l < np; ++l) {
            offsets[l] = run;
            run += totals[l];
        }
    }
}

// New id of every vertex: label offset + earlier chunks' count + rank inside the chunk.
__global__ void scatter_ids_kernel(const int32_t* labels, int64_t n, int32_t np, const int32_t* chunk_before,
                                   const int32_t* offsets, int32_t* old2new, int32_t* new2old) {
    __shared__ int32_t lab[kChunk];
    const int64_t lo = (int64_t)blockIdx.x * kChunk, hi = lo + kChunk < n ? lo + kChunk : n;
    const int cnt = (int)(hi - lo);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) lab[i] = labels[lo + i];
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int32_t l = lab[i];
        int rank = 0;
        for (int u = 0; u < i; ++u) rank += (lab[u] == l);
        const int32_t pos = offsets[l] + chunk_before[(int64_t)blockIdx.x * np + l] + rank;
        old2new[lo + i] = pos;
        new2old[pos] = (int32_t)(lo + i);
    }
}

__global__ void permute_rows_kernel(const float4* src, float4* dst, int64_t n, int32_t row4, const int32_t* new2old) {
    const int64_t total = n * row4;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / row4;
        const int c = (int)(t - p * row4);
        dst[t] = src[(int64_t)new2old[p] * row4 + c];
    }
}

// dst[v][j] = {internal id, caller id} of neighbour j of caller vertex v ({-1, -1} in padding).
__global__ void pair_adj_kernel(const int32_t* src, int2* dst, int64_t n, int32_t deg_pad, int32_t degree,
                                const int32_t* old2new) {
    const int64_t total = n * deg_pad;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % deg_pad);
        const int32_t v = j < degree ? src[t] : -1;
        dst[t] = v >= 0 ? make_int2(old2new[v], v) : make_int2(-1, -1);
    }
}

__global__ void pivot_ids_kernel(int32_t* pivots, int32_t np, int64_t stride) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) pivots[p] = (int32_t)(p * stride);
}

__global__ void map_ids_kernel(const int32_t* in, int32_t count, const int32_t* table, int32_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = in[i] >= 0 ? table[in[i]] : -1;     // -1: routing failed (the search reports it)
}

// Pivot ids for routed queries, and their work order: queries farther than tau from their pivot
// (they take the most hops; starting them first keeps them off the end of the batch) from the
// front, the others from the back. cursors[0..1] start at zero.
__global__ void route_ids_kernel(const int32_t* __restrict__ labels, const float* __restrict__ dists, int32_t count,
                                 const int32_t* __restrict__ table, float tau, int32_t* __restrict__ seeds,
                                 int32_t* __restrict__ order, int32_t* __restrict__ cursors) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    seeds[i] = labels[i] >= 0 ? table[labels[i]] : -1;
    if (!(dists[i] <= tau)) order[atomicAdd(cursors, 1)] = i;          // far, or a failed route
    else order[count - 1 - atomicAdd(cursors + 1, 1)] = i;
}

}  // namespace

int apply_locality_layout(DeviceIndex& ix, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = ix.n;
    const int32_t np = (int32_t)std::max<int64_t>(1, std::min<int64_t>(4096, n / 256));
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    int32_t *pivots = nullptr, *labels = nullptr, *chunk_hist = nullptr, *totals = nullptr, *offsets = nullptr;
    float *x2 = nullptr, *d2 = nullptr;
    int32_t* adj2 = nullptr;
    cudaError_t e;
    auto cleanup = [&]() {
        cudaFree(pivots); cudaFree(labels); cudaFree(chunk_hist); cudaFree(totals); cudaFree(offsets);
        cudaFree(x2); cudaFree(adj2); cudaFree(d2);
    };
    if ((e = cudaMalloc(&pivots, 4 * np)) != cudaSuccess || (e = cudaMalloc(&labels, 4 * n)) != cudaSuccess ||
        (e = cudaMalloc(&chunk_hist, 4 * nchunks * np)) != cudaSuccess || (e = cudaMalloc(&totals, 4 * np)) != cudaSuccess ||
        (e = cudaMalloc(&offsets, 4 * np)) != cudaSuccess || (e = cudaMalloc(&ix.old2new, 4 * n)) != cudaSuccess ||
        (e = cudaMalloc(&ix.new2old, 4 * n)) != cudaSuccess ||
        (e = cudaMalloc(&x2, sizeof(float) * n * ix.dim_pad)) != cudaSuccess ||
        (e = cudaMalloc(&adj2, sizeof(int2) * n * ix.deg_pad)) != cudaSuccess ||
        (e = cudaMalloc(&d2, sizeof(float) * n)) != cudaSuccess) {
        cleanup();
        return *why = std::string("layout buffers: ") + cudaGetErrorString(e), (int)e;
    }
    pivot_ids_kernel<<<(np + 255) / 256, 256, 0, st>>>(pivots, np, n / np);
    nearest_pivot_kernel<<<(unsigned)((n + kTile - 1) / kTile), 256, 0, st>>>(ix.x32, ix.dim_pad, ix.x32, n, ix.dim,
                                                                              ix.dim_pad, pivots, np, labels, d2);
    chunk_hist_kernel<<<(unsigned)nchunks, 256, 4 * np, st>>>(labels, n, np, chunk_hist);
    label_scan_kernel<<<(np + 127) / 128, 128, 0, st>>>(chunk_hist, nchunks, np, totals);
    offsets_kernel<<<1, 32, 0, st>>>(totals, np, offsets);
    scatter_ids_kernel<<<(unsigned)nchunks, 256, 0, st>>>(labels, n, np, chunk_hist, offsets, ix.old2new, ix.new2old);
    permute_rows_kernel<<<4096, 256, 0, st>>>(reinterpret_cast<const float4*>(ix.x32), reinterpret_cast<float4*>(x2), n,
                                              ix.dim_pad / 4, ix.new2old);
    pair_adj_kernel<<<4096, 256, 0, st>>>(ix.adj, reinterpret_cast<int2*>(adj2), n, ix.deg_pad, ix.degree, ix.old2new);
    if ((e = cudaGetLastError()) == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return *why = std::string("layout kernels: ") + cudaGetErrorString(e), (int)e;
    }
    std::swap(ix.x32, x2);
    std::swap(ix.adj, adj2);
    {
        // routed batches start with the queries farther from their pivot than 31/32 of the rows are
        std::vector<float> h((size_t)n);
        if ((e = cudaMemcpy(h.data(), d2, sizeof(float) * n, cudaMemcpyDeviceToHost)) != cudaSuccess) {
            cleanup();
            return *why = cudaGetErrorString(e), (int)e;
        }
        const size_t r = (size_t)std::min<int64_t>(n - 1, n - std::max<int64_t>(1, n / 32));
        std::nth_element(h.begin(), h.begin() + r, h.end());
        ix.far_tau = std::sqrt(std::max(h[r], 0.f));
    }
    // keep the pivots, as internal ids, for routing queries to an entry vertex
    if ((e = cudaMalloc(&ix.pivots, 4 * np)) != cudaSuccess) {
        cleanup();
        return *why = cudaGetErrorString(e), (int)e;
    }
    map_ids_kernel<<<(np + 255) / 256, 256, 0, st>>>(pivots, np, ix.old2new, ix.pivots);
    ix.npivots = np;
    // routing searches the pivots' rows (now in internal order) for each query's nearest
    knn_plan_destroy(ix.route_plan);
    ix.route_plan = nullptr;
    if (const int r = knn_plan_create(&ix.route_plan, ix.x32, ix.dim_pad, ix.pivots, np, ix.dim, 1, 256, stream, why)) {
        cleanup();
        return r;
    }
    int32_t entry_new = -1;
    if ((e = cudaMemcpy(&entry_new, ix.old2new + ix.entry, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) {
        cleanup();
        return *why = cudaGetErrorString(e), (int)e;
    }
    ix.entry_internal = entry_new;
    cleanup();  // frees the old rows and adjacency (swapped into x2 / adj2) and the scratch
    return 0;
}

}  // namespace deg

namespace deg {

int route_to_pivots(const DeviceIndex& ix, const float* queries, int64_t nq, int32_t* labels, int32_t* seeds,
                    float* dists, int32_t* order, int32_t* cursors, bool learned, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    KnnPlan* plan = learned ? ix.lroute_plan : ix.route_plan;
    const int32_t* pivots = learned ? ix.lpivots : ix.pivots;
    const float tau = learned ? ix.lfar_tau : ix.far_tau;
    if (!plan) return *why = learned ? "no learned entry points (deg_train_entry)" : "no routing plan (upload the index first)",
                      (int)cudaErrorInvalidValue;
    if (nq <= 0) return 0;
    // exact float32 nearest pivot (ties to the lower pivot index), tensor-core filtered
    if (const int r = knn_plan_run(plan, queries, nq, labels, dists, stream, why)) return r;
    if (order) {
        cudaMemsetAsync(cursors, 0, 2 * sizeof(int32_t), st);
        route_ids_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(labels, dists, (int32_t)nq, pivots, tau, seeds,
                                                                     order, cursors);
    } else {
        map_ids_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(labels, (int32_t)nq, pivots, seeds);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

}  // namespace deg

// ---- learned entry points (not in the paper) --------------------------------------------------
// The pivot routing starts each query at the pivot nearest to it. Here a second set of pivots is
// learned from the data instead of sampled: K centroids trained by Lloyd's algorithm (k-means:
// assign every row to its nearest centroid, move every centroid to the mean of its rows, repeat),
// each replaced by the base vertex nearest to it. With entry_mode 2 a query starts at the nearest
// of those vertices, found exactly as with the sampled pivots (entry_mode 1).
namespace deg {
namespace {

// sums[label][c] += row[c], counts[label] += 1 (one warp per row)
__global__ void centroid_sums_kernel(const float* __restrict__ x, int64_t n, int32_t dim, int32_t dim_pad,
                                     const int32_t* __restrict__ labels, float* __restrict__ sums, int32_t* __restrict__ counts) {
    const int lane = threadIdx.x & 31;
    for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
         v += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int32_t l = labels[v];
        for (int c = lane; c < dim; c += 32) atomicAdd(sums + (int64_t)l * dim_pad + c, x[v * dim_pad + c]);
        if (lane == 0) atomicAdd(counts + l, 1);
    }
}

// centroid = sums / count; an empty cluster keeps its centroid
__global__ void centroid_update_kernel(float* __restrict__ cent, const float* __restrict__ sums,
                                       const int32_t* __restrict__ counts, int32_t k, int32_t dim, int32_t dim_pad) {
    const int64_t total = (int64_t)k * dim;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / dim;
        const int d = (int)(i - c * dim);
        if (counts[c] > 0) cent[c * dim_pad + d] = sums[c * dim_pad + d] / (float)counts[c];
    }
}

// contiguous [k][dim] copy of [k][dim_pad] rows (the k-NN calls take row-major rows dim floats apart)
__global__ void compact_rows_kernel(const float* __restrict__ in, int32_t k, int32_t dim, int32_t dim_pad, float* __restrict__ out) {
    const int64_t total = (int64_t)k * dim;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[(i / dim) * dim_pad + i % dim];
}

}  // namespace

int train_entry_points(DeviceIndex& ix, int32_t k, int32_t iters, deg_stream_t stream, int64_t* sizes_out,
                       std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = ix.n;
    if (k < 1 || k > 4096 || k > n) return *why = "k must be in 1 ... min(4096, n)", (int)cudaErrorInvalidValue;
    if (ix.dim % 4 != 0) return *why = "learned entry points need a dimension divisible by 4", (int)cudaErrorInvalidValue;
    float *cent = nullptr, *sums = nullptr, *d2 = nullptr, *cdist = nullptr, *cflat = nullptr;
    int32_t *labels = nullptr, *counts = nullptr, *iota = nullptr, *med = nullptr;
    auto cleanup = [&]() {
        cudaFree(cent); cudaFree(sums); cudaFree(d2); cudaFree(cdist); cudaFree(cflat);
        cudaFree(labels); cudaFree(counts); cudaFree(iota); cudaFree(med);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&cent, sizeof(float) * k * ix.dim_pad)) != cudaSuccess ||
        (e = cudaMalloc(&sums, sizeof(float) * k * ix.dim_pad)) != cudaSuccess ||
        (e = cudaMalloc(&cflat, sizeof(float) * k * ix.dim)) != cudaSuccess ||
        (e = cudaMalloc(&d2, sizeof(float) * n)) != cudaSuccess || (e = cudaMalloc(&cdist, sizeof(float) * k)) != cudaSuccess ||
        (e = cudaMalloc(&labels, sizeof(int32_t) * n)) != cudaSuccess ||
        (e = cudaMalloc(&counts, sizeof(int32_t) * k)) != cudaSuccess ||
        (e = cudaMalloc(&iota, sizeof(int32_t) * k)) != cudaSuccess || (e = cudaMalloc(&med, sizeof(int32_t) * k)) != cudaSuccess) {
        cleanup();
        return *why = std::string("entry training buffers: ") + cudaGetErrorString(e), (int)e;
    }
    // start: k rows evenly spaced through the (layout-ordered) rows
    pivot_ids_kernel<<<(k + 255) / 256, 256, 0, st>>>(med, k, n / k);
    pivot_ids_kernel<<<(k + 255) / 256, 256, 0, st>>>(iota, k, 1);
    {
        // gather the start rows: cent[c] = x32[med[c]]
        std::vector<int32_t> h(k);
        if ((e = cudaMemcpyAsync(h.data(), med, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            cleanup();
            return *why = cudaGetErrorString(e), (int)e;
        }
        for (int32_t c = 0; c < k && e == cudaSuccess; ++c)
            e = cudaMemcpyAsync(cent + (int64_t)c * ix.dim_pad, ix.x32 + (int64_t)h[c] * ix.dim_pad,
                                sizeof(float) * ix.dim_pad, cudaMemcpyDeviceToDevice, st);
    }
    for (int32_t it = 0; it <= iters && e == cudaSuccess; ++it) {
        nearest_pivot_kernel<<<(unsigned)((n + kTile - 1) / kTile), 256, 0, st>>>(ix.x32, ix.dim_pad, cent, n, ix.dim,
                                                                                  ix.dim_pad, iota, k, labels, d2);
        if (it == iters) break;                           // the last assignment is the final one
        cudaMemsetAsync(sums, 0, sizeof(float) * k * ix.dim_pad, st);
        cudaMemsetAsync(counts, 0, sizeof(int32_t) * k, st);
        centroid_sums_kernel<<<2048, 256, 0, st>>>(ix.x32, n, ix.dim, ix.dim_pad, labels, sums, counts);
        centroid_update_kernel<<<512, 256, 0, st>>>(cent, sums, counts, k, ix.dim, ix.dim_pad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        cleanup();
        return *why = std::string("entry training: ") + cudaGetErrorString(e), (int)e;
    }
    // the vertex nearest to each centroid (exact k-NN over all rows, internal ids)
    compact_rows_kernel<<<256, 256, 0, st>>>(cent, k, ix.dim, ix.dim_pad, cflat);
    if (const int r = launch_knn_exact(ix.x32, n, cflat, k, ix.dim, 1, med, cdist, stream, why)) {
        cleanup();
        return r;
    }
    // routing over the new pivots' rows; the work order's threshold from the rows' centroid distances
    KnnPlan* plan = nullptr;
    if (const int r = knn_plan_create(&plan, ix.x32, ix.dim_pad, med, k, ix.dim, 1, 256, stream, why)) {
        cleanup();
        return r;
    }
    std::vector<float> h((size_t)n);
    std::vector<int32_t> hl(sizes_out ? (size_t)n : 0);
    if ((e = cudaMemcpy(h.data(), d2, sizeof(float) * n, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (sizes_out && (e = cudaMemcpy(hl.data(), labels, sizeof(int32_t) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)) {
        knn_plan_destroy(plan);
        cleanup();
        return *why = cudaGetErrorString(e), (int)e;
    }
    if (sizes_out) {
        for (int32_t c = 0; c < k; ++c) sizes_out[c] = 0;
        for (int64_t v = 0; v < n; ++v) ++sizes_out[hl[v]];
    }
    const size_t r = (size_t)std::min<int64_t>(n - 1, n - std::max<int64_t>(1, n / 32));
    std::nth_element(h.begin(), h.begin() + r, h.end());
    knn_plan_destroy(ix.lroute_plan);
    ix.lroute_plan = plan;
    cudaFree(ix.lpivots);
    ix.lpivots = med;
    med = nullptr;
    ix.lnpivots = k;
    ix.lfar_tau = std::sqrt(std::max(h[r], 0.f));
    cleanup();
    return 0;
}

}  // namespace deg
