// DEG construction on the device: batched ExtendGraph (paper Sec. 5.2, Alg. 3 with scheme C and
// the checkMRNG test of Alg. 2 in a first pass).
//
// The paper inserts one vertex at a time. Here vertices are inserted in batches of B (a small
// fraction of the vertices already in the graph):
//   1. the batch's rows are searched over the current graph with the library's own range-search
//      kernels (Alg. 1; seed vertex 0, k_ext results, eps_ext), all B queries in one launch;
//   2. one warp per new vertex v runs Alg. 3 on those results: walk the candidates b in order,
//      (first pass) keep b only if checkMRNG(v, b) holds with U as N(v), take the longest edge
//      (b, n) of b with n not in U, replace it by (v, b) and (v, n), until |U| = d; a second pass
//      drops the MRNG test.
// Concurrency. Two new vertices of a batch may want to rewire the same old vertex. Every old
// vertex whose row a warp changes (each b and each n) is claimed first for the batch with one
// atomicMax of the batch number on its lock word; a vertex already claimed in this batch is
// skipped (for n: the next longest edge of b is tried). A claimed row is changed only by its
// claimer, so each replacement keeps the graph even-regular, symmetric and connected (b reaches n
// through v). A vertex whose candidates run out before |U| = d undoes its replacements and is
// inserted again in a later batch (fresh search, twice the candidates), as the host builder
// searches again with twice k_ext.
// Differences from the sequential algorithm, by design: the vertices of a batch do not see each
// other during their search (B is at most 1/64 of the graph, so a vertex's neighbours are rarely
// in its own batch), contention can make a vertex take a later candidate or a shorter edge, and
// the result depends on which warp claims a vertex first. The optional optimizeEdge step of
// Alg. 3 is not run here (the paper's construction-only variant, App. G); the device refinement
// of Alg. 5 improves edges afterwards.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "deg_internal.h"

namespace deg {
namespace {

constexpr int kBuildWarps = 4;          // warps per block of the extension kernel
constexpr int kMaxBuildDegree = 128;    // the search kernels read at most 128 neighbours
constexpr int kPerLane = kMaxBuildDegree / 32;

// The graph while it is built: rows in caller order, adjacency as {id, id} pairs (the layout the
// search kernels read, with internal id = caller id), float32 edge weights beside it.
struct BuildGraph {
    const float* x;      // [n][dim_pad]
    int32_t dim_pad;
    int2* adj;           // [n][deg_pad]
    float* w;            // [n][deg_pad]
    int32_t* lock;       // [n] number of the last batch that claimed the vertex
    int32_t degree, deg_pad;
};

// Euclidean distance of rows a and b, warp-cooperative (every lane returns it).
__device__ float row_dist(const float* x, int32_t dim_pad, int32_t a, int32_t b, int lane) {
    const float4* pa = reinterpret_cast<const float4*>(x + (int64_t)a * dim_pad);
    const float4* pb = reinterpret_cast<const float4*>(x + (int64_t)b * dim_pad);
    float s = 0.f;
    for (int i = lane; i < dim_pad / 4; i += 32) {
        const float4 u = __ldg(pa + i), v = __ldg(pb + i);
        float t;
        t = u.x - v.x; s = fmaf(t, t, s);
        t = u.y - v.y; s = fmaf(t, t, s);
        t = u.z - v.z; s = fmaf(t, t, s);
        t = u.w - v.w; s = fmaf(t, t, s);
    }
#pragma unroll
    for (int m = 16; m; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    return sqrtf(s);
}

// The start graph: the complete graph on vertices 0..d (one warp per vertex), weights = distances.
__global__ void complete_graph_kernel(BuildGraph G) {
    const int lane = threadIdx.x & 31;
    const int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u > G.degree) return;
    int slot = 0;
    for (int v = 0; v <= G.degree; ++v) {
        if (v == u) continue;
        const float d = row_dist(G.x, G.dim_pad, u, v, lane);
        if (lane == 0) {
            G.adj[(int64_t)u * G.deg_pad + slot] = make_int2(v, v);
            G.w[(int64_t)u * G.deg_pad + slot] = d;
        }
        ++slot;
    }
}

// Row j-slots of vertex b in registers: slot j = lane + 32 i.
struct RowRegs {
    int32_t id[kPerLane];
    float w[kPerLane];
};

__device__ __forceinline__ void load_row(const BuildGraph& G, int32_t b, int lane, RowRegs& r) {
#pragma unroll
    for (int i = 0; i < kPerLane; ++i) {
        const int j = lane + 32 * i;
        r.id[i] = -1;
        r.w[i] = 0.f;
        if (j < G.degree) {
            r.id[i] = reinterpret_cast<volatile int*>(G.adj + (int64_t)b * G.deg_pad + j)[0];
            r.w[i] = reinterpret_cast<volatile float*>(G.w + (int64_t)b * G.deg_pad)[j];
        }
    }
}

// Index in U[0..nu) of vertex c, or -1 (each lane scans U; U is at most 128 long).
__device__ __forceinline__ int find_in(const int32_t* uid, int nu, int32_t c) {
    for (int k = 0; k < nu; ++k)
        if (uid[k] == c) return k;
    return -1;
}

// Claim vertex c for batch `tag`; returns the previous lock value if the claim succeeded, else -1.
__device__ __forceinline__ int claim(int32_t* lock, int32_t c, int32_t tag) {
    const int old = atomicMax(lock + c, tag);
    return old < tag ? old : -1;
}

__device__ __forceinline__ bool any_in(const int32_t* uid, int nu, int32_t c, int lane) {
    bool f = false;
    for (int k = lane; k < nu; k += 32) f |= uid[k] == c;
    return __any_sync(0xffffffffu, f);
}

__device__ __forceinline__ uint64_t warp_max64(uint64_t v) {
#pragma unroll
    for (int m = 16; m; m >>= 1) {
        const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
        const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
        v = max(v, ((uint64_t)hi << 32) | lo);
    }
    return v;
}

// Slot of vertex c in a row held in registers, or -1 (warp-uniform).
__device__ __forceinline__ int slot_of(const RowRegs& r, int32_t c, int lane) {
    int j = -1;
#pragma unroll
    for (int i = 0; i < kPerLane; ++i)
        if (r.id[i] == c) j = lane + 32 * i;
    const unsigned m = __ballot_sync(0xffffffffu, j >= 0);
    return m ? __shfl_sync(0xffffffffu, j, __ffs(m) - 1) : -1;
}

// Alg. 3 for the batch's vertices, one warp each. s_ids / s_d [nb][ks]: each vertex's range-search
// result (ids, Euclidean distances, ascending, -1 padded). status[t] = 0 inserted, 1 deferred.
__global__ void __launch_bounds__(kBuildWarps * 32) extend_kernel(BuildGraph G, const int32_t* __restrict__ batch,
                                                                  int32_t nb, const int32_t* __restrict__ s_ids,
                                                                  const float* __restrict__ s_d, int32_t ks,
                                                                  int32_t tag, int32_t* __restrict__ status) {
    __shared__ int32_t uid_s[kBuildWarps][kMaxBuildDegree];
    __shared__ float ud_s[kBuildWarps][kMaxBuildDegree];
    __shared__ int4 chg_s[kBuildWarps][kMaxBuildDegree / 2];
    __shared__ float wbn_s[kBuildWarps][kMaxBuildDegree / 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kBuildWarps + warp;
    if (t >= nb) return;
    int32_t* uid = uid_s[warp];
    float* ud = ud_s[warp];
    int4* chg = chg_s[warp];
    float* wbn = wbn_s[warp];
    const int32_t v = batch[t];
    const int d = G.degree;
    int nu = 0, nch = 0;
    for (int pass = 0; pass < 2 && nu < d; ++pass) {
        for (int i = 0; i < ks && nu < d; ++i) {
            const int32_t b = s_ids[(int64_t)t * ks + i];
            if (b < 0) break;
            const float db = s_d[(int64_t)t * ks + i];
            if (any_in(uid, nu, b, lane)) continue;                    // b already in U
            RowRegs r;
            if (pass == 0) {
                // checkMRNG(G, v, b) with N(v) = U: no common neighbour u with
                // delta(v, b) > max(delta(v, u), w(b, u))
                load_row(G, b, lane, r);
                bool bad = false;
#pragma unroll
                for (int k = 0; k < kPerLane; ++k)
                    if (r.id[k] >= 0) {
                        const int at = find_in(uid, nu, r.id[k]);
                        if (at >= 0 && db > fmaxf(ud[at], r.w[k])) bad = true;
                    }
                if (__any_sync(0xffffffffu, bad)) continue;
            }
            int ob = 0;
            if (lane == 0) ob = claim(G.lock, b, tag);
            ob = __shfl_sync(0xffffffffu, ob, 0);
            if (ob < 0) continue;                                       // another vertex of the batch has b
            load_row(G, b, lane, r);                                    // b's row no longer changes
            // n: the longest edge of b to a vertex outside U (ties to the lower id) that this warp
            // can claim
            uint64_t key[kPerLane];
#pragma unroll
            for (int k = 0; k < kPerLane; ++k)
                key[k] = (r.id[k] >= 0 && find_in(uid, nu, r.id[k]) < 0)
                             ? ((uint64_t)__float_as_uint(r.w[k]) << 32) | (uint32_t)(0x7fffffff - r.id[k]) : 0ull;
            int32_t n = -1;
            float wn = 0.f;
            for (;;) {
                uint64_t lb = 0;
#pragma unroll
                for (int k = 0; k < kPerLane; ++k) lb = max(lb, key[k]);
                const uint64_t best = warp_max64(lb);
                if (best == 0) break;
                const int32_t c = 0x7fffffff - (int32_t)(uint32_t)best;
                int got = 0;
                if (lane == 0) got = claim(G.lock, c, tag) >= 0;
                if (__shfl_sync(0xffffffffu, got, 0)) {
                    n = c;
                    wn = __uint_as_float((uint32_t)(best >> 32));
                    break;
                }
#pragma unroll
                for (int k = 0; k < kPerLane; ++k)
                    if (r.id[k] == c) key[k] = 0;
            }
            const int jb = n >= 0 ? slot_of(r, n, lane) : -1;
            int jn = -1;
            if (n >= 0) {
                RowRegs rn;
                load_row(G, n, lane, rn);
                jn = slot_of(rn, b, lane);
            }
            if (n < 0 || jb < 0 || jn < 0) {                            // give b (and n) back
                if (lane == 0) {
                    atomicCAS(G.lock + b, tag, ob);
                }
                continue;
            }
            const float dn = row_dist(G.x, G.dim_pad, v, n, lane);
            if (lane == 0) {
                G.adj[(int64_t)b * G.deg_pad + jb] = make_int2(v, v);
                G.w[(int64_t)b * G.deg_pad + jb] = db;
                G.adj[(int64_t)n * G.deg_pad + jn] = make_int2(v, v);
                G.w[(int64_t)n * G.deg_pad + jn] = dn;
                chg[nch] = make_int4(b, n, jb, jn);
                wbn[nch] = wn;
                uid[nu] = n;
                ud[nu] = dn;
                uid[nu + 1] = b;
                ud[nu + 1] = db;
            }
            ++nch;
            nu += 2;
            __syncwarp();
        }
    }
    if (nu < d) {
        // out of candidates: restore every replaced edge (b, n), newest first; v stays out
        if (lane == 0) {
            for (int c = nch - 1; c >= 0; --c) {
                const int4 e = chg[c];
                G.adj[(int64_t)e.x * G.deg_pad + e.z] = make_int2(e.y, e.y);
                G.w[(int64_t)e.x * G.deg_pad + e.z] = wbn[c];
                G.adj[(int64_t)e.y * G.deg_pad + e.w] = make_int2(e.x, e.x);
                G.w[(int64_t)e.y * G.deg_pad + e.w] = wbn[c];
            }
            status[t] = 1;
        }
        return;
    }
    for (int j = lane; j < d; j += 32) {
        G.adj[(int64_t)v * G.deg_pad + j] = make_int2(uid[j], uid[j]);
        G.w[(int64_t)v * G.deg_pad + j] = ud[j];
    }
    if (lane == 0) status[t] = 0;
}

// Gather the rows of the batch's vertices into contiguous query rows [nb][dim].
__global__ void gather_rows_kernel(const float* __restrict__ x, int32_t dim_pad, int32_t dim,
                                   const int32_t* __restrict__ batch, int32_t nb, float* __restrict__ out) {
    const int64_t total = (int64_t)nb * dim;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / dim;
        const int c = (int)(i - t * dim);
        out[i] = x[(int64_t)batch[t] * dim_pad + c];
    }
}

__global__ void iota_kernel(int32_t* a, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

// adjacency pairs -> [n][degree] int32
__global__ void compact_adj_kernel(const int2* __restrict__ adj, int64_t n, int32_t deg_pad, int32_t degree,
                                   int32_t* __restrict__ out) {
    const int64_t total = n * degree;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / degree;
        out[i] = adj[v * deg_pad + (i - v * degree)].x;
    }
}

}  // namespace

int build_graph_device(const float* x_host, int64_t n, int32_t dim, const deg_build_params& p, int32_t batch_div,
                       int32_t* adj_out, volatile int64_t* progress, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int32_t d = p.degree;
    if (d > kMaxBuildDegree) return *why = "degree above 128", (int)cudaErrorInvalidValue;
    if (p.k_ext > 1024) return *why = "k_ext above 1024", (int)cudaErrorInvalidValue;
    if (batch_div < 1) return *why = "batch_div must be positive", (int)cudaErrorInvalidValue;
    const int32_t dim_pad = (dim + 3) / 4 * 4, deg_pad = (d + 3) / 4 * 4;
    constexpr int64_t kMaxBatch = 8192;
    const int32_t kmax = std::min(1024, 4 * p.k_ext);
    float *x = nullptr, *w = nullptr, *qbuf = nullptr, *sd = nullptr;
    int2* adj = nullptr;
    int32_t *lock = nullptr, *iota = nullptr, *bids = nullptr, *sid = nullptr, *status = nullptr, *out = nullptr;
    Workspace ws;
    cudaError_t e = cudaSuccess;
    int rc = 0;
    auto cleanup = [&]() {
        cudaFree(x); cudaFree(w); cudaFree(qbuf); cudaFree(sd); cudaFree(adj); cudaFree(lock); cudaFree(iota);
        cudaFree(bids); cudaFree(sid); cudaFree(status); cudaFree(out);
        workspace_free(ws);
    };
    auto cuda_err = [&](const char* what) {
        *why = std::string(what) + ": " + cudaGetErrorString(e);
        cleanup();
        return (int)e;
    };
    if ((e = cudaMalloc(&x, sizeof(float) * n * dim_pad)) != cudaSuccess ||
        (e = cudaMalloc(&adj, sizeof(int2) * n * deg_pad)) != cudaSuccess ||
        (e = cudaMalloc(&w, sizeof(float) * n * deg_pad)) != cudaSuccess ||
        (e = cudaMalloc(&lock, sizeof(int32_t) * n)) != cudaSuccess ||
        (e = cudaMalloc(&iota, sizeof(int32_t) * n)) != cudaSuccess ||
        (e = cudaMalloc(&qbuf, sizeof(float) * kMaxBatch * dim)) != cudaSuccess ||
        (e = cudaMalloc(&bids, sizeof(int32_t) * kMaxBatch)) != cudaSuccess ||
        (e = cudaMalloc(&sid, sizeof(int32_t) * kMaxBatch * kmax)) != cudaSuccess ||
        (e = cudaMalloc(&sd, sizeof(float) * kMaxBatch * kmax)) != cudaSuccess ||
        (e = cudaMalloc(&status, sizeof(int32_t) * kMaxBatch)) != cudaSuccess)
        return cuda_err("build buffers");
    if ((e = cudaMemsetAsync(x, 0, sizeof(float) * n * dim_pad, st)) != cudaSuccess ||
        (e = cudaMemcpy2DAsync(x, sizeof(float) * dim_pad, x_host, sizeof(float) * dim, sizeof(float) * dim, n,
                               cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(adj, 0xff, sizeof(int2) * n * deg_pad, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(w, 0, sizeof(float) * n * deg_pad, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(lock, 0, sizeof(int32_t) * n, st)) != cudaSuccess)
        return cuda_err("build upload");
    iota_kernel<<<1024, 256, 0, st>>>(iota, n);
    BuildGraph G{x, dim_pad, adj, w, lock, d, deg_pad};
    complete_graph_kernel<<<(d + 1 + 3) / 4, 128, 0, st>>>(G);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err("start graph");

    // The graph as the search kernels see it: caller order, internal id = caller id, entry vertex 0.
    DeviceIndex view;
    view.n = n;
    view.dim = dim;
    view.dim_pad = dim_pad;
    view.degree = d;
    view.deg_pad = deg_pad;
    view.x32 = x;
    view.adj = reinterpret_cast<int32_t*>(adj);
    view.entry = 0;
    view.entry_internal = 0;
    view.old2new = iota;
    view.new2old = iota;
    if ((rc = workspace_reserve(ws, view, kMaxBatch, why)) != 0) {
        cleanup();
        return rc;
    }

    std::vector<int32_t> ids, deferred, st_h;
    int64_t next = d + 1, inserted = d + 1;
    int32_t tag = 0, stalls = 0;
    while (next < n || !deferred.empty()) {
        int32_t ks = p.k_ext;
        ids.clear();
        const bool retry = !deferred.empty();
        if (retry) {
            // vertices whose candidates ran out: search again with two (after a batch that inserted
            // nobody, four) times the candidates, on their own; each batch of them that inserts
            // nobody halves the next one, down to one vertex, which meets no contention
            ks = std::min<int32_t>(kmax, p.k_ext << std::min(stalls + 1, 2));
            const size_t take = std::min<size_t>(deferred.size(), (size_t)std::max<int64_t>(1, kMaxBatch >> stalls));
            ids.assign(deferred.begin(), deferred.begin() + take);
            deferred.erase(deferred.begin(), deferred.begin() + take);
        } else {
            const int64_t B = std::max<int64_t>(1, std::min<int64_t>({inserted / batch_div, kMaxBatch, n - next}));
            for (int64_t v = next; v < next + B; ++v) ids.push_back((int32_t)v);
            next += B;
        }
        const int32_t nb = (int32_t)ids.size();
        if ((e = cudaMemcpyAsync(bids, ids.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_err("batch ids");
        gather_rows_kernel<<<std::max(1, std::min(1024, (int)((int64_t)nb * dim / 256 + 1))), 256, 0, st>>>(
            x, dim_pad, dim, bids, nb, qbuf);
        SearchArgs a{};
        a.ix = &view;
        a.queries = qbuf;
        a.nq = nb;
        a.k = ks;
        a.eps = p.eps_ext;
        a.precision = DEG_F32;
        a.ids = sid;
        a.dists = sd;
        if ((rc = launch_search(a, ws, stream, why)) != 0) {
            cleanup();
            return rc;
        }
        ++tag;
        extend_kernel<<<(nb + kBuildWarps - 1) / kBuildWarps, kBuildWarps * 32, 0, st>>>(G, bids, nb, sid, sd, ks, tag,
                                                                                          status);
        st_h.resize(nb);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(st_h.data(), status, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_err("extension");
        const int64_t before = inserted;
        for (int32_t t = 0; t < nb; ++t) {
            if (st_h[t]) deferred.push_back(ids[t]);
            else ++inserted;
        }
        if (retry && inserted == before) {
            if (nb == 1 && ks == kmax) {
                cleanup();
                return *why = "a vertex found no d free neighbours among its candidates", (int)cudaErrorUnknown;
            }
            ++stalls;
        } else if (retry) {
            stalls = 0;
        }
        if (progress) *progress = inserted;
    }
    if ((e = cudaMalloc(&out, sizeof(int32_t) * n * d)) != cudaSuccess) return cuda_err("adjacency out");
    compact_adj_kernel<<<1024, 256, 0, st>>>(adj, n, deg_pad, d, out);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(adj_out, out, sizeof(int32_t) * n * d, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_err("adjacency copy");
    cleanup();
    return 0;
}

}  // namespace deg
