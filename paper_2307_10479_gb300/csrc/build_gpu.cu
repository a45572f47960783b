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
                                                                  int32_t tag, int32_t* __restrict__ status,
                                                                  int32_t* __restrict__ opt_u, int32_t* __restrict__ opt_cnt) {
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
    if (opt_u) {
        // the last line of Alg. 3: optimizeEdge(G, v, u) for u in U \ S, in the order of U
        int m = 0;
        for (int k = 0; k < d; ++k) {
            bool in_s = false;
            for (int i = lane; i < ks; i += 32) in_s |= s_ids[(int64_t)t * ks + i] == uid[k];
            if (!__any_sync(0xffffffffu, in_s)) {
                if (lane == 0) opt_u[(int64_t)t * d + m] = uid[k];
                ++m;
            }
        }
        if (lane == 0) opt_cnt[t] = m;
    }
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


// ---- optimizeEdge (Alg. 4) on the device ------------------------------------------------------
// Many edge optimisations run at once, one warp each, in lock step driven by the host: every step
// batches the range searches the running optimisations need into one launch of the search
// kernels (Alg. 1 from the seed pair the listing names), then one kernel takes each
// optimisation's decision. An optimisation claims (for the current wave) every vertex whose row
// it changes before changing it; a claim that fails, or an edge that another optimisation removed
// in between, reverts all its changes (state kAborted) and the host runs it again in a later wave.
// Each optimisation otherwise follows the sequential algorithm and its readings: i_opt bounds the
// iterations, case a adds (v1, v5) and (v1, v6), case b needs v1 and v4 not adjacent and a path
// found by either of the two searches, ties of the gain go to the first candidate in result and
// slot order, and all changes are reverted when no iteration succeeds.
constexpr int kMaxChanges = 16;         // 1 + 2 i_opt + 3 with i_opt <= 6
constexpr int kMaxOwned = 16;
enum OptState : int32_t { kSearchA = 0, kCaseA = 1, kCaseB = 2, kDone = 3, kFailed = 4, kAborted = 5 };

struct Change {
    int32_t u, v, su, sv;
    float w;
    int32_t added;
};

struct OptTask {
    int32_t v1, v2, v3, v4;
    int32_t mode;          // 0: optimise (v1, v2); 1: only if checkMRNG(v1, v2) fails; 2: v2 = v1's longest edge
    int32_t state, it, nch, nown;
    float gain, d14;
    int32_t owned[kMaxOwned];
    Change ch[kMaxChanges];
};

// ---- single-thread graph edits (lane 0 of a task's warp); rows of owned vertices are stable ----
__device__ int slot_scalar(const BuildGraph& G, int32_t u, int32_t c) {
    for (int j = 0; j < G.degree; ++j)
        if (G.adj[(int64_t)u * G.deg_pad + j].x == c) return j;
    return -1;
}
__device__ bool own(const BuildGraph& G, OptTask& T, int32_t c, int32_t tag) {
    for (int i = 0; i < T.nown; ++i)
        if (T.owned[i] == c) return true;
    if (T.nown == kMaxOwned || claim(G.lock, c, tag) < 0) return false;
    T.owned[T.nown++] = c;
    return true;
}
__device__ bool unlink_rec(const BuildGraph& G, OptTask& T, int32_t u, int32_t v) {
    const int su = slot_scalar(G, u, v), sv = slot_scalar(G, v, u);
    if (su < 0 || sv < 0 || T.nch == kMaxChanges) return false;
    T.ch[T.nch++] = Change{u, v, su, sv, G.w[(int64_t)u * G.deg_pad + su], 0};
    G.adj[(int64_t)u * G.deg_pad + su] = make_int2(-1, -1);
    G.adj[(int64_t)v * G.deg_pad + sv] = make_int2(-1, -1);
    return true;
}
__device__ bool link_rec(const BuildGraph& G, OptTask& T, int32_t u, int32_t v, float w) {
    if (u == v || slot_scalar(G, u, v) >= 0) return false;
    const int su = slot_scalar(G, u, -1), sv = slot_scalar(G, v, -1);
    if (su < 0 || sv < 0 || T.nch == kMaxChanges) return false;
    T.ch[T.nch++] = Change{u, v, su, sv, w, 1};
    G.adj[(int64_t)u * G.deg_pad + su] = make_int2(v, v);
    G.w[(int64_t)u * G.deg_pad + su] = w;
    G.adj[(int64_t)v * G.deg_pad + sv] = make_int2(u, u);
    G.w[(int64_t)v * G.deg_pad + sv] = w;
    return true;
}
__device__ void revert(const BuildGraph& G, OptTask& T, int32_t state) {
    for (int i = T.nch - 1; i >= 0; --i) {
        const Change c = T.ch[i];
        if (c.added) {
            G.adj[(int64_t)c.u * G.deg_pad + c.su] = make_int2(-1, -1);
            G.adj[(int64_t)c.v * G.deg_pad + c.sv] = make_int2(-1, -1);
        } else {
            G.adj[(int64_t)c.u * G.deg_pad + c.su] = make_int2(c.v, c.v);
            G.w[(int64_t)c.u * G.deg_pad + c.su] = c.w;
            G.adj[(int64_t)c.v * G.deg_pad + c.sv] = make_int2(c.u, c.u);
            G.w[(int64_t)c.v * G.deg_pad + c.sv] = c.w;
        }
    }
    T.nch = 0;
    T.state = state;
}
// checkMRNG (Alg. 2) of an existing edge (v1, v2): no common neighbour u with
// w(v1, v2) > max(w(v1, u), w(v2, u)).
__device__ bool mrng_ok(const BuildGraph& G, int32_t v1, int32_t v2) {
    const int s12 = slot_scalar(G, v1, v2);
    const float w12 = G.w[(int64_t)v1 * G.deg_pad + s12];
    for (int j = 0; j < G.degree; ++j) {
        const int32_t u = G.adj[(int64_t)v1 * G.deg_pad + j].x;
        if (u < 0) continue;
        const int s2u = slot_scalar(G, v2, u);
        if (s2u < 0) continue;
        if (w12 > fmaxf(G.w[(int64_t)v1 * G.deg_pad + j], G.w[(int64_t)v2 * G.deg_pad + s2u])) return false;
    }
    return true;
}
// After an iteration that connected nothing: shift the labels for the next one, or give up.
__device__ void next_iteration(const BuildGraph& G, OptTask& T, int32_t i_opt) {
    const int32_t v = T.v4;
    T.v4 = T.v3;
    T.v3 = T.v2;
    T.v2 = v;
    if (++T.it >= i_opt) revert(G, T, kFailed);
    else T.state = kSearchA;
}

// Start: claim v1 and v2, check the edge (and, by mode, its MRNG test), remove it.
__global__ void opt_init_kernel(BuildGraph G, OptTask* tasks, int32_t nt, int32_t tag) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    OptTask& T = tasks[t];
    T.state = kFailed;
    T.nch = T.nown = T.it = 0;
    if (!own(G, T, T.v1, tag)) { T.state = kAborted; return; }
    if (T.mode == 2) {                                            // the longest edge of v1, ties to the lower id
        int32_t far = -1;
        float wf = -1.f;
        for (int j = 0; j < G.degree; ++j) {
            const int32_t c = G.adj[(int64_t)T.v1 * G.deg_pad + j].x;
            const float w = G.w[(int64_t)T.v1 * G.deg_pad + j];
            if (c >= 0 && (w > wf || (w == wf && c < far))) { wf = w; far = c; }
        }
        T.v2 = far;
    }
    if (T.v2 < 0) return;
    if (!own(G, T, T.v2, tag)) { T.state = kAborted; return; }
    const int s12 = slot_scalar(G, T.v1, T.v2);
    if (s12 < 0) return;                                          // the edge is gone: nothing to do
    if (T.mode == 1 && mrng_ok(G, T.v1, T.v2)) return;
    T.gain = G.w[(int64_t)T.v1 * G.deg_pad + s12];
    unlink_rec(G, T, T.v1, T.v2);
    T.v3 = T.v4 = T.v1;
    T.state = kSearchA;
}

// The searches the tasks in `state` (kSearchA, or kCaseA and kCaseB together) need: one query
// per task (two for kCaseB), listed in list_task / qvert / seeds / seeds2; cnt[0] counts them.
__global__ void opt_gather_kernel(const OptTask* __restrict__ tasks, int32_t nt, int32_t phase, int32_t* list_task,
                                  int32_t* qvert, int32_t* seeds, int32_t* seeds2, int32_t* cnt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const OptTask& T = tasks[t];
    if (phase == 0 ? T.state != kSearchA : (T.state != kCaseA && T.state != kCaseB)) return;
    const int nq = T.state == kCaseB ? 2 : 1;
    const int at = atomicAdd(cnt, nq);
    for (int w = 0; w < nq; ++w) {
        list_task[at + w] = w == 0 ? t : -1;                      // the second query of a task follows its first
        if (T.state == kSearchA) {                                // RangeSearch(G, {v3, v4}, v2)
            qvert[at] = T.v2;
            seeds[at] = T.v3;
            seeds2[at] = T.v4 == T.v3 ? -1 : T.v4;
        } else {                                                  // RangeSearch(G, {v2, v3}, v1 or v4)
            qvert[at + w] = w == 0 ? T.v1 : T.v4;
            seeds[at + w] = T.v2;
            seeds2[at + w] = T.v3 == T.v2 ? -1 : T.v3;
        }
    }
}

// Best candidate of a warp: the largest gain, ties to the smallest scan order o (lane-local
// candidates arrive in increasing o, so each lane keeps its first maximum). Returns the owning
// lane, or -1 if no lane has one.
__device__ __forceinline__ int best_lane(float g, uint32_t o, bool has, int lane, uint64_t* key_out) {
    const uint64_t key = has ? ((uint64_t)__float_as_uint(g) << 32) | (0xffffffffu - o) : 0ull;
    const uint64_t best = warp_max64(key);
    *key_out = best;
    if (best == 0) return -1;
    return __ffs(__ballot_sync(0xffffffffu, key == best)) - 1;
}

// Alg. 4, the first half of an iteration: over the results s of RangeSearch(G, {v3, v4}, v2)
// (s not v1, v2 or a neighbour of v2) and their neighbours n != v2, the largest
// gain - delta(s, v2) + w(s, n) above gain; replace (s, n) by (v2, s).
__global__ void __launch_bounds__(kBuildWarps * 32) opt_step_a_kernel(BuildGraph G, OptTask* tasks,
                                                                      const int32_t* __restrict__ list_task, int32_t cnt,
                                                                      const int32_t* __restrict__ s_ids,
                                                                      const float* __restrict__ s_d, int32_t ks,
                                                                      int32_t tag, int32_t i_opt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * kBuildWarps + warp;
    if (e >= cnt) return;
    const int t = list_task[e];
    if (t < 0) return;
    OptTask& T = tasks[t];
    const int32_t v1 = T.v1, v2 = T.v2;
    const float gain = T.gain;
    RowRegs r2;
    load_row(G, v2, lane, r2);
    float bg = gain, bds = 0.f;
    uint32_t bo = 0;
    int32_t bs = -1, bn = -1;
    for (int i = 0; i < ks; ++i) {
        const int32_t s = s_ids[(int64_t)e * ks + i];
        if (s < 0) break;
        if (s == v1 || s == v2 || slot_of(r2, s, lane) >= 0) continue;
        const float ds = s_d[(int64_t)e * ks + i];
        for (int j = lane; j < G.degree; j += 32) {
            const int32_t n = reinterpret_cast<volatile int*>(G.adj + (int64_t)s * G.deg_pad + j)[0];
            if (n < 0 || n == v2) continue;
            const float g = gain - ds + reinterpret_cast<volatile float*>(G.w + (int64_t)s * G.deg_pad)[j];
            if (g > bg) { bg = g; bo = (uint32_t)(i * kMaxBuildDegree + j); bs = s; bn = n; bds = ds; }
        }
    }
    uint64_t key;
    const int src = best_lane(bg, bo, bs >= 0, lane, &key);
    int flag = 0;
    if (src >= 0) {
        bg = __shfl_sync(0xffffffffu, bg, src);
        bs = __shfl_sync(0xffffffffu, bs, src);
        bn = __shfl_sync(0xffffffffu, bn, src);
        bds = __shfl_sync(0xffffffffu, bds, src);
    }
    if (lane == 0) {
        if (src < 0) {
            revert(G, T, kFailed);                                  // no gain: undo everything
        } else if (!own(G, T, bs, tag) || !own(G, T, bn, tag) || !unlink_rec(G, T, bs, bn) ||
                   !link_rec(G, T, v2, bs, bds)) {
            revert(G, T, kAborted);
        } else {
            T.v3 = bs;
            T.v4 = bn;
            T.gain = bg;
            if (bn == v1) T.state = kCaseA;
            else if (slot_scalar(G, v1, bn) < 0) flag = 1;          // case b may apply: needs delta(v1, v4)
            else next_iteration(G, T, i_opt);
        }
    }
    flag = __shfl_sync(0xffffffffu, flag, 0);
    if (!flag) return;
    const float d14 = row_dist(G.x, G.dim_pad, v1, bn, lane);
    if (lane == 0) {
        if (bg - d14 > 0.f) {
            T.d14 = d14;
            T.state = kCaseB;
        } else {
            next_iteration(G, T, i_opt);
        }
    }
}

// Alg. 4, the second half. Case a (v4 = v1): over the results s of RangeSearch(G, {v2, v3}, v1)
// not adjacent to v1 and their neighbours n (not v1, not adjacent to v1), the largest
// gain + w(s, n) - delta(s, v1) - delta(n, v1) above zero; replace (s, n) by (v1, s), (v1, n).
// Case b: connect v1 and v4 if v1 is in the search for v1 or v4 in the search for v4 (a path).
__global__ void __launch_bounds__(kBuildWarps * 32) opt_step_b_kernel(BuildGraph G, OptTask* tasks,
                                                                      const int32_t* __restrict__ list_task, int32_t cnt,
                                                                      const int32_t* __restrict__ s_ids,
                                                                      const float* __restrict__ s_d, int32_t ks,
                                                                      int32_t tag, int32_t i_opt, int32_t dim) {
    extern __shared__ float sm_b[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * kBuildWarps + warp;
    if (e >= cnt) return;
    const int t = list_task[e];
    if (t < 0) return;
    OptTask& T = tasks[t];
    const int32_t v1 = T.v1;
    if (T.state == kCaseB) {
        bool path = false;
        for (int i = lane; i < ks; i += 32) {
            path |= s_ids[(int64_t)e * ks + i] == v1;
            path |= s_ids[(int64_t)(e + 1) * ks + i] == T.v4;
        }
        path = __any_sync(0xffffffffu, path);
        if (lane == 0) {
            if (!path) next_iteration(G, T, i_opt);
            else if (!link_rec(G, T, v1, T.v4, T.d14)) revert(G, T, kAborted);
            else T.state = kDone;
        }
        return;
    }
    // case a: v1's row and vector in shared memory (v1 is owned: its row does not change)
    int32_t* row1 = reinterpret_cast<int32_t*>(sm_b + warp * (kMaxBuildDegree + G.dim_pad));
    float* x1 = sm_b + warp * (kMaxBuildDegree + G.dim_pad) + kMaxBuildDegree;
    for (int j = lane; j < G.degree; j += 32) row1[j] = G.adj[(int64_t)v1 * G.deg_pad + j].x;
    for (int c = lane; c < G.dim_pad; c += 32) x1[c] = G.x[(int64_t)v1 * G.dim_pad + c];
    __syncwarp();
    const float gain = T.gain;
    float bg = 0.f, bds = 0.f, bdn = 0.f;
    uint32_t bo = 0;
    int32_t bs = -1, bn = -1;
    for (int i = 0; i < ks; ++i) {
        const int32_t s = s_ids[(int64_t)e * ks + i];
        if (s < 0) break;
        if (s == v1 || any_in(row1, G.degree, s, lane)) continue;
        const float ds = s_d[(int64_t)e * ks + i];
        for (int j = lane; j < G.degree; j += 32) {
            const int32_t n = reinterpret_cast<volatile int*>(G.adj + (int64_t)s * G.deg_pad + j)[0];
            if (n < 0 || n == v1 || find_in(row1, G.degree, n) >= 0) continue;
            const float ub = gain + reinterpret_cast<volatile float*>(G.w + (int64_t)s * G.deg_pad)[j] - ds;
            if (ub <= bg) continue;                                 // delta(n, v1) >= 0 cannot make it better
            const float4* xn = reinterpret_cast<const float4*>(G.x + (int64_t)n * G.dim_pad);
            float a = 0.f;
            for (int c = 0; c < G.dim_pad / 4; ++c) {
                const float4 u = __ldg(xn + c);
                float z;
                z = u.x - x1[4 * c]; a = fmaf(z, z, a);
                z = u.y - x1[4 * c + 1]; a = fmaf(z, z, a);
                z = u.z - x1[4 * c + 2]; a = fmaf(z, z, a);
                z = u.w - x1[4 * c + 3]; a = fmaf(z, z, a);
            }
            const float dn = sqrtf(a);
            const float g = ub - dn;
            if (g > bg) { bg = g; bo = (uint32_t)(i * kMaxBuildDegree + j); bs = s; bn = n; bds = ds; bdn = dn; }
        }
    }
    uint64_t key;
    const int src = best_lane(bg, bo, bs >= 0, lane, &key);
    if (src >= 0) {
        bs = __shfl_sync(0xffffffffu, bs, src);
        bn = __shfl_sync(0xffffffffu, bn, src);
        bds = __shfl_sync(0xffffffffu, bds, src);
        bdn = __shfl_sync(0xffffffffu, bdn, src);
    }
    if (lane == 0) {
        if (src < 0) next_iteration(G, T, i_opt);
        else if (!own(G, T, bs, tag) || !own(G, T, bn, tag) || !unlink_rec(G, T, bs, bn) ||
                 !link_rec(G, T, v1, bs, bds) || !link_rec(G, T, v1, bn, bdn))
            revert(G, T, kAborted);
        else T.state = kDone;
    }
    (void)dim;
}

// Tasks still running when the host's step budget ends: undo them.
__global__ void opt_finish_kernel(BuildGraph G, OptTask* tasks, int32_t nt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int s = tasks[t].state;
    if (s == kSearchA || s == kCaseA || s == kCaseB) revert(G, tasks[t], kFailed);
}

// Weights of an uploaded adjacency: w[u][j] = delta(u, adj[u][j]) (one warp per vertex).
__global__ void weights_kernel(BuildGraph G, int64_t n) {
    const int lane = threadIdx.x & 31;
    for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n;
         u += (int64_t)gridDim.x * (blockDim.x >> 5))
        for (int j = 0; j < G.degree; ++j) {
            const int32_t c = G.adj[u * G.deg_pad + j].x;
            const float d = c >= 0 ? row_dist(G.x, G.dim_pad, (int32_t)u, c, lane) : 0.f;
            if (lane == 0) G.w[u * G.deg_pad + j] = d;
        }
}

// [n][degree] int32 -> adjacency pairs
__global__ void expand_adj_kernel(const int32_t* __restrict__ in, int64_t n, int32_t deg_pad, int32_t degree,
                                  int2* __restrict__ adj) {
    const int64_t total = n * degree;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / degree;
        const int32_t c = in[i];
        adj[v * deg_pad + (i - v * degree)] = make_int2(c, c);
    }
}

// out[i][j] = neighbour j of vertex vs[i]
__global__ void gather_adj_rows_kernel(const int2* __restrict__ adj, int32_t deg_pad, int32_t degree,
                                       const int32_t* __restrict__ vs, int32_t cnt, int32_t* __restrict__ out) {
    const int64_t total = (int64_t)cnt * degree;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / degree;
        out[i] = adj[(int64_t)vs[r] * deg_pad + (i - r * degree)].x;
    }
}

constexpr int64_t kMaxBatch = 8192;

uint64_t splitmix64(uint64_t& s) {  // SplitMix64 (Steele, Lea, Flood 2014)
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The graph under construction and every buffer the batched steps use; the host side drives the
// batches and the optimisation waves.
class DeviceBuilder {
  public:
    DeviceBuilder(int64_t n, int32_t dim, int32_t degree, deg_stream_t stream)
        : n_(n), dim_(dim), d_(degree), dim_pad_((dim + 3) / 4 * 4), deg_pad_((degree + 3) / 4 * 4),
          stream_(stream), st_(reinterpret_cast<cudaStream_t>(stream)) {}
    ~DeviceBuilder() {
        for (void* p : {(void*)x_, (void*)w_, (void*)adj_, (void*)lock_, (void*)iota_, (void*)qbuf_, (void*)qvert_,
                        (void*)sid_, (void*)sd_, (void*)status_, (void*)opt_u_, (void*)opt_cnt_, (void*)tasks_,
                        (void*)list_, (void*)seeds_, (void*)seeds2_, (void*)cnt_, (void*)out_})
            cudaFree(p);
        workspace_free(ws_);
    }

    int init(const float* x_host, const int32_t* adj_host, int32_t kmax, std::string* why) {
        kmax_ = kmax;
        cudaError_t e;
        const int64_t nq = 2 * kMaxBatch;
        if ((e = cudaMalloc(&x_, sizeof(float) * n_ * dim_pad_)) != cudaSuccess ||
            (e = cudaMalloc(&adj_, sizeof(int2) * n_ * deg_pad_)) != cudaSuccess ||
            (e = cudaMalloc(&w_, sizeof(float) * n_ * deg_pad_)) != cudaSuccess ||
            (e = cudaMalloc(&lock_, sizeof(int32_t) * n_)) != cudaSuccess ||
            (e = cudaMalloc(&iota_, sizeof(int32_t) * n_)) != cudaSuccess ||
            (e = cudaMalloc(&qbuf_, sizeof(float) * nq * dim_)) != cudaSuccess ||
            (e = cudaMalloc(&qvert_, sizeof(int32_t) * nq)) != cudaSuccess ||
            (e = cudaMalloc(&sid_, sizeof(int32_t) * nq * kmax)) != cudaSuccess ||
            (e = cudaMalloc(&sd_, sizeof(float) * nq * kmax)) != cudaSuccess ||
            (e = cudaMalloc(&status_, sizeof(int32_t) * kMaxBatch)) != cudaSuccess ||
            (e = cudaMalloc(&opt_u_, sizeof(int32_t) * kMaxBatch * d_)) != cudaSuccess ||
            (e = cudaMalloc(&opt_cnt_, sizeof(int32_t) * kMaxBatch)) != cudaSuccess ||
            (e = cudaMalloc(&tasks_, sizeof(OptTask) * kMaxBatch)) != cudaSuccess ||
            (e = cudaMalloc(&list_, sizeof(int32_t) * nq)) != cudaSuccess ||
            (e = cudaMalloc(&seeds_, sizeof(int32_t) * nq)) != cudaSuccess ||
            (e = cudaMalloc(&seeds2_, sizeof(int32_t) * nq)) != cudaSuccess ||
            (e = cudaMalloc(&cnt_, sizeof(int32_t))) != cudaSuccess)
            return err(e, "build buffers", why);
        if ((e = cudaMemsetAsync(x_, 0, sizeof(float) * n_ * dim_pad_, st_)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(x_, sizeof(float) * dim_pad_, x_host, sizeof(float) * dim_, sizeof(float) * dim_, n_,
                                   cudaMemcpyHostToDevice, st_)) != cudaSuccess ||
            (e = cudaMemsetAsync(adj_, 0xff, sizeof(int2) * n_ * deg_pad_, st_)) != cudaSuccess ||
            (e = cudaMemsetAsync(w_, 0, sizeof(float) * n_ * deg_pad_, st_)) != cudaSuccess ||
            (e = cudaMemsetAsync(lock_, 0, sizeof(int32_t) * n_, st_)) != cudaSuccess)
            return err(e, "build upload", why);
        iota_kernel<<<1024, 256, 0, st_>>>(iota_, n_);
        G_ = BuildGraph{x_, dim_pad_, adj_, w_, lock_, d_, deg_pad_};
        if (adj_host) {
            // an existing graph: pairs and weights from its [n][degree] adjacency
            if ((e = cudaMalloc(&out_, sizeof(int32_t) * n_ * d_)) != cudaSuccess ||
                (e = cudaMemcpyAsync(out_, adj_host, sizeof(int32_t) * n_ * d_, cudaMemcpyHostToDevice, st_)) != cudaSuccess)
                return err(e, "adjacency upload", why);
            expand_adj_kernel<<<1024, 256, 0, st_>>>(out_, n_, deg_pad_, d_, adj_);
            weights_kernel<<<1024, 256, 0, st_>>>(G_, n_);
        } else {
            complete_graph_kernel<<<(d_ + 1 + 3) / 4, 128, 0, st_>>>(G_);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return err(e, "start graph", why);
        // the graph as the search kernels see it: caller order, internal id = caller id, entry 0
        view_.n = n_;
        view_.dim = dim_;
        view_.dim_pad = dim_pad_;
        view_.degree = d_;
        view_.deg_pad = deg_pad_;
        view_.x32 = x_;
        view_.adj = reinterpret_cast<int32_t*>(adj_);
        view_.entry = 0;
        view_.entry_internal = 0;
        view_.old2new = iota_;
        view_.new2old = iota_;
        return workspace_reserve(ws_, view_, nq, why);
    }

    // Range searches (Alg. 1, float32 rows) for the rows of vertices qvert_[0..nq) into sid_/sd_,
    // seeded at vertex 0, or at seeds_ (and seeds2_) when given.
    int search(int32_t nq, int32_t k, float eps, bool seeded, std::string* why) {
        gather_rows_kernel<<<std::max(1, std::min(1024, (int)((int64_t)nq * dim_ / 256 + 1))), 256, 0, st_>>>(
            x_, dim_pad_, dim_, qvert_, nq, qbuf_);
        SearchArgs a{};
        a.ix = &view_;
        a.queries = qbuf_;
        a.seeds = seeded ? seeds_ : nullptr;
        a.seeds2 = seeded ? seeds2_ : nullptr;
        a.nq = nq;
        a.k = k;
        a.eps = eps;
        a.precision = DEG_F32;
        a.ids = sid_;
        a.dists = sd_;
        return launch_search(a, ws_, stream_, why);
    }

    // Alg. 3 for the vertices ids (their searches run first); deferred gets the vertices to
    // insert again; with optimise, tasks gets (v, u) for u in U \ S of every inserted vertex.
    int extend(const std::vector<int32_t>& ids, int32_t ks, float eps, bool optimise, std::vector<int32_t>& deferred,
               std::vector<std::vector<int32_t>>* tasks, int64_t* inserted, std::string* why) {
        const int32_t nb = (int32_t)ids.size();
        cudaError_t e;
        if ((e = cudaMemcpyAsync(qvert_, ids.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st_)) != cudaSuccess)
            return err(e, "batch ids", why);
        if (const int rc = search(nb, ks, eps, false, why)) return rc;
        ++tag_;
        extend_kernel<<<(nb + kBuildWarps - 1) / kBuildWarps, kBuildWarps * 32, 0, st_>>>(
            G_, qvert_, nb, sid_, sd_, ks, tag_, status_, optimise ? opt_u_ : nullptr, opt_cnt_);
        st_h_.resize(nb);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(st_h_.data(), status_, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, st_)) != cudaSuccess)
            return err(e, "extension", why);
        if (optimise) {
            cnt_h_.resize(nb);
            u_h_.resize((size_t)nb * d_);
            if ((e = cudaMemcpyAsync(cnt_h_.data(), opt_cnt_, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, st_)) != cudaSuccess ||
                (e = cudaMemcpyAsync(u_h_.data(), opt_u_, sizeof(int32_t) * nb * d_, cudaMemcpyDeviceToHost, st_)) != cudaSuccess)
                return err(e, "optimisation tasks", why);
        }
        if ((e = cudaStreamSynchronize(st_)) != cudaSuccess) return err(e, "extension", why);
        for (int32_t t = 0; t < nb; ++t) {
            if (st_h_[t]) {
                deferred.push_back(ids[t]);
                continue;
            }
            ++*inserted;
            if (optimise) {
                std::vector<int32_t> q;
                for (int i = 0; i < cnt_h_[t]; ++i) q.push_back(ids[t]), q.push_back(u_h_[(size_t)t * d_ + i]), q.push_back(0);
                tasks->push_back(std::move(q));
            }
        }
        return 0;
    }

    // Runs task queues to completion: queue i holds (v1, v2, mode) triples run in order; a wave
    // takes the next task of every queue (queues share no v1, so their first claims do not
    // collide), aborted tasks go back to the front of their queue (at most 3 times).
    int optimise(std::vector<std::vector<int32_t>>& queues, int32_t i_opt, int32_t k_opt, float eps_opt,
                 std::string* why) {
        std::vector<size_t> pos(queues.size(), 0);
        std::vector<int> tries(queues.size(), 0);
        std::vector<OptTask> wave;
        std::vector<int32_t> owner;
        for (;;) {
            wave.clear();
            owner.clear();
            for (size_t i = 0; i < queues.size() && (int64_t)wave.size() < kMaxBatch; ++i) {
                if (pos[i] >= queues[i].size()) continue;
                OptTask T{};
                T.v1 = queues[i][pos[i]];
                T.v2 = queues[i][pos[i] + 1];
                T.mode = queues[i][pos[i] + 2];
                wave.push_back(T);
                owner.push_back((int32_t)i);
            }
            if (wave.empty()) return 0;
            if (const int rc = run_wave(wave, i_opt, k_opt, eps_opt, why)) return rc;
            for (size_t w = 0; w < wave.size(); ++w) {
                const int32_t i = owner[w];
                if (wave[w].state == kAborted && ++tries[i] <= 3) continue;   // same task again
                tries[i] = 0;
                pos[i] += 3;
                if (wave[w].state == kDone) ++improved_;
            }
        }
    }

    int run_wave(std::vector<OptTask>& wave, int32_t i_opt, int32_t k_opt, float eps_opt, std::string* why) {
        const int32_t nt = (int32_t)wave.size();
        cudaError_t e;
        if ((e = cudaMemcpyAsync(tasks_, wave.data(), sizeof(OptTask) * nt, cudaMemcpyHostToDevice, st_)) != cudaSuccess)
            return err(e, "tasks", why);
        ++tag_;
        opt_init_kernel<<<(nt + 127) / 128, 128, 0, st_>>>(G_, tasks_, nt, tag_);
        const size_t smem_b = sizeof(float) * kBuildWarps * (kMaxBuildDegree + dim_pad_);
        for (int step = 0; step < 2 * i_opt + 2; ++step) {
            int32_t c[2] = {0, 0};
            for (int phase = 0; phase < 2; ++phase) {
                if ((e = cudaMemsetAsync(cnt_, 0, sizeof(int32_t), st_)) != cudaSuccess) return err(e, "count", why);
                opt_gather_kernel<<<(nt + 127) / 128, 128, 0, st_>>>(tasks_, nt, phase, list_, qvert_, seeds_, seeds2_, cnt_);
                if ((e = cudaMemcpyAsync(&c[phase], cnt_, sizeof(int32_t), cudaMemcpyDeviceToHost, st_)) != cudaSuccess ||
                    (e = cudaStreamSynchronize(st_)) != cudaSuccess)
                    return err(e, "optimisation step", why);
                if (c[phase] == 0) continue;
                if (const int rc = search(c[phase], k_opt, eps_opt, true, why)) return rc;
                const int blocks = (c[phase] + kBuildWarps - 1) / kBuildWarps;
                if (phase == 0)
                    opt_step_a_kernel<<<blocks, kBuildWarps * 32, 0, st_>>>(G_, tasks_, list_, c[0], sid_, sd_, k_opt,
                                                                           tag_, i_opt);
                else
                    opt_step_b_kernel<<<blocks, kBuildWarps * 32, smem_b, st_>>>(G_, tasks_, list_, c[1], sid_, sd_,
                                                                                k_opt, tag_, i_opt, dim_);
            }
            if (c[0] == 0 && c[1] == 0) break;
        }
        opt_finish_kernel<<<(nt + 127) / 128, 128, 0, st_>>>(G_, tasks_, nt);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(wave.data(), tasks_, sizeof(OptTask) * nt, cudaMemcpyDeviceToHost, st_)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st_)) != cudaSuccess)
            return err(e, "optimisation wave", why);
        return 0;
    }

    // Rows of vertices vs (host), [count][degree] (gathered on the device, one copy out).
    int rows(const std::vector<int32_t>& vs, std::vector<int32_t>& out, std::string* why) {
        const int32_t cnt = (int32_t)vs.size();
        out.assign((size_t)cnt * d_, -1);
        cudaError_t e;
        if ((e = cudaMemcpyAsync(qvert_, vs.data(), sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, st_)) != cudaSuccess)
            return err(e, "rows", why);
        gather_adj_rows_kernel<<<256, 256, 0, st_>>>(adj_, deg_pad_, d_, qvert_, cnt, sid_);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(out.data(), sid_, sizeof(int32_t) * cnt * d_, cudaMemcpyDeviceToHost, st_)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st_)) != cudaSuccess)
            return err(e, "rows", why);
        return 0;
    }

    int download(int32_t* adj_host, std::string* why) {
        cudaError_t e;
        if (!out_ && (e = cudaMalloc(&out_, sizeof(int32_t) * n_ * d_)) != cudaSuccess) return err(e, "adjacency out", why);
        compact_adj_kernel<<<1024, 256, 0, st_>>>(adj_, n_, deg_pad_, d_, out_);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(adj_host, out_, sizeof(int32_t) * n_ * d_, cudaMemcpyDeviceToHost, st_)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st_)) != cudaSuccess)
            return err(e, "adjacency copy", why);
        return 0;
    }

    int64_t improved() const { return improved_; }

  private:
    static int err(cudaError_t e, const char* what, std::string* why) {
        *why = std::string(what) + ": " + cudaGetErrorString(e);
        return (int)e;
    }

    int64_t n_;
    int32_t dim_, d_, dim_pad_, deg_pad_, kmax_ = 0;
    deg_stream_t stream_;
    cudaStream_t st_;
    float *x_ = nullptr, *w_ = nullptr, *qbuf_ = nullptr, *sd_ = nullptr;
    int2* adj_ = nullptr;
    int32_t *lock_ = nullptr, *iota_ = nullptr, *qvert_ = nullptr, *sid_ = nullptr, *status_ = nullptr;
    int32_t *opt_u_ = nullptr, *opt_cnt_ = nullptr, *list_ = nullptr, *seeds_ = nullptr, *seeds2_ = nullptr;
    int32_t *cnt_ = nullptr, *out_ = nullptr;
    OptTask* tasks_ = nullptr;
    BuildGraph G_{};
    DeviceIndex view_;
    Workspace ws_;
    int32_t tag_ = 0;
    int64_t improved_ = 0;
    std::vector<int32_t> st_h_, cnt_h_, u_h_;
};

}  // namespace

namespace {

// dynamicEdgeOptimization (Alg. 5), `rounds` times: a random vertex v1 (SplitMix64), then
// optimizeEdge(v1, v2) for each neighbour v2 whose edge fails checkMRNG, then for v1's longest
// edge. Rounds run in batches of distinct vertices (at most 4,096 at once); each vertex's
// optimisations run in order, one per wave, and its neighbour list is taken when its batch starts
// (a neighbour that is no longer adjacent by its turn is skipped).
int refine_graph(DeviceBuilder& B, int64_t n, int32_t d, const deg_build_params& p, std::string* why) {
    uint64_t s = p.seed;
    std::vector<int32_t> vs, nb;
    std::vector<char> seen((size_t)n, 0);
    std::vector<std::vector<int32_t>> queues;
    for (int64_t done = 0; done < p.refine_rounds;) {
        vs.clear();
        const int64_t want = std::min<int64_t>(p.refine_rounds - done, 4096);
        while ((int64_t)vs.size() < want) {
            const int32_t v = (int32_t)(splitmix64(s) % (uint64_t)n);
            ++done;
            if (seen[v]) continue;                         // already in this batch: its turn is taken
            seen[v] = 1;
            vs.push_back(v);
            if (done >= p.refine_rounds) break;
        }
        for (int32_t v : vs) seen[v] = 0;
        if (const int rc = B.rows(vs, nb, why)) return rc;
        queues.assign(vs.size(), {});
        for (size_t i = 0; i < vs.size(); ++i) {
            for (int j = 0; j < d; ++j) {
                const int32_t u = nb[i * d + j];
                if (u >= 0) queues[i].insert(queues[i].end(), {vs[i], u, 1});
            }
            queues[i].insert(queues[i].end(), {vs[i], -1, 2});
        }
        if (const int rc = B.optimise(queues, p.i_opt, p.k_opt, p.eps_opt, why)) return rc;
    }
    return 0;
}

}  // namespace

int refine_graph_device(const float* x_host, const int32_t* adj_inout, int64_t n, int32_t dim, const deg_build_params& p,
                        int32_t* adj_out, int64_t* improved, deg_stream_t stream, std::string* why) {
    if (p.degree > kMaxBuildDegree) return *why = "degree above 128", (int)cudaErrorInvalidValue;
    if (p.k_opt > 1024 || p.i_opt > 6) return *why = "k_opt above 1024 or i_opt above 6", (int)cudaErrorInvalidValue;
    DeviceBuilder B(n, dim, p.degree, stream);
    if (const int rc = B.init(x_host, adj_inout, std::max(p.k_opt, p.degree), why)) return rc;
    if (const int rc = refine_graph(B, n, p.degree, p, why)) return rc;
    if (improved) *improved = B.improved();
    return B.download(adj_out, why);
}

namespace {

// Inserts vertices first .. n-1 (Alg. 3, with Alg. 4 for the new edges when p.i_opt > 0) into the
// graph on vertices 0 .. first-1, in batches of at most inserted / batch_div vertices.
int extend_vertices(DeviceBuilder& B, const deg_build_params& p, int64_t first, int64_t n, int32_t batch_div,
                    int32_t kmax, volatile int64_t* progress, std::string* why) {
    const bool optimise = p.i_opt > 0;
    std::vector<int32_t> ids, deferred;
    std::vector<std::vector<int32_t>> tasks;
    int64_t next = first, inserted = first;
    int32_t stalls = 0;
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
            const int64_t nb = std::max<int64_t>(1, std::min<int64_t>({inserted / batch_div, kMaxBatch, n - next}));
            for (int64_t v = next; v < next + nb; ++v) ids.push_back((int32_t)v);
            next += nb;
        }
        const int64_t before = inserted;
        if (const int rc = B.extend(ids, ks, p.eps_ext, optimise, deferred, &tasks, &inserted, why)) return rc;
        if (retry && inserted == before) {
            if (ids.size() == 1 && ks == kmax)
                return *why = "a vertex found no d free neighbours among its candidates", (int)cudaErrorUnknown;
            ++stalls;
        } else if (retry) {
            stalls = 0;
        }
        if (optimise && !tasks.empty()) {
            if (const int rc = B.optimise(tasks, p.i_opt, p.k_opt, p.eps_opt, why)) return rc;
            tasks.clear();
        }
        if (progress) *progress = inserted;
    }
    return 0;
}

int check_build_params(const deg_build_params& p, int32_t batch_div, std::string* why) {
    if (p.degree > kMaxBuildDegree) return *why = "degree above 128", (int)cudaErrorInvalidValue;
    if (p.k_ext > 1024 || p.k_opt > 1024) return *why = "k_ext and k_opt must be at most 1024", (int)cudaErrorInvalidValue;
    if (p.i_opt > 6) return *why = "i_opt above 6", (int)cudaErrorInvalidValue;
    if (batch_div < 1) return *why = "batch_div must be positive", (int)cudaErrorInvalidValue;
    return 0;
}

}  // namespace

int build_graph_device(const float* x_host, int64_t n, int32_t dim, const deg_build_params& p, int32_t batch_div,
                       int32_t* adj_out, volatile int64_t* progress, deg_stream_t stream, std::string* why) {
    if (const int rc = check_build_params(p, batch_div, why)) return rc;
    const int32_t kmax = std::min(1024, std::max({4 * p.k_ext, p.k_opt, p.degree}));
    DeviceBuilder B(n, dim, p.degree, stream);
    if (const int rc = B.init(x_host, nullptr, kmax, why)) return rc;
    if (const int rc = extend_vertices(B, p, p.degree + 1, n, batch_div, kmax, progress, why)) return rc;
    if (p.refine_rounds > 0)
        if (const int rc = refine_graph(B, n, p.degree, p, why)) return rc;
    return B.download(adj_out, why);
}

int insert_vertices_device(const float* x_host, int32_t* adj, int64_t n_old, int64_t n, int32_t dim,
                           const deg_build_params& p, int32_t batch_div, deg_stream_t stream, std::string* why) {
    if (const int rc = check_build_params(p, batch_div, why)) return rc;
    const int32_t kmax = std::min(1024, std::max({4 * p.k_ext, p.k_opt, p.degree}));
    DeviceBuilder B(n, dim, p.degree, stream);
    if (const int rc = B.init(x_host, adj, kmax, why)) return rc;
    if (const int rc = extend_vertices(B, p, n_old, n, batch_div, kmax, nullptr, why)) return rc;
    return B.download(adj, why);
}

}  // namespace deg
