// Batched range search (paper Alg. 1, Sec. 2.1) over a fixed-degree DEG, one warp per query.
//
// Per query the warp holds: the query vector in registers (each lane a slice of 16-byte chunks),
// the checked set C, the candidate set S and the result list R. One hop:
//   1. pop argmin_{S} (distance, id) with a warp reduction; stop if it exceeds r(1+eps)
//      (squared: d2 > r2 (1+eps)^2);
//   2. read the adjacency row (one coalesced load), test-and-insert every neighbour into C;
//   3. gather the unvisited neighbours' rows with 16-byte loads, G lanes per row and up to 16
//      rows in flight per warp, and reduce their squared distances with xor shuffles;
//   4. admit to S every neighbour with d2 <= r2 (1+eps)^2 and try every neighbour with
//      d2 <= r2 for R, both against the radius from before the hop.
// Evaluating a hop's neighbours together and admitting against the pre-hop radius returns the
// same R, the same expansions and the same checked set as the one-by-one loop of Alg. 1: R is
// always the k smallest (distance, id) seen so far, and an extra candidate admitted to S with
// the older, larger radius can only be popped when the search already stops. So the result
// is exact, not an approximation of Alg. 1.
//
// Readings of Alg. 1 (as in the rest of the library): seeds count as checked; exploration
// queries search from their own vertex but never return it; r = +inf until R first exceeds k;
// (distance, id) orders S and R, the lower id first.
//
// Three tiers, one result. The fast path keeps C as an open-addressing hash table, S as an
// unsorted pool (argmin by a warp reduction) and R as a sorted array, all in shared memory.
// A query that would overflow the hash table (load above 3/4) or the pool is rerun at once by
// the same warp in device-memory mode: C becomes an n-bit bitmap and S a larger pool in the
// warp's own slot of device memory. A query that overflows even that is recorded in an
// overflow list and finished by a second kernel whose pool has room for all n vertices.
// Every tier runs the same code on the same data, so the result does not depend on the tier.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "deg_internal.h"

namespace deg {
namespace {

constexpr int kWarpsPerBlock = 4;
constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint32_t kEmptySlot = 0xffffffffu;
constexpr int kMaxDegree = 128;
constexpr int kMaxK = 1024;
constexpr int kInlinePool = 32768;   // candidate pool of the device mode inside the fast kernel

__device__ __forceinline__ uint64_t make_key(float d2, int32_t id) {
    return ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)id;
}
__device__ __forceinline__ float key_d2(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ int32_t key_id(uint64_t k) { return (int32_t)(uint32_t)k; }

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
    for (int m = 16; m; m >>= 1) v = min(v, shfl_xor64(v, m));
    return v;
}

// ---- row storage formats ------------------------------------------------------------------
// A row is read as 16-byte chunks; each chunk holds EPC elements.
struct F32Rows {
    static constexpr int EPC = 4;
    __device__ static float scale(const float*, int32_t) { return 1.f; }
    __device__ static float acc(const uint4& c, const float* q, float s, float a) {
        (void)s;
        const float x0 = __uint_as_float(c.x), x1 = __uint_as_float(c.y);
        const float x2 = __uint_as_float(c.z), x3 = __uint_as_float(c.w);
        float t;
        t = q[0] - x0; a = fmaf(t, t, a);
        t = q[1] - x1; a = fmaf(t, t, a);
        t = q[2] - x2; a = fmaf(t, t, a);
        t = q[3] - x3; a = fmaf(t, t, a);
        return a;
    }
};
struct BF16Rows {
    static constexpr int EPC = 8;
    __device__ static float scale(const float*, int32_t) { return 1.f; }
    __device__ static float acc(const uint4& c, const float* q, float s, float a) {
        (void)s;
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float lo = __uint_as_float(w[i] << 16);          // bf16 -> f32 is exact
            const float hi = __uint_as_float(w[i] & 0xffff0000u);
            float t = q[2 * i] - lo;
            a = fmaf(t, t, a);
            t = q[2 * i + 1] - hi;
            a = fmaf(t, t, a);
        }
        return a;
    }
};
struct FP8Rows {
    static constexpr int EPC = 16;
    __device__ static float scale(const float* sc, int32_t id) { return __ldg(sc + id); }
    __device__ static float acc(const uint4& c, const float* q, float s, float a) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w[i] >> (16 * h)) & 0xffffu);
                const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);  // exact
                const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
                float t = fmaf(-s, f.x, q[4 * i + 2 * h]);
                a = fmaf(t, t, a);
                t = fmaf(-s, f.y, q[4 * i + 2 * h + 1]);
                a = fmaf(t, t, a);
            }
        }
        return a;
    }
};

struct Params {
    const uint8_t* rows;       // row base of the searched storage
    int64_t row_bytes;         // stride of that storage
    int32_t nchunk;            // 16-byte chunks per row
    const float* scale8;       // per-row scales (FP8) or null
    const float* x32;          // float32 rows (exploration queries, re-rank)
    int32_t dim_pad;           // float32 row stride (elements)
    const int32_t* adj;
    int32_t degree, deg_pad;
    int64_t n;
    int32_t entry;
    const float* queries;
    int32_t dim;
    const int32_t* seeds;
    int32_t explore;
    int32_t nq;
    int32_t k;                 // results returned
    int32_t ks;                // results kept during the search (k, or the re-rank width)
    int32_t kcap;              // power of two >= ks (sort width)
    int32_t rerank;            // 1: re-rank R on float32 rows before output
    float f;                   // (1 + eps)^2
    int32_t max_hops;
    // fast tier
    int32_t hcap, hshift, pcap;
    int32_t wpb;               // warps per block of the fast kernel
    // outputs
    int32_t* ids;
    float* dists;
    int32_t* status;
    int32_t* trace;
    // workspace
    int32_t* counters;         // [0] overflow count, [1] 2nd-kernel cursor, [2] fast cursor
    int32_t* overflow;
    int64_t words;             // 32-bit words of one visited bitmap (multiple of 4)
    uint32_t* ibitmaps;        // device mode inside the fast kernel: [islots][words]
    uint64_t* ipools;          //   [islots][ipcap]
    int32_t islots, ipcap;
    uint32_t* bitmaps;         // second kernel: [slots][words]
    uint64_t* pools;           //   [slots][n + 1]
    uint64_t* results;         //   [slots][kMaxK]
};

// Per-warp search state. All scalar members are warp-uniform (every lane holds the same value).
struct WarpState {
    uint32_t* hash;            // fast tier: hash table [hcap]
    uint32_t* bitmap;          // device tier: bitmap [words]
    uint64_t* pool;            // S
    uint64_t* res;             // R
    int32_t* cid;              // per-hop candidate ids [kMaxDegree]
    float* cd2;                // per-hop candidate distances [kMaxDegree]
    int32_t pcap;
    int32_t pool_n, res_n;
    bool trimmed;
    float r2;
    int32_t hops, evals, pool_hw;
};

template <class Rows, int G, int CPL>
struct Engine {
    static constexpr int EPC = Rows::EPC;
    static constexpr int RP = 32 / G;                                   // rows per pass
    static constexpr int U0 = 16 / RP > 0 ? 16 / RP : 1;
    static constexpr int U = (U0 * CPL > 16) ? (16 / CPL > 0 ? 16 / CPL : 1) : U0;   // passes in flight
    float q[CPL][EPC];

    __device__ void load_query(const float* qv, int dim, int lane) {
        const int p = lane % G;
#pragma unroll
        for (int j = 0; j < CPL; ++j)
#pragma unroll
            for (int e = 0; e < EPC; ++e) {
                const int i = (p + G * j) * EPC + e;
                q[j][e] = i < dim ? qv[i] : 0.f;
            }
    }

    // Squared distances of cid[0..cnt) into cd2[0..cnt).
    __device__ void distances(const Params& P, const int32_t* cid, float* cd2, int cnt, int lane) const {
        const int g = lane / G, p = lane % G;
        for (int i0 = 0; i0 < cnt; i0 += RP * U) {
            uint4 buf[U][CPL];
            float sc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * RP + g;
                sc[u] = 1.f;
                if (i < cnt) {
                    const int32_t id = cid[i];
                    const uint8_t* row = P.rows + (int64_t)id * P.row_bytes;
                    sc[u] = Rows::scale(P.scale8, id);
#pragma unroll
                    for (int j = 0; j < CPL; ++j) {
                        const int c = p + G * j;
                        buf[u][j] = c < P.nchunk ? __ldg(reinterpret_cast<const uint4*>(row) + c) : make_uint4(0, 0, 0, 0);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < CPL; ++j) buf[u][j] = make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float a = 0.f;
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    if (p + G * j < P.nchunk) a = Rows::acc(buf[u][j], q[j], sc[u], a);
                }
#pragma unroll
                for (int m = G / 2; m; m >>= 1) a += __shfl_xor_sync(0xffffffffu, a, m);
                const int i = i0 + u * RP + g;
                if (p == 0 && i < cnt) cd2[i] = a;
            }
        }
    }
};

// Exact float32 squared distance of one row (re-rank), one lane; rows are zero padded to a
// multiple of 4 floats and the query in shared memory likewise.
__device__ float exact_d2_lane(const float* x32, int32_t dim_pad, int32_t id, const float* qv) {
    const float4* row = reinterpret_cast<const float4*>(x32 + (int64_t)id * dim_pad);
    const float4* q4 = reinterpret_cast<const float4*>(qv);
    float a = 0.f;
    for (int i = 0; i < dim_pad / 4; ++i) {
        const float4 x = __ldg(row + i), y = q4[i];
        float t;
        t = y.x - x.x; a = fmaf(t, t, a);
        t = y.y - x.y; a = fmaf(t, t, a);
        t = y.z - x.z; a = fmaf(t, t, a);
        t = y.w - x.w; a = fmaf(t, t, a);
    }
    return a;
}

// Returns 1 if id was not in C (and inserts it), 0 if it was, -1 if the table is saturated.
__device__ __forceinline__ int visit_hash(uint32_t* tab, int hcap, int hshift, int32_t id) {
    uint32_t h = ((uint32_t)id * 0x9E3779B1u) >> hshift;
    const uint32_t mask = (uint32_t)hcap - 1;
    for (int t = 0; t < hcap; ++t) {
        const uint32_t old = atomicCAS(tab + h, kEmptySlot, (uint32_t)id);
        if (old == kEmptySlot) return 1;
        if (old == (uint32_t)id) return 0;
        h = (h + 1) & mask;
    }
    return -1;
}
__device__ __forceinline__ int visit_bitmap(uint32_t* bm, int32_t id) {
    const uint32_t bit = 1u << (id & 31);
    const uint32_t old = atomicOr(bm + (id >> 5), bit);
    return (old & bit) ? 0 : 1;
}

// Insert key c into R, kept sorted ascending in res[0..res_n) (Alg. 1: R <- R u {n}; if |R| > k,
// drop argmax and set r = max R). r stays +inf until R first overflows k.
__device__ __forceinline__ void result_insert(WarpState& W, int ks, uint64_t c, int lane) {
    int pos = 0;
    for (int i0 = 0; i0 < W.res_n; i0 += 32) {
        const int i = i0 + lane;
        pos += __popc(__ballot_sync(0xffffffffu, i < W.res_n && W.res[i] < c));
    }
    const bool full = W.res_n == ks;
    if (!full || pos < ks) {
        // shift [pos, last) up by one, top chunk first, then place c at pos
        const int last = full ? ks - 1 : W.res_n;
        for (int c0 = ((last - 1 - pos) / 32) * 32 + pos; c0 >= pos && last > pos; c0 -= 32) {
            const int i = c0 + lane;
            const uint64_t v = i < last ? W.res[i] : 0;
            __syncwarp();
            if (i < last) W.res[i + 1] = v;
            __syncwarp();
        }
        if (lane == 0) W.res[pos] = c;
        if (!full) ++W.res_n;
        __syncwarp();
    }
    if (full) {
        W.trimmed = true;
        W.r2 = key_d2(W.res[ks - 1]);
    }
}

// Remove pool entries above the current admission radius; returns the new size.
__device__ int pool_compact(WarpState& W, float thr, int lane) {
    int out = 0;
    for (int i0 = 0; i0 < W.pool_n; i0 += 32) {
        const int i = i0 + lane;
        const uint64_t v = i < W.pool_n ? W.pool[i] : kEmptyKey;
        const bool keep = i < W.pool_n && key_d2(v) <= thr;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) W.pool[out + __popc(m & ((1u << lane) - 1))] = v;
        out += __popc(m);
        __syncwarp();
    }
    return out;
}

// Sort R ascending (bitonic over kcap entries, padded with the empty key) and write the first k.
__device__ void finish_query(const Params& P, WarpState& W, int q, const float* qv, int status, int tier,
                             int lane) {
    // R is sorted already; a re-rank replaces its distances and sorts again.
    if (P.rerank) {
        // Re-rank: replace the reduced-precision distances by exact float32 ones.
        for (int i = lane; i < W.res_n; i += 32) {
            const int32_t id = key_id(W.res[i]);
            W.res[i] = make_key(exact_d2_lane(P.x32, P.dim_pad, id, qv), id);
        }
        __syncwarp();
    }
    for (int i = W.res_n + lane; i < P.kcap; i += 32) W.res[i] = kEmptyKey;
    __syncwarp();
    for (int size = 2; P.rerank && size <= P.kcap; size <<= 1) {
        for (int stride = size >> 1; stride; stride >>= 1) {
            for (int t = lane; t < P.kcap / 2; t += 32) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t a = W.res[lo], b = W.res[hi];
                if ((a > b) == up) { W.res[lo] = b; W.res[hi] = a; }
            }
            __syncwarp();
        }
    }
    for (int i = lane; i < P.k; i += 32) {
        const uint64_t v = i < W.res_n ? W.res[i] : kEmptyKey;
        const bool ok = i < W.res_n;
        P.ids[(int64_t)q * P.k + i] = ok ? key_id(v) : -1;
        P.dists[(int64_t)q * P.k + i] = ok ? sqrtf(key_d2(v)) : __int_as_float(0x7f800000);
    }
    if (lane == 0) {
        if (P.status) P.status[q] = status;
        if (P.trace) {
            P.trace[4 * (int64_t)q + 0] = W.hops;
            P.trace[4 * (int64_t)q + 1] = W.evals;
            P.trace[4 * (int64_t)q + 2] = W.pool_hw;
            P.trace[4 * (int64_t)q + 3] = tier;
        }
    }
}

// One query. Returns false if the fast tier overflowed (nothing written).
template <class Rows, int G, int CPL, bool DEVICE_TIER>
__device__ bool run_query(const Params& P, WarpState& W, int q, float* qv_smem, int tier, int lane) {
    Engine<Rows, G, CPL> eng;
    const int32_t seed = P.explore ? P.seeds[q] : (P.seeds ? P.seeds[q] : P.entry);
    const bool seed_ok = seed >= 0 && seed < P.n;
    const float* qsrc = P.explore ? P.x32 + (int64_t)(seed_ok ? seed : 0) * P.dim_pad : P.queries + (int64_t)q * P.dim;
    const int dim4 = (P.dim + 3) / 4 * 4;
    for (int i = lane; i < dim4; i += 32) qv_smem[i] = i < P.dim ? qsrc[i] : 0.f;
    __syncwarp();
    if (seed < 0 || seed >= P.n) {                                  // bad seed / vertex id
        W.res_n = 0;
        W.hops = W.evals = W.pool_hw = 0;
        finish_query(P, W, q, qv_smem, DEG_EINVAL, tier, lane);
        return true;
    }
    eng.load_query(qv_smem, P.dim, lane);

    // C <- {}: clear the visited structure.
    if (DEVICE_TIER) {
        uint4* b4 = reinterpret_cast<uint4*>(W.bitmap);
        for (int64_t i = lane; i < P.words / 4; i += 32) b4[i] = make_uint4(0, 0, 0, 0);
    } else {
        uint4* h4 = reinterpret_cast<uint4*>(W.hash);
        for (int i = lane; i < P.hcap / 4; i += 32) h4[i] = make_uint4(kEmptySlot, kEmptySlot, kEmptySlot, kEmptySlot);
    }
    W.pool_n = W.res_n = 0;
    W.trimmed = false;
    W.r2 = __int_as_float(0x7f800000);
    W.hops = W.evals = W.pool_hw = 0;
    __syncwarp();

    // Seed: S = {seed}, C = {seed}, R = {seed} (plain) or {} (exploration).
    if (lane == 0) W.cid[0] = seed;
    __syncwarp();
    eng.distances(P, W.cid, W.cd2, 1, lane);
    if (lane == 0) {
        if (DEVICE_TIER) visit_bitmap(W.bitmap, seed);
        else visit_hash(W.hash, P.hcap, P.hshift, seed);
    }
    __syncwarp();
    const uint64_t seed_key = make_key(W.cd2[0], seed);
    if (lane == 0) W.pool[0] = seed_key;
    W.pool_n = 1;
    W.pool_hw = 1;
    W.evals = 1;
    if (!P.explore) result_insert(W, P.ks, seed_key, lane);
    __syncwarp();

    const float inf = __int_as_float(0x7f800000);
    int status = DEG_OK;
    const int hlimit = P.hcap - P.hcap / 4;
    while (W.pool_n > 0) {
        // 1. pop argmin (distance, id) of S
        uint64_t best = kEmptyKey;
        int pos = 0;
        for (int i = lane; i < W.pool_n; i += 32) {
            const uint64_t v = W.pool[i];
            if (v < best) { best = v; pos = i; }
        }
        const uint64_t m = warp_min64(best);
        const unsigned who = __ballot_sync(0xffffffffu, best == m);
        pos = __shfl_sync(0xffffffffu, pos, __ffs(who) - 1);
        const float thr = W.trimmed ? W.r2 * P.f : inf;
        if (key_d2(m) > thr) break;                                 // too far: return R
        if (P.max_hops && W.hops >= P.max_hops) { status = DEG_EHOPLIMIT; break; }
        __syncwarp();
        if (lane == 0) W.pool[pos] = W.pool[W.pool_n - 1];
        --W.pool_n;
        ++W.hops;
        const int32_t s = key_id(m);

        // 2. N(G, s) \ C, then C <- C u N
        if (!DEVICE_TIER && W.evals + P.degree > hlimit) return false;
        int cnt = 0;
        for (int j0 = 0; j0 < P.degree; j0 += 32) {
            const int j = j0 + lane;
            const int32_t nb = j < P.degree ? __ldg(P.adj + (int64_t)s * P.deg_pad + j) : -1;
            int isnew = 0;
            if (nb >= 0) isnew = DEVICE_TIER ? visit_bitmap(W.bitmap, nb) : visit_hash(W.hash, P.hcap, P.hshift, nb);
            if (__any_sync(0xffffffffu, isnew < 0)) return false;
            const unsigned nm = __ballot_sync(0xffffffffu, isnew > 0);
            if (isnew > 0) W.cid[cnt + __popc(nm & ((1u << lane) - 1))] = nb;
            cnt += __popc(nm);
        }
        __syncwarp();
        if (cnt == 0) continue;
        W.evals += cnt;

        // 3. squared distances of the unvisited neighbours
        eng.distances(P, W.cid, W.cd2, cnt, lane);
        __syncwarp();

        // 4. admit against the radius from before the hop
        const float r2pre = W.trimmed ? W.r2 : inf;
        const float thrpre = W.trimmed ? W.r2 * P.f : inf;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            const bool valid = i < cnt;
            const float d2 = valid ? W.cd2[i] : inf;
            const int32_t id = valid ? W.cid[i] : -1;
            const uint64_t key = make_key(d2, id);
            const bool toS = valid && d2 <= thrpre;
            unsigned sm = __ballot_sync(0xffffffffu, toS);
            if (sm) {
                if (W.pool_n + __popc(sm) > W.pcap) {
                    W.pool_n = pool_compact(W, W.trimmed ? W.r2 * P.f : inf, lane);
                    if (W.pool_n + __popc(sm) > W.pcap) {
                        if (!DEVICE_TIER) return false;
                    }
                }
                if (toS) {
                    W.pool[W.pool_n + __popc(sm & ((1u << lane) - 1))] = key;
                    // its adjacency row is read if it is ever expanded: start pulling it into L2
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(P.adj + (int64_t)id * P.deg_pad));
                }
                W.pool_n += __popc(sm);
                W.pool_hw = max(W.pool_hw, W.pool_n);
            }
            unsigned rm = __ballot_sync(0xffffffffu, valid && d2 <= r2pre);
            __syncwarp();
            while (rm) {
                const int src = __ffs(rm) - 1;
                rm &= rm - 1;
                const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(key >> 32), src);
                const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)key, src);
                const uint64_t c = ((uint64_t)hi << 32) | lo;
                result_insert(W, P.ks, c, lane);
            }
        }
        __syncwarp();
    }
    finish_query(P, W, q, qv_smem, status, tier, lane);
    return true;
}

// Shared-memory bytes per warp of the fast tier.
__host__ __device__ inline int64_t fast_warp_bytes(int hcap, int pcap, int kcap, int dim) {
    const int64_t b = 4ll * hcap + 8ll * pcap + 8ll * kcap + (4 + 4) * kMaxDegree + 4ll * ((dim + 3) / 4 * 4);
    return (b + 15) / 16 * 16;
}

template <class Rows, int G, int CPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) search_fast_kernel(Params P) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t wb = fast_warp_bytes(P.hcap, P.pcap, P.kcap, P.dim);
    uint8_t* base = smem + warp * wb;
    WarpState W;
    W.hash = reinterpret_cast<uint32_t*>(base);
    W.pool = reinterpret_cast<uint64_t*>(base + 4ll * P.hcap);
    W.res = W.pool + P.pcap;
    W.cid = reinterpret_cast<int32_t*>(W.res + P.kcap);
    W.cd2 = reinterpret_cast<float*>(W.cid + kMaxDegree);
    float* qv = W.cd2 + kMaxDegree;
    W.bitmap = nullptr;
    const int slot = blockIdx.x * P.wpb + warp;
    uint64_t* const smem_pool = W.pool;
    for (;;) {
        int q = 0;
        if (lane == 0) q = atomicAdd(P.counters + 2, 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= P.nq) break;
        W.pool = smem_pool;
        W.pcap = P.pcap;
        bool done = run_query<Rows, G, CPL, false>(P, W, q, qv, 0, lane);
        if (!done && slot < P.islots) {
            // rerun in device-memory mode: bitmap C, larger pool in this warp's slot
            W.bitmap = P.ibitmaps + (int64_t)slot * P.words;
            W.pool = P.ipools + (int64_t)slot * P.ipcap;
            W.pcap = P.ipcap;
            done = run_query<Rows, G, CPL, true>(P, W, q, qv, 1, lane);
        }
        if (!done && lane == 0) P.overflow[atomicAdd(P.counters, 1)] = q;
        __syncwarp();
    }
}

template <class Rows, int G, int CPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) search_device_kernel(Params P, int slots) {
    __shared__ __align__(16) int32_t cid_s[kWarpsPerBlock][kMaxDegree];
    __shared__ __align__(16) float cd2_s[kWarpsPerBlock][kMaxDegree];
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = blockIdx.x * kWarpsPerBlock + warp;
    if (slot >= slots) return;
    float* qv = reinterpret_cast<float*>(smem) + warp * ((P.dim + 3) / 4 * 4);
    WarpState W;
    W.hash = nullptr;
    W.bitmap = P.bitmaps + slot * P.words;
    W.pool = P.pools + slot * (P.n + 1);
    W.res = P.results + (int64_t)slot * kMaxK;
    W.cid = cid_s[warp];
    W.cd2 = cd2_s[warp];
    W.pcap = (int32_t)(P.n + 1);
    const int count = *(volatile int32_t*)P.counters;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(P.counters + 1, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= count) break;
        run_query<Rows, G, CPL, true>(P, W, P.overflow[t], qv, 2, lane);
        __syncwarp();
    }
}

template <class Rows, int G, int CPL>
int launch_typed(Params P, Workspace& ws, cudaStream_t st, int64_t n, std::string* why) {
    cudaError_t e;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // Warps per block: as many (up to 4) as the per-warp state allows; shrink the visited table
    // if even one warp does not fit (queries beyond it finish in the device-memory kernel).
    int64_t wb = fast_warp_bytes(P.hcap, P.pcap, P.kcap, P.dim);
    while (wb > smem_max && P.hcap > 256) {
        P.hcap >>= 1;
        ++P.hshift;
        wb = fast_warp_bytes(P.hcap, P.pcap, P.kcap, P.dim);
    }
    if (wb > smem_max) return *why = "search state does not fit in shared memory", (int)cudaErrorInvalidValue;
    const int wpb = (int)std::min<int64_t>(kWarpsPerBlock, smem_max / wb);
    P.wpb = wpb;
    const int64_t smem = wb * wpb;
    auto fk = search_fast_kernel<Rows, G, CPL>;
    if ((e = cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) {
        *why = std::string("shared memory request too large: ") + cudaGetErrorString(e);
        return (int)e;
    }
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fk, wpb * 32, (size_t)smem)) != cudaSuccess)
        return *why = "occupancy query failed", (int)e;
    if (per_sm < 1) return *why = "search state does not fit in shared memory", (int)cudaErrorInvalidValue;
    const int64_t want = (P.nq + wpb - 1) / wpb;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * per_sm));
    if ((e = cudaMemsetAsync(P.counters, 0, 4 * sizeof(int32_t), st)) != cudaSuccess) return *why = "memset", (int)e;
    fk<<<grid, wpb * 32, smem, st>>>(P);
    if ((e = cudaGetLastError()) != cudaSuccess) return *why = std::string("fast kernel: ") + cudaGetErrorString(e), (int)e;
    auto dk = search_device_kernel<Rows, G, CPL>;
    const int64_t dsm = (int64_t)kWarpsPerBlock * ((P.dim + 3) / 4 * 4) * 4;
    if ((e = cudaFuncSetAttribute(dk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm)) != cudaSuccess)
        return *why = "device kernel attribute", (int)e;
    const int dgrid = (ws.slots + kWarpsPerBlock - 1) / kWarpsPerBlock;
    dk<<<dgrid, kWarpsPerBlock * 32, dsm, st>>>(P, ws.slots);
    if ((e = cudaGetLastError()) != cudaSuccess) return *why = std::string("device kernel: ") + cudaGetErrorString(e), (int)e;
    (void)n;
    return 0;
}

template <class Rows>
int dispatch_shape(Params P, Workspace& ws, cudaStream_t st, int64_t n, std::string* why) {
    const int nc = P.nchunk;
    if (nc <= 4) return launch_typed<Rows, 4, 1>(P, ws, st, n, why);
    if (nc <= 8) return launch_typed<Rows, 8, 1>(P, ws, st, n, why);
    if (nc <= 16) return launch_typed<Rows, 16, 1>(P, ws, st, n, why);
    if (nc <= 32) return launch_typed<Rows, 32, 1>(P, ws, st, n, why);
    if (nc <= 64) return launch_typed<Rows, 32, 2>(P, ws, st, n, why);
    if (nc <= 128) return launch_typed<Rows, 32, 4>(P, ws, st, n, why);
    if (nc <= 256) return launch_typed<Rows, 32, 8>(P, ws, st, n, why);
    *why = "row too wide (at most 4096 bytes)";
    return (int)cudaErrorInvalidValue;
}

int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

int workspace_reserve(Workspace& ws, const DeviceIndex& ix, int64_t nq, std::string* why) {
    cudaError_t e;
    if (!ws.counters) {
        if ((e = cudaMalloc(&ws.counters, 4 * sizeof(int32_t))) != cudaSuccess) return *why = "counters", (int)e;
    }
    if (ws.cap_q < nq) {
        cudaFree(ws.overflow);
        ws.overflow = nullptr;
        ws.cap_q = 0;
        if ((e = cudaMalloc(&ws.overflow, sizeof(int32_t) * nq)) != cudaSuccess) return *why = "overflow list", (int)e;
        ws.cap_q = nq;
    }
    if (!ws.pools) {
        // Second kernel: a bitmap of n bits, a pool of n + 1 keys and 1024 result keys per slot.
        const int64_t words = (ix.n + 127) / 128 * 4;
        const int64_t per_slot = words * 4 + 8 * (ix.n + 1) + 8 * kMaxK;
        int64_t slots = (1ll << 30) / per_slot;     // about 1 GiB of scratch
        slots = std::max<int64_t>(8, std::min<int64_t>(256, slots));
        slots = slots / kWarpsPerBlock * kWarpsPerBlock;
        // Device mode of the fast kernel: one slot per resident warp (up to 16 warps per SM),
        // a bitmap and a pool of kInlinePool keys each, within about 1.5 GiB.
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t iper = words * 4 + 8ll * kInlinePool;
        const int64_t islots = std::max<int64_t>(0, std::min<int64_t>((int64_t)sms * 16, (3ll << 29) / iper));
        if ((e = cudaMalloc(&ws.bitmaps, sizeof(uint32_t) * words * slots)) != cudaSuccess ||
            (e = cudaMalloc(&ws.pools, sizeof(uint64_t) * (ix.n + 1) * slots)) != cudaSuccess ||
            (e = cudaMalloc(&ws.results, sizeof(uint64_t) * kMaxK * slots)) != cudaSuccess ||
            (islots && (e = cudaMalloc(&ws.ibitmaps, sizeof(uint32_t) * words * islots)) != cudaSuccess) ||
            (islots && (e = cudaMalloc(&ws.ipools, sizeof(uint64_t) * kInlinePool * islots)) != cudaSuccess)) {
            workspace_free(ws);
            return *why = "device-memory scratch", (int)e;
        }
        ws.slots = (int32_t)slots;
        ws.words = words;
        ws.islots = (int32_t)islots;
        ws.ipcap = kInlinePool;
    }
    return 0;
}

void workspace_free(Workspace& ws) {
    cudaFree(ws.ibitmaps);
    cudaFree(ws.ipools);
    cudaFree(ws.counters);
    cudaFree(ws.overflow);
    cudaFree(ws.bitmaps);
    cudaFree(ws.pools);
    cudaFree(ws.results);
    cudaFree(ws.dq);
    cudaFree(ws.did);
    cudaFree(ws.dd);
    ws = Workspace{};
}

int launch_search(const SearchArgs& a, Workspace& ws, deg_stream_t stream, std::string* why) {
    const DeviceIndex& ix = *a.ix;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (ix.degree > kMaxDegree) return *why = "degree above 128", (int)cudaErrorInvalidValue;
    Params P{};
    P.x32 = ix.x32;
    P.dim_pad = ix.dim_pad;
    P.adj = ix.adj;
    P.degree = ix.degree;
    P.deg_pad = ix.deg_pad;
    P.n = ix.n;
    P.entry = ix.entry;
    P.queries = a.queries;
    P.dim = ix.dim;
    P.seeds = a.seeds;
    P.explore = a.explore;
    P.nq = (int32_t)a.nq;
    P.k = a.k;
    const bool reduced = a.precision != DEG_F32;
    P.ks = reduced && a.rerank ? std::max(a.rerank, a.k) : a.k;
    P.kcap = std::max(32, pow2_at_least(P.ks));
    P.rerank = reduced ? 1 : 0;
    const double f = (1.0 + (double)a.eps) * (1.0 + (double)a.eps);
    P.f = (float)f;
    P.max_hops = a.max_hops;
    // Fast-tier capacities: visited hash sized to the expected checked set, candidate pool.
    int hcap = a.visited_cap ? a.visited_cap : (P.ks <= 16 ? 4096 : P.ks <= 128 ? 8192 : 16384);
    hcap = std::max(hcap, pow2_at_least(4 * (ix.degree + 1)));
    int hs = 0;
    while ((1 << hs) < hcap) ++hs;
    P.hcap = hcap;
    P.hshift = 32 - hs;
    P.pcap = a.queue_cap ? std::max(a.queue_cap, 64) : std::max(1024, 2 * P.ks + 2 * ix.degree);
    P.pcap = (P.pcap + 31) / 32 * 32;
    P.ids = a.ids;
    P.dists = a.dists;
    P.status = a.status;
    P.trace = a.trace;
    P.counters = ws.counters;
    P.overflow = ws.overflow;
    P.bitmaps = ws.bitmaps;
    P.pools = ws.pools;
    P.results = ws.results;
    P.words = ws.words;
    P.ibitmaps = ws.ibitmaps;
    P.ipools = ws.ipools;
    P.islots = ws.islots;
    P.ipcap = ws.ipcap;
    if (a.precision == DEG_F32) {
        P.rows = reinterpret_cast<const uint8_t*>(ix.x32);
        P.row_bytes = 4ll * ix.dim_pad;
        P.nchunk = ix.dim_pad / 4;
        return dispatch_shape<F32Rows>(P, ws, st, ix.n, why);
    }
    if (a.precision == DEG_BF16) {
        P.rows = reinterpret_cast<const uint8_t*>(ix.xbf);
        P.row_bytes = 2ll * ix.dim_pad16;
        P.nchunk = ix.dim_pad16 / 8;
        return dispatch_shape<BF16Rows>(P, ws, st, ix.n, why);
    }
    P.rows = ix.x8;
    P.row_bytes = ix.dim_pad8;
    P.nchunk = ix.dim_pad8 / 16;
    P.scale8 = ix.scale8;
    return dispatch_shape<FP8Rows>(P, ws, st, ix.n, why);
}

}  // namespace deg
