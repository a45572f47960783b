// Batched range search (paper Alg. 1, Sec. 2.1) over a fixed-degree DEG, one warp per query.
//
// One hop of a query's warp:
//   1. pop the smallest (distance, id) of S; stop if it exceeds r(1+eps) (squared:
//      d2 > r2 (1+eps)^2);
//   2. read the adjacency row of the popped vertex (one coalesced load) and test-and-set every
//      neighbour in the visited bitmap C (one atomic per lane);
//   3. gather the rows of the unvisited neighbours with 16-byte loads, G lanes per row and up to
//      8 rows in flight, and reduce their squared distances with xor shuffles;
//   4. try every neighbour with d2 <= r2 for R (the radius from before the hop), keep the ks
//      smallest; then admit to S every neighbour with d2 <= r2 (1+eps)^2 for the radius after it.
// Evaluating a hop's neighbours together returns the same R, the same expansions and the same
// checked set as the one-by-one loop of Alg. 1: R is always the k smallest (distance, id) seen so
// far, and a candidate the one-by-one loop admits to S that the batch leaves out (it lies outside
// the radius after the hop) could only ever be popped to fail the stop test -- r never grows --
// and then the next key of S fails it too.
//
// Readings of Alg. 1 (as in the rest of the library): seeds count as checked; exploration
// queries search from their own vertex but never return it; r = +inf until R first exceeds k;
// (distance, id) orders S and R, the lower id first. The id in a key is the caller's id, so ties
// are broken exactly as Alg. 1 over the caller's numbering breaks them; the rows and the visited
// bitmap use internal ids (the locality layout), which the adjacency carries beside each caller id.
//
// State of one query. The checked set C is an n-bit bitmap in the warp's slot of device memory
// (cleared when the query starts). S is split in two: an unsorted "front" of at most F keys in
// shared memory, and a "back" pool of keys in the warp's device-memory slot, with a watermark w
// such that every front key < w <= every back key. So the front's minimum, found by a warp
// reduction, is the minimum of S. New candidates below w are appended to the front (the front's
// largest keys over F move to the back, and the smallest of them becomes the new w); those at or
// above w are appended to the back. When the front runs empty, it is refilled with the F
// smallest back keys, found exactly by an 8-bit-digit radix select over the 64-bit keys, and
// back keys above the current admission radius are dropped on the way (a candidate with
// d > r(1+eps) can never pass the stop test again, since r only shrinks). R is a sorted array
// in shared memory. A query whose back pool would overflow its slot is recorded in an overflow
// list and finished by a second kernel whose back pools have room for all n vertices; both
// kernels run the same code, so the result does not depend on which one finished the query.
#ifndef DEG_SEARCH_IMPL_CUH
#define DEG_SEARCH_IMPL_CUH

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "deg_internal.h"

namespace deg {
namespace sk {

constexpr int kWarpsPerBlock = 4;
#ifndef DEG_SEARCH_BLOCKS_PER_SM
#define DEG_SEARCH_BLOCKS_PER_SM 6
#endif
constexpr int kBlocksPerSM = DEG_SEARCH_BLOCKS_PER_SM;   // occupancy target: 24 warps per SM (85 registers)
constexpr uint64_t kEmptyKey = ~0ull;
constexpr int kMaxDegree = 128;
#ifndef DEG_SEARCH_FRONT
#define DEG_SEARCH_FRONT 128
#endif
#ifndef DEG_SEARCH_QUERY_IN_SMEM
#define DEG_SEARCH_QUERY_IN_SMEM 0
#endif
#ifndef DEG_SEARCH_ROW_PREFETCH_BYTES
#define DEG_SEARCH_ROW_PREFETCH_BYTES 256
#endif
constexpr int kFront = DEG_SEARCH_FRONT;  // sorted on-chip part of S (a power of two, >= 32)
constexpr int kBackPool = 32768;         // device-memory part of S in the main kernel
constexpr int kTouchCap = 8192;          // visited ids recorded per query for clearing C afterwards

// Key of a candidate: squared distance bits (non-negative floats order as unsigned integers) over
// the caller id of the vertex.
__device__ __forceinline__ uint64_t make_key(float d2, int32_t id) {
    return ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)id;
}
__device__ __forceinline__ float key_d2(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ int32_t key_id(uint64_t k) { return (int32_t)(uint32_t)k; }
__device__ __forceinline__ unsigned lanes_below(int lane) { return (1u << lane) - 1u; }

// (1 + eps)^2 as an unevaluated float sum hi + lo: Knuth's TwoSum for 1 + eps, then the square with
// its rounding error recovered by an FMA (Dekker's product). The error term err^2 is below 2^-46
// of hi and is dropped. Host code (the batch launch) and device code (the serving loop) run the
// same float operations, so both get the same pair for the same eps.
__host__ __device__ inline float2 eps_factor(float eps) {
    const float s = 1.f + eps;
    const float bb = s - 1.f;
    const float err = (1.f - (s - bb)) + (eps - bb);          // 1 + eps = s + err exactly
    const float p = s * s;
    const float pe = fmaf(s, s, -p);                          // s^2 = p + pe exactly
    return make_float2(p, fmaf(2.f * s, err, pe));
}

// The admission radius of Alg. 1, squared: d2 passes when d2 <= r2 (1 + eps)^2. The product is
// compared through hi + lo, so the test is exact to about 2^-46 of r2 instead of float32's
// rounding of r2 * (1 + eps)^2 (which differs from the real threshold by up to 2^-23 of it and
// could flip the test for an integer-valued distance next to it). r2 = +inf before the first trim.
struct Radius {
    float r2, hi, lo;
    __device__ __forceinline__ bool admits(float d2) const {
        return r2 == __int_as_float(0x7f800000) || fmaf(-r2, hi, d2) <= r2 * lo;
    }
};

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, src);
    const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
    for (int m = 16; m; m >>= 1) {
        const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
        const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
        v = min(v, ((uint64_t)hi << 32) | lo);
    }
    return v;
}

// ---- row storage formats ------------------------------------------------------------------
// A row is read as 16-byte chunks; each chunk holds EPC elements.
// Row formats. acc() folds one 16-byte chunk of a row into a lane's two partial sums (two
// independent FMA chains, even and odd elements, advanced together by paired float32
// instructions) and fin() turns the warp-reduced sum into the squared distance: float32 and bf16
// rows sum (q - x)^2 directly; FP8 rows sum q . x and expand ||q - s x||^2 = ||q||^2 - 2 s (q . x) +
// s^2 ||x||^2 with the row's s and s^2 ||x||^2 read from one float2 (one FMA per element instead
// of two).

// (a0, a1) += (x0, x1) * (y0, y1), and (a0, a1) += ((q0, q1) - (x0, x1))^2, each step one paired
// (.f32x2) instruction: per lane the same IEEE fma and subtraction as the scalar forms, so the sums
// are bit-identical to fmaf chains.
__device__ __forceinline__ void fma_pair(float& a0, float& a1, float x0, float x1, float y0, float y1) {
    unsigned long long a, x, y;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(x0), "f"(x1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(y0), "f"(y1));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a) : "l"(x), "l"(y));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(a));
}
__device__ __forceinline__ void sub_sq_pair(float& a0, float& a1, float q0, float q1, float x0, float x1) {
    unsigned long long a, q, x, t;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(q) : "f"(q0), "f"(q1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(x0), "f"(x1));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(q), "l"(x));
    asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(a) : "l"(t));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(a));
}

struct F32Rows {
    static constexpr int EPC = 4;
    __device__ static float2 scale(const float2*, int32_t) { return make_float2(1.f, 0.f); }
    __device__ static void acc(const uint4& c, const float* q, float& a0, float& a1) {
        sub_sq_pair(a0, a1, q[0], q[1], __uint_as_float(c.x), __uint_as_float(c.y));
        sub_sq_pair(a0, a1, q[2], q[3], __uint_as_float(c.z), __uint_as_float(c.w));
    }
    __device__ static float fin(float a, float2, float) { return a; }
};
struct BF16Rows {
    static constexpr int EPC = 8;
    __device__ static float2 scale(const float2*, int32_t) { return make_float2(1.f, 0.f); }
    __device__ static void acc(const uint4& c, const float* q, float& a0, float& a1) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            sub_sq_pair(a0, a1, q[2 * i], q[2 * i + 1], __uint_as_float(w[i] << 16), __uint_as_float(w[i] & 0xffff0000u));
    }
    __device__ static float fin(float a, float2, float) { return a; }
};
struct FP8Rows {
    static constexpr int EPC = 16;
    __device__ static float2 scale(const float2* sn, int32_t id) { return __ldg(sn + id); }
    __device__ static void acc(const uint4& c, const float* q, float& a0, float& a1) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w[i] >> (16 * h)) & 0xffffu);
                const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);  // exact
                const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
                fma_pair(a0, a1, q[4 * i + 2 * h], q[4 * i + 2 * h + 1], f.x, f.y);
            }
        }
    }
    // sn = {s, s^2 ||x||^2}; rounding can take a tiny true distance below zero: clamp
    __device__ static float fin(float dot, float2 sn, float qq) { return fmaxf(fmaf(-2.f * sn.x, dot, qq + sn.y), 0.f); }
};

struct Params {
    const uint8_t* rows;       // row base of the searched storage
    int64_t row_bytes;         // stride of that storage
    int32_t nchunk;            // 16-byte chunks per row
    const float2* norm8;       // FP8: per-row {scale s, s^2 ||x||^2}, or null
    const float* x32;          // float32 rows (exploration queries, re-rank)
    int32_t dim_pad;           // float32 row stride (elements)
    const int2* adj;           // [n][deg_pad] {internal id, caller id} of each neighbour, row = caller id
    int32_t degree, deg_pad;
    int64_t n;
    int32_t entry;             // internal id
    int32_t entry_caller;      // the same vertex's caller id
    const int32_t* old2new;    // caller id -> internal id
    const int32_t* new2old;    // internal id -> caller id
    const float* queries;
    int32_t dim;
    const int32_t* seeds;
    const int32_t* seeds2;     // a second seed per query (caller id, -1 = none), or null
    int32_t seeds_internal;    // 1: seeds are internal ids already (pivot routing)
    int32_t sorted_front;      // 1: keep S's front sorted (walks from the fixed entry vertex are long)
    const int32_t* order;      // work order of the main kernel (queries far from their pivot first), or null
    int32_t explore;
    int32_t nq;
    int32_t k;                 // results returned
    int32_t ks;                // results kept during the search (k, or the re-rank width)
    int32_t kcap;              // power of two >= ks (sort width of a re-rank)
    int32_t rerank;            // 1: re-rank R on float32 rows before output
    float f, f_lo;             // (1 + eps)^2 = f + f_lo (eps_factor)
    int32_t max_hops;
    int32_t wpb;               // warps per block
    // learned early stop (not in the paper): network weights, decision margin, trace recording
    const __nv_bfloat16* stop_w;   // inference layout (mlp.cu), or null
    float stop_logit;
    int32_t learned;           // 1: stop when the network's margin exceeds stop_logit
    float* rec_feats;          // training traces: [nq][rec_cap][kStopFeatures], or null
    int32_t* rec_labels;
    int32_t* rec_counts;
    int32_t rec_cap;
    // outputs
    int32_t* ids;
    float* dists;
    int32_t* status;
    int32_t* trace;
    // workspace
    int32_t* counters;         // [0] overflow count, [1] second-kernel cursor, [2] main cursor
    int32_t* overflow;
    int64_t words;             // 32-bit words of one visited bitmap (multiple of 4)
    uint32_t* bitmaps;         // main kernel: [slots][words], all zero between queries
    uint64_t* backs;           //   [slots][bstride]
    int32_t* touched;          //   [slots][kTouchCap] ids set in the bitmap by the running query
    int32_t slots, bcap, bstride;
    uint32_t* pbitmaps;        // second kernel: [pslots][words]
    uint64_t* pbacks;          //   [pslots][n + 1]
    int32_t pslots;
};

// Per-warp search state. Scalar members are warp-uniform (every lane holds the same value).
struct WarpState {
    uint32_t* bitmap;          // C
    int32_t* touched;          // ids visited by this query (main and serving kernels), or null
    int32_t tn;                // their number (above kTouchCap: clear the whole bitmap)
    uint64_t* fbuf;            // 32 keys of scratch for batched admission
    uint64_t* front;           // S, smallest part: unsorted [kFront + 32], or sorted descending [kFront]
    uint64_t* front2;          // sorted mode: the other front buffer (a merge writes it, then they swap)
    bool sorted;               // the front is kept sorted (long walks) or unsorted (short ones)
    uint64_t* back;            // S, the rest (device memory), [bcap]
    uint64_t* res;             // R, sorted ascending
    int32_t* cid;              // per-hop candidate internal ids [kMaxDegree] (also the refill histogram)
    float* cd2;                // per-hop candidate distances [kMaxDegree]
    int32_t* ccid;             // per-hop candidate caller ids [kMaxDegree]
    int32_t bcap;
    int32_t fn, back_n, res_n;
    uint64_t wmark;            // every front key < wmark <= every back key
    bool trimmed;
    float r2;
    int32_t hops, evals, peak;
    // for the learned stop's features
    int32_t last_change, evals_change;   // hop and evaluation count of the last change of the top k of R
    int32_t hop_rins;                    // insertions into R this hop
    float r2_first;
};

template <class Rows, int G, int CPL>
struct Engine {
    static constexpr int EPC = Rows::EPC;
    static constexpr int RP = 32 / G;                                      // rows per pass
    // rows in flight per warp: up to 16 FP8 rows with at most 4 chunks buffered per lane (16 rows
    // of 128 bytes), else up to 8 rows with at most 8 chunks per lane
    static constexpr int kRows = EPC == 16 ? 16 : 8, kBuf = EPC == 16 ? 4 : 8;
    static constexpr int UR = kRows / RP > 0 ? kRows / RP : 1;             // passes for kRows rows
    static constexpr int UC = kBuf / CPL > 0 ? kBuf / CPL : 1;             // register cap
    static constexpr int U = UR < UC ? UR : UC;                            // passes in flight
#if DEG_SEARCH_QUERY_IN_SMEM
    const float* qs;                                                       // the query in shared memory
#else
    float q[CPL][EPC];
#endif
    float qq;                                                              // ||q||^2 (FP8 expansion)

    // qv: the query in shared memory, zero padded to a multiple of 16 floats
    __device__ void load_query(const float* qv, int dim, int lane) {
        const int p = lane % G;
        float s = 0.f;
#if DEG_SEARCH_QUERY_IN_SMEM
        qs = qv;
#endif
#pragma unroll
        for (int j = 0; j < CPL; ++j)
#pragma unroll
            for (int e = 0; e < EPC; ++e) {
                const int i = (p + G * j) * EPC + e;
                const float v = i < dim ? qv[i] : 0.f;
#if !DEG_SEARCH_QUERY_IN_SMEM
                q[j][e] = v;
#endif
                s = fmaf(v, v, s);
            }
#pragma unroll
        for (int m = G / 2; m; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);  // one lane group holds all of q
        qq = s;
    }

    // Squared distances of cid[0..cnt) into cd2[0..cnt).
    __device__ void distances(const Params& P, const int32_t* cid, float* cd2, int cnt, int lane) const {
        const int g = lane / G, p = lane % G;
        for (int i0 = 0; i0 < cnt; i0 += RP * U) {
            uint4 buf[U][CPL];
            float2 sc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * RP + g;
                sc[u] = make_float2(1.f, 0.f);
#pragma unroll
                for (int j = 0; j < CPL; ++j) buf[u][j] = make_uint4(0, 0, 0, 0);
                if (i < cnt) {
                    const int32_t id = cid[i];
                    const uint8_t* row = P.rows + (int64_t)id * P.row_bytes;
                    sc[u] = Rows::scale(P.norm8, id);
#pragma unroll
                    for (int j = 0; j < CPL; ++j) {
                        const int c = p + G * j;
                        if (c < P.nchunk) buf[u][j] = __ldg(reinterpret_cast<const uint4*>(row) + c);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (i0 + u * RP < cnt) {                              // warp-uniform
                    float a0 = 0.f, a1 = 0.f;
#pragma unroll
                    for (int j = 0; j < CPL; ++j)
                        if (p + G * j < P.nchunk) {
#if DEG_SEARCH_QUERY_IN_SMEM
                            float qr[EPC];
                            const float4* q4 = reinterpret_cast<const float4*>(qs + (p + G * j) * EPC);
#pragma unroll
                            for (int e = 0; e < EPC / 4; ++e) {
                                const float4 t = q4[e];
                                qr[4 * e] = t.x;
                                qr[4 * e + 1] = t.y;
                                qr[4 * e + 2] = t.z;
                                qr[4 * e + 3] = t.w;
                            }
                            Rows::acc(buf[u][j], qr, a0, a1);
#else
                            Rows::acc(buf[u][j], q[j], a0, a1);
#endif
                        }
                    float a = a0 + a1;
#pragma unroll
                    for (int m = G / 2; m; m >>= 1) a += __shfl_xor_sync(0xffffffffu, a, m);
                    const int i = i0 + u * RP + g;
                    if (p == 0 && i < cnt) cd2[i] = Rows::fin(a, sc[u], qq);
                }
            }
        }
    }
};

// Exact float32 squared distance of one row (re-rank), one lane; rows are zero padded to a
// multiple of 4 floats and the query in shared memory likewise.
inline __device__ float exact_d2_lane(const float* x32, int32_t dim_pad, int32_t id, const float* qv) {
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

// Test-and-set of vertex id in C: 1 if it was not checked yet.
__device__ __forceinline__ int visit(uint32_t* bm, int32_t id) {
    const uint32_t bit = 1u << (id & 31);
    return (atomicOr(bm + (id >> 5), bit) & bit) ? 0 : 1;
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
        const int last = full ? ks - 1 : W.res_n;             // shift [pos, last) up by one
        for (int c0 = pos + ((last - 1 - pos) / 32) * 32; last > pos && c0 >= pos; c0 -= 32) {
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
    if (!full || pos < ks) {
        W.last_change = W.hops;
        W.evals_change = W.evals;
        ++W.hop_rins;
    }
    if (full) {
        if (!W.trimmed) W.r2_first = key_d2(W.res[ks - 1]);
        W.trimmed = true;
        W.r2 = key_d2(W.res[ks - 1]);
    }
}

// The front of S is unsorted: its minimum (the next pop) and its maximum (the key to evict) are
// found by a warp reduction. Keys are unique (a vertex enters S at most once), so the extreme key
// names its slot. fn > 0.
__device__ __forceinline__ int front_extreme(const WarpState& W, bool want_max, uint64_t* out, int lane) {
    uint64_t best = want_max ? 0ull : kEmptyKey;
    int bi = -1;
    for (int i = lane; i < W.fn; i += 32) {
        const uint64_t v = W.front[i];
        if (want_max ? v >= best : v <= best) {
            best = v;
            bi = i;
        }
    }
    uint64_t m = best;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)m, o);
        const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(m >> 32), o);
        const uint64_t t = ((uint64_t)hi << 32) | lo;
        m = want_max ? max(m, t) : min(m, t);
    }
    const unsigned own = __ballot_sync(0xffffffffu, bi >= 0 && best == m);
    *out = m;
    return __shfl_sync(0xffffffffu, bi, __ffs(own) - 1);
}

// ---- learned early stop -------------------------------------------------------------------
// Twelve warp-uniform features of the search state after a hop (the same code makes the
// training traces and feeds the network during a search).
__device__ __forceinline__ float stop_feature(const WarpState& W, int i, float d2_pop, int cnt, int adm, float f, int lane) {
    const float inf = __int_as_float(0x7f800000);
    switch (i) {
        case 0: return W.hops * (1.f / 64.f);
        case 1: return W.evals * (1.f / 1024.f);
        case 2: return log2f(1.f + (float)(W.fn + W.back_n)) * (1.f / 16.f);
        case 3: return W.trimmed ? 1.f : 0.f;
        case 4: return W.trimmed ? d2_pop / W.r2 : 0.f;
        case 5: {
            if (!W.trimmed) return 0.f;
            uint64_t fmin = kEmptyKey;
            if (W.fn > 0) {
                if (W.sorted) fmin = W.front[W.fn - 1];
                else front_extreme(W, false, &fmin, lane);
            }
            const float nxt = W.fn > 0 ? key_d2(fmin) : (W.back_n > 0 ? key_d2(W.wmark) : inf);
            return fminf(nxt / (W.r2 * f), 4.f);
        }
        case 6: return fminf((float)(W.hops - W.last_change), 256.f) * (1.f / 16.f);
        case 7: return W.hop_rins * 0.25f;
        case 8: return adm * 0.125f;
        case 9: return cnt * (1.f / 32.f);
        case 10: return W.trimmed ? W.r2 / W.r2_first : 1.f;
        default: return fminf((float)(W.evals - W.evals_change), 4096.f) * (1.f / 256.f);
    }
}

// logit(stop) - logit(continue) of the 12-64-64-2 network; bfloat16 weights in shared memory,
// inference layout W1t [12][64], b1, W2t [64][64], b2, W3 [2][64], b3. Warp-cooperative.
inline __device__ float stop_margin(const __nv_bfloat16* w, const float* x, int lane) {
    const __nv_bfloat16* W1t = w;
    const __nv_bfloat16* b1 = W1t + 12 * 64;
    const __nv_bfloat16* W2t = b1 + 64;
    const __nv_bfloat16* b2 = W2t + 64 * 64;
    const __nv_bfloat16* W3 = b2 + 64;
    const __nv_bfloat16* b3 = W3 + 2 * 64;
    float a0 = __bfloat162float(b1[lane]), a1 = __bfloat162float(b1[lane + 32]);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        a0 = fmaf(__bfloat162float(W1t[i * 64 + lane]), x[i], a0);
        a1 = fmaf(__bfloat162float(W1t[i * 64 + lane + 32]), x[i], a1);
    }
    a0 = fmaxf(a0, 0.f);
    a1 = fmaxf(a1, 0.f);
    float c0 = __bfloat162float(b2[lane]), c1 = __bfloat162float(b2[lane + 32]);
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
        const float v = __shfl_sync(0xffffffffu, a0, i);
        c0 = fmaf(__bfloat162float(W2t[i * 64 + lane]), v, c0);
        c1 = fmaf(__bfloat162float(W2t[i * 64 + lane + 32]), v, c1);
    }
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
        const float v = __shfl_sync(0xffffffffu, a1, i);
        c0 = fmaf(__bfloat162float(W2t[(32 + i) * 64 + lane]), v, c0);
        c1 = fmaf(__bfloat162float(W2t[(32 + i) * 64 + lane + 32]), v, c1);
    }
    c0 = fmaxf(c0, 0.f);
    c1 = fmaxf(c1, 0.f);
    float p = (__bfloat162float(W3[64 + lane]) - __bfloat162float(W3[lane])) * c0 +
              (__bfloat162float(W3[64 + lane + 32]) - __bfloat162float(W3[lane + 32])) * c1;
#pragma unroll
    for (int m = 16; m; m >>= 1) p += __shfl_xor_sync(0xffffffffu, p, m);
    return p + __bfloat162float(b3[1]) - __bfloat162float(b3[0]);
}

// Append to the back pool; on a full pool drop keys outside the radius first. False if still full.
__device__ __forceinline__ bool back_push(WarpState& W, uint64_t c, const Radius& thr, int lane) {
    if (W.back_n == W.bcap) {
        int out = 0;
        for (int i0 = 0; i0 < W.back_n; i0 += 32) {
            const int i = i0 + lane;
            const uint64_t v = i < W.back_n ? W.back[i] : kEmptyKey;
            const bool keep = i < W.back_n && thr.admits(key_d2(v));
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep) W.back[out + __popc(m & lanes_below(lane))] = v;
            out += __popc(m);
            __syncwarp();
        }
        W.back_n = out;
        if (W.back_n == W.bcap) return false;
    }
    if (lane == 0) W.back[W.back_n] = c;
    ++W.back_n;
    return true;
}

// Move front keys to the back pool, largest first, until the front holds kFront keys; wmark
// follows the smallest evicted key, so every front key < wmark <= every back key still holds.
// False if the back pool overflowed.
__device__ __forceinline__ bool trim_front(WarpState& W, const Radius& thr, int lane) {
    while (W.fn > kFront) {
        uint64_t kmax;
        const int i = front_extreme(W, true, &kmax, lane);
        __syncwarp();
        if (lane == 0) W.front[i] = W.front[W.fn - 1];
        --W.fn;
        __syncwarp();
        W.wmark = min(W.wmark, kmax);
        if (!back_push(W, kmax, thr, lane)) return false;
    }
    return true;
}

// Add candidate c (admitted to S). False if the back pool overflowed.
__device__ __forceinline__ bool s_insert(WarpState& W, uint64_t c, const Radius& thr, int lane) {
    if (c >= W.wmark) return back_push(W, c, thr, lane);
    if (lane == 0) W.front[W.fn] = c;
    ++W.fn;
    __syncwarp();
    return trim_front(W, thr, lane);
}

// Admit a batch of candidates (one per lane, where `take`) to S at once: keys below wmark are
// appended to the front, the others to the back pool, then the front's largest keys over its
// capacity move to the back pool. S ends as the same set as after one-by-one insertion and pops
// take its minimum, so pops are unchanged. A batch that could overflow the back pool takes the
// one-by-one path (which compacts the pool). False if the pool overflowed.
inline __device__ bool admit_batch(WarpState& W, uint64_t key, bool take, const Radius& thr, int lane) {
    const unsigned all = __ballot_sync(0xffffffffu, take);
    if (!all) return true;
    const bool toF = take && key < W.wmark;
    const unsigned mf = __ballot_sync(0xffffffffu, toF), mb = all & ~mf;
    const int m = __popc(mf), nb = __popc(mb);
    if (W.back_n + nb + m > W.bcap) {
        unsigned rest = all;
        while (rest) {
            const int src = __ffs(rest) - 1;
            rest &= rest - 1;
            if (!s_insert(W, shfl64(key, src), thr, lane)) return false;
        }
        return true;
    }
    if (take && !toF) W.back[W.back_n + __popc(mb & lanes_below(lane))] = key;
    if (toF) W.front[W.fn + __popc(mf & lanes_below(lane))] = key;
    W.back_n += nb;
    W.fn += m;
    __syncwarp();
    return trim_front(W, thr, lane);
}

// ---- the sorted front (for long walks) ----------------------------------------------------------
// The same S kept with its front sorted descending in two buffers: a pop reads the front's last
// key, and a batch is merged in by rank. Cheaper than the unsorted front when S is large and pops
// are many (walks from the fixed entry vertex: about 1,500 hops), dearer for short walks.
// Add candidate c (admitted to S). False if the back pool overflowed.
__device__ __forceinline__ bool s_insert_sorted(WarpState& W, uint64_t c, const Radius& thr, int lane) {
    if (c >= W.wmark) return back_push(W, c, thr, lane);
    // position in the descending front: number of keys greater than c
    int pos = 0;
    for (int i0 = 0; i0 < W.fn; i0 += 32) {
        const int i = i0 + lane;
        pos += __popc(__ballot_sync(0xffffffffu, i < W.fn && W.front[i] > c));
    }
    if (W.fn < kFront) {
        // shift [pos, fn) up by one, top chunk first
        for (int c0 = pos + ((W.fn - 1 - pos) / 32) * 32; W.fn > pos && c0 >= pos; c0 -= 32) {
            const int i = c0 + lane;
            const uint64_t v = i < W.fn ? W.front[i] : 0;
            __syncwarp();
            if (i < W.fn) W.front[i + 1] = v;
            __syncwarp();
        }
        if (lane == 0) W.front[pos] = c;
        ++W.fn;
        __syncwarp();
        return true;
    }
    if (pos == 0) {                                           // c above every front key
        W.wmark = c;
        return back_push(W, c, thr, lane);
    }
    // full: evict the largest key front[0] to the back, shift [1, pos) down, place c at pos-1
    const uint64_t evicted = W.front[0];
    for (int c0 = 1; c0 < pos; c0 += 32) {
        const int i = c0 + lane;
        const uint64_t v = i < pos ? W.front[i] : 0;
        __syncwarp();
        if (i < pos) W.front[i - 1] = v;
        __syncwarp();
    }
    if (lane == 0) W.front[pos - 1] = c;
    __syncwarp();
    W.wmark = evicted;
    return back_push(W, evicted, thr, lane);
}

// Admit a batch of candidates (one per lane, where `take`) to S at once: merge them with the
// sorted front, the largest overflow keys go to the back pool, and wmark becomes the smallest of
// those. S ends as the same set as after one-by-one insertion, and every front key stays below
// wmark <= every back key, so pops are unchanged. A batch that would overflow the back pool takes
// the one-by-one path (which compacts the pool). False if the pool overflowed.
inline __device__ bool admit_batch_sorted(WarpState& W, uint64_t key, bool take, const Radius& thr, int lane) {
    const unsigned all = __ballot_sync(0xffffffffu, take);
    if (!all) return true;
    const bool toF = take && key < W.wmark;
    const unsigned mf = __ballot_sync(0xffffffffu, toF), mb = all & ~mf;
    const int m = __popc(mf), nb = __popc(mb), fn = W.fn;
    const int E = max(0, fn + m - kFront);                    // evicted: the E largest of the merge
    if (W.back_n + nb + E > W.bcap) {
        unsigned rest = all;
        while (rest) {
            const int src = __ffs(rest) - 1;
            rest &= rest - 1;
            if (!s_insert_sorted(W, shfl64(key, src), thr, lane)) return false;
        }
        return true;
    }
    if (take && !toF) W.back[W.back_n + __popc(mb & lanes_below(lane))] = key;
    if (m > 0) {
        uint64_t* fb = W.fbuf;
        if (toF) fb[__popc(mf & lanes_below(lane))] = key;
        __syncwarp();
        int knew = -1;                                        // merged (descending) index of key
        if (toF) {
            int r = 0;
            for (int j = 0; j < m; ++j) r += fb[j] > key;
            int lo = 0;                                       // front keys above key (fixed steps)
#pragma unroll
            for (int step = kFront; step; step >>= 1)
                if (lo + step <= fn && W.front[lo + step - 1] > key) lo += step;
            knew = r + lo;
        }
        // the merge goes to the second buffer (the first is still read), which then becomes the front.
        // The new keys' merged indices, as a bit mask one 32-index word at a time, place the front
        // keys: merged index p that no new key holds takes front key p - (new keys below p).
        const int64_t ev0 = W.back_n + nb;                    // evicted keys land after the direct ones
        const int total = fn + m;                             // <= kFront + 32
        uint64_t last = kEmptyKey;                            // merged index E - 1: the new wmark
        uint64_t* dst = W.front2;
        int below = 0;                                        // new keys at merged indices under word c
#pragma unroll
        for (int c = 0; c < kFront / 32 + 1; ++c) {
            if (32 * c >= total) break;                       // warp-uniform
            const unsigned word = __reduce_or_sync(0xffffffffu, (knew >> 5) == c ? 1u << (knew & 31) : 0u);
            const int p = 32 * c + lane;
            if (p < total && !((word >> lane) & 1u)) {
                const uint64_t v = W.front[p - below - __popc(word & lanes_below(lane))];
                if (p >= E) dst[p - E] = v;
                else W.back[ev0 + p] = v;
                if (p == E - 1) last = v;
            }
            below += __popc(word);
        }
        if (knew >= E) dst[knew - E] = key;
        else if (knew >= 0) W.back[ev0 + knew] = key;
        if (toF && knew == E - 1) last = key;
        if (E > 0) W.wmark = warp_min64(last);
        W.front2 = W.front;
        W.front = dst;
    }
    W.fn = fn + m - E;
    W.back_n += nb + E;
    __syncwarp();
    return true;
}

// Add a batch of result candidates (one per lane, where `take`) to R, sorted ascending: merge,
// keep the ks smallest. The same R, radius and trim as one-by-one insertion (Alg. 1 admits them
// all against the radius from before the hop). For the learned stop, a key landing among the
// first k (the results returned) marks this hop as the last change of the top k.
inline __device__ void result_batch(WarpState& W, int ks, int k, uint64_t key, bool take, int lane) {
    const unsigned mr = __ballot_sync(0xffffffffu, take);
    if (!mr) return;
    const int m = __popc(mr), rn = W.res_n;
    uint64_t* fb = W.fbuf;
    if (take) fb[__popc(mr & lanes_below(lane))] = key;
    __syncwarp();
    int knew = -1;
    if (take) {
        int r = 0;
        for (int j = 0; j < m; ++j) r += fb[j] < key;
        int lo = 0;                                           // R keys below key (warp-uniform steps)
        for (int step = rn > 0 ? 1 << (31 - __clz(rn)) : 0; step; step >>= 1)
            if (lo + step <= rn && W.res[lo + step - 1] < key) lo += step;
        knew = r + lo;
    }
    // existing keys fill the merged indices (below ks) that no new key holds, in order: index p
    // takes R key p - (new keys below p). Top word first, all reads of a word before its writes.
    const int total = min(rn + m, ks);
    for (int c = (total - 1) >> 5; c >= 0; --c) {
        const unsigned word = __reduce_or_sync(0xffffffffu, (knew >> 5) == c ? 1u << (knew & 31) : 0u);
        const int below = __popc(__ballot_sync(0xffffffffu, knew >= 0 && knew < 32 * c));
        const int p = 32 * c + lane;
        const bool mine = p < total && !((word >> lane) & 1u);
        uint64_t v = 0;
        if (mine) v = W.res[p - below - __popc(word & lanes_below(lane))];
        __syncwarp();
        if (mine) W.res[p] = v;
        __syncwarp();
    }
    if (knew >= 0 && knew < ks) W.res[knew] = key;
    const int added = __popc(__ballot_sync(0xffffffffu, knew >= 0 && knew < ks));
    const bool top = __any_sync(0xffffffffu, knew >= 0 && knew < k);
    W.res_n = min(rn + m, ks);
    __syncwarp();
    W.hop_rins += added;
    if (top) {
        W.last_change = W.hops;
        W.evals_change = W.evals;
    }
    if (rn + m > ks) {                                        // R overflowed k: r = max R
        if (!W.trimmed) W.r2_first = key_d2(W.res[ks - 1]);
        W.trimmed = true;
        W.r2 = key_d2(W.res[ks - 1]);
    }
}

// The front is empty: move the (up to) kFront smallest back keys into it, dropping back keys
// outside the radius. Exact: the boundary is the (kFront+1)-th smallest key, found by radix select.
inline __device__ void refill(WarpState& W, const Radius& thr, int lane) {
    int out = 0;                                              // drop keys above the radius
    for (int i0 = 0; i0 < W.back_n; i0 += 32) {
        const int i = i0 + lane;
        const uint64_t v = i < W.back_n ? W.back[i] : kEmptyKey;
        const bool keep = i < W.back_n && thr.admits(key_d2(v));
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) W.back[out + __popc(m & lanes_below(lane))] = v;
        out += __popc(m);
        __syncwarp();
    }
    W.back_n = out;
    uint64_t boundary = kEmptyKey;                            // keys < boundary go to the front
    if (W.back_n > kFront) {
        uint32_t* hist = reinterpret_cast<uint32_t*>(W.cid);  // 256 counters (cid + cd2 = 1 KiB)
        uint64_t prefix = 0;
        uint32_t rank = kFront;                               // 0-based rank of the boundary key
        for (int pass = 0; pass < 8; ++pass) {
            const int shift = 56 - 8 * pass;
            const uint64_t hmask = pass == 0 ? 0ull : (~0ull << (shift + 8));
            for (int i = lane; i < 256; i += 32) hist[i] = 0;
            __syncwarp();
            for (int i = lane; i < W.back_n; i += 32) {
                const uint64_t v = W.back[i];
                if ((v & hmask) == prefix) atomicAdd(hist + ((v >> shift) & 0xffu), 1u);
            }
            __syncwarp();
            // the digit holding the wanted rank: warp prefix sum over 8 bins per lane
            uint32_t c8[8], sum = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) { c8[b] = hist[lane * 8 + b]; sum += c8[b]; }
            uint32_t incl = sum;
#pragma unroll
            for (int m = 1; m < 32; m <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, m);
                if (lane >= m) incl += t;
            }
            const uint32_t excl = incl - sum;
            const unsigned owner = __ballot_sync(0xffffffffu, excl <= rank && rank < incl);
            const int src = __ffs(owner) - 1;                 // exists: rank < keys with the prefix
            int digit = 0;
            uint32_t before = 0;
            if (lane == src) {
                uint32_t acc = excl;
                int b = 0;
                for (; b < 7; ++b) {
                    if (acc + c8[b] > rank) break;
                    acc += c8[b];
                }
                digit = lane * 8 + b;
                before = acc;
            }
            digit = __shfl_sync(0xffffffffu, digit, src);
            before = __shfl_sync(0xffffffffu, before, src);
            rank -= before;
            prefix |= (uint64_t)digit << shift;
            __syncwarp();
        }
        boundary = prefix;                                    // the (kFront+1)-th smallest key
    }
    // split: keys below the boundary to the front (min(back_n, kFront) of them), the rest stays
    int fo = 0, bo = 0;
    uint64_t wm = kEmptyKey;
    for (int i0 = 0; i0 < W.back_n; i0 += 32) {
        const int i = i0 + lane;
        const bool valid = i < W.back_n;
        const uint64_t v = valid ? W.back[i] : kEmptyKey;
        const bool tof = valid && v < boundary;
        const bool tob = valid && !tof;
        const unsigned mf = __ballot_sync(0xffffffffu, tof), mb = __ballot_sync(0xffffffffu, tob);
        __syncwarp();
        if (tof) W.front[fo + __popc(mf & lanes_below(lane))] = v;
        if (tob) W.back[bo + __popc(mb & lanes_below(lane))] = v;
        if (tob) wm = min(wm, v);
        fo += __popc(mf);
        bo += __popc(mb);
        __syncwarp();
    }
    W.fn = fo;
    W.back_n = bo;
    W.wmark = warp_min64(wm);
    if (W.sorted) {
        // sort the front descending (bitonic over kFront slots, padded with key 0, the smallest)
        for (int i = fo + lane; i < kFront; i += 32) W.front[i] = 0;
        __syncwarp();
        for (int size = 2; size <= kFront; size <<= 1)
            for (int stride = size >> 1; stride; stride >>= 1) {
                for (int t = lane; t < kFront / 2; t += 32) {
                    const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                    const bool desc = (lo & size) == 0;
                    const uint64_t a = W.front[lo], b = W.front[hi];
                    if ((a < b) == desc) { W.front[lo] = b; W.front[hi] = a; }
                }
                __syncwarp();
            }
    }
}

// Re-rank if asked, then write R (already sorted) to the outputs.
inline __device__ void finish_query(const Params& P, WarpState& W, int q, const float* qv, int status, int tier, int lane) {
    if (P.rerank) {
        for (int i = lane; i < W.res_n; i += 32) {
            const int32_t id = key_id(W.res[i]);
            W.res[i] = make_key(exact_d2_lane(P.x32, P.dim_pad, __ldg(P.old2new + id), qv), id);
        }
        for (int i = W.res_n + lane; i < P.kcap; i += 32) W.res[i] = kEmptyKey;
        __syncwarp();
        for (int size = 2; size <= P.kcap; size <<= 1)
            for (int stride = size >> 1; stride; stride >>= 1) {
                for (int t = lane; t < P.kcap / 2; t += 32) {
                    const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const uint64_t a = W.res[lo], b = W.res[hi];
                    if ((a > b) == up) { W.res[lo] = b; W.res[hi] = a; }
                }
                __syncwarp();
            }
    }
    for (int i = lane; i < P.k; i += 32) {
        const bool ok = i < W.res_n;
        const uint64_t v = ok ? W.res[i] : kEmptyKey;
        P.ids[(int64_t)q * P.k + i] = ok ? key_id(v) : -1;
        P.dists[(int64_t)q * P.k + i] = ok ? sqrtf(key_d2(v)) : __int_as_float(0x7f800000);
    }
    if (P.rec_feats) {
        // label of the hop recorded in slot t (hop t+1): 1 if the top k of R never changed after it
        const int rec = min(W.hops, P.rec_cap);
        for (int t = lane; t < rec; t += 32) P.rec_labels[(int64_t)q * P.rec_cap + t] = (t + 1 >= W.last_change) ? 1 : 0;
        if (lane == 0) P.rec_counts[q] = rec;
    }
    if (lane == 0) {
        if (P.status) P.status[q] = status;
        if (P.trace) {
            P.trace[4 * (int64_t)q + 0] = W.hops;
            P.trace[4 * (int64_t)q + 1] = W.evals;
            P.trace[4 * (int64_t)q + 2] = W.peak;
            P.trace[4 * (int64_t)q + 3] = tier;
        }
    }
}

// One query. Returns false if its back pool overflowed (nothing written).
// Clear the bitmap words the finished query set (the whole bitmap when it visited more than
// kTouchCap vertices), so the slot's next query starts from C = {}.
inline __device__ void clear_visited(WarpState& W, const Params& P, int lane) {
    __syncwarp();
    if (W.tn <= kTouchCap) {
        for (int i = lane; i < W.tn; i += 32) W.bitmap[W.touched[i] >> 5] = 0u;
    } else {
        uint4* b4 = reinterpret_cast<uint4*>(W.bitmap);
        for (int64_t i = lane; i < P.words / 4; i += 32) b4[i] = make_uint4(0, 0, 0, 0);
    }
    W.tn = 0;
    __syncwarp();
}

// Which front a query's S keeps: sorted for long walks (from the fixed entry vertex, or with 64 or
// more results kept, or eps of 0.02 or more: hundreds to thousands of pops), unsorted for short
// ones (measured on the 1M x 128 workload: the unsorted front is 6% faster for the 34-hop routed
// walks and 6-13% slower for the long ones).
__host__ __device__ inline bool sorted_front_for(bool fixed_entry, int ks, float eps) {
    return fixed_entry || ks >= 64 || eps >= 0.02f;
}

// Mode: 0 the front of S unsorted, 1 sorted, 2 as P.sorted_front says (one kernel serving both).
template <class Rows, int G, int CPL, int Mode>
__device__ bool run_query(const Params& P, WarpState& W, int q, float* qv_smem, int tier, int lane) {
    // seeds and exploration vertices come in caller ids (routed seeds in internal ids); rows are
    // read by internal id, keys carry the caller id
    const bool given = P.explore || P.seeds;
    const int32_t seed_in = given ? P.seeds[q] : 0;
    const bool seed_ok = !given || (seed_in >= 0 && seed_in < P.n);
    const int32_t seed = !given ? P.entry : (!seed_ok ? 0 : P.seeds_internal ? seed_in : __ldg(P.old2new + seed_in));
    const int32_t seed_c = !given ? P.entry_caller : (!seed_ok ? 0 : P.seeds_internal ? __ldg(P.new2old + seed_in) : seed_in);
    const float* qsrc = P.explore ? P.x32 + (int64_t)(seed_ok ? seed : 0) * P.dim_pad : P.queries + (int64_t)q * P.dim;
    const int dim16 = (P.dim + 15) / 16 * 16;                  // zero padded to whole 16-element chunks
    for (int i = lane; i < dim16; i += 32) qv_smem[i] = i < P.dim ? qsrc[i] : 0.f;
    W.fn = W.back_n = W.res_n = 0;
    const bool sorted = Mode == 2 ? P.sorted_front != 0 : Mode == 1;
    W.sorted = sorted;
    W.wmark = kEmptyKey;
    W.trimmed = false;
    W.r2 = __int_as_float(0x7f800000);
    W.hops = W.evals = W.peak = 0;
    W.last_change = W.evals_change = W.hop_rins = 0;
    W.r2_first = 1.f;
    __syncwarp();
    if (!seed_ok) {                                            // bad seed / vertex id
        finish_query(P, W, q, qv_smem, DEG_EINVAL, tier, lane);
        return true;
    }
    Engine<Rows, G, CPL> eng;
    eng.load_query(qv_smem, P.dim, lane);

    // C <- {}: the main and serving kernels find the bitmap clear (each query clears the words it
    // set when it ends); the second kernel clears it whole
    if (!W.touched) {
        uint4* b4 = reinterpret_cast<uint4*>(W.bitmap);
        for (int64_t i = lane; i < P.words / 4; i += 32) b4[i] = make_uint4(0, 0, 0, 0);
    } else if (lane == 0) {
        W.touched[0] = seed;
    }
    W.tn = 1;
    __syncwarp();

    // Seed: S = {seed}, C = {seed}, R = {seed} (plain) or {} (exploration).
    if (lane == 0) W.cid[0] = seed;
    __syncwarp();
    eng.distances(P, W.cid, W.cd2, 1, lane);
    if (lane == 0) visit(W.bitmap, seed);
    __syncwarp();
    const uint64_t seed_key = make_key(W.cd2[0], seed_c);
    if (lane == 0) W.front[0] = seed_key;
    W.fn = 1;
    W.peak = 1;
    W.evals = 1;
    if (!P.explore) result_insert(W, P.ks, seed_key, lane);
    __syncwarp();
    if (P.seeds2) {
        // a second seed (Alg. 1 takes a seed set; the device builder's optimizeEdge searches from
        // two vertices): S, C and R get it too, unless it is absent (-1), out of range or the first
        const int32_t s2c = P.seeds2[q];
        if (s2c >= 0 && s2c < P.n && s2c != seed_c) {
            const int32_t s2 = __ldg(P.old2new + s2c);
            if (lane == 0) {
                W.cid[0] = s2;
                if (W.touched) W.touched[1] = s2;
            }
            __syncwarp();
            eng.distances(P, W.cid, W.cd2, 1, lane);
            if (lane == 0) visit(W.bitmap, s2);
            __syncwarp();
            const uint64_t k2 = make_key(W.cd2[0], s2c);
            if (lane == 0) {                                  // a sorted front stays descending
                if (!sorted || k2 < W.front[0]) W.front[1] = k2;
                else { W.front[1] = W.front[0]; W.front[0] = k2; }
            }
            W.fn = 2;
            W.peak = 2;
            W.evals = 2;
            W.tn = 2;
            __syncwarp();
            if (!P.explore) result_insert(W, P.ks, k2, lane);
            __syncwarp();
        }
    }

    const float inf = __int_as_float(0x7f800000);
    int status = DEG_OK;
    for (;;) {
        const Radius thr{W.trimmed ? W.r2 : inf, P.f, P.f_lo};
        if (W.fn == 0) {
            if (W.back_n == 0) break;                          // S empty
            refill(W, thr, lane);
            if (W.fn == 0) break;
        }
        // 1. pop the minimum of S (the front's minimum: its last key when sorted)
        uint64_t m;
        const int mi = sorted ? W.fn - 1 : front_extreme(W, false, &m, lane);
        if (sorted) m = W.front[mi];
        if (!thr.admits(key_d2(m))) break;                     // too far: return R
        if (P.max_hops && W.hops >= P.max_hops) { status = DEG_EHOPLIMIT; break; }
        __syncwarp();
        if (lane == 0 && !sorted) W.front[mi] = W.front[W.fn - 1];
        --W.fn;
        ++W.hops;
        const int32_t s = key_id(m);                           // caller id: the adjacency row
        __syncwarp();

        // 2. N(G, s) \ C, then C <- C u N
        int cnt = 0;
        for (int j0 = 0; j0 < P.degree; j0 += 32) {
            const int j = j0 + lane;
            const int2 e = j < P.degree ? __ldg(P.adj + (int64_t)s * P.deg_pad + j) : make_int2(-1, -1);
            const int32_t nb = e.x;
            if (nb >= 0 && P.row_bytes <= DEG_SEARCH_ROW_PREFETCH_BYTES) {
                // start pulling the row into L2 while the visited test is in flight (a visited
                // neighbour's row is usually there already); float32 rows (four lines) lose by it
                const uint8_t* row = P.rows + (int64_t)nb * P.row_bytes;
                for (int64_t b = 0; b < P.row_bytes; b += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + b));
                if (P.norm8) asm volatile("prefetch.global.L2 [%0];" ::"l"(P.norm8 + nb));
            }
            const int isnew = nb >= 0 ? visit(W.bitmap, nb) : 0;
            const unsigned nm = __ballot_sync(0xffffffffu, isnew);
            if (isnew) {
                const int at = cnt + __popc(nm & lanes_below(lane));
                W.cid[at] = nb;
                W.ccid[at] = e.y;
            }
            cnt += __popc(nm);
        }
        __syncwarp();
        if (cnt == 0) continue;
        W.evals += cnt;
        if (W.touched && W.tn + cnt <= kTouchCap)
            for (int i = lane; i < cnt; i += 32) W.touched[W.tn + i] = W.cid[i];
        W.tn += cnt;

        // 3. squared distances of the unvisited neighbours
        eng.distances(P, W.cid, W.cd2, cnt, lane);
        __syncwarp();

        // 4. R <- R u {n : d(n) <= r} against the radius from before the hop, keeping the ks smallest
        const float r2pre = W.trimmed ? W.r2 : inf;
        W.hop_rins = 0;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            const bool valid = i < cnt;
            const float d2 = valid ? W.cd2[i] : inf;
            result_batch(W, P.ks, P.k, make_key(d2, valid ? W.ccid[i] : -1), valid && d2 <= r2pre, lane);
        }
        // 5. S <- S u {n : d(n) <= r (1 + eps)} against the radius after the hop: a candidate outside
        //    it could only ever be popped to fail the stop test (r never grows), and the next key
        //    of S would fail it as well, so leaving it out changes no pop and no result
        const Radius thr_post{W.trimmed ? W.r2 : inf, P.f, P.f_lo};
        int adm = 0;
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            const bool valid = i < cnt;
            const float d2 = valid ? W.cd2[i] : inf;
            const int32_t id = valid ? W.ccid[i] : -1;
            const bool toS = valid && thr_post.admits(d2);
            if (toS)  // its adjacency row is read if it is ever expanded: start pulling it into L2
                asm volatile("prefetch.global.L2 [%0];" ::"l"(P.adj + (int64_t)id * P.deg_pad));
            adm += __popc(__ballot_sync(0xffffffffu, toS));
            if (!(sorted ? admit_batch_sorted(W, make_key(d2, id), toS, thr_post, lane)
                           : admit_batch(W, make_key(d2, id), toS, thr_post, lane)))
                return false;
        }
        W.peak = max(W.peak, W.fn + W.back_n);
        __syncwarp();
        // the learned stop is asked every fourth hop, and only once the top k of R have not changed
        // for two hops (while they still change, more expansion is evidently still paying)
        const bool ask = P.learned && (W.hops & 3) == 0 && W.hops - W.last_change >= 2;
        if (ask || P.rec_feats) {
            float x[kStopFeatures];
#pragma unroll
            for (int i = 0; i < kStopFeatures; ++i) x[i] = stop_feature(W, i, key_d2(m), cnt, adm, P.f, lane);
            if (P.rec_feats && W.hops <= P.rec_cap && lane < kStopFeatures) {
                float v = x[0];
#pragma unroll
                for (int i = 1; i < kStopFeatures; ++i) v = lane == i ? x[i] : v;
                P.rec_feats[((int64_t)q * P.rec_cap + (W.hops - 1)) * kStopFeatures + lane] = v;
            }
            if (ask && stop_margin(P.stop_w, x, lane) > P.stop_logit) break;
        }
    }
    finish_query(P, W, q, qv_smem, status, tier, lane);
    return true;
}

// Shared-memory bytes per warp.
__host__ __device__ inline int64_t warp_bytes(int kcap, int dim) {
    const int64_t b = 16ll * kFront + 8ll * kcap + (4 + 4 + 4) * kMaxDegree + 8ll * 32 + 4ll * ((dim + 15) / 16 * 16);
    return (b + 15) / 16 * 16;
}

__device__ __forceinline__ float* bind_smem(WarpState& W, uint8_t* base, const Params& P) {
    W.front = reinterpret_cast<uint64_t*>(base);
    W.front2 = W.front + kFront;                              // the unsorted front uses both halves
    W.res = W.front + 2 * kFront;
    W.cid = reinterpret_cast<int32_t*>(W.res + P.kcap);
    W.cd2 = reinterpret_cast<float*>(W.cid + kMaxDegree);
    W.ccid = reinterpret_cast<int32_t*>(W.cd2 + kMaxDegree);
    W.fbuf = reinterpret_cast<uint64_t*>(W.ccid + kMaxDegree);
    return reinterpret_cast<float*>(W.fbuf + 32);
}

// Bytes of shared memory for the learned-stop weights at the head of a block (0 if off).
__host__ __device__ inline int64_t stop_bytes(int learned) { return learned ? (2ll * kStopParams + 15) / 16 * 16 : 0; }

__device__ __forceinline__ uint8_t* load_stop_weights(Params& P, uint8_t* smem) {
    if (!P.learned) return smem;
    __nv_bfloat16* w = reinterpret_cast<__nv_bfloat16*>(smem);
    for (int i = threadIdx.x; i < kStopParams; i += blockDim.x) w[i] = P.stop_w[i];
    __syncthreads();
    P.stop_w = w;
    return smem + stop_bytes(1);
}

template <class Rows, int G, int CPL, int Mode>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, kBlocksPerSM) search_fast_kernel(Params P) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = blockIdx.x * P.wpb + warp;
    uint8_t* wbase = load_stop_weights(P, smem);
    WarpState W;
    float* qv = bind_smem(W, wbase + warp * warp_bytes(P.kcap, P.dim), P);
    W.bitmap = P.bitmaps + (int64_t)slot * P.words;
    W.touched = P.touched + (int64_t)slot * kTouchCap;
    W.tn = 0;
    W.back = P.backs + (int64_t)slot * P.bstride;
    W.bcap = P.bcap;
    for (;;) {
        int q = 0;
        if (lane == 0) {
            q = atomicAdd(P.counters + 2, 1);
            if (q < P.nq && P.order) q = P.order[q];
            else if (q >= P.nq) q = P.nq;
        }
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= P.nq) break;
        const bool done = run_query<Rows, G, CPL, Mode>(P, W, q, qv, 0, lane);
        clear_visited(W, P, lane);
        if (!done && lane == 0) P.overflow[atomicAdd(P.counters, 1)] = q;
        __syncwarp();
    }
}

template <class Rows, int G, int CPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) search_device_kernel(Params P) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = blockIdx.x * kWarpsPerBlock + warp;
    uint8_t* wbase = load_stop_weights(P, smem);
    if (slot >= P.pslots) return;
    WarpState W;
    float* qv = bind_smem(W, wbase + warp * warp_bytes(P.kcap, P.dim), P);
    W.bitmap = P.pbitmaps + (int64_t)slot * P.words;
    W.touched = nullptr;                                      // cleared whole at each query start
    W.tn = 0;
    W.back = P.pbacks + (int64_t)slot * (P.n + 1);
    W.bcap = (int32_t)(P.n + 1);
    const int count = *(volatile int32_t*)P.counters;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(P.counters + 1, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= count) break;
        run_query<Rows, G, CPL, 1>(P, W, P.overflow[t], qv, 1, lane);   // queries with a large S: sorted front
        __syncwarp();
    }
}

// ---- serving: a persistent kernel over a request ring ----------------------------------------
// Requests are posted by the host into a ring in mapped host memory; every warp of the kernel
// claims the next request number, waits (bounded by %globaltimer) until the host has posted it,
// runs it with the same per-query code as a batch search (so a request's result does not depend
// on what else is in flight), writes the result into the ring and publishes it with a release
// store of its sequence number. The kernel ends when the host raises the stop flag, or with
// DEG_ETIMEOUT when no request arrives for idle_ns.
struct ServeRing {
    const float* vecs;                    // [cap][dim] query vectors
    const int4* meta;                     // [cap] {k, eps bits, vertex (-1: vector query), seq}
    int32_t* ids;                         // [cap][kmax]
    float* dists;                         // [cap][kmax]
    int32_t* status;                      // [cap]
    int32_t* trace;                       // [cap][4]
    uint32_t* done;                       // [cap]: seq + 1 once the result is written
    unsigned long long* times;            // [cap][2]: %globaltimer when the request was taken, when done
    const unsigned long long* tail;       // requests posted so far
    const int32_t* stop;
    int32_t* kstatus;                     // kernel status (device memory)
    unsigned long long* claim;            // next request number (device memory)
    int32_t cap, kmax, entry_mode;
    unsigned long long idle_ns;
    int32_t max_blocks;                   // 0: as many resident blocks as fit
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_sys(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Nearest pivot (float32 distance, tie -> lower pivot index) to the query in shared memory.
inline __device__ int32_t route_one(const Params& P, const int32_t* pivots, int np, const float* qv, int lane) {
    uint64_t best = kEmptyKey;
    for (int p = lane; p < np; p += 32) best = min(best, make_key(exact_d2_lane(P.x32, P.dim_pad, __ldg(pivots + p), qv), p));
    best = warp_min64(best);
    return __ldg(pivots + key_id(best));
}

template <class Rows, int G, int CPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, kBlocksPerSM) serve_kernel(Params P, ServeRing S,
                                                                                  const int32_t* pivots, int np) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int32_t seed_s[kWarpsPerBlock];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = blockIdx.x * P.wpb + warp;
    uint8_t* wbase = load_stop_weights(P, smem);
    WarpState W;
    float* qv = bind_smem(W, wbase + warp * warp_bytes(P.kcap, P.dim), P);
    W.bitmap = P.bitmaps + (int64_t)slot * P.words;
    W.touched = P.touched + (int64_t)slot * kTouchCap;
    W.tn = 0;
    W.back = P.backs + (int64_t)slot * P.bstride;
    W.bcap = P.bcap;
    const int dim16 = (P.dim + 15) / 16 * 16;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(S.claim, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        // wait until request i is posted, the host asks to stop, or nothing arrives for idle_ns. The
        // ring lives in host memory, and thousands of waiting warps polling it back to back load
        // the link to it: the wait backs off from 256 ns to 4 us, and the stop flag is read on
        // every eighth poll only.
        const unsigned long long t0 = global_ns();
        int state = 0;                                        // 1 posted, 2 stop, 3 timeout
        unsigned sleep_ns = 256;
        for (unsigned poll = 0; state == 0; ++poll) {
            if (lane == 0) {
                if (ld_acquire_sys(S.tail) > i) state = 1;
                else if ((poll & 7) == 7 && ld_acquire_sys(S.stop)) state = 2;
                else if (global_ns() - t0 > S.idle_ns) state = 3;
            }
            state = __shfl_sync(0xffffffffu, state, 0);
            if (state == 0) {
                __nanosleep(sleep_ns);
                sleep_ns = min(sleep_ns * 2, 4096u);
            }
        }
        if (state == 3 && lane == 0) atomicExch(S.kstatus, (int)DEG_ETIMEOUT);
        if (state != 1) return;
        const int r = (int)(i % (unsigned long long)S.cap);
        if (lane == 0) S.times[2 * r] = global_ns();
        const int4 m = S.meta[r];
        Params Q = P;
        Q.k = m.x;
        Q.ks = P.rerank ? max(P.ks, m.x) : m.x;
        const float2 fe = eps_factor(__int_as_float(m.y));
        Q.f = fe.x;
        Q.f_lo = fe.y;
        Q.nq = 1;
        Q.ids = S.ids + (int64_t)r * S.kmax;
        Q.dists = S.dists + (int64_t)r * S.kmax;
        Q.status = S.status + r;
        Q.trace = S.trace + 4 * (int64_t)r;
        Q.seeds_internal = 0;
        Q.sorted_front = sorted_front_for(m.z < 0 && S.entry_mode == 0, Q.ks, __int_as_float(m.y)) ? 1 : 0;
        if (m.z >= 0) {                                       // exploration from vertex m.z
            Q.explore = 1;
            Q.seeds = reinterpret_cast<const int32_t*>(S.meta + r) + 2;
            Q.queries = nullptr;
        } else {
            Q.explore = 0;
            Q.queries = S.vecs + (int64_t)r * P.dim;
            Q.seeds = nullptr;
            if (S.entry_mode >= 1) {
                for (int d = lane; d < dim16; d += 32) qv[d] = d < P.dim ? Q.queries[d] : 0.f;
                __syncwarp();
                const int32_t sd = route_one(P, pivots, np, qv, lane);
                if (lane == 0) seed_s[warp] = sd;
                __syncwarp();
                Q.seeds = seed_s + warp;
                Q.seeds_internal = 1;
            }
        }
        const bool done = run_query<Rows, G, CPL, 2>(Q, W, 0, qv, 0, lane);
        clear_visited(W, Q, lane);
        if (!done) {
            for (int j = lane; j < m.x; j += 32) { Q.ids[j] = -1; Q.dists[j] = __int_as_float(0x7f800000); }
            if (lane == 0) *Q.status = DEG_EOVERFLOW;
        }
        __syncwarp();
        if (lane == 0) S.times[2 * r + 1] = global_ns();
        __threadfence_system();
        if (lane == 0) st_release_sys(S.done + r, (uint32_t)(i + 1));
    }
}

template <class Rows, int G, int CPL>
int launch_serve(Params P, const ServeRing& S, const int32_t* pivots, int np, cudaStream_t st, int* warps,
                 std::string* why) {
    cudaError_t e;
    int dev = 0, smem_max = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t wb = warp_bytes(P.kcap, P.dim), sb = stop_bytes(P.learned);
    if (wb * kWarpsPerBlock + sb > smem_max) return *why = "serving state does not fit", (int)cudaErrorInvalidValue;
    P.wpb = kWarpsPerBlock;
    const int64_t smem = sb + wb * kWarpsPerBlock;
    auto k = serve_kernel<Rows, G, CPL>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return *why = std::string("serve attribute: ") + cudaGetErrorString(e), (int)e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWarpsPerBlock * 32, (size_t)smem)) != cudaSuccess)
        return *why = "occupancy query failed", (int)e;
    // every block must be resident at once (persistent); never more warps than device slots, nor
    // more blocks than the caller allows (the rest of the GPU stays free for other work)
    int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, (int64_t)P.slots / kWarpsPerBlock));
    if (S.max_blocks > 0) grid = std::min<int64_t>(grid, S.max_blocks);
    *warps = (int)(grid * kWarpsPerBlock);
    k<<<(unsigned)grid, kWarpsPerBlock * 32, smem, st>>>(P, S, pivots, np);
    if ((e = cudaGetLastError()) != cudaSuccess) return *why = std::string("serve kernel: ") + cudaGetErrorString(e), (int)e;
    return 0;
}

template <class Rows>
int dispatch_serve(Params P, const ServeRing& S, const int32_t* pivots, int np, cudaStream_t st, int* warps,
                   std::string* why) {
    const int nc = P.nchunk;
    if (nc <= 4) return launch_serve<Rows, 4, 1>(P, S, pivots, np, st, warps, why);
    if (nc <= 8) return launch_serve<Rows, 8, 1>(P, S, pivots, np, st, warps, why);
    if (nc <= 16) return launch_serve<Rows, 16, 1>(P, S, pivots, np, st, warps, why);
    if (nc <= 32) return launch_serve<Rows, 32, 1>(P, S, pivots, np, st, warps, why);
    *why = "serving supports rows of at most 512 bytes";
    return (int)cudaErrorInvalidValue;
}

template <class Rows, int G, int CPL>
int launch_typed(Params P, cudaStream_t st, void* timer_start, void* timer_end, std::string* why) {
    cudaError_t e;
    int dev = 0, smem_max = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t wb = warp_bytes(P.kcap, P.dim), sb = stop_bytes(P.learned);
    if (wb + sb > smem_max) return *why = "search state does not fit in shared memory", (int)cudaErrorInvalidValue;
    const int wpb = (int)std::min<int64_t>(kWarpsPerBlock, (smem_max - sb) / wb);
    P.wpb = wpb;
    const int64_t smem = sb + wb * wpb;
    auto fk = P.sorted_front ? search_fast_kernel<Rows, G, CPL, 1> : search_fast_kernel<Rows, G, CPL, 0>;
    if ((e = cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return *why = std::string("shared memory attribute: ") + cudaGetErrorString(e), (int)e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fk, wpb * 32, (size_t)smem)) != cudaSuccess)
        return *why = "occupancy query failed", (int)e;
    if (per_sm < 1) return *why = "search state does not fit", (int)cudaErrorInvalidValue;
    // one device-memory slot per warp of the grid: the grid never exceeds the slots
    const int64_t want = (P.nq + wpb - 1) / wpb;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)sms * per_sm, (int64_t)P.slots / wpb}));
    if ((e = cudaMemsetAsync(P.counters, 0, 4 * sizeof(int32_t), st)) != cudaSuccess) return *why = "memset", (int)e;
    if (timer_start && (e = cudaEventRecord(static_cast<cudaEvent_t>(timer_start), st)) != cudaSuccess)
        return *why = "timer event", (int)e;
    fk<<<(unsigned)grid, wpb * 32, smem, st>>>(P);
    if ((e = cudaGetLastError()) != cudaSuccess) return *why = std::string("main kernel: ") + cudaGetErrorString(e), (int)e;
    auto dk = search_device_kernel<Rows, G, CPL>;
    const int64_t dsm = sb + wb * kWarpsPerBlock;
    if (dsm > smem_max) return *why = "second kernel state does not fit", (int)cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(dk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm)) != cudaSuccess)
        return *why = "second kernel attribute", (int)e;
    dk<<<(P.pslots + kWarpsPerBlock - 1) / kWarpsPerBlock, kWarpsPerBlock * 32, dsm, st>>>(P);
    if ((e = cudaGetLastError()) != cudaSuccess) return *why = std::string("second kernel: ") + cudaGetErrorString(e), (int)e;
    if (timer_end && (e = cudaEventRecord(static_cast<cudaEvent_t>(timer_end), st)) != cudaSuccess)
        return *why = "timer event", (int)e;
    return 0;
}

template <class Rows>
int dispatch_shape(Params P, cudaStream_t st, void* t0, void* t1, std::string* why) {
    const int nc = P.nchunk;
    if (nc <= 4) return launch_typed<Rows, 4, 1>(P, st, t0, t1, why);
    if (nc <= 8) return launch_typed<Rows, 8, 1>(P, st, t0, t1, why);
    if (nc <= 16) return launch_typed<Rows, 16, 1>(P, st, t0, t1, why);
    if (nc <= 32) return launch_typed<Rows, 32, 1>(P, st, t0, t1, why);
    if (nc <= 64) return launch_typed<Rows, 32, 2>(P, st, t0, t1, why);
    if (nc <= 128) return launch_typed<Rows, 32, 4>(P, st, t0, t1, why);
    if (nc <= 256) return launch_typed<Rows, 32, 8>(P, st, t0, t1, why);
    *why = "row too wide (at most 4096 bytes)";
    return (int)cudaErrorInvalidValue;
}

// The launchers, one translation unit per row format (search_f32.cu, search_bf16.cu, search_fp8.cu),
// so the kernels of the three formats compile in parallel.
int dispatch_search_f32(Params P, cudaStream_t st, void* t0, void* t1, std::string* why);
int dispatch_search_bf16(Params P, cudaStream_t st, void* t0, void* t1, std::string* why);
int dispatch_search_fp8(Params P, cudaStream_t st, void* t0, void* t1, std::string* why);
int dispatch_serve_f32(Params P, const ServeRing& S, const int32_t* pivots, int np, cudaStream_t st, int* warps,
                       std::string* why);
int dispatch_serve_bf16(Params P, const ServeRing& S, const int32_t* pivots, int np, cudaStream_t st, int* warps,
                        std::string* why);
int dispatch_serve_fp8(Params P, const ServeRing& S, const int32_t* pivots, int np, cudaStream_t st, int* warps,
                       std::string* why);

}  // namespace sk
}  // namespace deg

#endif
