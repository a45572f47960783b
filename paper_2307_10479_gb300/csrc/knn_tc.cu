// Exact k nearest neighbours (paper Eq. 1) with the distance contraction on the 5th-generation
// tensor cores. The result equals the CUDA-core path's bit for bit: the same float32 distances
// sum_d fmaf(q_d - x_d, q_d - x_d, .) in dimension order, ties ordered by id.
//
// Per chunk of queries:
//   1. bfloat16 copies of rows and queries (K padded to a multiple of 64), with float32 squared
//      norms and the norms of the rounding residuals x - bf16(x);
//   2. sample pass: approximate squared distances a = |q|^2 + |x|^2 - 2 bf16(q).bf16(x) of every
//      query against every s-th row (tcgen05.mma.kind::f16, float32 accumulators in tensor memory),
//      reduced to the minimum of each group of 16 sampled rows; t_s = the k-th smallest group
//      minimum. k groups hold k distinct rows with a <= t_s, so t_s is at least the k-th smallest a
//      over all rows;
//   3. filter pass: a against every row; a row is a candidate when a <= t_s + 2b, where b bounds
//      |a - e| for the float32 distance e (bfloat16 rounding, accumulation and norm rounding; see
//      error_bound). If e_k is the k-th smallest e, the k rows with the smallest a have e <= t + b
//      (t = k-th smallest a), so e_k <= t + b and every row with e <= e_k has a <= t + 2b <= t_s + 2b:
//      all true neighbours, ties included, are candidates;
//   4. re-rank: per query, t = the k-th smallest a among the candidates (it is the global one), the
//      rows with a <= t + 2b get e computed exactly, sorted by (e, id), the first k returned.
// A query with more candidates than the buffer holds is recomputed by the CUDA-core path.
//
// The distance kernel is a persistent, warp-specialised tcgen05 pipeline, one CTA per SM:
//   warp 0  TMA producer: 128 queries x 64 and 256 rows x 64 bf16 tiles (128-byte swizzle) into a
//           4-stage shared-memory ring, completion counted on the stage's mbarrier;
//   warp 1  MMA issuer: one thread issues tcgen05.mma (M = 128, N = 256, K = 16) into one of two
//           256-column tensor-memory accumulators, commits each stage back to the producer and each
//           finished tile to the epilogue;
//   warps 2-17 epilogue: tcgen05.ld of the finished accumulator (four warps per 32-lane quarter, 64
//           columns each), approximate distances, group minima (sample pass) or candidate appends
//           (filter pass), then the accumulator is handed back, so the next tile's MMAs overlap this
//           epilogue.
// Work items are (query tile, row tile) pairs, the query tile varying fastest, so the CTAs running
// at one time read the same row tiles (each row tile leaves DRAM once, the rest are L2 hits).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "deg_internal.h"

namespace deg {
namespace {

constexpr int TM = 128, TN = 256, KC = 64;
constexpr int kStages = 4;
constexpr int kStageA = TM * KC * 2;                    // 16 KiB of queries
constexpr int kStageB = TN * KC * 2;                    // 32 KiB of rows
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kSmemDyn = kStages * kStageBytes + 1024;  // + alignment slack: one CTA per SM
constexpr int kEpiWarps = 16;                           // epilogue warps: four per lane quarter
constexpr int kEpiCols = TN * 4 / kEpiWarps;            // accumulator columns per epilogue warp
static_assert(kEpiCols == 64, "the epilogue reads two 32-column halves per warp");
constexpr int kTcThreads = 32 * (2 + kEpiWarps);        // producer, MMA, epilogue
constexpr int kTmemCols = 2 * TN;                       // two accumulators
constexpr int64_t kSampleMax = 65536;                   // sample rows per query
constexpr int kGroup = 16;                              // sampled rows per group minimum
constexpr int kCandCapMax = 8192;                       // candidates per query, at most
constexpr int64_t kPlanRowsMax = 4096;                  // rows of a k-NN plan (inline fallback in shared memory)
constexpr int kSelThreads = 256;
constexpr int kRerankThreads = 512;
constexpr unsigned long long kWaitNs = 2000000000ull;   // bounded wait on the tensor core: 2 s

// Instruction descriptor, kind::f16: D float32 (bits 4-5 = 1), A and B bfloat16 (bits 7-9, 10-12
// = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle layout that TMA
// writes (8-row groups of 128-byte rows, 1024 bytes apart): start address >> 4, leading byte
// offset 16 (unused for this layout), stride byte offset 1024, descriptor version 1 (bit 46),
// layout type 2 = 128-byte swizzle (bits 61-63). A K step of 16 elements moves the start by 32 bytes.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int32_t x, int32_t y, uint32_t mbar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(mbar) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the given phase of the barrier; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    const uint64_t start = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
        if (done) return true;
        if (global_ns() - start > kWaitNs) return false;
    }
}

// Order-preserving map of a float to an unsigned key (negative approximate distances occur).
__device__ __forceinline__ uint32_t okey(float v) {
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_okey(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Upper bound on |a - e| for one query against any row, with u = 2^-24:
//  - bfloat16 rounding of the dot product: with q = bq + rq, x = bx + rx,
//    |q.x - bq.bx| <= |q||rx| + |rq||x| + |rq||rx|, doubled by the factor 2 of a;
//  - float32 accumulation of the exact bf16 products: <= (K + 2) 2^-22 sum |bq_d bx_d|
//    (four times the per-addition error of a truncating adder), doubled;
//  - rounding of |q|^2, |x|^2 (K u each, relative), of their combination (2u each), and of e
//    itself ((K + 3) u relative to |q - x|^2 <= (|q| + |x|)^2): (3K + 8) u (|q| + |x|)^2;
//  - coordinates below 2^-126, flushed to zero in the bf16 copies: 2^-126 (|q| + |x|) each, doubled.
// K is the padded dimension. |x| and |rx| are replaced by their maxima over the rows; a 1%
// margin covers the float32 evaluation of the bound.
__device__ __forceinline__ float error_bound(float qn, float rq, float xmax2, float rmax, int kpad) {
    const float u = 5.9604645e-08f;
    const float grow = 1.f + (float)(kpad + 2) * u;
    const float Q = sqrtf(qn * grow) * 1.0001f, X = sqrtf(xmax2 * grow) * 1.0001f;
    const float RQ = rq * 1.001f, R = rmax * 1.001f;
    const float rounding = 2.f * (Q * R + RQ * X + RQ * R);
    const float accumulate = 2.f * (float)(kpad + 2) * 2.3841858e-07f * (Q + RQ) * (X + R);
    const float sums = (3.f * (float)kpad + 8.f) * u * (Q + X) * (Q + X);
    const float flushed = 2.f * (float)kpad * 1.1754944e-38f * (Q + X);       // coordinates below 2^-126
    return 1.01f * (rounding + accumulate + sums + flushed) + 1e-30f;
}

// t + 2b, rounded up past the float32 rounding of the sum.
__device__ __forceinline__ float window_limit(float t, float b) {
    return t + 2.f * b + (fabsf(t) + 2.f * b) * 4.7683716e-07f;
}

// bfloat16 copy with zero padding to kpad columns; norms = float32 sum of squares; resid = norm
// of x - bf16(x).
__global__ void bf16_rows_kernel(const float* __restrict__ x, int64_t rows, int32_t dim, int32_t kpad,
                                 __nv_bfloat16* __restrict__ out, float* __restrict__ norms, float* __restrict__ resid) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows; r += nw) {
        float s = 0.f, e = 0.f;
        for (int i = lane; i < kpad; i += 32) {
            const float v = i < dim ? x[r * dim + i] : 0.f;
            // subnormal bf16 values are flushed here, so that the residual accounts for them
            const __nv_bfloat16 b = fabsf(v) < 1.17549435e-38f ? __float2bfloat16_rn(0.f) : __float2bfloat16_rn(v);
            out[r * kpad + i] = b;
            const float d = v - __bfloat162float(b);
            s = fmaf(v, v, s);
            e = fmaf(d, d, e);
        }
#pragma unroll
        for (int m = 16; m; m >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, m);
            e += __shfl_xor_sync(0xffffffffu, e, m);
        }
        if (lane == 0) {
            norms[r] = s;
            resid[r] = sqrtf(e);
        }
    }
}

// out[0] = max norms, out[1] = max resid (both non-negative: int ordering of the bits works).
__global__ void row_maxima_kernel(const float* norms, const float* resid, int64_t n, float* out) {
    float a = 0.f, b = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a = fmaxf(a, norms[i]);
        b = fmaxf(b, resid[i]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<int*>(out), __float_as_int(a));
        atomicMax(reinterpret_cast<int*>(out) + 1, __float_as_int(b));
    }
}

// 32 consecutive accumulator columns of this warp's 32 lanes (one register per column).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                   "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr) : "memory");
}

// (u0, u1) = (x0 - 2 v0, x1 - 2 v1) in one paired float32 FMA (each lane rounded once).
__device__ __forceinline__ void xn_minus_2v(float x0, float x1, uint32_t v0, uint32_t v1, float& u0, float& u1) {
    unsigned long long vv, xx, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(vv) : "r"(v0), "r"(v1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(xx) : "f"(x0), "f"(x1));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(vv), "l"(0xC0000000C0000000ull), "l"(xx));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(u0), "=f"(u1) : "l"(r));
}

// Waits for this thread's tcgen05.ld; v is tied to the wait, so the compiler treats the registers
// as written here (not at the load) and touches them only afterwards.
__device__ __forceinline__ void tmem_wait_ld(uint32_t* v) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]),
                   "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]),
                   "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :: "memory");
}

// min(a, b, c) in one three-input min (sm_100 and later).
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

struct TcArgs {
    int32_t q_row0;                // first query of this chunk (tensor-map row)
    int32_t nq;                    // queries in this chunk
    int32_t qblocks;               // ceil(nq / 128)
    int64_t ncols;                 // rows in this pass
    int64_t tiles;                 // ceil(ncols / 256)
    int32_t nk;                    // kpad / 64
    const float* qn;               // [nq] squared norms of this chunk's queries
    const float* xn;               // squared norms of this pass's rows, zero-padded to tiles * 256
    float* gmin;                   // sample pass: [nq][ceil(ncols / 16)] group minima
    const float* limit;            // filter pass: [nq]
    unsigned long long* cand;      // filter pass: [nq][cap] keys okey(a) << 32 | row
    int32_t* cnt;                  // filter pass: [nq]
    int32_t cap;
    int32_t* error;                // set to 1 when a wait ran out
};

// One 32-column half of an epilogue warp's accumulator block: lane = query row qrow, column j =
// row xc + 32 c + j. Per column u = |x|^2 - 2 q.x (one paired FMA; rows past the end get +inf,
// which no filter or group minimum takes); the filter pass appends the rows with u <= T, the sample
// pass writes the two group-of-16 minima |q|^2 + min u.
template <bool kFilter>
__device__ __forceinline__ void epilogue_half(const TcArgs& a, const uint32_t* v, const float4* xs4, int c, int64_t xc,
                                              int64_t qrow, bool qvalid, float qnorm, float T, int ng) {
    const int64_t xg = xc + c * 32;
    if (!qvalid || xg >= a.ncols) return;
    float u[32];
#pragma unroll
    for (int j4 = 0; j4 < 8; ++j4) {
        const float4 xv = xs4[c * 8 + j4];
        xn_minus_2v(xv.x, xv.y, v[j4 * 4], v[j4 * 4 + 1], u[j4 * 4], u[j4 * 4 + 1]);
        xn_minus_2v(xv.z, xv.w, v[j4 * 4 + 2], v[j4 * 4 + 3], u[j4 * 4 + 2], u[j4 * 4 + 3]);
    }
    if (xg + 32 > a.ncols) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (xg + j >= a.ncols) u[j] = __int_as_float(0x7f800000);
    }
    if (kFilter) {
        float m[11];
#pragma unroll
        for (int j = 0; j < 10; ++j) m[j] = min3f(u[3 * j], u[3 * j + 1], u[3 * j + 2]);
        m[10] = fminf(u[30], u[31]);
        const float lo = fminf(min3f(min3f(m[0], m[1], m[2]), min3f(m[3], m[4], m[5]), min3f(m[6], m[7], m[8])),
                               fminf(m[9], m[10]));
        if (lo <= T) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (u[j] <= T && xg + j < a.ncols) {
                    const int p = atomicAdd(a.cnt + qrow, 1);
                    if (p < a.cap)
                        a.cand[qrow * a.cap + p] = ((unsigned long long)okey(qnorm + u[j]) << 32) | (uint32_t)(xg + j);
                }
            }
        }
    } else {
        float g[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float* w = u + 16 * h;
            const float t0 = min3f(w[0], w[1], w[2]), t1 = min3f(w[3], w[4], w[5]), t2 = min3f(w[6], w[7], w[8]);
            const float t3 = min3f(w[9], w[10], w[11]), t4 = min3f(w[12], w[13], w[14]);
            g[h] = min3f(min3f(t0, t1, t2), fminf(t3, t4), w[15]);
        }
        a.gmin[qrow * ng + xg / 16] = qnorm + g[0];
        if (xg + 16 < a.ncols) a.gmin[qrow * ng + xg / 16 + 1] = qnorm + g[1];
    }
}

template <bool kFilter>
__global__ void __launch_bounds__(kTcThreads, 1) dist_tc_kernel(const __grid_constant__ CUtensorMap tq,
                                                               const __grid_constant__ CUtensorMap tx, const TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(16) float xn_tile[kEpiWarps][kEpiCols];   // each epilogue warp's row norms
    const uint32_t ring = smem_u32(smem_raw) + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t items = (uint32_t)(a.qblocks * a.tiles);      // < 2^31: checked by the caller
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull_bar[b]), 1);
            mbar_init(smem_u32(&tempty_bar[b]), kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool failed = false;
    if (warp == 0) {
        // ---- TMA producer ----
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(&tq) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&tx) : "memory");
            int s = 0;
            uint32_t ph = 0;
            for (uint32_t w = blockIdx.x; w < items && !failed; w += gridDim.x) {
                const int32_t qy = a.q_row0 + (int32_t)(w % (uint32_t)a.qblocks) * TM;
                const int32_t xy = (int32_t)(w / (uint32_t)a.qblocks) * TN;
                for (int kc = 0; kc < a.nk; ++kc) {
                    if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u)) {
                        failed = true;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    mbar_expect_tx(fb, kStageBytes);
                    const uint32_t dst = ring + s * kStageBytes;
                    tma_load_2d(dst, &tq, kc * KC, qy, fb);
                    tma_load_2d(dst + kStageA, &tx, kc * KC, xy, fb);
                    if (++s == kStages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int s = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            for (uint32_t w = blockIdx.x; w < items && !failed; w += gridDim.x) {
                if (!mbar_wait(smem_u32(&tempty_bar[acc]), aph ^ 1u)) {
                    failed = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * TN);
                for (int kc = 0; kc < a.nk; ++kc) {
                    if (!mbar_wait(smem_u32(&full_bar[s]), ph)) {
                        failed = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = ring + s * kStageBytes, sb = sa + kStageA;
#pragma unroll
                    for (int k16 = 0; k16 < KC / 16; ++k16) {
                        const uint64_t ad = sw128_desc(sa + k16 * 32), bd = sw128_desc(sb + k16 * 32);
                        const uint32_t accumulate = (kc > 0 || k16 > 0) ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                     ::"r"(d), "l"(ad), "l"(bd), "r"(kIdesc), "r"(accumulate) : "memory");
                    }
                    mma_commit(smem_u32(&empty_bar[s]));        // the stage is free once these MMAs finish
                    if (++s == kStages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (failed) break;
                mma_commit(smem_u32(&tfull_bar[acc]));          // the tile is ready for the epilogue
                if (++acc == 2) {
                    acc = 0;
                    aph ^= 1u;
                }
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue warps 2-17: tensor-memory lanes 32 * (warp % 4) ... + 31, accumulator columns
        // 64 * ((warp - 2) / 4) ... + 63. Per column u = |x|^2 - 2 q.x (one paired FMA) and
        // a = |q|^2 + u. The filter compares u with T = limit - |q|^2 rounded up, so a row passes
        // whenever a <= limit; stored keys and group minima are |q|^2 + u. Both roundings are
        // inside the error bound.
        const int quarter = warp & 3, cgroup = (warp - 2) >> 2;
        const float4* xs4 = reinterpret_cast<const float4*>(xn_tile[warp - 2]);
        const int ng = (int)((a.ncols + 15) / 16);
        int acc = 0;
        uint32_t aph = 0;
        for (uint32_t w = blockIdx.x; w < items; w += gridDim.x) {
            const int64_t qrow = (int64_t)(w % (uint32_t)a.qblocks) * TM + quarter * 32 + lane;
            const int64_t xc = (int64_t)(w / (uint32_t)a.qblocks) * TN + cgroup * kEpiCols;
            const bool qvalid = qrow < a.nq;
            float4 xpre = make_float4(0.f, 0.f, 0.f, 0.f);
            if (lane < kEpiCols / 4) xpre = __ldg(reinterpret_cast<const float4*>(a.xn + xc) + lane);   // norms are padded
            const float qnorm = qvalid ? a.qn[qrow] : 0.f;
            float T = 0.f;
            if (kFilter && qvalid) {
                const float d = a.limit[qrow] - qnorm;
                T = d + fabsf(d) * 2.3841858e-07f;
            }
            const bool ok = mbar_wait(smem_u32(&tfull_bar[acc]), aph);
            if (!__all_sync(0xffffffffu, ok)) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (lane < kEpiCols / 4) reinterpret_cast<float4*>(xn_tile[warp - 2])[lane] = xpre;
            __syncwarp();
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * TN + cgroup * kEpiCols);
            // the second half's tcgen05.ld is in flight while the first half is processed; once both
            // are in registers the accumulator goes back to the MMA warp, before the second half's work
            uint32_t v0[32], v1[32];
            tmem_ld32(tbase, v0);
            tmem_wait_ld(v0);
            tmem_ld32(tbase + 32u, v1);
            epilogue_half<kFilter>(a, v0, xs4, 0, xc, qrow, qvalid, qnorm, T, ng);
            tmem_wait_ld(v1);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[acc]));
            epilogue_half<kFilter>(a, v1, xs4, 1, xc, qrow, qvalid, qnorm, T, ng);
            if (++acc == 2) {
                acc = 0;
                aph ^= 1u;
            }
        }
    }
    if (failed && lane == 0) atomicExch(a.error, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Radix select over `count` 32-bit keys: the key of rank `rank` (0-based), keys read through
// get(i); four passes of 8-bit digits. Lanes of a warp that hit the same bin add once (keys of
// one query crowd into a few bins).
template <int kThreads, typename Get>
__device__ uint32_t radix_select32(int count, uint32_t rank, Get get, uint32_t* hist, uint32_t* prefix_s, uint32_t* rank_s) {
    if (threadIdx.x == 0) {
        *prefix_s = 0;
        *rank_s = rank;
    }
    for (int pass = 0; pass < 4; ++pass) {
        for (int i = threadIdx.x; i < 256; i += kThreads) hist[i] = 0;
        __syncthreads();
        const int shift = 24 - 8 * pass;
        const uint32_t want = *prefix_s;
        const uint32_t hmask = pass == 0 ? 0u : (0xffffffffu << (shift + 8));
        for (int i0 = 0; i0 < count; i0 += kThreads) {
            const int i = i0 + (int)threadIdx.x;
            uint32_t bin = 256u;
            if (i < count) {
                const uint32_t kv = get(i);
                if ((kv & hmask) == (want & hmask)) bin = (kv >> shift) & 0xffu;
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, bin);
            if (bin < 256u && (threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t acc = 0, r = *rank_s;
            int dg = 0;
            for (; dg < 255; ++dg) {
                if (acc + hist[dg] > r) break;
                acc += hist[dg];
            }
            *rank_s = r - acc;
            *prefix_s = want | ((uint32_t)dg << shift);
        }
        __syncthreads();
    }
    return *prefix_s;
}

// limit[q] = window_limit(k-th smallest group minimum, b_q); +inf when there are fewer than k
// groups (every row is then a candidate).
__global__ void __launch_bounds__(kSelThreads) sample_limit_kernel(const float* __restrict__ gmin, int ng, int k,
                                                                  const float* __restrict__ qn, const float* __restrict__ rq,
                                                                  const float* __restrict__ maxima, int32_t kpad,
                                                                  float* __restrict__ limit) {
    __shared__ uint32_t skeys[kSampleMax / kGroup];
    __shared__ uint32_t hist[256], prefix_s, rank_s;
    const int64_t q = blockIdx.x;
    if (ng < k) {
        if (threadIdx.x == 0) limit[q] = __int_as_float(0x7f800000);
        return;
    }
    for (int i = threadIdx.x; i < ng; i += kSelThreads) skeys[i] = okey(gmin[q * ng + i]);
    __syncthreads();
    const uint32_t tk = radix_select32<kSelThreads>(ng, (uint32_t)(k - 1), [&](int i) { return skeys[i]; }, hist,
                                                    &prefix_s, &rank_s);
    if (threadIdx.x == 0) limit[q] = window_limit(from_okey(tk), error_bound(qn[q], rq[q], maxima[0], maxima[1], kpad));
}

// Exact float32 squared distance of row x, summed in dimension order (as the CUDA-core path).
__device__ __forceinline__ float exact_row_d2(const float* qv, const float* __restrict__ xf, int64_t x, int32_t dim, bool vec) {
    const float* xv = xf + x * dim;
    float e = 0.f;
    int j = 0;
    if (vec)
        for (; j < dim; j += 4) {
            const float4 r = __ldg(reinterpret_cast<const float4*>(xv + j));
            float t = qv[j] - r.x;
            e = fmaf(t, t, e);
            t = qv[j + 1] - r.y;
            e = fmaf(t, t, e);
            t = qv[j + 2] - r.z;
            e = fmaf(t, t, e);
            t = qv[j + 3] - r.w;
            e = fmaf(t, t, e);
        }
    for (; j < dim; ++j) {
        const float t = qv[j] - xv[j];
        e = fmaf(t, t, e);
    }
    return e;
}

// Ascending block-wide bitonic sort of P keys (P a power of two) in shared memory.
template <int kThreads>
__device__ void bitonic_sort(unsigned long long* a, int P) {
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += kThreads) {
                const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long u = a[lo], w = a[hi];
                if ((u > w) == up) {
                    a[lo] = w;
                    a[hi] = u;
                }
            }
            __syncthreads();
        }
}

struct RerankArgs {
    const unsigned long long* cand;   // [nq][cap] candidate keys okey(a) << 32 | row
    const int32_t* cnt;               // [nq]
    int32_t cap, k;
    const float* qf;                  // [nq][dim] float32 queries
    const float* xf;                  // [rows][dim] float32 rows
    int32_t dim;
    const float* qn;                  // [nq]
    const float* rq;                  // [nq]
    const float* maxima;              // [2]
    int32_t kpad;
    int32_t* ids;                     // [nq][k]
    float* dists;                     // [nq][k]
    int32_t* ov;                      // [0] count, [1..] queries left for the CUDA-core path
    int32_t inline_n;                 // > 0: such a query is finished here, exactly, over all inline_n rows
    const int32_t* error;             // nonzero: a tensor-core wait ran out; the results are ids -1
};

// Re-rank (step 4). Dynamic shared memory: the query row, then two arrays of `cap` 64-bit keys
// (cap a power of 2), or, for the inline fallback, the keys of all rows.
__global__ void __launch_bounds__(kRerankThreads) rerank_kernel(const RerankArgs A) {
    extern __shared__ __align__(16) unsigned long long rk[];
    const int dim4 = (A.dim + 3) & ~3;
    float* qv = reinterpret_cast<float*>(rk);
    unsigned long long* keys = rk + dim4 / 2;
    unsigned long long* sel = keys + A.cap;
    __shared__ uint32_t hist[256], prefix_s, rank_s;
    __shared__ int m_s;
    const int64_t q = blockIdx.x;
    const int k = A.k;
    if (A.error && *A.error) {
        for (int i = threadIdx.x; i < k; i += kRerankThreads) {
            A.ids[q * k + i] = -1;
            A.dists[q * k + i] = __int_as_float(0x7f800000);
        }
        return;
    }
    const int c = A.cnt[q];
    if (c > A.cap && A.inline_n == 0) {                  // recomputed by the CUDA-core path
        if (threadIdx.x == 0) A.ov[1 + atomicAdd(A.ov, 1)] = (int32_t)q;
        return;
    }
    for (int j = threadIdx.x; j < A.dim; j += kRerankThreads) qv[j] = A.qf[q * A.dim + j];
    const bool vec = (A.dim & 3) == 0 && (reinterpret_cast<uintptr_t>(A.xf) & 15) == 0;
    if (c > A.cap) {                                     // every row, exactly
        __syncthreads();
        int P = 1;
        while (P < A.inline_n) P <<= 1;
        for (int i = threadIdx.x; i < P; i += kRerankThreads)
            keys[i] = i < A.inline_n ? ((unsigned long long)__float_as_uint(exact_row_d2(qv, A.xf, i, A.dim, vec)) << 32) | (uint32_t)i
                                     : ~0ull;
        __syncthreads();
        bitonic_sort<kRerankThreads>(keys, P);
        for (int i = threadIdx.x; i < k; i += kRerankThreads) {
            A.ids[q * k + i] = (int32_t)(uint32_t)keys[i];
            A.dists[q * k + i] = sqrtf(__uint_as_float((uint32_t)(keys[i] >> 32)));
        }
        return;
    }
    for (int i = threadIdx.x; i < c; i += kRerankThreads) keys[i] = A.cand[q * A.cap + i];
    if (threadIdx.x == 0) m_s = 0;
    __syncthreads();
    const uint32_t tk = radix_select32<kRerankThreads>(c, (uint32_t)(k - 1), [&](int i) { return (uint32_t)(keys[i] >> 32); },
                                                       hist, &prefix_s, &rank_s);
    const float lim = window_limit(from_okey(tk), error_bound(A.qn[q], A.rq[q], A.maxima[0], A.maxima[1], A.kpad));
    for (int i = threadIdx.x; i < c; i += kRerankThreads) {
        const unsigned long long key = keys[i];
        if (from_okey((uint32_t)(key >> 32)) > lim) continue;
        const uint32_t x = (uint32_t)key;
        const float e = exact_row_d2(qv, A.xf, x, A.dim, vec);
        sel[atomicAdd(&m_s, 1)] = ((unsigned long long)__float_as_uint(e) << 32) | x;
    }
    __syncthreads();
    const int m = m_s;
    int P = 1;
    while (P < m) P <<= 1;
    for (int i = m + threadIdx.x; i < P; i += kRerankThreads) sel[i] = ~0ull;
    __syncthreads();
    bitonic_sort<kRerankThreads>(sel, P);
    for (int i = threadIdx.x; i < k; i += kRerankThreads) {
        A.ids[q * k + i] = (int32_t)(uint32_t)sel[i];
        A.dists[q * k + i] = sqrtf(__uint_as_float((uint32_t)(sel[i] >> 32)));
    }
}

// k = 1, one warp per query: limit = window_limit(min of the group minima, b_q).
__global__ void nearest_limit_kernel(const float* __restrict__ gmin, int ng, int64_t nq, const float* __restrict__ qn,
                                     const float* __restrict__ rq, const float* __restrict__ maxima, int32_t kpad,
                                     float* __restrict__ limit) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nq) return;
    float m = __int_as_float(0x7f800000);
    for (int i = lane; i < ng; i += 32) m = fminf(m, gmin[q * ng + i]);
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) limit[q] = window_limit(m, error_bound(qn[q], rq[q], maxima[0], maxima[1], kpad));
}

// k = 1, one warp per query: the exact (distance, row) minimum over the candidates, or over every
// row when they overflowed. All candidates are scored, so no selection is needed.
__global__ void nearest_finish_kernel(const unsigned long long* __restrict__ cand, const int32_t* __restrict__ cnt, int cap,
                                      const float* __restrict__ qf, const float* __restrict__ xf, int32_t dim, int64_t n,
                                      int64_t nq, int32_t* __restrict__ ids, float* __restrict__ dists,
                                      const int32_t* __restrict__ error) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nq) return;
    if (*error) {
        if (lane == 0) {
            ids[q] = -1;
            dists[q] = __int_as_float(0x7f800000);
        }
        return;
    }
    const float* qv = qf + q * dim;
    const bool vec = (dim & 3) == 0 && (reinterpret_cast<uintptr_t>(xf) & 15) == 0 && (reinterpret_cast<uintptr_t>(qf) & 15) == 0;
    const int c = cnt[q];
    unsigned long long best = ~0ull;
    if (c <= cap) {
        for (int i = lane; i < c; i += 32) {
            const uint32_t x = (uint32_t)cand[q * cap + i];
            best = min(best, ((unsigned long long)__float_as_uint(exact_row_d2(qv, xf, x, dim, vec)) << 32) | x);
        }
    } else {
        for (int64_t x = lane; x < n; x += 32)
            best = min(best, ((unsigned long long)__float_as_uint(exact_row_d2(qv, xf, x, dim, vec)) << 32) | (uint32_t)x);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
        best = min(best, t);
    }
    if (lane == 0) {
        ids[q] = (int32_t)(uint32_t)best;
        dists[q] = sqrtf(__uint_as_float((uint32_t)(best >> 32)));
    }
}

// Smem bytes of rerank_kernel.
int rerank_smem_bytes(int cap, int dim, int inline_n) {
    int P = 1;
    while (P < inline_n) P <<= 1;
    return 4 * ((dim + 3) & ~3) + 8 * std::max(2 * cap, inline_n > 0 ? P : 0);
}

__global__ void gather_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ list, int count, int32_t dim,
                                   float* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)count * dim;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[(int64_t)list[i / dim] * dim + i % dim];
}

__global__ void scatter_results_kernel(const int32_t* __restrict__ gid, const float* __restrict__ gd,
                                       const int32_t* __restrict__ list, int count, int k, int32_t* __restrict__ ids,
                                       float* __restrict__ dists) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)count * k;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = list[i / k];
        ids[q * k + i % k] = gid[i];
        dists[q * k + i % k] = gd[i];
    }
}

// xs[j] = xn[j * stride] for j < ns; zero up to `padded`.
__global__ void strided_norms_kernel(const float* __restrict__ xn, int64_t stride, int64_t ns, int64_t padded,
                                     float* __restrict__ xs) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < padded; j += (int64_t)gridDim.x * blockDim.x)
        xs[j] = j < ns ? xn[j * stride] : 0.f;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                   const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no link to libcuda).
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// 2-D bf16 map over `rows` rows of `kpad` elements, `row_bytes` apart; box 64 x box_rows with the
// 128-byte swizzle; rows past the end read as zero.
bool make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t kpad, uint64_t row_bytes, uint32_t box_rows) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {kpad, rows};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)KC, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// dst[i][0 .. dim) = src[(ids ? ids[i] : i) * stride + 0 .. dim)
__global__ void gather_plan_rows_kernel(const float* __restrict__ src, int64_t stride, const int32_t* __restrict__ ids,
                                        int64_t n, int32_t dim, float* __restrict__ dst) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * dim; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / dim;
        dst[t] = src[(ids ? (int64_t)ids[i] : i) * stride + t % dim];
    }
}

// The dynamic shared-memory limit is one process-wide setting per kernel: raise it, once, to the
// device's opt-in maximum (occupancy follows the bytes each launch asks for, not this limit).
template <typename F>
cudaError_t open_smem_limit(F* f, int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

cudaError_t open_smem_limits() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = open_smem_limit(dist_tc_kernel<false>, optin);
    if (e == cudaSuccess) e = open_smem_limit(dist_tc_kernel<true>, optin);
    if (e == cudaSuccess) e = open_smem_limit(rerank_kernel, optin);
    return e;
}

struct Scratch {
    void* p[13] = {};
    ~Scratch() {
        for (void* q : p) cudaFree(q);
    }
};

// launch_knn_exact's scratch, kept between calls: per device, grown when a call needs more, made
// again in a new context of the device (the old context's memory went with it). The lock is held
// for the whole call, which ends with its stream synchronised, so no call's kernels use a buffer
// that another call frees or grows.
struct KnnScratch {
    std::mutex mu;
    unsigned long long ctx = 0;
    void* p[13] = {};
    size_t bytes[13] = {};
};
KnnScratch g_knn_scratch[64];

}  // namespace

int launch_knn_exact(const float* base, int64_t n, const float* queries, int64_t nq, int32_t dim, int32_t k,
                     int32_t* ids, float* dists, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (k > n) return *why = "k larger than n", (int)cudaErrorInvalidValue;
    if (nq == 0) return 0;
    if (n > INT32_MAX - TN) return *why = "n too large", (int)cudaErrorInvalidValue;   // work items fit 31 bits
    const int32_t kpad = (dim + KC - 1) / KC * KC;
    const int64_t stride = (n + kSampleMax - 1) / kSampleMax;
    const int64_t ns = (n + stride - 1) / stride;
    const int64_t ng = (ns + kGroup - 1) / kGroup;
    const int64_t chunk = std::min<int64_t>((nq + TM - 1) / TM * TM, 16384);
    // about k * stride rows fall below the sampled threshold; room for twice that
    int cap = 1024;
    while (cap < kCandCapMax && (int64_t)cap < 2 * (int64_t)k * stride) cap <<= 1;
    const int64_t tiles_n = (n + TN - 1) / TN, tiles_s = (ns + TN - 1) / TN;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    if (dev < 0 || dev >= 64) return *why = "device index above 63", (int)cudaErrorInvalidValue;
    KnnScratch& s = g_knn_scratch[dev];
    std::lock_guard<std::mutex> lock(s.mu);
    unsigned long long ctx = current_context_id();
    if (ctx == 0) {
        cudaFree(nullptr);                                   // makes the device's context current
        ctx = current_context_id();
    }
    if (ctx == 0 || ctx != s.ctx) {
        for (int i = 0; i < 13; ++i) {
            s.p[i] = nullptr;
            s.bytes[i] = 0;
        }
        s.ctx = ctx;
    }
    const size_t sizes[] = {2ull * n * kpad, 4ull * tiles_n * TN, 4ull * n, 2ull * nq * kpad, 4ull * nq, 4ull * nq, 16,
                            4ull * chunk * ng, 4ull * chunk, 8ull * chunk * cap, 4ull * chunk, 4ull * (chunk + 2),
                            4ull * tiles_s * TN};
    for (int i = 0; i < 13 && e == cudaSuccess; ++i) {
        const size_t need = std::max<size_t>(sizes[i], 16);
        if (s.bytes[i] >= need) continue;
        if (s.p[i]) cudaFree(s.p[i]);
        s.p[i] = nullptr;
        s.bytes[i] = 0;
        if ((e = cudaMalloc(&s.p[i], need)) == cudaSuccess) s.bytes[i] = need;
    }
    if (e != cudaSuccess) return *why = std::string("knn scratch: ") + cudaGetErrorString(e), (int)e;
    auto* xb = static_cast<__nv_bfloat16*>(s.p[0]);
    auto* xn = static_cast<float*>(s.p[1]);
    auto* xr = static_cast<float*>(s.p[2]);
    auto* qb = static_cast<__nv_bfloat16*>(s.p[3]);
    auto* qn = static_cast<float*>(s.p[4]);
    auto* qr = static_cast<float*>(s.p[5]);
    auto* maxima = static_cast<float*>(s.p[6]);
    auto* gmin = static_cast<float*>(s.p[7]);
    auto* limit = static_cast<float*>(s.p[8]);
    auto* cand = static_cast<unsigned long long*>(s.p[9]);
    auto* cnt = static_cast<int32_t*>(s.p[10]);
    auto* ov = static_cast<int32_t*>(s.p[11]);         // [0] overflow count, [1..chunk] queries, [chunk+1] error
    auto* xs = static_cast<float*>(s.p[12]);
    int32_t* err = ov + chunk + 1;
    const int rerank_smem = rerank_smem_bytes(cap, dim, 0);
    if ((e = open_smem_limits()) != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    CUtensorMap tq, tx_all, tx_sample;
    if (!make_map(&tq, qb, nq, kpad, 2ull * kpad, TM) || !make_map(&tx_all, xb, n, kpad, 2ull * kpad, TN) ||
        !make_map(&tx_sample, xb, ns, kpad, 2ull * kpad * stride, TN))
        return *why = "tensor map encoding failed", (int)cudaErrorInvalidValue;
    cudaMemsetAsync(maxima, 0, 16, st);
    cudaMemsetAsync(xn, 0, 4ull * tiles_n * TN, st);
    bf16_rows_kernel<<<2048, 256, 0, st>>>(base, n, dim, kpad, xb, xn, xr);
    bf16_rows_kernel<<<1024, 256, 0, st>>>(queries, nq, dim, kpad, qb, qn, qr);
    row_maxima_kernel<<<304, 256, 0, st>>>(xn, xr, n, maxima);
    strided_norms_kernel<<<256, 256, 0, st>>>(xn, stride, ns, tiles_s * TN, xs);
    for (int64_t q0 = 0; q0 < nq && e == cudaSuccess; q0 += chunk) {
        const int64_t qc = std::min(chunk, nq - q0);
        const int32_t qblocks = (int32_t)((qc + TM - 1) / TM);
        auto grid = [&](int64_t tiles) { return (unsigned)std::min<int64_t>((int64_t)qblocks * tiles, sms); };
        const TcArgs sa{(int32_t)q0, (int32_t)qc, qblocks, ns, tiles_s, kpad / KC, qn + q0, xs, gmin, nullptr, nullptr, nullptr, 0, err};
        const TcArgs fa{(int32_t)q0, (int32_t)qc, qblocks, n, tiles_n, kpad / KC, qn + q0, xn, nullptr, limit, cand, cnt, cap, err};
        cudaMemsetAsync(ov, 0, 4ull * (chunk + 2), st);
        cudaMemsetAsync(cnt, 0, 4ull * qc, st);
        dist_tc_kernel<false><<<grid(tiles_s), kTcThreads, kSmemDyn, st>>>(tq, tx_sample, sa);
        sample_limit_kernel<<<(unsigned)qc, kSelThreads, 0, st>>>(gmin, (int)ng, k, qn + q0, qr + q0, maxima, kpad, limit);
        dist_tc_kernel<true><<<grid(tiles_n), kTcThreads, kSmemDyn, st>>>(tq, tx_all, fa);
        const RerankArgs ra{cand, cnt, cap, k, queries + q0 * dim, base, dim, qn + q0, qr + q0, maxima, kpad,
                            ids + q0 * k, dists + q0 * k, ov, 0, nullptr};
        rerank_kernel<<<(unsigned)qc, kRerankThreads, rerank_smem, st>>>(ra);
        int32_t flags[2] = {0, 0};
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(&flags[0], ov, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(&flags[1], err, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        if (flags[1]) return *why = "a tensor-core wait exceeded its limit", (int)cudaErrorLaunchTimeout;
        if (flags[0] > 0) {                              // too many candidates: the CUDA-core path
            const int nov = flags[0];
            Scratch g;
            if ((e = cudaMalloc(&g.p[0], 4ull * nov * dim)) != cudaSuccess || (e = cudaMalloc(&g.p[1], 4ull * nov * k)) != cudaSuccess ||
                (e = cudaMalloc(&g.p[2], 4ull * nov * k)) != cudaSuccess)
                break;
            gather_rows_kernel<<<256, 256, 0, st>>>(queries + q0 * dim, ov + 1, nov, dim, static_cast<float*>(g.p[0]));
            const int r = launch_knn_simt(base, n, static_cast<float*>(g.p[0]), nov, dim, k, static_cast<int32_t*>(g.p[1]),
                                          static_cast<float*>(g.p[2]), stream, why);
            if (r != 0) return r;
            scatter_results_kernel<<<256, 256, 0, st>>>(static_cast<int32_t*>(g.p[1]), static_cast<float*>(g.p[2]), ov + 1,
                                                        nov, k, ids + q0 * k, dists + q0 * k);
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        }
    }
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

// ---- k-NN plan over a small fixed row set (entry routing) ------------------------------------
// The same pipeline as launch_knn_exact, with the rows' bfloat16 copy, norms and tensor map made
// once, scratch kept between calls, and no host synchronisation: a query with more candidates
// than `cap` is finished exactly inside the re-rank kernel over all rows (at most kPlanRowsMax).
struct KnnPlan {
    int64_t n = 0;
    int32_t dim = 0, kpad = 0, k = 0, cap = 0, sms = 0, rerank_smem = 0;
    int64_t tiles = 0, ng = 0;
    float* x32 = nullptr;             // [n][dim] contiguous float32 rows
    __nv_bfloat16* xb = nullptr;      // [n][kpad]
    float* xn = nullptr;              // [tiles * 256], zero padded
    float* xr = nullptr;              // [n]
    float* maxima = nullptr;          // [2]
    CUtensorMap tx;
    int64_t cap_q = 0;                // queries the scratch below holds
    __nv_bfloat16* qb = nullptr;
    float *qn = nullptr, *qr = nullptr, *gmin = nullptr, *limit = nullptr, *dscr = nullptr;
    unsigned long long* cand = nullptr;
    int32_t *cnt = nullptr, *flags = nullptr;   // flags: [0] error, [1] unused overflow count
};

namespace {
void plan_free_scratch(KnnPlan* p) {
    cudaFree(p->qb);
    cudaFree(p->qn);
    cudaFree(p->qr);
    cudaFree(p->gmin);
    cudaFree(p->limit);
    cudaFree(p->dscr);
    cudaFree(p->cand);
    cudaFree(p->cnt);
    cudaFree(p->flags);
    p->qb = nullptr;
    p->qn = p->qr = p->gmin = p->limit = p->dscr = nullptr;
    p->cand = nullptr;
    p->cnt = p->flags = nullptr;
    p->cap_q = 0;
}
}  // namespace

void knn_plan_destroy(KnnPlan* p) {
    if (!p) return;
    plan_free_scratch(p);
    cudaFree(p->x32);
    cudaFree(p->xb);
    cudaFree(p->xn);
    cudaFree(p->xr);
    cudaFree(p->maxima);
    delete p;
}

int knn_plan_create(KnnPlan** out, const float* rows, int64_t row_stride, const int32_t* row_ids, int64_t n, int32_t dim,
                    int32_t k, int32_t cap, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    *out = nullptr;
    if (n < 1 || n > kPlanRowsMax || k < 1 || k > n || dim < 1 || cap < 1 || (cap & (cap - 1)))
        return *why = "knn plan: bad sizes", (int)cudaErrorInvalidValue;
    KnnPlan* p = new KnnPlan;
    p->n = n;
    p->dim = dim;
    p->kpad = (dim + KC - 1) / KC * KC;
    p->k = k;
    p->cap = cap;
    p->tiles = (n + TN - 1) / TN;
    p->ng = (n + 15) / 16;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev);
    p->rerank_smem = rerank_smem_bytes(cap, dim, (int)n);
    cudaError_t e;
    if ((e = cudaMalloc(&p->x32, 4ull * n * dim)) != cudaSuccess || (e = cudaMalloc(&p->xb, 2ull * n * p->kpad)) != cudaSuccess ||
        (e = cudaMalloc(&p->xn, 4ull * p->tiles * TN)) != cudaSuccess || (e = cudaMalloc(&p->xr, 4ull * n)) != cudaSuccess ||
        (e = cudaMalloc(&p->maxima, 16)) != cudaSuccess || (e = open_smem_limits()) != cudaSuccess) {
        knn_plan_destroy(p);
        return *why = std::string("knn plan: ") + cudaGetErrorString(e), (int)e;
    }
    cudaMemsetAsync(p->xn, 0, 4ull * p->tiles * TN, st);
    cudaMemsetAsync(p->maxima, 0, 16, st);
    gather_plan_rows_kernel<<<256, 256, 0, st>>>(rows, row_stride, row_ids, n, dim, p->x32);
    bf16_rows_kernel<<<256, 256, 0, st>>>(p->x32, n, dim, p->kpad, p->xb, p->xn, p->xr);
    row_maxima_kernel<<<64, 256, 0, st>>>(p->xn, p->xr, n, p->maxima);
    if (!make_map(&p->tx, p->xb, n, p->kpad, 2ull * p->kpad, TN)) {
        knn_plan_destroy(p);
        return *why = "knn plan: tensor map encoding failed", (int)cudaErrorInvalidValue;
    }
    if ((e = cudaGetLastError()) == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        knn_plan_destroy(p);
        return *why = std::string("knn plan: ") + cudaGetErrorString(e), (int)e;
    }
    *out = p;
    return 0;
}

int knn_plan_run(KnnPlan* p, const float* queries, int64_t nq, int32_t* ids, float* dists, deg_stream_t stream,
                 std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (nq <= 0) return 0;
    if (nq > (int64_t)1 << 24) return *why = "knn plan: too many queries", (int)cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (nq > p->cap_q) {                                  // grow the scratch (the only allocation)
        plan_free_scratch(p);
        const int64_t c = std::max<int64_t>(1024, (nq + TM - 1) / TM * TM);
        if ((e = cudaMalloc(&p->qb, 2ull * c * p->kpad)) != cudaSuccess || (e = cudaMalloc(&p->qn, 4ull * c)) != cudaSuccess ||
            (e = cudaMalloc(&p->qr, 4ull * c)) != cudaSuccess || (e = cudaMalloc(&p->gmin, 4ull * c * p->ng)) != cudaSuccess ||
            (e = cudaMalloc(&p->limit, 4ull * c)) != cudaSuccess || (e = cudaMalloc(&p->dscr, 4ull * c * p->k)) != cudaSuccess ||
            (e = cudaMalloc(&p->cand, 8ull * c * p->cap)) != cudaSuccess || (e = cudaMalloc(&p->cnt, 4ull * c)) != cudaSuccess ||
            (e = cudaMalloc(&p->flags, 16)) != cudaSuccess) {
            plan_free_scratch(p);
            return *why = std::string("knn plan scratch: ") + cudaGetErrorString(e), (int)e;
        }
        p->cap_q = c;
    }
    CUtensorMap tq;
    if (!make_map(&tq, p->qb, nq, p->kpad, 2ull * p->kpad, TM))
        return *why = "knn plan: tensor map encoding failed", (int)cudaErrorInvalidValue;
    const int32_t qblocks = (int32_t)((nq + TM - 1) / TM);
    const unsigned grid = (unsigned)std::min<int64_t>((int64_t)qblocks * p->tiles, p->sms);
    cudaMemsetAsync(p->flags, 0, 16, st);
    cudaMemsetAsync(p->cnt, 0, 4ull * nq, st);
    bf16_rows_kernel<<<256, 256, 0, st>>>(queries, nq, p->dim, p->kpad, p->qb, p->qn, p->qr);
    const TcArgs sa{0, (int32_t)nq, qblocks, p->n, p->tiles, p->kpad / KC, p->qn, p->xn, p->gmin, nullptr, nullptr, nullptr, 0,
                    p->flags};
    const TcArgs fa{0, (int32_t)nq, qblocks, p->n, p->tiles, p->kpad / KC, p->qn, p->xn, nullptr, p->limit, p->cand, p->cnt,
                    p->cap, p->flags};
    dist_tc_kernel<false><<<grid, kTcThreads, kSmemDyn, st>>>(tq, p->tx, sa);
    const unsigned wblocks = (unsigned)((nq + 7) / 8);   // one warp per query, 8 per block
    if (p->k == 1)
        nearest_limit_kernel<<<wblocks, 256, 0, st>>>(p->gmin, (int)p->ng, nq, p->qn, p->qr, p->maxima, p->kpad, p->limit);
    else
        sample_limit_kernel<<<(unsigned)nq, kSelThreads, 0, st>>>(p->gmin, (int)p->ng, p->k, p->qn, p->qr, p->maxima, p->kpad,
                                                                  p->limit);
    dist_tc_kernel<true><<<grid, kTcThreads, kSmemDyn, st>>>(tq, p->tx, fa);
    if (p->k == 1) {
        nearest_finish_kernel<<<wblocks, 256, 0, st>>>(p->cand, p->cnt, p->cap, queries, p->x32, p->dim, p->n, nq, ids,
                                                       dists ? dists : p->dscr, p->flags);
    } else {
        const RerankArgs ra{p->cand, p->cnt, p->cap, p->k, queries, p->x32, p->dim, p->qn, p->qr, p->maxima, p->kpad,
                            ids, dists ? dists : p->dscr, p->flags + 1, (int32_t)p->n, p->flags};
        rerank_kernel<<<(unsigned)nq, kRerankThreads, p->rerank_smem, st>>>(ra);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

}  // namespace deg
