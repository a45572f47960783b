// Exact k nearest neighbours (paper Eq. 1) with the distance contraction on the 5th-generation
// tensor cores. The result equals the CUDA-core path's bit for bit: the same float32 distances
// sum_d fmaf(q_d - x_d, q_d - x_d, .) in dimension order, ties ordered by id.
//
// Per chunk of queries:
//   1. bfloat16 copies of rows and queries (K padded to a multiple of 64), with float32 squared
//      norms and the norms of the rounding residuals x - bf16(x);
//   2. sample pass: approximate squared distances a = |q|^2 + |x|^2 - 2 bf16(q).bf16(x) of every
//      query against every s-th row (tcgen05.mma.kind::f16, float32 accumulators in tensor memory);
//      t_s = the k-th smallest of them is at least the k-th smallest a over all rows;
//   3. filter pass: a against every row; a row is a candidate when a <= t_s + 2b, where b bounds
//      |a - e| for the float32 distance e (bfloat16 rounding, accumulation and norm rounding; see
//      error_bound). If e_k is the k-th smallest e, the k rows with the smallest a have e <= t + b
//      (t = k-th smallest a), so e_k <= t + b and every row with e <= e_k has a <= t + 2b <= t_s + 2b:
//      all true neighbours, ties included, are candidates;
//   4. re-rank: per query, t = the k-th smallest a among the candidates (it is the global one), the
//      rows with a <= t + 2b get e computed exactly, sorted by (e, id), the first k returned.
// A query with more candidates than the buffer holds is recomputed by the CUDA-core path.
//
// Tensor-core tile: M = 128 queries (tensor-memory lanes) x N = 256 rows (tensor-memory columns),
// K staged 64 at a time in the no-swizzle K-major layout of 8-row x 16-byte core matrices. Two
// CTAs per SM (shared memory sized for it) so that one stages while the other multiplies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "deg_internal.h"

namespace deg {
namespace {

constexpr int TM = 128, TN = 256, KC = 64, KC8 = KC / 8;
constexpr int kTcThreads = 128;
constexpr int kAResident = 256;                         // query K extent kept resident in shared memory
constexpr int kSmemA = TM * kAResident * 2;             // 64 KiB
constexpr int kSmemB = TN * KC * 2;                     // 32 KiB
constexpr int kSmemDyn = kSmemA + kSmemB + 1024;        // + alignment slack; caps residency at 2 CTAs/SM
constexpr int kChunkBytes = TM * KC * 2;                // one K chunk of the query tile
constexpr int64_t kSampleMax = 32768;                   // sample rows per query
constexpr int kCandCap = 8192;                          // candidates per query
constexpr int kSelThreads = 1024;
constexpr int kRerankThreads = 512;
constexpr unsigned long long kWaitNs = 2000000000ull;   // bounded wait on the tensor core: 2 s

// Instruction descriptor, kind::f16: D float32 (bits 4-5 = 1), A and B bfloat16 (bits 7-9, 10-12
// = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading byte offset (between core matrices
// along K), stride byte offset (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
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

// Copies rows [row0, row0 + rows) x columns [k0, k0 + KC) of a bf16 matrix (row r at
// src + r * stride * kpad) into the core-matrix layout: core (r / 8, c / 8) at
// ((r / 8) * KC8 + c / 8) * 128 bytes, row r % 8 of it at + (r % 8) * 16. Consecutive threads
// write consecutive 16-byte pieces; rows beyond `valid` are zero.
__device__ __forceinline__ void stage(uint8_t* dst, const __nv_bfloat16* __restrict__ src, int64_t row0, int64_t valid,
                                      int64_t stride, int rows, int32_t kpad, int k0) {
    for (int t = threadIdx.x; t < rows * KC8; t += kTcThreads) {
        const int r8 = t & 7, kc = (t >> 3) % KC8, m8 = (t >> 3) / KC8;
        const int64_t row = row0 + m8 * 8 + r8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (row < valid) v = *reinterpret_cast<const uint4*>(src + row * stride * kpad + k0 + kc * 8);
        *reinterpret_cast<uint4*>(dst + t * 16) = v;
    }
}

struct TcArgs {
    const __nv_bfloat16* qb;       // [nq][kpad]
    const float* qn;               // [nq]
    int64_t nq;
    const __nv_bfloat16* xb;       // rows, row c of this pass at xb + c * row_stride * kpad
    const float* xn;               // row norms, same indexing
    int64_t ncols;                 // rows in this pass
    int64_t row_stride;
    int32_t kpad;
    float* D;                      // sample pass: [nq][ncols]
    const float* limit;            // filter pass: [nq]
    unsigned long long* cand;      // filter pass: [nq][cap] keys okey(a) << 32 | row
    int32_t* cnt;                  // filter pass: [nq]
    int32_t cap;
    int32_t* error;                // set to 1 when a tensor-core wait ran out
};

// Grid: x = query tile (128 queries), y = column stripe; CTA (x, y) walks column tiles y, y + gy, ...
// The query tile's K extent stays in shared memory when kpad <= 256, else it is staged per chunk.
template <bool kFilter>
__global__ void __launch_bounds__(kTcThreads, 2) dist_tc_kernel(TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    uint8_t* As = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* Bs = As + kSmemA;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q0 = (int64_t)blockIdx.x * TM;
    const uint32_t mb = smem_u32(&mbar);
    const int nk = a.kpad / KC;
    const bool a_resident = a.kpad <= kAResident;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (a_resident)
        for (int kc = 0; kc < nk; ++kc) stage(As + kc * kChunkBytes, a.qb, q0, a.nq, 1, TM, a.kpad, kc * KC);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const int64_t qrow = q0 + warp * 32 + lane;           // the query in this thread's tensor-memory lane
    const bool qvalid = qrow < a.nq;
    const float qnorm = qvalid ? a.qn[qrow] : 0.f;
    const float lim = (kFilter && qvalid) ? a.limit[qrow] : 0.f;
    const int64_t tiles = (a.ncols + TN - 1) / TN;
    uint32_t phase = 0;
    bool failed = false;
    for (int64_t tile = blockIdx.y; tile < tiles && !failed; tile += gridDim.y) {
        const int64_t x0 = tile * TN;
        for (int kc = 0; kc < nk; ++kc) {
            const uint8_t* Ak = a_resident ? As + kc * kChunkBytes : As;
            if (!a_resident) stage(As, a.qb, q0, a.nq, 1, TM, a.kpad, kc * KC);
            stage(Bs, a.xb, x0, a.ncols, a.row_stride, TN, a.kpad, kc * KC);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");      // generic writes -> tensor core
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int s = 0; s < KC / 16; ++s) {
                    const uint64_t ad = make_desc(smem_u32(Ak) + s * 256, 128, KC8 * 128);
                    const uint64_t bd = make_desc(smem_u32(Bs) + s * 256, 128, KC8 * 128);
                    const uint32_t accumulate = (kc > 0 || s > 0) ? 1u : 0u;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                 ::"r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(accumulate) : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                             : "memory");
            }
            const bool ok = mbar_wait(mb, phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {                  // block-uniform decision
                failed = true;
                break;
            }
        }
        if (failed) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                           "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                         : "r"(taddr) : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (!qvalid) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int64_t x = x0 + c0 + j;
                if (x >= a.ncols) break;
                const float d = qnorm + __ldg(a.xn + x * a.row_stride) - 2.f * __uint_as_float(v[j]);
                if (kFilter) {
                    if (d <= lim) {
                        const int p = atomicAdd(a.cnt + qrow, 1);
                        if (p < a.cap) a.cand[qrow * a.cap + p] = ((unsigned long long)okey(d) << 32) | (uint32_t)x;
                    }
                } else {
                    a.D[qrow * a.ncols + x] = d;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (failed) {
        // the last commit may still be outstanding: wait for it once more (bounded), then free
        const bool ok = mbar_wait(mb, phase ^ 1u);
        (void)ok;
        if (threadIdx.x == 0) atomicExch(a.error, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
}

// Radix select over `count` 32-bit keys: the key of rank `rank` (0-based), keys read through
// get(i); four passes of 8-bit digits.
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
        for (int i = threadIdx.x; i < count; i += kThreads) {
            const uint32_t kv = get(i);
            if ((kv & hmask) == (want & hmask)) atomicAdd(&hist[(kv >> shift) & 0xffu], 1u);
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

// limit[q] = window_limit(k-th smallest sampled a, b_q). Dynamic shared memory: ns keys.
__global__ void __launch_bounds__(kSelThreads) sample_limit_kernel(const float* __restrict__ Ds, int64_t ns, int k,
                                                                  const float* __restrict__ qn, const float* __restrict__ rq,
                                                                  const float* __restrict__ maxima, int32_t kpad,
                                                                  float* __restrict__ limit) {
    extern __shared__ uint32_t skeys[];
    __shared__ uint32_t hist[256], prefix_s, rank_s;
    const int64_t q = blockIdx.x;
    for (int64_t i = threadIdx.x; i < ns; i += kSelThreads) skeys[i] = okey(Ds[q * ns + i]);
    __syncthreads();
    const uint32_t tk = radix_select32<kSelThreads>((int)ns, (uint32_t)(k - 1), [&](int i) { return skeys[i]; }, hist,
                                                    &prefix_s, &rank_s);
    if (threadIdx.x == 0) limit[q] = window_limit(from_okey(tk), error_bound(qn[q], rq[q], maxima[0], maxima[1], kpad));
}

// Re-rank (step 4). Dynamic shared memory: two arrays of kCandCap 64-bit keys.
__global__ void __launch_bounds__(kRerankThreads) rerank_kernel(const unsigned long long* __restrict__ cand,
                                                               const int32_t* __restrict__ cnt, int k,
                                                               const float* __restrict__ qf, const float* __restrict__ xf,
                                                               int32_t dim, const float* __restrict__ qn,
                                                               const float* __restrict__ rq, const float* __restrict__ maxima,
                                                               int32_t kpad, int32_t* __restrict__ ids,
                                                               float* __restrict__ dists, int32_t* __restrict__ ov) {
    extern __shared__ unsigned long long rk[];
    unsigned long long* keys = rk;
    unsigned long long* sel = rk + kCandCap;
    __shared__ uint32_t hist[256], prefix_s, rank_s;
    __shared__ int m_s;
    const int64_t q = blockIdx.x;
    const int c = cnt[q];
    if (c > kCandCap) {                                  // recomputed by the CUDA-core path
        if (threadIdx.x == 0) ov[1 + atomicAdd(ov, 1)] = (int32_t)q;
        return;
    }
    for (int i = threadIdx.x; i < c; i += kRerankThreads) keys[i] = cand[q * kCandCap + i];
    if (threadIdx.x == 0) m_s = 0;
    __syncthreads();
    const uint32_t tk = radix_select32<kRerankThreads>(c, (uint32_t)(k - 1), [&](int i) { return (uint32_t)(keys[i] >> 32); },
                                                       hist, &prefix_s, &rank_s);
    const float lim = window_limit(from_okey(tk), error_bound(qn[q], rq[q], maxima[0], maxima[1], kpad));
    const float* qv = qf + q * dim;
    for (int i = threadIdx.x; i < c; i += kRerankThreads) {
        const unsigned long long key = keys[i];
        if (from_okey((uint32_t)(key >> 32)) > lim) continue;
        const uint32_t x = (uint32_t)key;
        const float* xv = xf + (int64_t)x * dim;
        float e = 0.f;
        for (int j = 0; j < dim; ++j) {                  // dimension order, as the CUDA-core path
            const float u = qv[j] - xv[j];
            e = fmaf(u, u, e);
        }
        sel[atomicAdd(&m_s, 1)] = ((unsigned long long)__float_as_uint(e) << 32) | x;
    }
    __syncthreads();
    const int m = m_s;
    int P = 1;
    while (P < m) P <<= 1;
    for (int i = m + threadIdx.x; i < P; i += kRerankThreads) sel[i] = ~0ull;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += kRerankThreads) {
                const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long u = sel[lo], w = sel[hi];
                if ((u > w) == up) {
                    sel[lo] = w;
                    sel[hi] = u;
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < k; i += kRerankThreads) {
        ids[q * k + i] = (int32_t)(uint32_t)sel[i];
        dists[q * k + i] = sqrtf(__uint_as_float((uint32_t)(sel[i] >> 32)));
    }
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

struct Scratch {
    void* p[12] = {};
    ~Scratch() {
        for (void* q : p) cudaFree(q);
    }
};

}  // namespace

int launch_knn_exact(const float* base, int64_t n, const float* queries, int64_t nq, int32_t dim, int32_t k,
                     int32_t* ids, float* dists, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (k > n) return *why = "k larger than n", (int)cudaErrorInvalidValue;
    if (nq == 0) return 0;
    const int32_t kpad = (dim + KC - 1) / KC * KC;
    const int64_t stride = (n + kSampleMax - 1) / kSampleMax;
    const int64_t ns = (n + stride - 1) / stride;
    const int64_t chunk = std::min<int64_t>((nq + TM - 1) / TM * TM, 16384);
    Scratch s;
    cudaError_t e = cudaSuccess;
    const size_t sizes[] = {2ull * n * kpad, 4ull * n, 4ull * n, 2ull * nq * kpad, 4ull * nq, 4ull * nq, 16,
                            4ull * chunk * ns, 4ull * chunk, 8ull * chunk * kCandCap, 4ull * chunk, 4ull * (chunk + 2)};
    for (int i = 0; i < 12 && e == cudaSuccess; ++i) e = cudaMalloc(&s.p[i], std::max<size_t>(sizes[i], 16));
    if (e != cudaSuccess) return *why = std::string("knn scratch: ") + cudaGetErrorString(e), (int)e;
    auto* xb = static_cast<__nv_bfloat16*>(s.p[0]);
    auto* xn = static_cast<float*>(s.p[1]);
    auto* xr = static_cast<float*>(s.p[2]);
    auto* qb = static_cast<__nv_bfloat16*>(s.p[3]);
    auto* qn = static_cast<float*>(s.p[4]);
    auto* qr = static_cast<float*>(s.p[5]);
    auto* maxima = static_cast<float*>(s.p[6]);
    auto* Ds = static_cast<float*>(s.p[7]);
    auto* limit = static_cast<float*>(s.p[8]);
    auto* cand = static_cast<unsigned long long*>(s.p[9]);
    auto* cnt = static_cast<int32_t*>(s.p[10]);
    auto* ov = static_cast<int32_t*>(s.p[11]);         // [0] overflow count, [1..chunk] queries, [chunk+1] error
    int32_t* err = ov + chunk + 1;
    const int sample_smem = (int)(4 * ns), rerank_smem = 2 * kCandCap * 8;
    if ((e = cudaFuncSetAttribute(dist_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(dist_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(sample_limit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, sample_smem)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(rerank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rerank_smem)) != cudaSuccess)
        return *why = cudaGetErrorString(e), (int)e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaMemsetAsync(maxima, 0, 16, st);
    bf16_rows_kernel<<<2048, 256, 0, st>>>(base, n, dim, kpad, xb, xn, xr);
    bf16_rows_kernel<<<1024, 256, 0, st>>>(queries, nq, dim, kpad, qb, qn, qr);
    row_maxima_kernel<<<304, 256, 0, st>>>(xn, xr, n, maxima);
    for (int64_t q0 = 0; q0 < nq && e == cudaSuccess; q0 += chunk) {
        const int64_t qc = std::min(chunk, nq - q0);
        const int64_t qblocks = (qc + TM - 1) / TM;
        auto stripes = [&](int64_t cols) {
            const int64_t tiles = (cols + TN - 1) / TN;
            return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (2ll * sms) / qblocks));
        };
        const TcArgs sa{qb + q0 * kpad, qn + q0, qc, xb, xn, ns, stride, kpad, Ds, nullptr, nullptr, nullptr, 0, err};
        const TcArgs fa{qb + q0 * kpad, qn + q0, qc, xb, xn, n, 1, kpad, nullptr, limit, cand, cnt, kCandCap, err};
        cudaMemsetAsync(ov, 0, 4ull * (chunk + 2), st);
        cudaMemsetAsync(cnt, 0, 4ull * qc, st);
        dist_tc_kernel<false><<<dim3((unsigned)qblocks, stripes(ns)), kTcThreads, kSmemDyn, st>>>(sa);
        sample_limit_kernel<<<(unsigned)qc, kSelThreads, sample_smem, st>>>(Ds, ns, k, qn + q0, qr + q0, maxima, kpad, limit);
        dist_tc_kernel<true><<<dim3((unsigned)qblocks, stripes(n)), kTcThreads, kSmemDyn, st>>>(fa);
        rerank_kernel<<<(unsigned)qc, kRerankThreads, rerank_smem, st>>>(cand, cnt, k, queries + q0 * dim, base, dim, qn + q0,
                                                                        qr + q0, maxima, kpad, ids + q0 * k, dists + q0 * k, ov);
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

}  // namespace deg
