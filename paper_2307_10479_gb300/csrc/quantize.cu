// Reduced-precision copies of the float32 rows, made once at upload.
//   BF16: each element rounded to the nearest bfloat16 (ties to even); rows padded to 8 elements.
//   FP8 : per row s = max_i |x_i| / 448 (448 = largest finite E4M3 value; s = 1 for an all-zero
//         row), codes c_i = E4M3(x_i / s) rounded to nearest even and saturated to +-448;
//         the row is read back as s * c_i. Rows padded to 16 codes.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <string>

#include "deg_internal.h"

namespace deg {
namespace {

__global__ void bf16_kernel(const float* x, int64_t n, int32_t dim, int32_t dim_pad, __nv_bfloat16* out,
                            int32_t out_pad) {
    const int64_t total = n * out_pad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / out_pad;
        const int c = (int)(i - r * out_pad);
        out[i] = __float2bfloat16_rn(c < dim ? x[r * dim_pad + c] : 0.f);
    }
}

// E4M3 codes of each row with its scale s, and {s, s^2 ||decoded codes||^2} for the search's distance
// expansion (the decoded codes are exact in float32; their squares are summed in float32).
__global__ void fp8_kernel(const float* x, int64_t n, int32_t dim, int32_t dim_pad, __nv_fp8_storage_t* out,
                           int32_t out_pad, float* scale, float2* norm) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nw) {
        const float* row = x + r * dim_pad;
        float m = 0.f;
        for (int i = lane; i < dim; i += 32) m = fmaxf(m, fabsf(row[i]));
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float s = m > 0.f ? m / 448.f : 1.f;
        float xx = 0.f;
        for (int i = lane; i < out_pad; i += 32) {
            const __nv_fp8_storage_t c = i < dim ? __nv_cvt_float_to_fp8(row[i] / s, __NV_SATFINITE, __NV_E4M3) : 0;
            out[r * out_pad + i] = c;
            const float v = __half2float(__half(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3)));
            xx = fmaf(v, v, xx);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) xx += __shfl_xor_sync(0xffffffffu, xx, o);
        if (lane == 0) {
            scale[r] = s;
            norm[r] = make_float2(s, s * s * xx);
        }
    }
}

}  // namespace

int make_bf16_copy(DeviceIndex& ix, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ix.dim_pad16 = (ix.dim + 7) / 8 * 8;
    cudaError_t e = cudaMalloc(&ix.xbf, sizeof(uint16_t) * ix.n * ix.dim_pad16);
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    bf16_kernel<<<4096, 256, 0, st>>>(ix.x32, ix.n, ix.dim, ix.dim_pad, reinterpret_cast<__nv_bfloat16*>(ix.xbf),
                                      ix.dim_pad16);
    if ((e = cudaGetLastError()) != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

int make_fp8_copy(DeviceIndex& ix, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ix.dim_pad8 = (ix.dim + 15) / 16 * 16;
    cudaError_t e = cudaMalloc(&ix.x8, (size_t)ix.n * ix.dim_pad8);
    if (e == cudaSuccess) e = cudaMalloc(&ix.scale8, sizeof(float) * ix.n);
    if (e == cudaSuccess) e = cudaMalloc(&ix.norm8, 2 * sizeof(float) * ix.n);
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    fp8_kernel<<<2048, 256, 0, st>>>(ix.x32, ix.n, ix.dim, ix.dim_pad, ix.x8, ix.dim_pad8, ix.scale8,
                                      reinterpret_cast<float2*>(ix.norm8));
    if ((e = cudaGetLastError()) != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

}  // namespace deg
