// Learned early stop of the search (not in the paper; the paper stops by the eps test only).
// A 12 -> 64 -> 64 -> 2 perceptron with ReLU scores, after every hop, whether the result list
// can still change; the search stops when the "stop" logit beats "continue" by a threshold, and
// the eps test of Alg. 1 still stops it no later than the plain method would.
//
// Training kernels (float32), all deterministic: one block runs forward and backward for up to
// 128 samples with every activation in shared memory, then sums each parameter's gradient over
// its samples in a fixed order; a second kernel sums the block partials in block order and a
// third applies Adam. Parameter layout (5,122 floats): W1 [64][12], b1, W2 [64][64], b2,
// W3 [2][64], b3 (logit 0 = continue, logit 1 = stop); loss = mean softmax cross-entropy.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "deg_internal.h"

namespace deg {
namespace {

constexpr int IN = kStopFeatures, H = 64, OUT = 2;
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + OUT * H;
constexpr int NP = OB3 + OUT;
static_assert(NP == kStopParams, "parameter count");
constexpr int BS = 128;       // samples (and threads) per block
constexpr int LD = H + 1;     // padded row stride of the activation tiles (no bank conflicts)

__global__ void __launch_bounds__(BS) mlp_fwd_bwd_kernel(const float* __restrict__ w, const float* __restrict__ x,
                                                         const int32_t* __restrict__ labels, int64_t count,
                                                         float* __restrict__ partial, float* __restrict__ loss_partial) {
    extern __shared__ float sm[];
    float* ws = sm;                       // NP
    float* xs = ws + NP;                  // [BS][IN]
    float* h1 = xs + BS * IN;             // [BS][LD]
    float* h2 = h1 + BS * LD;
    float* d1 = h2 + BS * LD;
    float* d2 = d1 + BS * LD;
    float* dz = d2 + BS * LD;             // [BS][OUT]
    float* lsum = dz + BS * OUT;          // [BS]
    const int t = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * BS;
    for (int i = t; i < NP; i += BS) ws[i] = w[i];
    for (int i = t; i < BS * IN; i += BS) {
        const int64_t s = s0 + i / IN;
        xs[i] = s < count ? x[s0 * IN + i] : 0.f;
    }
    __syncthreads();
    const bool live = s0 + t < count;
    // forward
    for (int j = 0; j < H; ++j) {
        float a = ws[OB1 + j];
        for (int i = 0; i < IN; ++i) a = fmaf(ws[OW1 + j * IN + i], xs[t * IN + i], a);
        h1[t * LD + j] = fmaxf(a, 0.f);
    }
    for (int j = 0; j < H; ++j) {
        float a = ws[OB2 + j];
        for (int i = 0; i < H; ++i) a = fmaf(ws[OW2 + j * H + i], h1[t * LD + i], a);
        h2[t * LD + j] = fmaxf(a, 0.f);
    }
    float z[OUT];
    for (int o = 0; o < OUT; ++o) {
        float a = ws[OB3 + o];
        for (int i = 0; i < H; ++i) a = fmaf(ws[OW3 + o * H + i], h2[t * LD + i], a);
        z[o] = a;
    }
    const float m = fmaxf(z[0], z[1]);
    const float lse = m + logf(expf(z[0] - m) + expf(z[1] - m));
    const int y = live ? labels[s0 + t] : 0;
    lsum[t] = live ? lse - z[y] : 0.f;
    // backward: dz = softmax - onehot (the 1/count of the mean is applied at the reduction)
    for (int o = 0; o < OUT; ++o) dz[t * OUT + o] = live ? expf(z[o] - lse) - (o == y ? 1.f : 0.f) : 0.f;
    for (int i = 0; i < H; ++i) {
        float g = 0.f;
        for (int o = 0; o < OUT; ++o) g = fmaf(ws[OW3 + o * H + i], dz[t * OUT + o], g);
        d2[t * LD + i] = h2[t * LD + i] > 0.f ? g : 0.f;
    }
    for (int i = 0; i < H; ++i) {
        float g = 0.f;
        for (int j = 0; j < H; ++j) g = fmaf(ws[OW2 + j * H + i], d2[t * LD + j], g);
        d1[t * LD + i] = h1[t * LD + i] > 0.f ? g : 0.f;
    }
    __syncthreads();
    // per-parameter sums over this block's samples, in sample order
    float* out = partial + (int64_t)blockIdx.x * NP;
    for (int p = t; p < NP; p += BS) {
        float g = 0.f;
        if (p < OB1) {
            const int j = p / IN, i = p % IN;
            for (int s = 0; s < BS; ++s) g = fmaf(d1[s * LD + j], xs[s * IN + i], g);
        } else if (p < OW2) {
            const int j = p - OB1;
            for (int s = 0; s < BS; ++s) g += d1[s * LD + j];
        } else if (p < OB2) {
            const int j = (p - OW2) / H, i = (p - OW2) % H;
            for (int s = 0; s < BS; ++s) g = fmaf(d2[s * LD + j], h1[s * LD + i], g);
        } else if (p < OW3) {
            const int j = p - OB2;
            for (int s = 0; s < BS; ++s) g += d2[s * LD + j];
        } else if (p < OB3) {
            const int o = (p - OW3) / H, i = (p - OW3) % H;
            for (int s = 0; s < BS; ++s) g = fmaf(dz[s * OUT + o], h2[s * LD + i], g);
        } else {
            const int o = p - OB3;
            for (int s = 0; s < BS; ++s) g += dz[s * OUT + o];
        }
        out[p] = g;
    }
    if (t == 0) {
        float l = 0.f;
        for (int s = 0; s < BS; ++s) l += lsum[s];
        loss_partial[blockIdx.x] = l;
    }
}

__global__ void mlp_reduce_kernel(const float* __restrict__ partial, const float* __restrict__ loss_partial,
                                  int nblocks, int64_t count, float* __restrict__ grad, float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const float inv = 1.f / (float)count;
    if (p < NP) {
        float g = 0.f;
        for (int b = 0; b < nblocks; ++b) g += partial[(int64_t)b * NP + p];
        grad[p] = g * inv;
    }
    if (p == 0 && loss) {
        float l = 0.f;
        for (int b = 0; b < nblocks; ++b) l += loss_partial[b];
        *loss = l * inv;
    }
}

__global__ void mlp_adam_kernel(float* w, float* m, float* v, const float* g, int step, float lr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mp = b1 * m[p] + (1.f - b1) * g[p];
    const float vp = b2 * v[p] + (1.f - b2) * g[p] * g[p];
    m[p] = mp;
    v[p] = vp;
    const float mh = mp / (1.f - powf(b1, (float)step));
    const float vh = vp / (1.f - powf(b2, (float)step));
    w[p] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void mlp_predict_kernel(const float* __restrict__ w, const float* __restrict__ x, int64_t count,
                                   float* __restrict__ p_stop) {
    __shared__ float ws[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) ws[i] = w[i];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    float xi[IN], h1[H], z[OUT];
    for (int i = 0; i < IN; ++i) xi[i] = x[s * IN + i];
    for (int j = 0; j < H; ++j) {
        float a = ws[OB1 + j];
        for (int i = 0; i < IN; ++i) a = fmaf(ws[OW1 + j * IN + i], xi[i], a);
        h1[j] = fmaxf(a, 0.f);
    }
    for (int o = 0; o < OUT; ++o) z[o] = ws[OB3 + o];
    for (int j = 0; j < H; ++j) {
        float a = ws[OB2 + j];
        for (int i = 0; i < H; ++i) a = fmaf(ws[OW2 + j * H + i], h1[i], a);
        a = fmaxf(a, 0.f);
        for (int o = 0; o < OUT; ++o) z[o] = fmaf(ws[OW3 + o * H + j], a, z[o]);
    }
    p_stop[s] = 1.f / (1.f + expf(z[0] - z[1]));
}

// bfloat16 copy for inference inside the search, with W1 and W2 transposed ([in][out]) so the
// 32 lanes of a warp read consecutive outputs: W1t [12][64], b1, W2t [64][64], b2, W3, b3.
__global__ void pack_inference_kernel(const float* w, __nv_bfloat16* out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    int src = p;
    if (p < OB1) {
        const int i = p / H, j = p % H;      // out position [i][j] <- W1[j][i]
        src = OW1 + j * IN + i;
    } else if (p >= OW2 && p < OB2) {
        const int i = (p - OW2) / H, j = (p - OW2) % H;
        src = OW2 + j * H + i;
    }
    out[p] = __float2bfloat16_rn(w[src]);
}

size_t fwd_bwd_smem() { return sizeof(float) * (NP + BS * IN + 4 * BS * LD + BS * OUT + BS); }

}  // namespace

int mlp_loss_grad(const float* w, const float* x, const int32_t* labels, int64_t count, float* grad, float* loss,
                  float* scratch, deg_stream_t stream, std::string* why) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nb = (int)((count + BS - 1) / BS);
    float* partial = scratch;
    float* lpart = scratch + (int64_t)nb * NP;
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fwd_bwd_smem());
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    mlp_fwd_bwd_kernel<<<nb, BS, fwd_bwd_smem(), st>>>(w, x, labels, count, partial, lpart);
    mlp_reduce_kernel<<<(NP + 255) / 256, 256, 0, st>>>(partial, lpart, nb, count, grad, loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

int64_t mlp_scratch_floats(int64_t count) {
    const int64_t nb = (count + BS - 1) / BS;
    return nb * NP + nb;
}

int mlp_adam(float* w, float* m, float* v, const float* g, int step, float lr, deg_stream_t stream, std::string* why) {
    mlp_adam_kernel<<<(NP + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(w, m, v, g, step, lr);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

int mlp_predict(const float* w, const float* x, int64_t count, float* p_stop, deg_stream_t stream, std::string* why) {
    mlp_predict_kernel<<<(unsigned)((count + 127) / 128), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(w, x, count, p_stop);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

int mlp_pack_inference(const float* w, uint16_t* out, deg_stream_t stream, std::string* why) {
    pack_inference_kernel<<<(NP + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        w, reinterpret_cast<__nv_bfloat16*>(out));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return *why = cudaGetErrorString(e), (int)e;
    return 0;
}

}  // namespace deg
