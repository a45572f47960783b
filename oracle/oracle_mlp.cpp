// CPU oracle (test infrastructure only): the learned early-stop network of the library, in FP64.
// Not from the paper (the paper's stop rule is the eps test of Alg. 1); it follows the plain
// definition of a 2-hidden-layer perceptron with ReLU and a softmax cross-entropy loss:
//   h1 = relu(W1 x + b1)   W1 [64][12]
//   h2 = relu(W2 h1 + b2)  W2 [64][64]
//   z  = W3 h2 + b3        W3 [2][64]   (z[0] = continue, z[1] = stop)
//   loss = mean over samples of -log softmax(z)[label]
// Parameters are one flat array: W1, b1, W2, b2, W3, b3 (5122 values), row-major.
#include <cmath>
#include <cstdint>
#include <vector>

namespace {
constexpr int IN = 12, H = 64, OUT = 2;
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + OUT * H;
constexpr int NPARAM = OB3 + OUT;
}  // namespace

extern "C" int oracle_mlp_nparams() { return NPARAM; }

// Mean loss over `count` samples; if grad != NULL, also the gradient of the mean loss.
extern "C" double oracle_mlp_loss_grad(const double* w, const float* x, const int32_t* labels, int64_t count,
                                       double* grad) {
    if (grad)
        for (int i = 0; i < NPARAM; ++i) grad[i] = 0.0;
    double total = 0.0;
    std::vector<double> h1(H), h2(H), d1(H), d2(H);
    for (int64_t s = 0; s < count; ++s) {
        const float* xs = x + s * IN;
        for (int j = 0; j < H; ++j) {
            double a = w[OB1 + j];
            for (int i = 0; i < IN; ++i) a += w[OW1 + j * IN + i] * (double)xs[i];
            h1[j] = a > 0 ? a : 0;
        }
        for (int j = 0; j < H; ++j) {
            double a = w[OB2 + j];
            for (int i = 0; i < H; ++i) a += w[OW2 + j * H + i] * h1[i];
            h2[j] = a > 0 ? a : 0;
        }
        double z[OUT];
        for (int o = 0; o < OUT; ++o) {
            double a = w[OB3 + o];
            for (int i = 0; i < H; ++i) a += w[OW3 + o * H + i] * h2[i];
            z[o] = a;
        }
        const double m = z[0] > z[1] ? z[0] : z[1];
        const double lse = m + std::log(std::exp(z[0] - m) + std::exp(z[1] - m));
        const int y = labels[s];
        total += lse - z[y];
        if (!grad) continue;
        // d loss / d z = softmax(z) - onehot(y), divided by count for the mean
        double dz[OUT];
        for (int o = 0; o < OUT; ++o) dz[o] = (std::exp(z[o] - lse) - (o == y ? 1.0 : 0.0)) / (double)count;
        for (int o = 0; o < OUT; ++o) {
            grad[OB3 + o] += dz[o];
            for (int i = 0; i < H; ++i) grad[OW3 + o * H + i] += dz[o] * h2[i];
        }
        for (int i = 0; i < H; ++i) {
            double g = 0;
            for (int o = 0; o < OUT; ++o) g += w[OW3 + o * H + i] * dz[o];
            d2[i] = h2[i] > 0 ? g : 0;
        }
        for (int j = 0; j < H; ++j) {
            grad[OB2 + j] += d2[j];
            for (int i = 0; i < H; ++i) grad[OW2 + j * H + i] += d2[j] * h1[i];
        }
        for (int i = 0; i < H; ++i) {
            double g = 0;
            for (int j = 0; j < H; ++j) g += w[OW2 + j * H + i] * d2[j];
            d1[i] = h1[i] > 0 ? g : 0;
        }
        for (int j = 0; j < H; ++j) {
            grad[OB1 + j] += d1[j];
            for (int i = 0; i < IN; ++i) grad[OW1 + j * IN + i] += d1[j] * (double)xs[i];
        }
    }
    return total / (double)count;
}

// Probability of "stop" (softmax(z)[1]) per sample.
extern "C" void oracle_mlp_predict(const double* w, const float* x, int64_t count, double* p_stop) {
    std::vector<double> h1(H), h2(H);
    for (int64_t s = 0; s < count; ++s) {
        const float* xs = x + s * IN;
        for (int j = 0; j < H; ++j) {
            double a = w[OB1 + j];
            for (int i = 0; i < IN; ++i) a += w[OW1 + j * IN + i] * (double)xs[i];
            h1[j] = a > 0 ? a : 0;
        }
        for (int j = 0; j < H; ++j) {
            double a = w[OB2 + j];
            for (int i = 0; i < H; ++i) a += w[OW2 + j * H + i] * h1[i];
            h2[j] = a > 0 ? a : 0;
        }
        double z[OUT];
        for (int o = 0; o < OUT; ++o) {
            double a = w[OB3 + o];
            for (int i = 0; i < H; ++i) a += w[OW3 + o * H + i] * h2[i];
            z[o] = a;
        }
        p_stop[s] = 1.0 / (1.0 + std::exp(z[0] - z[1]));
    }
}
