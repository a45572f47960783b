// CPU oracle (test infrastructure only): reduced-precision storage of the base rows and the
// search over it. The paper stores float32 features only (Sec. 5.4); the BF16 and FP8 stores
// with a float32 re-rank are the library's extension, so these functions follow the format
// definitions rather than a passage of the paper:
//   bfloat16: the upper 16 bits of the float32 pattern, rounded to nearest, ties to even.
//   FP8 E4M3 ("FN" variant): 1 sign, 4 exponent (bias 7), 3 mantissa bits; no infinities;
//     subnormals m * 2^-9; largest finite 448; conversion rounds to nearest even and
//     saturates to +-448. A row is stored as codes c_i = E4M3(x_i / s) with the float32 scale
//     s = max_i |x_i| / 448 (s = 1 for an all-zero row) and read back as s * c_i.
// The search runs Alg. 1 on the decoded rows (FP64 distances), keeping `keep` results, then
// re-ranks those on the float32 rows (FP64 distances) and returns the k best by (distance, id).
#include "deg_oracle.h"
#include "oracle_common.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

namespace {

uint16_t bf16_rne(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (uint16_t)((u >> 16) | 0x40);  // NaN
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

double bf16_value(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

double round_half_even(double v) {
    const double f = std::floor(v);
    const double r = v - f;
    if (r > 0.5) return f + 1.0;
    if (r < 0.5) return f;
    return std::fmod(f, 2.0) == 0.0 ? f : f + 1.0;
}

uint8_t e4m3_rne_sat(float xf) {
    const double x = (double)xf;
    const uint8_t sign = std::signbit(x) ? 0x80 : 0x00;
    double a = std::fabs(x);
    if (std::isnan(x)) return 0x7f;
    if (a == 0.0) return sign;
    // spacing of representable values around a: subnormal spacing 2^-9 below 2^-6, else 2^(e-3)
    int E;
    std::frexp(a, &E);                   // a = f * 2^E, f in [0.5, 1) -> a in [2^(E-1), 2^E)
    const int e = E - 1;
    const double quantum = e < -6 ? std::ldexp(1.0, -9) : std::ldexp(1.0, e - 3);
    double v = round_half_even(a / quantum) * quantum;
    if (v > 448.0) v = 448.0;            // saturate
    if (v == 0.0) return sign;
    if (v < std::ldexp(1.0, -6)) {       // subnormal: m * 2^-9
        const int m = (int)(v / std::ldexp(1.0, -9));
        return (uint8_t)(sign | m);
    }
    int E2;
    const double f2 = std::frexp(v, &E2);   // v = f2 * 2^E2
    const int e2 = E2 - 1;
    const int m = (int)((f2 * 2.0 - 1.0) * 8.0);
    return (uint8_t)(sign | ((e2 + 7) << 3) | m);
}

double e4m3_value(uint8_t c) {
    const double s = (c & 0x80) ? -1.0 : 1.0;
    const int ef = (c >> 3) & 0xf, m = c & 7;
    if (ef == 0) return s * m * std::ldexp(1.0, -9);
    return s * (1.0 + m / 8.0) * std::ldexp(1.0, ef - 7);
}

}  // namespace

extern "C" int oracle_quantize_bf16(const float* x, int64_t n, int32_t dim, uint16_t* out) {
    for (int64_t i = 0; i < n * dim; ++i) out[i] = bf16_rne(x[i]);
    return 0;
}

extern "C" int oracle_quantize_fp8(const float* x, int64_t n, int32_t dim, uint8_t* codes, float* scales) {
    for (int64_t r = 0; r < n; ++r) {
        const float* row = x + r * dim;
        float m = 0.f;
        for (int32_t i = 0; i < dim; ++i) m = std::max(m, std::fabs(row[i]));
        const float s = m > 0.f ? m / 448.0f : 1.0f;          // float32 division
        scales[r] = s;
        for (int32_t i = 0; i < dim; ++i) codes[r * dim + i] = e4m3_rne_sat(row[i] / s);
    }
    return 0;
}

extern "C" int oracle_decode(int32_t precision, const void* codes, const float* scales, int64_t n, int32_t dim,
                             double* out) {
    for (int64_t r = 0; r < n; ++r)
        for (int32_t i = 0; i < dim; ++i) {
            const int64_t j = r * dim + i;
            out[j] = precision == 1 ? bf16_value(static_cast<const uint16_t*>(codes)[j])
                                    : (double)scales[r] * e4m3_value(static_cast<const uint8_t*>(codes)[j]);
        }
    return 0;
}

extern "C" int oracle_range_search_decoded(const double* dec, const float* base, int64_t n, int32_t dim,
                                           const int32_t* adj, int32_t degree, const float* queries,
                                           const int32_t* seeds, int64_t nq, int32_t explore, int32_t keep,
                                           int32_t k, double eps, int32_t* ids, double* dists, int32_t nthreads) {
    using namespace oracle;
    if (!dec || !base || !adj || !seeds || !ids || !dists || keep < k || k < 1) return -1;
    if (!explore && !queries) return -1;
    Graph g{n, degree, adj};
    parallel_for(nq, nthreads, [&](int64_t q) {
        const float* qv = explore ? base + (int64_t)seeds[q] * dim : queries + q * dim;
        auto dq = [&](int32_t v) {
            double s = 0.0;
            for (int32_t i = 0; i < dim; ++i) {
                const double t = dec[(int64_t)v * dim + i] - (double)qv[i];
                s += t * t;
            }
            return std::sqrt(s);
        };
        std::vector<Cand> R = range_search(g, dq, {seeds[q]}, keep, eps, !explore, nullptr);
        for (Cand& c : R) c.d = distance(base + (int64_t)c.id * dim, qv, dim);   // re-rank
        std::sort(R.begin(), R.end());
        for (int32_t j = 0; j < k; ++j) {
            ids[q * k + j] = j < (int32_t)R.size() ? R[j].id : -1;
            dists[q * k + j] = j < (int32_t)R.size() ? R[j].d : std::numeric_limits<double>::infinity();
        }
    });
    return 0;
}
