// The search and serving kernels for BF16 rows (search_impl.cuh), compiled on their own.
#include "search_impl.cuh"

namespace deg {
namespace sk {

int dispatch_search_bf16(Params P, cudaStream_t st, void* t0, void* t1, std::string* why) {
    return dispatch_shape<BF16Rows>(P, st, t0, t1, why);
}

int dispatch_serve_bf16(Params P, const ServeRing& S, const int32_t* pivots, int np, cudaStream_t st, int* warps,
                       std::string* why) {
    return dispatch_serve<BF16Rows>(P, S, pivots, np, st, warps, why);
}

}  // namespace sk
}  // namespace deg
