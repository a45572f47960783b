// The search and serving kernels for float32 rows (search_impl.cuh), compiled on their own.
#include "search_impl.cuh"

namespace deg {
namespace sk {

int dispatch_search_f32(Params P, cudaStream_t st, void* t0, void* t1, std::string* why) {
    return dispatch_shape<F32Rows>(P, st, t0, t1, why);
}

int dispatch_serve_f32(Params P, const ServeRing& S, const int32_t* pivots, int np, cudaStream_t st, int* warps,
                       std::string* why) {
    return dispatch_serve<F32Rows>(P, S, pivots, np, st, warps, why);
}

}  // namespace sk
}  // namespace deg
