/* CPU oracle for the Dynamic Exploration Graph (DEG) search path -- TEST INFRASTRUCTURE.
 *
 * Plain, slow, FP64 restatement of the paper's definitions and algorithms, used only by the
 * tests, the smoke check and the CPU-baseline leg of the benchmark. It shares no code with
 * the CUDA library and the library never calls it.
 *
 * Conventions: feature rows are float32 [n][dim] row-major (the data as stored); every
 * distance is computed in double. Adjacency is int32 [n][degree] row-major. Result lists are
 * sorted ascending by (distance, id); missing entries are id -1 / distance +inf.
 */
#ifndef DEG_ORACLE_H
#define DEG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Eq. 1: exact k nearest neighbours of each query by exhaustive FP64 L2 distance.
 * exclude[q] (nullable) is a base id left out for query q (-1 for none). */
int oracle_knn_bruteforce(const float* base, int64_t n, int32_t dim,
                          const float* queries, int64_t nq, int32_t k,
                          const int32_t* exclude, int32_t* ids, double* dists,
                          int32_t nthreads);

/* Alg. 1 RangeSearch, one query per call site, batched over queries.
 *  queries  : [nq][dim] query vectors; NULL in exploration mode (query = base row seeds[q]).
 *  seeds    : [nq] seed vertex per query.
 *  explore  : 0 = plain search (seed enters R), 1 = exploration (seed excluded from R).
 *  trace    : nullable [nq][4] int64: hops H, evaluations E (= |C|), max |S|, final |C|.
 * Returns 0, or -1 on invalid arguments. */
int oracle_range_search(const float* base, int64_t n, int32_t dim,
                        const int32_t* adj, int32_t degree,
                        const float* queries, const int32_t* seeds, int64_t nq,
                        int32_t explore, int32_t k, double eps,
                        int32_t* ids, double* dists, int64_t* trace, int32_t nthreads);

/* Fixed entry vertex (the median vertex, Sec. 5.4): the base row nearest (FP64,
 * tie -> lower id) to the coordinate-wise lower median of all base rows. */
int32_t oracle_median_vertex(const float* base, int64_t n, int32_t dim);

/* DEG construction (Alg. 2-5) in FP64 with stored edge weights. Vertices are inserted in id
 * order starting from the complete graph K_{d+1} on ids 0..d. adj_out: [n][degree] int32;
 * weights_out (nullable): [n][degree] double. Returns 0 or a negative error code. */
int deg_build_oracle(const float* base, int64_t n, int32_t dim, int32_t degree,
                     int32_t k_ext, double eps_ext, int32_t k_opt, double eps_opt,
                     int32_t i_opt, int32_t refine_rounds, uint64_t seed,
                     int32_t* adj_out, double* weights_out);

/* Structural invariants of a DEG (Sec. 5.1). Returns a bit mask of violations:
 *  1 degree slot empty/out of range, 2 self loop, 4 duplicate edge, 8 asymmetric,
 *  16 disconnected (BFS), 32 odd or < 4 degree, 64 has a bridge (only tested if n <= bridge_max_n). */
int32_t oracle_check_graph(const int32_t* adj, int64_t n, int32_t degree, int64_t bridge_max_n);

/* Eq. 4: average neighbour distance AND(V) of the whole graph, FP64. */
double oracle_average_neighbor_distance(const float* base, int64_t n, int32_t dim,
                                        const int32_t* adj, int32_t degree);

/* Eq. 3: graph quality GQ from precomputed exact neighbour lists knn [n][degree] (self excluded). */
double oracle_graph_quality(const int32_t* adj, const int32_t* knn, int64_t n, int32_t degree);

/* Building blocks exposed for pinning tests (operate on a graph with stored weights). */
/* Alg. 2 checkMRNG on an existing graph: 1 if the edge (v1,v2) passes, 0 otherwise. */
int32_t oracle_check_mrng(const float* base, int64_t n, int32_t dim, const int32_t* adj,
                          int32_t degree, int32_t v1, int32_t v2);

/* Alg. 4 optimizeEdge applied to one edge of a given graph (in place). Returns 1 if the graph
 * changed, 0 if the attempt was reverted, negative on error. */
int32_t oracle_optimize_edge(const float* base, int64_t n, int32_t dim, int32_t* adj,
                             int32_t degree, int32_t v1, int32_t v2, int32_t i_opt,
                             int32_t k_opt, double eps_opt);

/* Reduced-precision stores (format definitions: bfloat16 RNE; FP8 E4M3 with a per-row scale
 * s = max|x|/448, codes RNE and saturated) and the search over them with an FP64 re-rank. */
int oracle_quantize_bf16(const float* x, int64_t n, int32_t dim, uint16_t* out);
int oracle_quantize_fp8(const float* x, int64_t n, int32_t dim, uint8_t* codes, float* scales);
/* precision 1 = bf16 codes (uint16), 2 = fp8 codes (uint8) with scales -> FP64 values [n][dim]. */
int oracle_decode(int32_t precision, const void* codes, const float* scales, int64_t n, int32_t dim, double* out);
/* Alg. 1 over the decoded rows keeping `keep` results, then re-rank on the float32 rows. */
int oracle_range_search_decoded(const double* dec, const float* base, int64_t n, int32_t dim,
                                const int32_t* adj, int32_t degree, const float* queries,
                                const int32_t* seeds, int64_t nq, int32_t explore, int32_t keep,
                                int32_t k, double eps, int32_t* ids, double* dists, int32_t nthreads);

#ifdef __cplusplus
}
#endif
#endif
