/* deg.h -- C ABI of libdeg: batched Dynamic Exploration Graph (DEG) search on one GB300.
 *
 * The paper (arXiv 2307.10479) defines the method:
 *   - Alg. 1 RangeSearch(G, S, q, k, eps) (Sec. 2.1)      -> deg_search / deg_explore
 *   - exploration queries seeded at the query's own vertex (Sec. 6.7) -> deg_explore
 *   - Eq. 1, the exact k nearest neighbours                -> knn_exact
 *   - Sec. 5 construction (Alg. 2-5)                       -> deg_build (host, not the GPU path)
 *   - Sec. 5.4: search graphs drop edge weights and start at the "median vertex"
 *                                                          -> deg_upload / deg_entry_vertex
 *
 * Conventions for every call:
 *   - Distances are Euclidean (L2, not squared). Result lists are sorted ascending by
 *     (distance, id), ties going to the lower id; a list shorter than k is padded with
 *     id -1 and distance +inf.
 *   - Pointers named *_dev are device pointers (cudaMalloc'd or torch tensors); *_host are
 *     host pointers. The caller owns every buffer it passes; the library owns a deg_index and
 *     the device copies it makes. `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - Device work is asynchronous on `stream`: the return value reports argument validation
 *     and launch errors only. Per-query outcomes go to the optional status_dev array.
 *   - On failure a call returns a negative deg_status, leaves outputs unspecified and records
 *     a message for deg_last_error() (thread-local).
 *   - Searches on one index may run concurrently on different streams only when each passes
 *     its own `workspace` (deg_search_ex); the convenience calls share the index's workspace
 *     and must be ordered by the caller (same stream or explicit synchronisation).
 */
#ifndef DEG_H
#define DEG_H

#include <stdint.h>

#if defined(__GNUC__)
#define DEG_API __attribute__((visibility("default")))
#else
#define DEG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DEG_OK = 0,
    DEG_EINVAL = -1,      /* invalid argument (k < 1, eps < 0 or NaN, ids out of range, ...) */
    DEG_ENOMEM = -2,      /* host or device allocation failed                                */
    DEG_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed                     */
    DEG_EIO = -4,         /* file could not be read or written, or has a bad format          */
    DEG_EOVERFLOW = -5,   /* per query: a bounded structure overflowed (result not exact)    */
    DEG_EHOPLIMIT = -6,   /* per query: stopped at deg_search_params.max_hops expansions     */
    DEG_ETIMEOUT = -7,    /* a bounded device wait expired                                   */
    DEG_EGRAPH = -8,      /* graph violates a DEG invariant (degree, symmetry, loops)        */
    DEG_ENOTREADY = -9    /* index not uploaded to the device (call deg_upload first)        */
} deg_status;

typedef enum {
    DEG_F32 = 0,          /* rows stored as float32                                          */
    DEG_BF16 = 1,         /* rows stored as bfloat16 (round to nearest even), no scale       */
    DEG_FP8 = 2           /* rows stored as FP8 E4M3 codes with a per-row float32 scale      */
} deg_precision;

/* Construction parameters (paper Table 2): even degree d >= 4; k_ext >= d and eps_ext for the
 * search of a new vertex (Alg. 3); k_opt, eps_opt, i_opt for edge optimisation (Alg. 4);
 * refine_rounds calls of Alg. 5 after the last insertion, drawing vertices from `seed`. */
typedef struct {
    int32_t degree;
    int32_t k_ext;
    float eps_ext;
    int32_t k_opt;
    float eps_opt;
    int32_t i_opt;
    int32_t refine_rounds;
    uint64_t seed;
} deg_build_params;

typedef struct deg_index deg_index;   /* opaque, owned by the library */

/* ---- index lifecycle ------------------------------------------------------------------- */

/* Build a DEG over base_host [n][dim] float32 on the host (paper Sec. 5.2-5.3, Alg. 2-5).
 * Copies the vectors. n >= degree + 1. Single-threaded; minutes to hours at n = 10^6.
 * progress (nullable) receives the number of vertices inserted so far. */
DEG_API deg_status deg_build(const float* base_host, int64_t n, int32_t dim, const deg_build_params* p,
                     volatile int64_t* progress, deg_index** out);

/* Build a DEG over base_host [n][dim] float32 on the current GPU: ExtendGraph (Sec. 5.2, Alg. 3,
 * scheme C with the checkMRNG test of Alg. 2 in a first pass) for batches of new vertices at a
 * time. Each batch is searched over the graph built so far by the library's search kernels
 * (Alg. 1: seed vertex 0, k_ext results, eps_ext); one warp per new vertex then replaces edges
 * (b, n) by (v, b), (v, n). A batch holds at most 1/batch_div of the vertices already inserted
 * (at least 1, at most 8,192), so the vertices of a batch rarely fall in each other's
 * neighbourhoods; old vertices are claimed per batch, so two new vertices never rewire the same
 * vertex in one batch, and a vertex that runs out of free candidates is inserted again later with
 * more candidates. With i_opt > 0, each batch then runs the optional last line of Alg. 3,
 * optimizeEdge (Alg. 4; k_opt, eps_opt, i_opt iterations) for every new edge (v, u) with u outside
 * v's search result: all of a batch's optimisations at once, one per new vertex at a time, their
 * searches batched; an optimisation claims each vertex it rewires and is undone and repeated
 * later if another holds one. i_opt = 0 gives the paper's construction-only graph (App. G).
 * refine_rounds > 0 then runs that many rounds of Alg. 5 (as deg_refine_device). The graph is an
 * even-regular, symmetric, connected graph without loops or duplicates (checked before
 * returning; DEG_EGRAPH otherwise), but not the graph the sequential builder makes: which batch
 * member claims a vertex first depends on the order the warps run in. Copies the vectors; device
 * memory about n * (4 dim + 12 degree) bytes plus the search scratch, all freed before returning.
 * Synchronises `stream`. DEG_EINVAL when dim is outside 1 ... 1024, degree is odd or outside
 * 4 ... 128, n < degree + 1 or above 2^31 - 1, k_ext is outside degree ... 1024, i_opt is outside
 * 0 ... 6, k_opt outside 1 ... 1024 (with i_opt > 0), refine_rounds < 0 or > 0 with i_opt = 0, an
 * eps < 0 or batch_div < 1; DEG_ECUDA on a device error. progress (nullable) receives the number
 * of vertices inserted so far. */
DEG_API deg_status deg_build_device(const float* base_host, int64_t n, int32_t dim, const deg_build_params* p,
                                    int32_t batch_div, volatile int64_t* progress, deg_index** out, void* stream);

/* Grow an index by m vectors new_host [m][dim] float32 on the current GPU: they become vertices
 * n .. n+m-1 and are inserted as deg_build_device inserts vertices (Sec. 5.2, Alg. 3 in batches of
 * at most 1/batch_div of the graph, seeded at vertex 0; Alg. 4 for the new edges when p->i_opt >
 * 0). The paper builds a graph by exactly such insertions; this makes the index grow after it is
 * built. Copies the vectors. The host adjacency is replaced and the device copy released (upload
 * again before searching); on an error the index is unchanged. p->degree must equal the index's.
 * DEG_EINVAL on bad parameters (as deg_build_device), DEG_ECUDA on a device error, DEG_EGRAPH if
 * the result violates a graph invariant. */
DEG_API deg_status deg_insert_device(deg_index* idx, const float* new_host, int64_t m, const deg_build_params* p,
                                     int32_t batch_div, void* stream);

/* dynamicEdgeOptimization (Sec. 5.3, Alg. 5) on the current GPU over the index's graph:
 * p->refine_rounds rounds, each taking a random vertex v1 (SplitMix64 from p->seed) and running
 * optimizeEdge (Alg. 4; p->i_opt, p->k_opt, p->eps_opt) on each edge (v1, v2) that fails
 * checkMRNG (Alg. 2) and then on v1's longest edge. Up to 4,096 rounds run at once, on distinct
 * vertices, with the same claims as deg_build_device; so the rounds are not the sequential
 * order's. The graph keeps its invariants (checked; DEG_EGRAPH otherwise). *improved (nullable)
 * receives the number of optimisations that changed the graph. The host adjacency is replaced and
 * the device copy released: upload again before searching. p->degree must equal the index's. */
DEG_API deg_status deg_refine_device(deg_index* idx, const deg_build_params* p, int64_t* improved, void* stream);

/* Remove vertex v (0 <= v < n) from the index on the host. The paper leaves removal open (App. A)
 * while calling the graph fully dynamic; this removal keeps every invariant. v's d edges go; its
 * former neighbours, each one edge short, are joined in pairs by new edges, closest non-adjacent
 * pairs first (ties by ids); a pair left that is already adjacent is joined through a nearby edge
 * (x, y), replaced by (a, x) and (b, y), x a neighbour of a neighbour of a, minimising
 * |a-x| + |b-y| - |x-y|. The graph stays connected exactly when the former neighbours still reach
 * one another, which is checked. Then the last vertex n-1 takes id v (its vector and edges move;
 * *moved_from (nullable) = n-1, or -1 if v was n-1) and n shrinks by one, so ids stay 0 .. n-2.
 * The device copy is released (upload again before searching). DEG_EINVAL (index unchanged) if v
 * is out of range, if fewer than degree + 1 vertices would remain, or if no reconnection keeps the graph
 * connected; DEG_EGRAPH if the result violates an invariant. */
DEG_API deg_status deg_remove(deg_index* idx, int32_t v, int32_t* moved_from);

/* Wrap an existing graph: base_host [n][dim] float32 and adj_host [n][degree] int32 are copied.
 * The adjacency is checked (every entry in [0,n), no self-loops, no duplicates, symmetric,
 * degree even and >= 4): DEG_EGRAPH if it is not a valid undirected regular graph. */
DEG_API deg_status deg_index_from_arrays(const float* base_host, const int32_t* adj_host, int64_t n,
                                 int32_t dim, int32_t degree, deg_index** out);

/* Graph file: header, adjacency [n][degree] int32 and, if with_vectors, the vectors. Edge
 * weights are not stored (Sec. 5.4: search drops them; they are recomputed when needed).
 * A file without vectors carries a checksum of them; deg_load then requires base_host
 * (otherwise ignored, may be NULL) and fails with DEG_EIO if the checksum differs. */
DEG_API deg_status deg_save(const deg_index* idx, const char* path, int32_t with_vectors);
DEG_API deg_status deg_load(const char* path, const float* base_host, deg_index** out);

/* Shape queries; deg_get_adjacency copies the graph out to adj_host [n][degree]. */
DEG_API deg_status deg_index_info(const deg_index* idx, int64_t* n, int32_t* dim, int32_t* degree);
DEG_API deg_status deg_get_adjacency(const deg_index* idx, int32_t* adj_host);

/* Make the index resident on the current CUDA device: float32 rows (always, padded to a
 * multiple of 4 floats), the adjacency, and the reduced-precision copies named in
 * precision_mask (bit 1 << DEG_BF16, bit 1 << DEG_FP8). Computes the fixed entry vertex on the
 * device: the row nearest to the per-coordinate lower median (rank floor((n-1)/2)) of all rows
 * -- the paper's "median vertex" (Sec. 5.4). Synchronises `stream` before returning. */
DEG_API deg_status deg_upload(deg_index* idx, int32_t precision_mask, void* stream);

/* Copy the device's reduced-precision rows out to the host, unpadded: precision DEG_BF16 ->
 * codes_host [n][dim] uint16 (bfloat16 bit patterns); DEG_FP8 -> codes_host [n][dim] uint8
 * (E4M3 codes) and scales_host [n] float32. DEG_ENOTREADY if that copy was not uploaded. */
DEG_API deg_status deg_export_codes(const deg_index* idx, int32_t precision, void* codes_host, float* scales_host);

/* Learned entry points (not in the paper): a second set of routing pivots (entry_mode 2) of k
 * vertices learned from the data; the sampled pivots (entry_mode 1) stay. Lloyd's algorithm (k-means) runs `iters` rounds on the device
 * from k rows spaced evenly through the stored order (every row to its nearest centroid, every
 * centroid to the mean of its rows; an empty cluster keeps its centroid); each centroid is then
 * replaced by the base vertex nearest to it, and those vertices are the learned pivots, used by
 * the batch routing and the serving loop alike. Training again replaces them. sizes_host (nullable) [k] gets the final cluster
 * sizes. Needs an uploaded index and a dimension divisible by 4. Synchronises `stream`.
 * DEG_EINVAL when k is outside 1 ... min(4096, n) or iters outside 0 ... 1000; DEG_ENOTREADY
 * before deg_upload; DEG_ECUDA on a device error. */
DEG_API deg_status deg_train_entry(deg_index* idx, int32_t k, int32_t iters, int64_t* sizes_host, void* stream);

/* The routing pivots as caller ids: the sampled ones (learned = 0, chosen at upload) or the learned
 * ones (learned = 1, deg_train_entry). Returns their number (0 if there are none, -1 on a NULL
 * index or a device error); ids_host [cap] is filled only when cap is at least that number. */
DEG_API int32_t deg_get_pivots(const deg_index* idx, int32_t learned, int32_t* ids_host, int32_t cap);

/* The entry vertex computed by deg_upload, or -1 before it. */
DEG_API int32_t deg_entry_vertex(const deg_index* idx);

/* Release every host and device resource of the index (NULL is a no-op). */
DEG_API void deg_free(deg_index* idx);

/* ---- search (Alg. 1) ---------------------------------------------------------------------- */

typedef struct {
    int32_t k;            /* results per query, 1 <= k <= 1024 and k <= n (k <= n-1 to explore) */
    float eps;            /* range factor eps >= 0 of Alg. 1                                  */
    int32_t precision;    /* DEG_F32 | DEG_BF16 | DEG_FP8 (the copy must have been uploaded)  */
    int32_t rerank;       /* precision != F32: keep this many candidates (>= k, <= 1024) and
                             re-rank them on the float32 rows; 0 = k (no widening); -1 = no
                             re-rank: the k results and distances of the reduced-precision
                             search as computed (to measure the format's distance error)     */
    int32_t max_hops;     /* 0 = unlimited; else a query stops after this many expansions and
                             reports DEG_EHOPLIMIT with its current result list               */
    int32_t visited_cap;  /* reserved, must be 0 (the checked set is an n-bit bitmap)          */
    int32_t queue_cap;    /* candidates a query may hold in its device-memory pool in the
                             main kernel, 0 = 32768 (the maximum); a query needing more is
                             finished by a second kernel with room for all n vertices          */
    int32_t entry_mode;   /* plain searches with no seeds: 0 = the fixed entry vertex (paper,
                             Sec. 5.4); 1 = per query, the nearest of the index's pivot vertices
                             (about n/256, at most 4096, chosen at upload); 2 = the nearest of
                             the learned entry points (deg_train_entry) -- 1 and 2 are not in
                             the paper */
    int32_t learned_stop; /* 1: every fourth hop, once R has not changed for two hops, the
                             index's stop network (deg_set_stop_model) may end the search
                             early; the eps test still applies. Not in the paper; 0 = the
                             plain method */
} deg_search_params;

/* Plain search: one Alg. 1 run per query q of queries_dev [nq][dim] float32, seeded at
 * seeds_dev[q] (int32, nullable: NULL = the entry vertex of deg_upload). Seeds enter the result
 * list (Alg. 1 initialises R with the seeds). Writes ids_dev [nq][k] int32 and dists_dev
 * [nq][k] float32; status_dev (nullable) [nq] int32 gets DEG_OK or a per-query status. Exact: a
 * query whose candidate pool outgrows its slot is finished by a second kernel with room for all
 * n vertices, with an identical result. */
DEG_API deg_status deg_search(deg_index* idx, const float* queries_dev, int64_t nq, int32_t k, float eps,
                      const int32_t* seeds_dev, int32_t* ids_dev, float* dists_dev,
                      int32_t* status_dev, void* stream);

/* Instrumentation, not in the paper: every later search call on idx records start_event on its
 * stream just before the main search kernel (after any entry routing) and end_event just after
 * the second kernel, so cudaEventElapsedTime gives the search kernels' own time. The events are
 * cudaEvent_t handles the caller creates and owns; NULL, NULL stops the recording. DEG_EINVAL if
 * only one is NULL. Not thread-safe against concurrent searches on the same index. */
DEG_API deg_status deg_set_kernel_timer(deg_index* idx, void* start_event, void* end_event);

/* Exploration (Sec. 6.7): query q is the indexed vertex vertex_ids_dev[q]; the search starts
 * at that vertex and never returns it (the user has already seen it). */
DEG_API deg_status deg_explore(deg_index* idx, const int32_t* vertex_ids_dev, int64_t nq, int32_t k,
                       float eps, int32_t* ids_dev, float* dists_dev, int32_t* status_dev,
                       void* stream);

/* Full form of both. queries_dev is NULL iff explore != 0 (then seeds_dev holds the vertex
 * ids). trace_dev (nullable) [nq][4] int32 receives per query: hops H (expansions), vertices
 * evaluated E (= |C|), the largest size of the candidate set S, and 1 if the query was
 * finished by the second kernel. */
DEG_API deg_status deg_search_ex(deg_index* idx, const deg_search_params* p, const float* queries_dev,
                         const int32_t* seeds_dev, int32_t explore, int64_t nq, int32_t* ids_dev,
                         float* dists_dev, int32_t* status_dev, int32_t* trace_dev, void* stream);

/* End-to-end form with HOST buffers: copies queries_host [nq][dim] (or the vertex ids in
 * seeds_host when explore != 0) to the device, searches, copies ids/dists back into
 * ids_host [nq][k] / dists_host [nq][k], and synchronises `stream` before returning. Uses
 * device buffers cached in the index (grown on demand). */
DEG_API deg_status deg_search_host(deg_index* idx, const deg_search_params* p, const float* queries_host,
                           const int32_t* seeds_host, int32_t explore, int64_t nq,
                           int32_t* ids_host, float* dists_host, void* stream);

/* ---- learned early stop (library extension; the paper stops by the eps test alone) --------
 * A 12-64-64-2 perceptron (ReLU; 5,122 float32 parameters laid out W1 [64][12], b1 [64],
 * W2 [64][64], b2 [64], W3 [2][64], b3 [2]; logit 1 = stop) reads 12 features of the search state
 * after each hop and predicts whether the result list is already final. */

#define DEG_STOP_FEATURES 12
#define DEG_STOP_PARAMS 5122

/* Training traces: run the plain search (p->learned_stop ignored) and record, for each of the
 * first `cap` hops of query q, the 12 features (feats_dev [nq][cap][12] float32) and the label
 * 1 if the result list never changed after that hop, else 0 (labels_dev [nq][cap] int32);
 * counts_dev [nq] int32 gets the number of hops recorded. Slots past the count are untouched. */
DEG_API deg_status deg_stop_record(deg_index* idx, const deg_search_params* p, const float* queries_dev,
                                   int64_t nq, int32_t cap, float* feats_dev, int32_t* labels_dev,
                                   int32_t* counts_dev, void* stream);

/* Mean softmax cross-entropy of `count` samples x_dev [count][12] with labels_dev [count] and its
 * gradient grad_dev [5122] (loss_dev [1], nullable). scratch_dev holds
 * deg_mlp_scratch_floats(count) floats. Deterministic (fixed summation order). */
DEG_API deg_status deg_mlp_loss_grad(const float* w_dev, const float* x_dev, const int32_t* labels_dev, int64_t count,
                                     float* grad_dev, float* loss_dev, float* scratch_dev, void* stream);
DEG_API int64_t deg_mlp_scratch_floats(int64_t count);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) of w_dev with moments m_dev, v_dev (all [5122]);
 * step counts from 1. */
DEG_API deg_status deg_mlp_adam(float* w_dev, float* m_dev, float* v_dev, const float* grad_dev, int32_t step,
                                float lr, void* stream);

/* p_stop_dev [count] = softmax(network(x))[stop]. */
DEG_API deg_status deg_mlp_predict(const float* w_dev, const float* x_dev, int64_t count, float* p_stop_dev,
                                   void* stream);

/* Install a trained network on an uploaded index (stored in bfloat16 for the search) with the
 * decision threshold: stop when P(stop) > threshold, 0 < threshold < 1. */
DEG_API deg_status deg_set_stop_model(deg_index* idx, const float* w_dev, float threshold, void* stream);

/* ---- serving (library extension: continuous batching) ---------------------------------------
 * A persistent kernel keeps the index resident and serves requests from a ring in mapped host
 * memory: each of its warps takes the next request as soon as it is free, so requests posted
 * while others run are admitted as warps free up and run concurrently with them. Requests mix
 * k, eps and kind (vector query or exploration from a vertex). A request's result equals the
 * result of the same search run alone (the same per-query code; nothing is shared between
 * queries). Every device wait is bounded: when no request arrives for idle_timeout_s the kernel
 * ends and deg_serve_stop reports DEG_ETIMEOUT. */

typedef struct deg_server deg_server;

typedef struct {
    int32_t capacity;        /* ring slots (requests posted and not yet collected), >= 1          */
    int32_t kmax;            /* largest k of any request, 1..1024                                 */
    int32_t precision;       /* DEG_F32 | DEG_BF16 | DEG_FP8 (uploaded)                           */
    int32_t rerank;          /* reduced precision: re-rank width (0 = k)                          */
    int32_t entry_mode;      /* vector requests: 0 fixed entry vertex, 1 nearest pivot, 2 nearest
                                learned entry point                                               */
    int32_t learned_stop;    /* 1: use the index's stop network                                    */
    double idle_timeout_s;   /* end the kernel when no request arrives for this long (> 0)         */
    int32_t max_blocks;      /* 0: as many blocks of 4 warps as fit on the GPU; else at most this
                                many, leaving the rest of the GPU to other kernels                  */
} deg_serve_config;

/* Launch the serving kernel on its own (non-blocking) stream. The index must stay alive, and must
 * not be uploaded again or freed, until deg_serve_stop. The request ring (vectors, parameters,
 * results) lives in mapped pinned host memory owned by the server. *out is NULL on any error:
 * DEG_EINVAL for a NULL argument or a bad config (capacity < 1, kmax outside 1..1024,
 * idle_timeout_s <= 0, entry_mode outside 0..2, rerank outside 0..1024, max_blocks < 0);
 * DEG_ENOTREADY if the index, or its copy in the chosen precision, is not uploaded, or if
 * learned_stop is set without a stop model; DEG_ENOMEM / DEG_ECUDA if an allocation or the launch
 * fails (entry_mode 2 without learned entry points is a launch failure). */
DEG_API deg_status deg_serve_start(deg_index* idx, const deg_serve_config* cfg, deg_server** out);

/* Post one request: vec_host [dim] float32 for a vector query (vertex = -1), or vec_host NULL
 * and vertex = a vertex id for an exploration request; 1 <= k <= kmax; eps >= 0. *seq_out gets
 * its sequence number. DEG_EOVERFLOW (nothing posted) when its ring slot still holds an
 * uncollected request: poll earlier requests and retry. */
DEG_API deg_status deg_serve_submit(deg_server* srv, const float* vec_host, int32_t vertex, int32_t k, float eps,
                                    int64_t* seq_out);

/* 1 and the result (ids_host / dists_host [k], status_host [1], each nullable) if request seq is
 * finished, 0 if not yet, negative deg_status on error. Collecting frees its ring slot. */
DEG_API int32_t deg_serve_poll(deg_server* srv, int64_t seq, int32_t* ids_host, float* dists_host,
                               int32_t* status_host);

/* Replay a request trace: request i is posted at arrival_s[i] seconds after the call starts (or
 * as soon as its ring slot frees), results go to ids_out / dists_out [count][kmax] and
 * status_out [count], and latency_s_out[i] = completion time - arrival_s[i] as seen by the host.
 * vecs_host [count][dim] (rows of exploration requests are ignored), vertices [count] (-1 for a
 * vector query), ks [count], epss [count]. Fails with DEG_ETIMEOUT after timeout_s seconds.
 * device_s_out (nullable) [count] gets each request's device time: from the warp taking the posted
 * request to its result being published (%globaltimer), so latency minus device time is the time
 * spent waiting to be posted, waiting for a free warp and being collected by the host. */
DEG_API deg_status deg_serve_run_trace(deg_server* srv, const float* vecs_host, const int32_t* vertices,
                                       const int32_t* ks, const float* epss, const double* arrival_s, int64_t count,
                                       double* latency_s_out, int32_t* ids_out, float* dists_out,
                                       int32_t* status_out, double* device_s_out, double timeout_s);

/* Number of warps (concurrent requests) of the running kernel. */
DEG_API int32_t deg_serve_slots(const deg_server* srv);

/* Ask the kernel to finish, wait for it (bounded: in-flight requests complete first), free the
 * server. Returns DEG_OK, or DEG_ETIMEOUT if the kernel had ended on its idle timeout. */
DEG_API deg_status deg_serve_stop(deg_server* srv);

/* ---- exact ground truth (Eq. 1) ----------------------------------------------------------- */

/* Exact k nearest neighbours of queries_dev [nq][dim] among base_dev [n][dim] (float32 rows,
 * row-major, dim floats apart), 1 <= k <= 1024. Distances are the float32 Euclidean distances
 * the library's search uses; ties go to the lower id. Up to k = 256 the distances come from
 * bfloat16 tensor-core products and every row within a proven rounding bound is re-scored in
 * float32; above 256 every distance is computed in float32 on the CUDA cores. Both give the same
 * result. Synchronises the stream before it returns. The tensor-core path keeps its device scratch
 * (the bfloat16 copy of the rows, norms and per-query candidate lists: about 2 * n * dim rounded up
 * to 64, plus tens of KiB per query) from one call to the next, per device, growing it when a call
 * needs more and holding it until the process exits; calls on one device are serialised by a
 * lock. */
DEG_API deg_status knn_exact(const float* base_dev, int64_t n, const float* queries_dev, int64_t nq,
                     int32_t dim, int32_t k, int32_t* ids_dev, float* dists_dev, void* stream);

/* knn_exact without any device allocation. The paper has no counterpart: this is a library
 * service for callers that cannot allocate device memory while they run -- for instance a
 * process whose device memory is entirely reserved by another allocator (a framework's caching
 * allocator, a fixed memory budget), or a loop that cannot accept the device-wide
 * synchronisation that cudaMalloc/cudaFree imply. The caller still owns every input and output.
 * Same arguments, results and errors as knn_exact, except:
 *  - the distances live in one static device array of 32 MiB (8,388,608 float32) held by every
 *    GPU that loads the library until the process exits; n must be at most 8,388,608 (else
 *    DEG_EINVAL) and queries are processed in chunks of 8,388,608 / n (at most 4,194,240);
 *  - the device address is cached with the id of the CUDA context it was looked up in; a call in
 *    a new context of the device (after cudaDeviceReset, say) looks it up again;
 *  - the first call on a device looks up that array's device address (cudaGetSymbolAddress, with
 *    the device current) and caches it: make that first call before any stream capture;
 *  - all calls share the array and it keeps the last call's contents; two calls whose work
 *    overlaps on the GPU (different streams, or different host threads) race on it and give
 *    undefined results: order them on one stream or synchronise between them;
 *  - the call does not synchronise the stream (knn_exact does). */
DEG_API deg_status knn_exact_noalloc(const float* base_dev, int64_t n, const float* queries_dev, int64_t nq,
                                     int32_t dim, int32_t k, int32_t* ids_dev, float* dists_dev, void* stream);

/* Nearest row (k = 1 of Eq. 1) among a small set: for each query of queries_dev [nq][dim], the
 * index in [0, n) of the nearest of rows_dev [n][dim] (float32, row-major), 1 <= n <= 4096, and
 * its float32 distance. This is the search the pivot entry routing runs (entry_mode 1). Results
 * are exact: the same float32 distances as knn_exact, ties to the lower index. Distances come
 * from bfloat16 tensor-core products, and every row within a proven rounding bound of the
 * smallest is re-scored exactly. `cap` (a power of two, 1 ... 4096) bounds the rows re-scored per
 * query. A query with more rows inside the bound is scored exactly against all n rows instead,
 * with the same result. Allocates its scratch and synchronises the stream. DEG_EINVAL when n is
 * outside 1 ... 4096, dim is not positive, nq is negative or above 2^24, a pointer is NULL, or
 * cap is not a power of two in 1 ... 4096; DEG_ECUDA on a device error. nq = 0 does nothing. */
DEG_API deg_status deg_nearest_rows(const float* rows_dev, int64_t n, int32_t dim, const float* queries_dev, int64_t nq,
                                    int32_t cap, int32_t* ids_dev, float* dists_dev, void* stream);

/* Message of the last failed call on this thread ("" if none). */
DEG_API const char* deg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DEG_H */
