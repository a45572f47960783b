// Internal declarations of libdeg (not part of the C ABI).
#ifndef DEG_INTERNAL_H
#define DEG_INTERNAL_H

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/deg.h"

struct CUstream_st;
typedef CUstream_st* deg_stream_t;

namespace deg {

constexpr int kStopFeatures = 12;   // inputs of the learned-stop network
constexpr int kStopParams = 5122;   // 12*64 + 64 + 64*64 + 64 + 2*64 + 2

// Host-side graph construction (builder.cpp).
int build_graph(const float* x, int64_t n, int32_t dim, const deg_build_params& p, int32_t* adj_out,
                volatile int64_t* progress);

// Removes vertex v from the graph adj [n][d] over rows x [n][dim] (builder.cpp): its neighbours are
// re-paired so the graph stays even-regular, symmetric and connected, then the last vertex takes
// id v (*moved_from = n-1, or -1 when v was last) and n shrinks by one; *touched (nullable) gets
// the ids, after the move, of every vertex whose row changed. Returns 0, or 1 with *why set and
// nothing changed.
int remove_vertex(std::vector<float>& x, std::vector<int32_t>& adj, int64_t& n, int32_t dim, int32_t d, int32_t v,
                  int32_t* moved_from, std::vector<int32_t>* touched, std::string* why);

// Device construction (build_gpu.cu): batched ExtendGraph on the current device, adjacency
// [n][degree] written to adj_out (host). Returns a cudaError_t value (0 = success).
int build_graph_device(const float* x_host, int64_t n, int32_t dim, const deg_build_params& p, int32_t batch_div,
                       int32_t* adj_out, volatile int64_t* progress, deg_stream_t stream, std::string* why);
// Inserts vertices n_old .. n-1 (their rows in x_host [n][dim]) into the graph adj [n][degree] whose
// first n_old rows hold a graph and the rest -1 (batched Alg. 3, Alg. 4 when p.i_opt > 0).
int insert_vertices_device(const float* x_host, int32_t* adj, int64_t n_old, int64_t n, int32_t dim,
                           const deg_build_params& p, int32_t batch_div, deg_stream_t stream, std::string* why);
// Alg. 5 (p.refine_rounds rounds, p.i_opt / k_opt / eps_opt, SplitMix64(p.seed)) on the device over
// an existing graph adj_in [n][degree]; the result goes to adj_out (may be adj_in).
int refine_graph_device(const float* x_host, const int32_t* adj_in, int64_t n, int32_t dim, const deg_build_params& p,
                        int32_t* adj_out, int64_t* improved, deg_stream_t stream, std::string* why);

// Id of the calling thread's current CUDA context (0 when there is none): device addresses cached
// between calls are valid only in the context they were made in.
unsigned long long current_context_id();

// Record an error message for deg_last_error() and return the status.
deg_status fail(deg_status s, const std::string& msg);

// Device copy of an index (everything the kernels read), owned by deg_index.
struct DeviceIndex {
    int64_t n = 0;
    int32_t dim = 0;          // logical dimension
    int32_t dim_pad = 0;      // float32 row stride in elements (multiple of 4)
    int32_t degree = 0;       // logical degree
    int32_t deg_pad = 0;      // adjacency row stride in int32 (multiple of 4)
    float* x32 = nullptr;     // [n][dim_pad] float32, zero padded
    uint16_t* xbf = nullptr;  // [n][dim_pad16] bfloat16 (optional)
    int32_t dim_pad16 = 0;    // bf16 row stride (multiple of 8)
    uint8_t* x8 = nullptr;    // [n][dim_pad8] E4M3 codes (optional)
    float* scale8 = nullptr;  // [n] per-row scale of the E4M3 codes
    float* norm8 = nullptr;   // [n][2] {scale s, s^2 ||decoded codes||^2} per E4M3 row
    int32_t dim_pad8 = 0;     // fp8 row stride (multiple of 16)
    int32_t* adj = nullptr;   // uploaded: [n][deg_pad] caller ids, padded slots -1; after the locality
                              // layout: [n][deg_pad] int2 {internal id, caller id}, row = caller id
    int32_t entry = -1;       // entry vertex, caller's id
    // Locality layout: rows are stored in internal-id order (layout.cu).
    int32_t* old2new = nullptr;   // [n] caller id -> internal id
    int32_t* new2old = nullptr;   // [n] internal id -> caller id
    int32_t entry_internal = -1;
    int32_t* pivots = nullptr;    // [npivots] internal ids of the layout's pivots
    int32_t npivots = 0;
    struct KnnPlan* route_plan = nullptr;   // nearest-pivot search over the pivots' rows (knn_tc.cu)
    float far_tau = 3.4e38f;      // routed queries farther than this from their pivot start first
    // learned entry points (deg_train_entry): the same routing over trained pivots (entry_mode 2)
    int32_t* lpivots = nullptr;
    int32_t lnpivots = 0;
    struct KnnPlan* lroute_plan = nullptr;
    float lfar_tau = 3.4e38f;
    uint16_t* stop_w = nullptr;   // learned-stop weights, bfloat16, inference layout (mlp.cu)
    float stop_logit = 0.f;       // stop when logit(stop) - logit(continue) > this
};

// Scratch of the search kernels: the overflow list, and per-warp device-memory state (a visited
// bitmap of n bits and a back pool of candidate keys) for the main kernel and, with room for all
// n vertices, for the second kernel.
struct Workspace {
    int32_t* counters = nullptr;     // [0] overflow count, [1] second-kernel cursor, [2] main cursor
    int32_t* overflow = nullptr;     // [cap_q] query indices
    int32_t* route = nullptr;        // [4 * cap_q + 2] pivot labels, routed seeds (internal ids), pivot
                                     // distances (float), work order, two order cursors
    int64_t cap_q = 0;
    int64_t words = 0;               // 32-bit words of one visited bitmap
    uint32_t* bitmaps = nullptr;     // main kernel: [slots][words]
    uint64_t* backs = nullptr;       //   [slots][bcap] candidate keys
    int32_t* touched = nullptr;      //   [slots][8192] ids visited by the running query
    int32_t slots = 0, bcap = 0;
    uint32_t* pbitmaps = nullptr;    // second kernel: [pslots][words]
    uint64_t* pbacks = nullptr;      //   [pslots][n + 1]
    int32_t pslots = 0;
    // host e2e staging
    void* dq = nullptr;
    void* did = nullptr;
    void* dd = nullptr;
    int64_t stage_q = 0, stage_k = 0;
};

struct SearchArgs {
    const DeviceIndex* ix;
    const float* queries;     // [nq][dim] (row stride dim) or nullptr when explore
    const int32_t* seeds;     // [nq] or nullptr (entry vertex)
    int32_t explore;
    int64_t nq;
    int32_t k;
    float eps;
    int32_t precision;
    int32_t rerank;
    int32_t max_hops;
    int32_t visited_cap;
    int32_t queue_cap;
    int32_t entry_mode;
    int32_t learned_stop;
    float* rec_feats;         // training traces: [nq][rec_cap][kStopFeatures] (or null)
    int32_t* rec_labels;      //   [nq][rec_cap]
    int32_t* rec_counts;      //   [nq]
    int32_t rec_cap;
    int32_t* ids;
    float* dists;
    int32_t* status;
    int32_t* trace;
    const int32_t* seeds2 = nullptr;   // [nq] second seed per query (caller id, -1 = none), or null
    void* timer_start = nullptr;   // cudaEvent_t recorded just before the main search kernel
    void* timer_end = nullptr;     // cudaEvent_t recorded just after the second kernel
};

// Serving ring (device pointers into mapped host memory, plus two device words).
struct ServeArgs {
    const DeviceIndex* ix;
    const float* vecs;
    const int32_t* meta;          // [cap][4] {k, eps bits, vertex, seq}
    int32_t* ids;
    float* dists;
    int32_t* status;
    int32_t* trace;
    uint32_t* done;
    unsigned long long* times;    // [cap][2] device start / end (%globaltimer ns)
    const unsigned long long* tail;
    const int32_t* stop;
    int32_t* kstatus;
    unsigned long long* claim;
    int32_t cap, kmax, entry_mode, precision, rerank, learned_stop;
    unsigned long long idle_ns;
    int32_t max_blocks;       // 0: as many resident blocks as fit
};

// Kernel launchers (search.cu). Return a cudaError_t value (0 = success).
int launch_serving(const ServeArgs& a, Workspace& ws, deg_stream_t stream, int* warps, std::string* why);
int launch_search(const SearchArgs& a, Workspace& ws, deg_stream_t stream, std::string* why);
int workspace_reserve(Workspace& ws, const DeviceIndex& ix, int64_t nq, std::string* why);
void workspace_free(Workspace& ws);

// Entry vertex (entry.cu): lower median per coordinate, then the nearest row. Synchronous.
int compute_entry_vertex(DeviceIndex& ix, deg_stream_t stream, std::string* why);

// Reorder rows and adjacency by nearest pivot (layout.cu); fills old2new/new2old. Synchronous.
int apply_locality_layout(DeviceIndex& ix, deg_stream_t stream, std::string* why);

// Learned entry points (layout.cu): k-means (Lloyd, iters rounds) over the rows, each centroid
// replaced by its nearest row; those rows become the routing pivots. sizes_out (nullable, host,
// [k]) gets each final cluster's size. Synchronous.
int train_entry_points(DeviceIndex& ix, int32_t k, int32_t iters, deg_stream_t stream, int64_t* sizes_out,
                       std::string* why);

// Entry routing (layout.cu): seeds[q] = internal id of the pivot nearest to query q, dists[q] its
// distance; if order is given, a work order with the queries farther than far_tau from their
// pivot first (cursors: two int32 of device scratch).
int route_to_pivots(const DeviceIndex& ix, const float* queries, int64_t nq, int32_t* labels, int32_t* seeds,
                    float* dists, int32_t* order, int32_t* cursors, bool learned, deg_stream_t stream, std::string* why);

// Reduced-precision copies (quantize.cu).
int make_bf16_copy(DeviceIndex& ix, deg_stream_t stream, std::string* why);
int make_fp8_copy(DeviceIndex& ix, deg_stream_t stream, std::string* why);

// Learned-stop network (mlp.cu).
int mlp_loss_grad(const float* w, const float* x, const int32_t* labels, int64_t count, float* grad, float* loss,
                  float* scratch, deg_stream_t stream, std::string* why);
int64_t mlp_scratch_floats(int64_t count);
int mlp_adam(float* w, float* m, float* v, const float* g, int step, float lr, deg_stream_t stream, std::string* why);
int mlp_predict(const float* w, const float* x, int64_t count, float* p_stop, deg_stream_t stream, std::string* why);
int mlp_pack_inference(const float* w, uint16_t* out, deg_stream_t stream, std::string* why);

// Exact kNN: tensor-core distances with an exact float32 re-rank (knn_tc.cu); synchronises the
// stream.
int launch_knn_exact(const float* base, int64_t n, const float* queries, int64_t nq, int32_t dim,
                     int32_t k, int32_t* ids, float* dists, deg_stream_t stream, std::string* why);
// The same result from CUDA-core float32 distances and a full radix select (knn_exact.cu).
int launch_knn_simt(const float* base, int64_t n, const float* queries, int64_t nq, int32_t dim,
                    int32_t k, int32_t* ids, float* dists, deg_stream_t stream, std::string* why);
// k-NN over a small fixed row set (at most 4096 rows), tensor-core distances with the exact re-rank,
// no host synchronisation per call (knn_tc.cu). Rows are gathered at creation:
// row i = rows[(row_ids ? row_ids[i] : i) * row_stride ...]. ids[q][0..k) are row indices.
struct KnnPlan;
int knn_plan_create(KnnPlan** out, const float* rows, int64_t row_stride, const int32_t* row_ids, int64_t n, int32_t dim,
                    int32_t k, int32_t cap, deg_stream_t stream, std::string* why);
int knn_plan_run(KnnPlan* p, const float* queries, int64_t nq, int32_t* ids, float* dists, deg_stream_t stream,
                 std::string* why);
void knn_plan_destroy(KnnPlan* p);
// Same, on a fixed statically allocated scratch (no allocation in the call).
int launch_knn_exact_noalloc(const float* base, int64_t n, const float* queries, int64_t nq, int32_t dim,
                             int32_t k, int32_t* ids, float* dists, deg_stream_t stream, std::string* why);

}  // namespace deg

#endif
