// C ABI of libdeg: argument validation, index lifecycle, graph files and the host side of the
// search and kNN calls. Every compute step runs in the library's CUDA kernels; this file only
// checks, allocates, copies and launches.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "deg_internal.h"

struct deg_index {
    int64_t n = 0;
    int32_t dim = 0;
    int32_t degree = 0;
    std::vector<float> x;        // [n][dim]
    std::vector<int32_t> adj;    // [n][degree]
    deg::DeviceIndex dev;
    deg::Workspace ws;
    int device = -1;
    int32_t uploaded_mask = 0;
    void* timer_start = nullptr;  // cudaEvent_t pair recorded around the search kernels (or null)
    void* timer_end = nullptr;
};

namespace deg {
namespace {
thread_local std::string g_last_error;

constexpr char kMagic[8] = {'D', 'E', 'G', 'G', 'R', 'A', 'P', 'H'};
constexpr uint32_t kVersion = 1;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t flags;          // bit 0: vectors follow the adjacency
    int64_t n;
    int32_t dim;
    int32_t degree;
    uint64_t vec_checksum;   // FNV-1a 64 over the float32 bytes of the vectors
    uint64_t reserved[3];
};
static_assert(sizeof(FileHeader) == 64, "header layout");

uint64_t fnv1a(const void* p, size_t bytes) {
    const uint8_t* b = static_cast<const uint8_t*>(p);
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < bytes; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

deg_status cuda_fail(cudaError_t e, const char* what) {
    return fail(DEG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Graph invariants of Sec. 5.1 that the search relies on (entries in range, no loops, no
// duplicates, symmetric, even degree >= 4). Connectivity is not required by the search.
deg_status check_graph(const int32_t* adj, int64_t n, int32_t d) {
    if (d < 4 || d % 2) return fail(DEG_EGRAPH, "degree must be even and >= 4");
    for (int64_t u = 0; u < n; ++u) {
        const int32_t* r = adj + u * d;
        for (int32_t j = 0; j < d; ++j) {
            const int32_t v = r[j];
            if (v < 0 || v >= n) return fail(DEG_EGRAPH, "neighbour id out of range at vertex " + std::to_string(u));
            if (v == u) return fail(DEG_EGRAPH, "self loop at vertex " + std::to_string(u));
            for (int32_t i = 0; i < j; ++i)
                if (r[i] == v) return fail(DEG_EGRAPH, "duplicate edge at vertex " + std::to_string(u));
            const int32_t* b = adj + (int64_t)v * d;
            bool back = false;
            for (int32_t i = 0; i < d && !back; ++i) back = (b[i] == u);
            if (!back) return fail(DEG_EGRAPH, "asymmetric edge " + std::to_string(u) + "-" + std::to_string(v));
        }
    }
    return DEG_OK;
}

// check_graph over the rows of the vertices `rows` only (a local edit keeps the rest as it was).
deg_status check_rows(const int32_t* adj, int64_t n, int32_t d, const std::vector<int32_t>& rows) {
    for (const int32_t u : rows) {
        const int32_t* r = adj + (int64_t)u * d;
        for (int32_t j = 0; j < d; ++j) {
            const int32_t v = r[j];
            if (v < 0 || v >= n) return fail(DEG_EGRAPH, "neighbour id out of range at vertex " + std::to_string(u));
            if (v == u) return fail(DEG_EGRAPH, "self loop at vertex " + std::to_string(u));
            for (int32_t i = 0; i < j; ++i)
                if (r[i] == v) return fail(DEG_EGRAPH, "duplicate edge at vertex " + std::to_string(u));
            const int32_t* b = adj + (int64_t)v * d;
            bool back = false;
            for (int32_t i = 0; i < d && !back; ++i) back = (b[i] == u);
            if (!back) return fail(DEG_EGRAPH, "asymmetric edge " + std::to_string(u) + "-" + std::to_string(v));
        }
    }
    return DEG_OK;
}

void free_device(deg_index* idx) {
    DeviceIndex& d = idx->dev;
    cudaFree(d.x32);
    cudaFree(d.xbf);
    cudaFree(d.x8);
    cudaFree(d.scale8);
    cudaFree(d.norm8);
    cudaFree(d.adj);
    cudaFree(d.old2new);
    cudaFree(d.new2old);
    cudaFree(d.pivots);
    knn_plan_destroy(d.route_plan);
    d.route_plan = nullptr;
    knn_plan_destroy(d.lroute_plan);
    d.lroute_plan = nullptr;
    cudaFree(d.lpivots);
    cudaFree(d.stop_w);
    d = DeviceIndex{};
    workspace_free(idx->ws);
    idx->uploaded_mask = 0;
}

deg_index* new_index(int64_t n, int32_t dim, int32_t degree) {
    deg_index* idx = new (std::nothrow) deg_index;
    if (!idx) return nullptr;
    try {
        idx->n = n;
        idx->dim = dim;
        idx->degree = degree;
        idx->x.resize((size_t)n * dim);
        idx->adj.resize((size_t)n * degree);
    } catch (const std::bad_alloc&) {
        delete idx;
        return nullptr;
    }
    return idx;
}

}  // namespace

deg_status fail(deg_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

}  // namespace deg

using namespace deg;

extern "C" const char* deg_last_error(void) { return g_last_error.c_str(); }

extern "C" deg_status deg_build(const float* base_host, int64_t n, int32_t dim, const deg_build_params* p,
                                volatile int64_t* progress, deg_index** out) {
    if (!out) return fail(DEG_EINVAL, "deg_build: out is NULL");
    *out = nullptr;
    if (!base_host || !p) return fail(DEG_EINVAL, "deg_build: NULL argument");
    if (dim <= 0) return fail(DEG_EINVAL, "deg_build: dim must be positive");
    if (p->degree < 4 || p->degree % 2) return fail(DEG_EINVAL, "deg_build: degree must be even and >= 4");
    if (p->degree > 256) return fail(DEG_EINVAL, "deg_build: degree must be <= 256");
    if (n < p->degree + 1) return fail(DEG_EINVAL, "deg_build: need n >= degree + 1");
    if (n > INT32_MAX) return fail(DEG_EINVAL, "deg_build: n must fit in int32");
    if (p->k_ext < p->degree || p->k_opt < 1 || p->i_opt < 0 || p->refine_rounds < 0)
        return fail(DEG_EINVAL, "deg_build: need k_ext >= degree, k_opt >= 1, i_opt >= 0");
    if (!(p->eps_ext >= 0.f) || !(p->eps_opt >= 0.f)) return fail(DEG_EINVAL, "deg_build: eps must be >= 0");
    deg_index* idx = new_index(n, dim, p->degree);
    if (!idx) return fail(DEG_ENOMEM, "deg_build: host allocation failed");
    std::memcpy(idx->x.data(), base_host, sizeof(float) * (size_t)n * dim);
    try {
        build_graph(idx->x.data(), n, dim, *p, idx->adj.data(), progress);
    } catch (const std::exception& e) {
        delete idx;
        return fail(DEG_EGRAPH, std::string("deg_build: ") + e.what());
    }
    *out = idx;
    return DEG_OK;
}

extern "C" deg_status deg_build_device(const float* base_host, int64_t n, int32_t dim, const deg_build_params* p,
                                       int32_t batch_div, volatile int64_t* progress, deg_index** out, void* stream) {
    if (!out) return fail(DEG_EINVAL, "deg_build_device: out is NULL");
    *out = nullptr;
    if (!base_host || !p) return fail(DEG_EINVAL, "deg_build_device: NULL argument");
    if (dim <= 0 || dim > 1024) return fail(DEG_EINVAL, "deg_build_device: dim must be in [1, 1024]");
    if (p->degree < 4 || p->degree % 2 || p->degree > 128)
        return fail(DEG_EINVAL, "deg_build_device: degree must be even and in [4, 128]");
    if (n < p->degree + 1) return fail(DEG_EINVAL, "deg_build_device: need n >= degree + 1");
    if (n > INT32_MAX) return fail(DEG_EINVAL, "deg_build_device: n must fit in int32");
    if (p->k_ext < p->degree || p->k_ext > 1024) return fail(DEG_EINVAL, "deg_build_device: need degree <= k_ext <= 1024");
    if (p->i_opt < 0 || p->i_opt > 6 || (p->i_opt > 0 && (p->k_opt < 1 || p->k_opt > 1024)) || p->refine_rounds < 0)
        return fail(DEG_EINVAL, "deg_build_device: need 0 <= i_opt <= 6, 1 <= k_opt <= 1024, refine_rounds >= 0");
    if (p->refine_rounds > 0 && p->i_opt == 0) return fail(DEG_EINVAL, "deg_build_device: refine_rounds needs i_opt >= 1");
    if (!(p->eps_ext >= 0.f) || !(p->eps_opt >= 0.f)) return fail(DEG_EINVAL, "deg_build_device: eps must be >= 0");
    if (batch_div < 1) return fail(DEG_EINVAL, "deg_build_device: batch_div must be >= 1");
    deg_index* idx = new_index(n, dim, p->degree);
    if (!idx) return fail(DEG_ENOMEM, "deg_build_device: host allocation failed");
    std::memcpy(idx->x.data(), base_host, sizeof(float) * (size_t)n * dim);
    std::string why;
    const int e = build_graph_device(idx->x.data(), n, dim, *p, batch_div, idx->adj.data(), progress,
                                     static_cast<deg_stream_t>(stream), &why);
    if (e != 0) {
        delete idx;
        return fail(e == cudaErrorInvalidValue ? DEG_EINVAL : DEG_ECUDA, "deg_build_device: " + why);
    }
    const deg_status s = check_graph(idx->adj.data(), n, p->degree);
    if (s != DEG_OK) {
        delete idx;
        return s;
    }
    *out = idx;
    return DEG_OK;
}

extern "C" deg_status deg_insert_device(deg_index* idx, const float* new_host, int64_t m, const deg_build_params* p,
                                        int32_t batch_div, void* stream) {
    if (!idx || !p || (m > 0 && !new_host)) return fail(DEG_EINVAL, "deg_insert_device: NULL argument");
    if (m < 0 || idx->n + m > INT32_MAX) return fail(DEG_EINVAL, "deg_insert_device: bad count");
    if (p->degree != idx->degree || idx->degree > 128) return fail(DEG_EINVAL, "deg_insert_device: params.degree differs from the index's, or above 128");
    if (p->k_ext < p->degree || p->k_ext > 1024 || p->i_opt < 0 || p->i_opt > 6 ||
        (p->i_opt > 0 && (p->k_opt < 1 || p->k_opt > 1024)) || !(p->eps_ext >= 0.f) || !(p->eps_opt >= 0.f) || batch_div < 1)
        return fail(DEG_EINVAL, "deg_insert_device: need degree <= k_ext <= 1024, 0 <= i_opt <= 6, 1 <= k_opt <= 1024, eps >= 0, batch_div >= 1");
    if (m == 0) return DEG_OK;
    const int64_t n_old = idx->n, n = n_old + m;
    try {
        idx->x.resize((size_t)n * idx->dim);
        idx->adj.resize((size_t)n * idx->degree, -1);
    } catch (const std::bad_alloc&) {
        idx->x.resize((size_t)n_old * idx->dim);
        idx->adj.resize((size_t)n_old * idx->degree);
        return fail(DEG_ENOMEM, "deg_insert_device: host allocation failed");
    }
    std::memcpy(idx->x.data() + (size_t)n_old * idx->dim, new_host, sizeof(float) * (size_t)m * idx->dim);
    std::string why;
    const int e = insert_vertices_device(idx->x.data(), idx->adj.data(), n_old, n, idx->dim, *p, batch_div,
                                         static_cast<deg_stream_t>(stream), &why);
    if (e != 0) {
        idx->x.resize((size_t)n_old * idx->dim);
        idx->adj.resize((size_t)n_old * idx->degree);
        return fail(e == cudaErrorInvalidValue ? DEG_EINVAL : DEG_ECUDA, "deg_insert_device: " + why);
    }
    idx->n = n;
    free_device(idx);                                          // the device copy shows the old graph
    return check_graph(idx->adj.data(), idx->n, idx->degree);
}

extern "C" deg_status deg_refine_device(deg_index* idx, const deg_build_params* p, int64_t* improved, void* stream) {
    if (!idx || !p) return fail(DEG_EINVAL, "deg_refine_device: NULL argument");
    if (p->degree != idx->degree) return fail(DEG_EINVAL, "deg_refine_device: params.degree differs from the index's");
    if (idx->degree > 128) return fail(DEG_EINVAL, "deg_refine_device: degree above 128");
    if (p->refine_rounds < 0 || p->i_opt < 1 || p->i_opt > 6 || p->k_opt < 1 || p->k_opt > 1024 || !(p->eps_opt >= 0.f))
        return fail(DEG_EINVAL, "deg_refine_device: need refine_rounds >= 0, 1 <= i_opt <= 6, 1 <= k_opt <= 1024, eps_opt >= 0");
    if (p->refine_rounds == 0) {
        if (improved) *improved = 0;
        return DEG_OK;
    }
    std::string why;
    const int e = refine_graph_device(idx->x.data(), idx->adj.data(), idx->n, idx->dim, *p, idx->adj.data(), improved,
                                      static_cast<deg_stream_t>(stream), &why);
    if (e != 0) return fail(e == cudaErrorInvalidValue ? DEG_EINVAL : DEG_ECUDA, "deg_refine_device: " + why);
    const deg_status s = check_graph(idx->adj.data(), idx->n, idx->degree);
    if (s != DEG_OK) return s;
    free_device(idx);                                          // the device copy shows the old graph
    return DEG_OK;
}

extern "C" deg_status deg_remove(deg_index* idx, int32_t v, int32_t* moved_from) {
    if (!idx) return fail(DEG_EINVAL, "deg_remove: NULL index");
    if (v < 0 || v >= idx->n) return fail(DEG_EINVAL, "deg_remove: vertex out of range");
    std::string why;
    int32_t moved = -1;
    std::vector<int32_t> touched;
    if (deg::remove_vertex(idx->x, idx->adj, idx->n, idx->dim, idx->degree, v, &moved, &touched, &why) != 0)
        return fail(DEG_EINVAL, "deg_remove: " + why);
    if (moved_from) *moved_from = moved;
    free_device(idx);                                          // the device copy shows the old graph
    return check_rows(idx->adj.data(), idx->n, idx->degree, touched);
}

extern "C" deg_status deg_index_from_arrays(const float* base_host, const int32_t* adj_host, int64_t n,
                                            int32_t dim, int32_t degree, deg_index** out) {
    if (!out) return fail(DEG_EINVAL, "deg_index_from_arrays: out is NULL");
    *out = nullptr;
    if (!base_host || !adj_host || n <= 0 || dim <= 0) return fail(DEG_EINVAL, "deg_index_from_arrays: bad arguments");
    if (n > INT32_MAX) return fail(DEG_EINVAL, "deg_index_from_arrays: n must fit in int32");
    if (degree > 256) return fail(DEG_EINVAL, "deg_index_from_arrays: degree must be <= 256");
    deg_status s = check_graph(adj_host, n, degree);
    if (s != DEG_OK) return s;
    deg_index* idx = new_index(n, dim, degree);
    if (!idx) return fail(DEG_ENOMEM, "deg_index_from_arrays: host allocation failed");
    std::memcpy(idx->x.data(), base_host, sizeof(float) * (size_t)n * dim);
    std::memcpy(idx->adj.data(), adj_host, sizeof(int32_t) * (size_t)n * degree);
    *out = idx;
    return DEG_OK;
}

extern "C" deg_status deg_save(const deg_index* idx, const char* path, int32_t with_vectors) {
    if (!idx || !path) return fail(DEG_EINVAL, "deg_save: NULL argument");
    FileHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.flags = with_vectors ? 1u : 0u;
    h.n = idx->n;
    h.dim = idx->dim;
    h.degree = idx->degree;
    h.vec_checksum = fnv1a(idx->x.data(), sizeof(float) * idx->x.size());
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(DEG_EIO, std::string("deg_save: cannot open ") + path);
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 &&
              std::fwrite(idx->adj.data(), sizeof(int32_t), idx->adj.size(), f) == idx->adj.size();
    if (ok && with_vectors) ok = std::fwrite(idx->x.data(), sizeof(float), idx->x.size(), f) == idx->x.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? DEG_OK : fail(DEG_EIO, std::string("deg_save: write failed for ") + path);
}

extern "C" deg_status deg_load(const char* path, const float* base_host, deg_index** out) {
    if (!out || !path) return fail(DEG_EINVAL, "deg_load: NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(DEG_EIO, std::string("deg_load: cannot open ") + path);
    FileHeader h{};
    if (std::fread(&h, sizeof h, 1, f) != 1 || std::memcmp(h.magic, kMagic, 8) || h.version != kVersion ||
        h.n <= 0 || h.n > INT32_MAX || h.dim <= 0 || h.degree < 4 || h.degree > 256) {
        std::fclose(f);
        return fail(DEG_EIO, std::string("deg_load: bad header in ") + path);
    }
    const bool has_vec = h.flags & 1u;
    if (!has_vec && !base_host) {
        std::fclose(f);
        return fail(DEG_EINVAL, "deg_load: file has no vectors and base_host is NULL");
    }
    deg_index* idx = new_index(h.n, h.dim, h.degree);
    if (!idx) {
        std::fclose(f);
        return fail(DEG_ENOMEM, "deg_load: host allocation failed");
    }
    bool ok = std::fread(idx->adj.data(), sizeof(int32_t), idx->adj.size(), f) == idx->adj.size();
    if (ok && has_vec) ok = std::fread(idx->x.data(), sizeof(float), idx->x.size(), f) == idx->x.size();
    std::fclose(f);
    if (!ok) {
        delete idx;
        return fail(DEG_EIO, std::string("deg_load: truncated file ") + path);
    }
    if (!has_vec) {
        std::memcpy(idx->x.data(), base_host, sizeof(float) * idx->x.size());
        if (fnv1a(idx->x.data(), sizeof(float) * idx->x.size()) != h.vec_checksum) {
            delete idx;
            return fail(DEG_EIO, "deg_load: base_host does not match the vectors the graph was built on");
        }
    }
    deg_status s = check_graph(idx->adj.data(), idx->n, idx->degree);
    if (s != DEG_OK) {
        delete idx;
        return s;
    }
    *out = idx;
    return DEG_OK;
}

extern "C" deg_status deg_index_info(const deg_index* idx, int64_t* n, int32_t* dim, int32_t* degree) {
    if (!idx) return fail(DEG_EINVAL, "deg_index_info: NULL index");
    if (n) *n = idx->n;
    if (dim) *dim = idx->dim;
    if (degree) *degree = idx->degree;
    return DEG_OK;
}

extern "C" deg_status deg_get_adjacency(const deg_index* idx, int32_t* adj_host) {
    if (!idx || !adj_host) return fail(DEG_EINVAL, "deg_get_adjacency: NULL argument");
    std::memcpy(adj_host, idx->adj.data(), sizeof(int32_t) * idx->adj.size());
    return DEG_OK;
}

extern "C" deg_status deg_upload(deg_index* idx, int32_t precision_mask, void* stream) {
    if (!idx) return fail(DEG_EINVAL, "deg_upload: NULL index");
    if (precision_mask & ~((1 << DEG_BF16) | (1 << DEG_FP8) | (1 << DEG_F32)))
        return fail(DEG_EINVAL, "deg_upload: unknown precision bit");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "deg_upload: cudaGetDevice");
    if (idx->dev.x32 && idx->device != dev) free_device(idx);
    DeviceIndex& d = idx->dev;
    std::string why;
    if (!d.x32) {
        d.n = idx->n;
        d.dim = idx->dim;
        d.dim_pad = (idx->dim + 3) / 4 * 4;
        d.degree = idx->degree;
        d.deg_pad = (idx->degree + 3) / 4 * 4;
        const size_t xb = sizeof(float) * (size_t)d.n * d.dim_pad;
        const size_t ab = sizeof(int32_t) * (size_t)d.n * d.deg_pad;
        if ((e = cudaMalloc(&d.x32, xb)) != cudaSuccess || (e = cudaMalloc(&d.adj, ab)) != cudaSuccess) {
            free_device(idx);
            return fail(DEG_ENOMEM, std::string("deg_upload: cudaMalloc: ") + cudaGetErrorString(e));
        }
        // Strided 2-D copies place each row at its padded stride; padding is zero / -1.
        if ((e = cudaMemsetAsync(d.x32, 0, xb, st)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(d.x32, sizeof(float) * d.dim_pad, idx->x.data(), sizeof(float) * d.dim,
                                   sizeof(float) * d.dim, d.n, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d.adj, 0xff, ab, st)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(d.adj, sizeof(int32_t) * d.deg_pad, idx->adj.data(), sizeof(int32_t) * d.degree,
                                   sizeof(int32_t) * d.degree, d.n, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            free_device(idx);
            return cuda_fail(e, "deg_upload: copy");
        }
        idx->device = dev;
        idx->uploaded_mask = 1 << DEG_F32;
        if (compute_entry_vertex(d, st, &why) != 0) {
            free_device(idx);
            return fail(DEG_ECUDA, "deg_upload: entry vertex: " + why);
        }
        if (apply_locality_layout(d, st, &why) != 0) {
            free_device(idx);
            return fail(DEG_ECUDA, "deg_upload: layout: " + why);
        }
    }
    if ((precision_mask & (1 << DEG_BF16)) && !d.xbf) {
        if (make_bf16_copy(d, st, &why) != 0) return fail(DEG_ECUDA, "deg_upload: bf16 copy: " + why);
        idx->uploaded_mask |= 1 << DEG_BF16;
    }
    if ((precision_mask & (1 << DEG_FP8)) && !d.x8) {
        if (make_fp8_copy(d, st, &why) != 0) return fail(DEG_ECUDA, "deg_upload: fp8 copy: " + why);
        idx->uploaded_mask |= 1 << DEG_FP8;
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "deg_upload: synchronize");
    return DEG_OK;
}

extern "C" int32_t deg_entry_vertex(const deg_index* idx) { return idx ? idx->dev.entry : -1; }

extern "C" int32_t deg_get_pivots(const deg_index* idx, int32_t learned, int32_t* ids_host, int32_t cap) {
    if (!idx) return -1;
    const DeviceIndex& d = idx->dev;
    const int32_t* piv = learned ? d.lpivots : d.pivots;
    const int32_t np = learned ? d.lnpivots : d.npivots;
    if (!piv) return 0;
    if (!ids_host || cap < np) return np;
    // internal ids -> caller ids
    std::vector<int32_t> in((size_t)np), n2o((size_t)d.n);
    if (cudaMemcpy(in.data(), piv, sizeof(int32_t) * np, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(n2o.data(), d.new2old, sizeof(int32_t) * d.n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    for (int32_t i = 0; i < np; ++i) ids_host[i] = n2o[in[i]];
    return np;
}

extern "C" deg_status deg_train_entry(deg_index* idx, int32_t k, int32_t iters, int64_t* sizes_host, void* stream) {
    if (!idx) return fail(DEG_EINVAL, "deg_train_entry: NULL index");
    if (!idx->dev.x32) return fail(DEG_ENOTREADY, "deg_train_entry: upload the index first");
    if (k < 1 || k > 4096 || k > idx->n || iters < 0 || iters > 1000)
        return fail(DEG_EINVAL, "deg_train_entry: need 1 <= k <= min(4096, n), 0 <= iters <= 1000");
    std::string why;
    const int e = train_entry_points(idx->dev, k, iters, static_cast<deg_stream_t>(stream), sizes_host, &why);
    if (e != 0) return fail(e == cudaErrorInvalidValue ? DEG_EINVAL : DEG_ECUDA, "deg_train_entry: " + why);
    return DEG_OK;
}

extern "C" deg_status deg_export_codes(const deg_index* idx, int32_t precision, void* codes_host, float* scales_host) {
    if (!idx || !codes_host) return fail(DEG_EINVAL, "deg_export_codes: NULL argument");
    const DeviceIndex& d = idx->dev;
    if (precision != DEG_BF16 && precision != DEG_FP8)
        return fail(DEG_EINVAL, "deg_export_codes: precision must be DEG_BF16 or DEG_FP8");
    if (precision == DEG_BF16 ? !d.xbf : !d.x8) return fail(DEG_ENOTREADY, "deg_export_codes: copy not uploaded");
    if (precision == DEG_FP8 && !scales_host) return fail(DEG_EINVAL, "deg_export_codes: scales_host is NULL");
    // The device stores rows in internal (layout) order: copy them out, then put them back in the
    // caller's order.
    const size_t eb = precision == DEG_BF16 ? 2 : 1;
    std::vector<uint8_t> rows;
    std::vector<float> sc;
    std::vector<int32_t> o2n;
    try {
        rows.resize(eb * d.dim * d.n);
        o2n.resize(d.n);
        if (precision == DEG_FP8) sc.resize(d.n);
    } catch (const std::bad_alloc&) {
        return fail(DEG_ENOMEM, "deg_export_codes: host allocation failed");
    }
    cudaError_t e = precision == DEG_BF16
        ? cudaMemcpy2D(rows.data(), eb * d.dim, d.xbf, 2 * (size_t)d.dim_pad16, eb * d.dim, d.n, cudaMemcpyDeviceToHost)
        : cudaMemcpy2D(rows.data(), eb * d.dim, d.x8, (size_t)d.dim_pad8, eb * d.dim, d.n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(o2n.data(), d.old2new, 4 * d.n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && precision == DEG_FP8) e = cudaMemcpy(sc.data(), d.scale8, 4 * d.n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "deg_export_codes");
    uint8_t* out = static_cast<uint8_t*>(codes_host);
    for (int64_t v = 0; v < d.n; ++v) {
        std::memcpy(out + v * eb * d.dim, rows.data() + (size_t)o2n[v] * eb * d.dim, eb * d.dim);
        if (precision == DEG_FP8) scales_host[v] = sc[o2n[v]];
    }
    return DEG_OK;
}

extern "C" void deg_free(deg_index* idx) {
    if (!idx) return;
    free_device(idx);
    delete idx;
}

namespace {

deg_status validate_search(const deg_index* idx, const deg_search_params* p, const float* queries,
                           const int32_t* seeds, int32_t explore, int64_t nq) {
    if (!idx || !p) return fail(DEG_EINVAL, "search: NULL index or params");
    if (!idx->dev.x32) return fail(DEG_ENOTREADY, "search: index not uploaded (call deg_upload)");
    if (nq < 0 || nq > INT32_MAX) return fail(DEG_EINVAL, "search: nq out of range");
    if (p->k < 1 || p->k > 1024) return fail(DEG_EINVAL, "search: k must be in [1, 1024]");
    if (explore ? p->k > idx->n - 1 : p->k > idx->n) return fail(DEG_EINVAL, "search: k larger than the candidates");
    if (!(p->eps >= 0.f) || std::isinf(p->eps)) return fail(DEG_EINVAL, "search: eps must be finite and >= 0");
    if (p->precision < DEG_F32 || p->precision > DEG_FP8) return fail(DEG_EINVAL, "search: unknown precision");
    if (!(idx->uploaded_mask & (1 << p->precision))) return fail(DEG_ENOTREADY, "search: precision copy not uploaded");
    if (p->rerank < -1 || p->rerank > 1024 || (p->rerank > 0 && p->rerank < p->k))
        return fail(DEG_EINVAL, "search: rerank must be -1, 0 or in [k, 1024]");
    if (p->max_hops < 0) return fail(DEG_EINVAL, "search: max_hops must be >= 0");
    if (p->visited_cap != 0) return fail(DEG_EINVAL, "search: visited_cap is reserved and must be 0");
    if (p->queue_cap < 0 || p->queue_cap > 32768) return fail(DEG_EINVAL, "search: queue_cap must be in [0, 32768]");
    if (p->entry_mode < 0 || p->entry_mode > 2) return fail(DEG_EINVAL, "search: entry_mode must be 0, 1 or 2");
    if (p->entry_mode == 2 && !idx->dev.lpivots) return fail(DEG_ENOTREADY, "search: no learned entry points (deg_train_entry)");
    if (p->learned_stop != 0 && p->learned_stop != 1) return fail(DEG_EINVAL, "search: learned_stop must be 0 or 1");
    if (p->entry_mode >= 1 && (explore || seeds)) return fail(DEG_EINVAL, "search: entry_mode 1 or 2 needs query vectors and no seeds");
    if (explore ? (queries != nullptr || seeds == nullptr) : (queries == nullptr && nq > 0))
        return fail(DEG_EINVAL, "search: explore needs vertex ids and no query vectors; search needs vectors");
    return DEG_OK;
}

}  // namespace

extern "C" deg_status deg_search_ex(deg_index* idx, const deg_search_params* p, const float* queries_dev,
                                    const int32_t* seeds_dev, int32_t explore, int64_t nq, int32_t* ids_dev,
                                    float* dists_dev, int32_t* status_dev, int32_t* trace_dev, void* stream) {
    deg_status s = validate_search(idx, p, queries_dev, seeds_dev, explore, nq);
    if (s != DEG_OK) return s;
    if (nq == 0) return DEG_OK;
    if (!ids_dev || !dists_dev) return fail(DEG_EINVAL, "search: NULL output");
    std::string why;
    if (workspace_reserve(idx->ws, idx->dev, nq, &why) != 0) return fail(DEG_ENOMEM, "search: workspace: " + why);
    if (p->learned_stop && !idx->dev.stop_w) return fail(DEG_ENOTREADY, "search: no stop model (deg_set_stop_model)");
    SearchArgs a{&idx->dev, queries_dev, seeds_dev, explore ? 1 : 0, nq, p->k, p->eps, p->precision,
                 p->rerank, p->max_hops, p->visited_cap, p->queue_cap, p->entry_mode, p->learned_stop ? 1 : 0,
                 nullptr, nullptr, nullptr, 0, ids_dev, dists_dev, status_dev, trace_dev};
    a.timer_start = idx->timer_start;
    a.timer_end = idx->timer_end;
    const int e = launch_search(a, idx->ws, static_cast<deg_stream_t>(stream), &why);
    if (e != 0) return fail(e == cudaErrorInvalidValue ? DEG_EINVAL : DEG_ECUDA, "search: " + why);
    return DEG_OK;
}

extern "C" deg_status deg_set_kernel_timer(deg_index* idx, void* start_event, void* end_event) {
    if (!idx) return fail(DEG_EINVAL, "set_kernel_timer: NULL index");
    if ((start_event == nullptr) != (end_event == nullptr))
        return fail(DEG_EINVAL, "set_kernel_timer: give both events or neither");
    idx->timer_start = start_event;
    idx->timer_end = end_event;
    return DEG_OK;
}

extern "C" deg_status deg_search(deg_index* idx, const float* queries_dev, int64_t nq, int32_t k, float eps,
                                 const int32_t* seeds_dev, int32_t* ids_dev, float* dists_dev,
                                 int32_t* status_dev, void* stream) {
    deg_search_params p{k, eps, DEG_F32, 0, 0, 0, 0, 0, 0};
    return deg_search_ex(idx, &p, queries_dev, seeds_dev, 0, nq, ids_dev, dists_dev, status_dev, nullptr, stream);
}

extern "C" deg_status deg_explore(deg_index* idx, const int32_t* vertex_ids_dev, int64_t nq, int32_t k,
                                  float eps, int32_t* ids_dev, float* dists_dev, int32_t* status_dev,
                                  void* stream) {
    deg_search_params p{k, eps, DEG_F32, 0, 0, 0, 0, 0, 0};
    return deg_search_ex(idx, &p, nullptr, vertex_ids_dev, 1, nq, ids_dev, dists_dev, status_dev, nullptr, stream);
}

extern "C" deg_status deg_search_host(deg_index* idx, const deg_search_params* p, const float* queries_host,
                                      const int32_t* seeds_host, int32_t explore, int64_t nq, int32_t* ids_host,
                                      float* dists_host, void* stream) {
    deg_status s = validate_search(idx, p, queries_host, seeds_host, explore, nq);
    if (s != DEG_OK) return s;
    if (nq == 0) return DEG_OK;
    if (!ids_host || !dists_host) return fail(DEG_EINVAL, "search_host: NULL output");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Workspace& ws = idx->ws;
    cudaError_t e;
    const int64_t row = explore ? 0 : idx->dim;
    if (ws.stage_q < nq || ws.stage_k < p->k) {
        cudaFree(ws.dq);
        cudaFree(ws.did);
        cudaFree(ws.dd);
        ws.dq = ws.did = ws.dd = nullptr;
        ws.stage_q = ws.stage_k = 0;
        const size_t qb = std::max<size_t>(sizeof(float) * (size_t)nq * idx->dim, sizeof(int32_t) * (size_t)nq);
        if ((e = cudaMalloc(&ws.dq, qb)) != cudaSuccess || (e = cudaMalloc(&ws.did, sizeof(int32_t) * nq * p->k)) != cudaSuccess ||
            (e = cudaMalloc(&ws.dd, sizeof(float) * nq * p->k)) != cudaSuccess)
            return fail(DEG_ENOMEM, std::string("search_host: cudaMalloc: ") + cudaGetErrorString(e));
        ws.stage_q = nq;
        ws.stage_k = p->k;
    }
    if (!explore && seeds_host) return fail(DEG_EINVAL, "search_host: per-query seeds are not supported with host buffers");
    const size_t in_bytes = explore ? sizeof(int32_t) * nq : sizeof(float) * nq * row;
    if ((e = cudaMemcpyAsync(ws.dq, explore ? (const void*)seeds_host : (const void*)queries_host, in_bytes,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "search_host: H2D");
    const float* q = explore ? nullptr : static_cast<const float*>(ws.dq);
    const int32_t* sd = explore ? static_cast<const int32_t*>(ws.dq) : nullptr;
    s = deg_search_ex(idx, p, q, sd, explore, nq, static_cast<int32_t*>(ws.did), static_cast<float*>(ws.dd),
                      nullptr, nullptr, stream);
    if (s != DEG_OK) return s;
    if ((e = cudaMemcpyAsync(ids_host, ws.did, sizeof(int32_t) * nq * p->k, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dists_host, ws.dd, sizeof(float) * nq * p->k, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "search_host: D2H");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "search_host: synchronize");
    return DEG_OK;
}

extern "C" deg_status knn_exact(const float* base_dev, int64_t n, const float* queries_dev, int64_t nq,
                                int32_t dim, int32_t k, int32_t* ids_dev, float* dists_dev, void* stream) {
    if (n <= 0 || n > INT32_MAX || nq < 0 || nq > INT32_MAX || dim <= 0) return fail(DEG_EINVAL, "knn_exact: bad sizes");
    if (k < 1 || k > 1024) return fail(DEG_EINVAL, "knn_exact: k must be in [1, 1024]");
    if (k > n) return fail(DEG_EINVAL, "knn_exact: k larger than n");
    if (nq == 0) return DEG_OK;
    if (!base_dev || !queries_dev || !ids_dev || !dists_dev) return fail(DEG_EINVAL, "knn_exact: NULL argument");
    std::string why;
    // k above 256 (ground truth for long lists): the CUDA-core path, whose result the tensor-core
    // path reproduces bit for bit at k <= 256
    const int e = k <= 256 ? launch_knn_exact(base_dev, n, queries_dev, nq, dim, k, ids_dev, dists_dev,
                                              static_cast<deg_stream_t>(stream), &why)
                           : launch_knn_simt(base_dev, n, queries_dev, nq, dim, k, ids_dev, dists_dev,
                                             static_cast<deg_stream_t>(stream), &why);
    if (e != 0) return fail(DEG_ECUDA, "knn_exact: " + why);
    return DEG_OK;
}

extern "C" deg_status knn_exact_noalloc(const float* base_dev, int64_t n, const float* queries_dev, int64_t nq,
                                        int32_t dim, int32_t k, int32_t* ids_dev, float* dists_dev, void* stream) {
    if (n <= 0 || n > INT32_MAX || nq < 0 || nq > INT32_MAX || dim <= 0)
        return fail(DEG_EINVAL, "knn_exact_noalloc: bad sizes");
    if (k < 1 || k > 1024) return fail(DEG_EINVAL, "knn_exact_noalloc: k must be in [1, 1024]");
    if (k > n) return fail(DEG_EINVAL, "knn_exact_noalloc: k larger than n");
    if (n > (8ll << 20)) return fail(DEG_EINVAL, "knn_exact_noalloc: n exceeds the static scratch (at most 8388608 base rows)");
    if (nq == 0) return DEG_OK;
    if (!base_dev || !queries_dev || !ids_dev || !dists_dev) return fail(DEG_EINVAL, "knn_exact_noalloc: NULL argument");
    std::string why;
    const int e = launch_knn_exact_noalloc(base_dev, n, queries_dev, nq, dim, k, ids_dev, dists_dev,
                                           static_cast<deg_stream_t>(stream), &why);
    if (e != 0) return fail(e == cudaErrorInvalidValue ? DEG_EINVAL : DEG_ECUDA, "knn_exact_noalloc: " + why);
    return DEG_OK;
}

extern "C" deg_status deg_nearest_rows(const float* rows_dev, int64_t n, int32_t dim, const float* queries_dev, int64_t nq,
                                       int32_t cap, int32_t* ids_dev, float* dists_dev, void* stream) {
    if (n < 1 || n > 4096 || dim < 1 || nq < 0 || nq > (1ll << 24)) return fail(DEG_EINVAL, "nearest_rows: bad sizes");
    if (cap < 1 || cap > 4096 || (cap & (cap - 1))) return fail(DEG_EINVAL, "nearest_rows: cap must be a power of two in [1, 4096]");
    if (nq == 0) return DEG_OK;
    if (!rows_dev || !queries_dev || !ids_dev || !dists_dev) return fail(DEG_EINVAL, "nearest_rows: NULL argument");
    const deg_stream_t st = static_cast<deg_stream_t>(stream);
    std::string why;
    KnnPlan* plan = nullptr;
    int e = knn_plan_create(&plan, rows_dev, dim, nullptr, n, dim, 1, cap, st, &why);
    if (e == 0) e = knn_plan_run(plan, queries_dev, nq, ids_dev, dists_dev, st, &why);
    if (e == 0) e = (int)cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    knn_plan_destroy(plan);
    if (e != 0) return fail(DEG_ECUDA, "nearest_rows: " + (why.empty() ? std::string(cudaGetErrorString((cudaError_t)e)) : why));
    return DEG_OK;
}

extern "C" deg_status deg_stop_record(deg_index* idx, const deg_search_params* p, const float* queries_dev,
                                      int64_t nq, int32_t cap, float* feats_dev, int32_t* labels_dev,
                                      int32_t* counts_dev, void* stream) {
    deg_status s = validate_search(idx, p, queries_dev, nullptr, 0, nq);
    if (s != DEG_OK) return s;
    if (cap < 1) return fail(DEG_EINVAL, "stop_record: cap must be >= 1");
    if (nq == 0) return DEG_OK;
    if (!feats_dev || !labels_dev || !counts_dev) return fail(DEG_EINVAL, "stop_record: NULL output");
    std::string why;
    if (workspace_reserve(idx->ws, idx->dev, nq, &why) != 0) return fail(DEG_ENOMEM, "stop_record: workspace: " + why);
    // results of the recording run are not needed: reuse the e2e staging buffers
    Workspace& ws = idx->ws;
    if (ws.stage_q < nq || ws.stage_k < p->k) {
        cudaFree(ws.dq); cudaFree(ws.did); cudaFree(ws.dd);
        ws.dq = ws.did = ws.dd = nullptr;
        ws.stage_q = ws.stage_k = 0;
        cudaError_t e;
        const size_t qb = std::max<size_t>(sizeof(float) * (size_t)nq * idx->dim, sizeof(int32_t) * (size_t)nq);
        if ((e = cudaMalloc(&ws.dq, qb)) != cudaSuccess || (e = cudaMalloc(&ws.did, sizeof(int32_t) * nq * p->k)) != cudaSuccess ||
            (e = cudaMalloc(&ws.dd, sizeof(float) * nq * p->k)) != cudaSuccess)
            return fail(DEG_ENOMEM, std::string("stop_record: cudaMalloc: ") + cudaGetErrorString(e));
        ws.stage_q = nq;
        ws.stage_k = p->k;
    }
    SearchArgs a{&idx->dev, queries_dev, nullptr, 0, nq, p->k, p->eps, p->precision, p->rerank, p->max_hops,
                 p->visited_cap, p->queue_cap, p->entry_mode, 0, feats_dev, labels_dev, counts_dev, cap,
                 static_cast<int32_t*>(ws.did), static_cast<float*>(ws.dd), nullptr, nullptr};
    const int e = launch_search(a, idx->ws, static_cast<deg_stream_t>(stream), &why);
    if (e != 0) return fail(DEG_ECUDA, "stop_record: " + why);
    return DEG_OK;
}

extern "C" int64_t deg_mlp_scratch_floats(int64_t count) { return count > 0 ? mlp_scratch_floats(count) : 0; }

extern "C" deg_status deg_mlp_loss_grad(const float* w_dev, const float* x_dev, const int32_t* labels_dev, int64_t count,
                                        float* grad_dev, float* loss_dev, float* scratch_dev, void* stream) {
    if (!w_dev || !x_dev || !labels_dev || !grad_dev || !scratch_dev || count < 1)
        return fail(DEG_EINVAL, "mlp_loss_grad: bad arguments");
    std::string why;
    if (mlp_loss_grad(w_dev, x_dev, labels_dev, count, grad_dev, loss_dev, scratch_dev,
                      static_cast<deg_stream_t>(stream), &why) != 0)
        return fail(DEG_ECUDA, "mlp_loss_grad: " + why);
    return DEG_OK;
}

extern "C" deg_status deg_mlp_adam(float* w_dev, float* m_dev, float* v_dev, const float* grad_dev, int32_t step,
                                   float lr, void* stream) {
    if (!w_dev || !m_dev || !v_dev || !grad_dev || step < 1 || !(lr > 0.f)) return fail(DEG_EINVAL, "mlp_adam: bad arguments");
    std::string why;
    if (mlp_adam(w_dev, m_dev, v_dev, grad_dev, step, lr, static_cast<deg_stream_t>(stream), &why) != 0)
        return fail(DEG_ECUDA, "mlp_adam: " + why);
    return DEG_OK;
}

extern "C" deg_status deg_mlp_predict(const float* w_dev, const float* x_dev, int64_t count, float* p_stop_dev,
                                      void* stream) {
    if (count == 0) return DEG_OK;
    if (!w_dev || !x_dev || !p_stop_dev || count < 0) return fail(DEG_EINVAL, "mlp_predict: bad arguments");
    std::string why;
    if (mlp_predict(w_dev, x_dev, count, p_stop_dev, static_cast<deg_stream_t>(stream), &why) != 0)
        return fail(DEG_ECUDA, "mlp_predict: " + why);
    return DEG_OK;
}

extern "C" deg_status deg_set_stop_model(deg_index* idx, const float* w_dev, float threshold, void* stream) {
    if (!idx || !w_dev) return fail(DEG_EINVAL, "set_stop_model: NULL argument");
    if (!(threshold > 0.f && threshold < 1.f)) return fail(DEG_EINVAL, "set_stop_model: threshold must be in (0, 1)");
    if (!idx->dev.x32) return fail(DEG_ENOTREADY, "set_stop_model: index not uploaded");
    cudaError_t e;
    if (!idx->dev.stop_w && (e = cudaMalloc(&idx->dev.stop_w, 2 * kStopParams)) != cudaSuccess)
        return cuda_fail(e, "set_stop_model");
    std::string why;
    if (mlp_pack_inference(w_dev, idx->dev.stop_w, static_cast<deg_stream_t>(stream), &why) != 0)
        return fail(DEG_ECUDA, "set_stop_model: " + why);
    idx->dev.stop_logit = std::log(threshold / (1.f - threshold));
    if ((e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream))) != cudaSuccess) return cuda_fail(e, "set_stop_model");
    return DEG_OK;
}

// ---- serving ------------------------------------------------------------------------------------

struct deg_server {
    deg_index* idx = nullptr;
    cudaStream_t stream = nullptr;
    int32_t cap = 0, kmax = 0, dim = 0, warps = 0;
    // mapped pinned host memory (host views)
    float* vecs = nullptr;
    int32_t* meta = nullptr;               // [cap][4]
    int32_t* ids = nullptr;
    float* dists = nullptr;
    int32_t* status = nullptr;
    int32_t* trace = nullptr;
    uint32_t* done = nullptr;
    unsigned long long* times = nullptr;   // [cap][2] device start / end of each request (ns)
    unsigned long long* tail = nullptr;
    int32_t* stop = nullptr;
    // device words
    int32_t* kstatus = nullptr;
    unsigned long long* claim = nullptr;
    int64_t posted = 0;
    std::vector<int64_t> held;             // per slot: sequence number occupying it, -1 if free
};

namespace {

void server_free(deg_server* s) {
    cudaFreeHost(s->vecs); cudaFreeHost(s->meta); cudaFreeHost(s->ids); cudaFreeHost(s->dists);
    cudaFreeHost(s->status); cudaFreeHost(s->trace); cudaFreeHost(s->done); cudaFreeHost(s->tail);
    cudaFreeHost(s->stop); cudaFreeHost(s->times);
    cudaFree(s->kstatus); cudaFree(s->claim);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

template <class T>
cudaError_t host_alloc(T** p, size_t count) {
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(p), sizeof(T) * count, cudaHostAllocMapped);
    if (e == cudaSuccess) std::memset(*p, 0, sizeof(T) * count);
    return e;
}

template <class T>
T* dev_view(T* host) {
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, host, 0) != cudaSuccess) return nullptr;   // caller checks
    return static_cast<T*>(d);
}

}  // namespace

extern "C" deg_status deg_serve_start(deg_index* idx, const deg_serve_config* cfg, deg_server** out) {
    if (!out) return fail(DEG_EINVAL, "serve_start: out is NULL");
    *out = nullptr;
    if (!idx || !cfg) return fail(DEG_EINVAL, "serve_start: NULL argument");
    if (!idx->dev.x32) return fail(DEG_ENOTREADY, "serve_start: index not uploaded");
    if (cfg->capacity < 1 || cfg->kmax < 1 || cfg->kmax > 1024 || !(cfg->idle_timeout_s > 0))
        return fail(DEG_EINVAL, "serve_start: need capacity >= 1, 1 <= kmax <= 1024, idle_timeout_s > 0");
    if (cfg->precision < DEG_F32 || cfg->precision > DEG_FP8 || !(idx->uploaded_mask & (1 << cfg->precision)))
        return fail(DEG_ENOTREADY, "serve_start: precision copy not uploaded");
    if (cfg->entry_mode < 0 || cfg->entry_mode > 2) return fail(DEG_EINVAL, "serve_start: entry_mode must be 0, 1 or 2");
    if (cfg->learned_stop && !idx->dev.stop_w) return fail(DEG_ENOTREADY, "serve_start: no stop model");
    if (cfg->rerank < 0 || cfg->rerank > 1024) return fail(DEG_EINVAL, "serve_start: rerank out of range");
    if (cfg->max_blocks < 0) return fail(DEG_EINVAL, "serve_start: max_blocks must be >= 0");
    std::string why;
    if (workspace_reserve(idx->ws, idx->dev, 1, &why) != 0) return fail(DEG_ENOMEM, "serve_start: workspace: " + why);
    deg_server* s = new (std::nothrow) deg_server;
    if (!s) return fail(DEG_ENOMEM, "serve_start: host allocation failed");
    s->idx = idx;
    s->cap = cfg->capacity;
    s->kmax = cfg->kmax;
    s->dim = idx->dim;
    cudaError_t e;
    const size_t cap = (size_t)s->cap;
    if ((e = host_alloc(&s->vecs, cap * s->dim)) != cudaSuccess || (e = host_alloc(&s->meta, cap * 4)) != cudaSuccess ||
        (e = host_alloc(&s->ids, cap * s->kmax)) != cudaSuccess || (e = host_alloc(&s->dists, cap * s->kmax)) != cudaSuccess ||
        (e = host_alloc(&s->status, cap)) != cudaSuccess || (e = host_alloc(&s->trace, cap * 4)) != cudaSuccess ||
        (e = host_alloc(&s->done, cap)) != cudaSuccess || (e = host_alloc(&s->times, 2 * cap)) != cudaSuccess ||
        (e = host_alloc(&s->tail, 1)) != cudaSuccess ||
        (e = host_alloc(&s->stop, 1)) != cudaSuccess || (e = cudaMalloc(&s->kstatus, 4)) != cudaSuccess ||
        (e = cudaMalloc(&s->claim, 8)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        server_free(s);
        return fail(DEG_ENOMEM, std::string("serve_start: ") + cudaGetErrorString(e));
    }
    s->held.assign(cap, -1);
    if ((e = cudaMemsetAsync(s->kstatus, 0, 4, s->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(s->claim, 0, 8, s->stream)) != cudaSuccess) {
        server_free(s);
        return cuda_fail(e, "serve_start");
    }
    ServeArgs a{&idx->dev, dev_view(s->vecs), dev_view(s->meta), dev_view(s->ids), dev_view(s->dists),
                dev_view(s->status), dev_view(s->trace), dev_view(s->done), dev_view(s->times), dev_view(s->tail),
                dev_view(s->stop),
                s->kstatus, s->claim, s->cap, s->kmax, cfg->entry_mode, cfg->precision, cfg->rerank,
                cfg->learned_stop ? 1 : 0, (unsigned long long)(cfg->idle_timeout_s * 1e9), cfg->max_blocks};
    if (!a.vecs || !a.meta || !a.ids || !a.dists || !a.status || !a.trace || !a.done || !a.times || !a.tail || !a.stop) {
        server_free(s);
        return fail(DEG_ECUDA, "serve_start: no device view of the mapped ring");
    }
    if (launch_serving(a, idx->ws, reinterpret_cast<deg_stream_t>(s->stream), &s->warps, &why) != 0) {
        server_free(s);
        return fail(DEG_ECUDA, "serve_start: " + why);
    }
    *out = s;
    return DEG_OK;
}

extern "C" int32_t deg_serve_slots(const deg_server* srv) { return srv ? srv->warps : 0; }

extern "C" deg_status deg_serve_submit(deg_server* s, const float* vec_host, int32_t vertex, int32_t k, float eps,
                                       int64_t* seq_out) {
    if (!s || !seq_out) return fail(DEG_EINVAL, "serve_submit: NULL argument");
    if (k < 1 || k > s->kmax || !(eps >= 0.f) || std::isinf(eps)) return fail(DEG_EINVAL, "serve_submit: bad k or eps");
    if (vertex >= 0 ? (vertex >= s->idx->n || vec_host) : (!vec_host || vertex != -1))
        return fail(DEG_EINVAL, "serve_submit: give a vector (vertex -1) or a vertex id (vector NULL)");
    if (vertex >= 0 && k > s->idx->n - 1) return fail(DEG_EINVAL, "serve_submit: k larger than the candidates");
    const int64_t seq = s->posted;
    const size_t r = (size_t)(seq % s->cap);
    if (s->held[r] >= 0) return fail(DEG_EOVERFLOW, "serve_submit: ring slot busy (collect earlier results)");
    if (vec_host) std::memcpy(s->vecs + r * s->dim, vec_host, sizeof(float) * s->dim);
    int32_t eb;
    std::memcpy(&eb, &eps, 4);
    s->meta[4 * r + 0] = k;
    s->meta[4 * r + 1] = eb;
    s->meta[4 * r + 2] = vertex;
    s->meta[4 * r + 3] = (int32_t)seq;
    s->held[r] = seq;
    ++s->posted;
    std::atomic_thread_fence(std::memory_order_release);
    __atomic_store_n(s->tail, (unsigned long long)s->posted, __ATOMIC_RELEASE);
    *seq_out = seq;
    return DEG_OK;
}

// A finished request's device time (from taking it to publishing it), read after its completion was
// seen and before its ring slot takes another request.
static double device_seconds(const deg_server* s, size_t r) {
    const unsigned long long a = __atomic_load_n(s->times + 2 * r, __ATOMIC_ACQUIRE);
    const unsigned long long b = __atomic_load_n(s->times + 2 * r + 1, __ATOMIC_ACQUIRE);
    return b >= a ? (double)(b - a) * 1e-9 : 0.0;
}

extern "C" int32_t deg_serve_poll(deg_server* s, int64_t seq, int32_t* ids_host, float* dists_host,
                                  int32_t* status_host) {
    if (!s || seq < 0 || seq >= s->posted) return fail(DEG_EINVAL, "serve_poll: unknown request");
    const size_t r = (size_t)(seq % s->cap);
    if (s->held[r] != seq) return fail(DEG_EINVAL, "serve_poll: request already collected");
    if (__atomic_load_n(s->done + r, __ATOMIC_ACQUIRE) != (uint32_t)(seq + 1)) return 0;
    const int32_t k = s->meta[4 * r + 0];
    if (ids_host) std::memcpy(ids_host, s->ids + r * s->kmax, sizeof(int32_t) * k);
    if (dists_host) std::memcpy(dists_host, s->dists + r * s->kmax, sizeof(float) * k);
    if (status_host) *status_host = s->status[r];
    s->held[r] = -1;
    return 1;
}

extern "C" deg_status deg_serve_run_trace(deg_server* s, const float* vecs_host, const int32_t* vertices,
                                          const int32_t* ks, const float* epss, const double* arrival_s, int64_t count,
                                          double* latency_s_out, int32_t* ids_out, float* dists_out,
                                          int32_t* status_out, double* device_s_out, double timeout_s) {
    if (!s || !vecs_host || !vertices || !ks || !epss || !arrival_s || !latency_s_out || count < 0)
        return fail(DEG_EINVAL, "serve_run_trace: NULL argument");
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    std::vector<int64_t> seq_of(count, -1);
    std::vector<int64_t> outstanding;
    outstanding.reserve(1 << 16);
    int64_t next = 0, finished = 0;
    while (finished < count) {
        const double t = now();
        if (t > timeout_s) return fail(DEG_ETIMEOUT, "serve_run_trace: trace did not finish in time");
        // post every request whose arrival time has come (while ring slots are free)
        while (next < count && arrival_s[next] <= t) {
            int64_t seq;
            const bool vq = vertices[next] < 0;
            const deg_status st = deg_serve_submit(s, vq ? vecs_host + next * (int64_t)s->dim : nullptr,
                                                   vq ? -1 : vertices[next], ks[next], epss[next], &seq);
            if (st == DEG_EOVERFLOW) break;
            if (st != DEG_OK) return st;
            seq_of[next] = seq;
            outstanding.push_back(next);
            ++next;
        }
        // collect finished requests
        for (size_t j = 0; j < outstanding.size();) {
            const int64_t i = outstanding[j];
            int32_t stv = 0;
            const int32_t got = deg_serve_poll(s, seq_of[i], ids_out ? ids_out + i * s->kmax : nullptr,
                                               dists_out ? dists_out + i * s->kmax : nullptr, &stv);
            if (got < 0) return (deg_status)got;
            if (got == 1) {
                latency_s_out[i] = now() - arrival_s[i];
                if (status_out) status_out[i] = stv;
                if (device_s_out) device_s_out[i] = device_seconds(s, (size_t)(seq_of[i] % s->cap));
                ++finished;
                outstanding[j] = outstanding.back();
                outstanding.pop_back();
            } else {
                ++j;
            }
        }
    }
    return DEG_OK;
}

extern "C" deg_status deg_serve_stop(deg_server* s) {
    if (!s) return fail(DEG_EINVAL, "serve_stop: NULL server");
    __atomic_store_n(s->stop, 1, __ATOMIC_RELEASE);
    cudaError_t e = cudaStreamSynchronize(s->stream);
    int32_t ks = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&ks, s->kstatus, 4, cudaMemcpyDeviceToHost);
    server_free(s);
    if (e != cudaSuccess) return cuda_fail(e, "serve_stop");
    return ks == DEG_ETIMEOUT ? fail(DEG_ETIMEOUT, "serve_stop: the kernel ended on its idle timeout") : DEG_OK;
}
