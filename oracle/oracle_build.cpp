// CPU oracle (test infrastructure only): DEG construction -- checkMRNG (Alg. 2),
// ExtendGraph (Alg. 3, scheme C with RNG checks), optimizeEdge (Alg. 4, scheme D gain) and
// dynamicEdgeOptimization (Alg. 5) -- plus the structural invariants of Sec. 5.1, AND (Eq. 4)
// and GQ (Eq. 3). FP64 distances and stored FP64 edge weights w(u,v) = delta(u,v).
//
// Readings where the algorithms are silent or garbled:
//  B1 insertion order = vertex id; the start graph is K_{d+1} on ids 0..d; the ExtendGraph
//     search seed is vertex 0 (Sec. 5.2 step 1 allows any vertex).
//  B2 checkMRNG(G, v, b) inside ExtendGraph treats the tentative set U as N(v) with
//     w(v,u) = delta(v,u) (v itself has no edges until the end of Alg. 3).
//  B3 a b already in U, or whose neighbours are all in U, is skipped; n = the neighbour of b
//     with the longest edge, tie -> lower id; if both passes leave |U| < d the search is
//     repeated with k_ext doubled.
//  B5 i_opt bounds the iterations of Alg. 4 (the prose's "after a few iterations").
//  B6 case b requires v1 and v4 NOT adjacent (prose), not adjacent as the listing prints.
//  B7 case a adds (v1, v5) and (v1, v6) (prose: va-ve, va-vf) and requires both outside N(v1).
//  B8 case b's path exists iff v1 is in S1 or v4 is in S4.
//  B10 Alg. 5 draws its random vertex with SplitMix64(seed); N(v1) is snapshotted first and a
//     v2 that is no longer adjacent is skipped.
// Edges are removed before the edge that replaces them is added, so no vertex ever holds more
// than d edges; every modification records its exact slots so a revert is bit-identical.
#include "deg_oracle.h"
#include "oracle_common.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <queue>
#include <stdexcept>
#include <vector>

namespace oracle {
namespace {

struct Mod {
    bool added;
    int32_t u, v;
    int32_t su, sv;
    double w;
};

uint64_t splitmix64(uint64_t& x) {  // Steele, Lea, Flood (2014)
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

class Builder {
  public:
    Builder(const float* base, int64_t n, int dim, int d)
        : base_(base), n_(n), dim_(dim), d_(d), adj_(n * d, -1), w_(n * d, 0.0) {}

    const float* base_;
    int64_t n_;
    int dim_, d_;
    std::vector<int32_t> adj_;
    std::vector<double> w_;

    double delta(int32_t a, int32_t b) const {
        return distance(base_ + (int64_t)a * dim_, base_ + (int64_t)b * dim_, dim_);
    }
    int slot(int32_t u, int32_t v) const {
        for (int j = 0; j < d_; ++j)
            if (adj_[(int64_t)u * d_ + j] == v) return j;
        return -1;
    }
    bool adjacent(int32_t u, int32_t v) const { return slot(u, v) >= 0; }
    double weight(int32_t u, int32_t v) const { return w_[(int64_t)u * d_ + slot(u, v)]; }
    std::vector<int32_t> neighbors(int32_t u) const {
        std::vector<int32_t> out;
        for (int j = 0; j < d_; ++j)
            if (adj_[(int64_t)u * d_ + j] >= 0) out.push_back(adj_[(int64_t)u * d_ + j]);
        return out;
    }
    int free_slot(int32_t u) const { return slot(u, -1); }

    Mod add_edge(int32_t u, int32_t v, double w) {
        const int su = free_slot(u), sv = free_slot(v);
        if (su < 0 || sv < 0 || u == v || adjacent(u, v)) throw std::runtime_error("add_edge");
        adj_[(int64_t)u * d_ + su] = v; w_[(int64_t)u * d_ + su] = w;
        adj_[(int64_t)v * d_ + sv] = u; w_[(int64_t)v * d_ + sv] = w;
        return {true, u, v, su, sv, w};
    }
    Mod remove_edge(int32_t u, int32_t v) {
        const int su = slot(u, v), sv = slot(v, u);
        if (su < 0 || sv < 0) throw std::runtime_error("remove_edge");
        const double w = w_[(int64_t)u * d_ + su];
        adj_[(int64_t)u * d_ + su] = -1; w_[(int64_t)u * d_ + su] = 0.0;
        adj_[(int64_t)v * d_ + sv] = -1; w_[(int64_t)v * d_ + sv] = 0.0;
        return {false, u, v, su, sv, w};
    }
    void undo(const Mod& m) {
        if (m.added) {
            adj_[(int64_t)m.u * d_ + m.su] = -1; w_[(int64_t)m.u * d_ + m.su] = 0.0;
            adj_[(int64_t)m.v * d_ + m.sv] = -1; w_[(int64_t)m.v * d_ + m.sv] = 0.0;
        } else {
            adj_[(int64_t)m.u * d_ + m.su] = m.v; w_[(int64_t)m.u * d_ + m.su] = m.w;
            adj_[(int64_t)m.v * d_ + m.sv] = m.u; w_[(int64_t)m.v * d_ + m.sv] = m.w;
        }
    }

    // Alg. 1 on the current graph, query = the feature vector of vertex x.
    std::vector<Cand> search(std::vector<int32_t> seeds, int32_t x, int k, double eps) const {
        std::sort(seeds.begin(), seeds.end());
        seeds.erase(std::unique(seeds.begin(), seeds.end()), seeds.end());
        Graph g{n_, d_, adj_.data()};
        return range_search(g, [&](int32_t v) { return delta(v, x); }, seeds, k, eps, true, nullptr);
    }

    // Alg. 2 on an existing edge (v1, v2): false if a common neighbour u lies in the lune.
    bool check_mrng(int32_t v1, int32_t v2) const {
        const double w12 = delta(v1, v2);
        for (int32_t u : neighbors(v1)) {
            if (!adjacent(v2, u)) continue;
            if (w12 > std::max(weight(v1, u), weight(v2, u))) return false;
        }
        return true;
    }

    // Alg. 2 for the vertex v under construction (reading B2: N(v) := U).
    bool check_mrng_tentative(int32_t v, int32_t b, const std::vector<int32_t>& U) const {
        const double wvb = delta(v, b);
        for (int32_t u : U) {
            if (!adjacent(b, u)) continue;
            if (wvb > std::max(delta(v, u), weight(b, u))) return false;
        }
        return true;
    }

    // Alg. 4 optimizeEdge(G, v1, v2, i_opt, k_opt, eps_opt). Returns true if the graph changed.
    bool optimize_edge(int32_t v1, int32_t v2, int i_opt, int k_opt, double eps_opt) {
        if (!adjacent(v1, v2)) return false;
        std::vector<Mod> M;
        double gain = weight(v1, v2);
        M.push_back(remove_edge(v1, v2));
        int32_t v3 = v1, v4 = v1;
        for (int it = 0; it < i_opt; ++it) {
            // Find s (result of a search for v2) and n in N(s) maximising
            // gain - delta(s, v2) + w(s, n): replace (s, n) by (v2, s).
            double b = gain;
            int32_t best_s = -1, best_n = -1;
            for (const Cand& c : search({v3, v4}, v2, k_opt, eps_opt)) {
                const int32_t s = c.id;
                if (s == v1 || s == v2 || adjacent(v2, s)) continue;
                for (int32_t nb : neighbors(s)) {
                    if (nb == v2) continue;
                    const double g2 = gain - delta(s, v2) + weight(s, nb);
                    if (b < g2) { b = g2; best_s = s; best_n = nb; }
                }
            }
            if (b == gain) break;                       // no improving swap
            v3 = best_s;
            v4 = best_n;
            gain = b;
            M.push_back(remove_edge(v3, v4));
            M.push_back(add_edge(v2, v3, delta(v2, v3)));

            if (v1 == v4) {
                // Case a: v1 misses two edges; replace an edge (v5, v6) by (v1, v5), (v1, v6).
                double b2 = 0.0;
                int32_t v5 = -1, v6 = -1;
                for (const Cand& c : search({v2, v3}, v1, k_opt, eps_opt)) {
                    const int32_t s = c.id;
                    if (s == v1 || adjacent(v1, s)) continue;
                    for (int32_t nb : neighbors(s)) {
                        if (nb == v1 || adjacent(v1, nb)) continue;
                        const double g2 = gain + weight(s, nb) - delta(s, v1) - delta(nb, v1);
                        if (b2 < g2) { b2 = g2; v5 = s; v6 = nb; }
                    }
                }
                if (b2 > 0.0) {
                    remove_edge(v5, v6);
                    add_edge(v1, v5, delta(v1, v5));
                    add_edge(v1, v6, delta(v1, v6));
                    return true;
                }
            } else if (!adjacent(v1, v4) && 0.0 < gain - delta(v1, v4)) {
                // Case b: connect v1 and v4 if a path links them to {v2, v3}.
                const auto S1 = search({v2, v3}, v1, k_opt, eps_opt);
                const auto S4 = search({v2, v3}, v4, k_opt, eps_opt);
                bool path = false;
                for (const Cand& c : S1) path |= (c.id == v1);
                for (const Cand& c : S4) path |= (c.id == v4);
                if (path) {
                    add_edge(v1, v4, delta(v1, v4));
                    return true;
                }
            }
            const int32_t t = v4;                       // next iteration: v2 is the vertex
            v4 = v3;                                    // that lost an edge, seeds the two
            v3 = v2;                                    // previous vertices
            v2 = t;
        }
        for (auto it = M.rbegin(); it != M.rend(); ++it) undo(*it);
        return false;
    }

    // Alg. 3 ExtendGraph(G, d, v, {0}, k_ext, eps_ext) followed by optimizeEdge for u in U \ S.
    void extend(int32_t v, int k_ext, double eps_ext, int i_opt, int k_opt, double eps_opt) {
        int kk = k_ext;
        std::vector<Cand> S = search({0}, v, kk, eps_ext);
        std::vector<int32_t> U;
        auto inU = [&](int32_t x) { return std::find(U.begin(), U.end(), x) != U.end(); };
        bool skip_rng = false;
        while ((int)U.size() < d_) {
            for (size_t i = 0; i < S.size() && (int)U.size() < d_; ++i) {
                const int32_t b = S[i].id;          // closest remaining b in B = S \ U
                if (inU(b)) continue;
                if (!skip_rng && !check_mrng_tentative(v, b, U)) continue;
                int32_t n = -1;
                double wn = -1.0;
                for (int32_t c : neighbors(b)) {    // N(G, b) \ U, longest edge (scheme C)
                    if (inU(c)) continue;
                    const double w = weight(b, c);
                    if (w > wn || (w == wn && c < n)) { wn = w; n = c; }
                }
                if (n < 0) continue;
                U.push_back(n);
                U.push_back(b);
                remove_edge(n, b);
            }
            if (skip_rng && (int)U.size() < d_) {  // both passes failed: widen the search
                if (kk > 4 * n_) throw std::runtime_error("extend: no candidates left");
                kk *= 2;
                S = search({0}, v, kk, eps_ext);
            }
            skip_rng = true;
        }
        for (int32_t e : U) add_edge(v, e, delta(v, e));
        for (int32_t u : U) {
            bool inS = false;
            for (const Cand& c : S) inS |= (c.id == u);
            if (!inS && adjacent(v, u)) optimize_edge(v, u, i_opt, k_opt, eps_opt);
        }
    }

    // Alg. 5 dynamicEdgeOptimization for one random vertex.
    void dynamic_edge_optimization(uint64_t& rng, int64_t count, int i_opt, int k_opt, double eps_opt) {
        const int32_t v1 = (int32_t)(splitmix64(rng) % (uint64_t)count);
        for (int32_t v2 : neighbors(v1))
            if (adjacent(v1, v2) && !check_mrng(v1, v2)) optimize_edge(v1, v2, i_opt, k_opt, eps_opt);
        int32_t far = -1;
        double wf = -1.0;
        for (int32_t c : neighbors(v1)) {
            const double w = weight(v1, c);
            if (w > wf || (w == wf && c < far)) { wf = w; far = c; }
        }
        if (far >= 0) optimize_edge(v1, far, i_opt, k_opt, eps_opt);
    }

    void init_weights_from_adjacency() {
        for (int64_t u = 0; u < n_; ++u)
            for (int j = 0; j < d_; ++j) {
                const int32_t v = adj_[u * d_ + j];
                w_[u * d_ + j] = v >= 0 ? delta((int32_t)u, v) : 0.0;
            }
    }
};

}  // namespace
}  // namespace oracle

using namespace oracle;

extern "C" int deg_build_oracle(const float* base, int64_t n, int32_t dim, int32_t degree,
                                int32_t k_ext, double eps_ext, int32_t k_opt, double eps_opt,
                                int32_t i_opt, int32_t refine_rounds, uint64_t seed,
                                int32_t* adj_out, double* weights_out) {
    // Even regularity, d >= 4 (Sec. 5.1); the smallest DEG_d is K_{d+1}.
    if (!base || !adj_out || dim <= 0 || degree < 4 || degree % 2 || n < degree + 1) return -1;
    if (k_ext < degree || k_opt < 1 || i_opt < 0 || eps_ext < 0 || eps_opt < 0) return -1;
    try {
        Builder B(base, n, dim, degree);
        for (int32_t u = 0; u <= degree; ++u)
            for (int32_t v = u + 1; v <= degree; ++v) B.add_edge(u, v, B.delta(u, v));
        for (int64_t v = degree + 1; v < n; ++v)
            B.extend((int32_t)v, k_ext, eps_ext, i_opt, k_opt, eps_opt);
        uint64_t rng = seed;
        for (int32_t r = 0; r < refine_rounds; ++r) B.dynamic_edge_optimization(rng, n, i_opt, k_opt, eps_opt);
        std::copy(B.adj_.begin(), B.adj_.end(), adj_out);
        if (weights_out) std::copy(B.w_.begin(), B.w_.end(), weights_out);
    } catch (const std::exception&) {
        return -2;
    }
    return 0;
}

extern "C" int32_t oracle_check_mrng(const float* base, int64_t n, int32_t dim, const int32_t* adj,
                                     int32_t degree, int32_t v1, int32_t v2) {
    Builder B(base, n, dim, degree);
    std::copy(adj, adj + n * degree, B.adj_.begin());
    B.init_weights_from_adjacency();
    return B.check_mrng(v1, v2) ? 1 : 0;
}

extern "C" int32_t oracle_optimize_edge(const float* base, int64_t n, int32_t dim, int32_t* adj,
                                        int32_t degree, int32_t v1, int32_t v2, int32_t i_opt,
                                        int32_t k_opt, double eps_opt) {
    try {
        Builder B(base, n, dim, degree);
        std::copy(adj, adj + n * degree, B.adj_.begin());
        B.init_weights_from_adjacency();
        if (!B.adjacent(v1, v2)) return -1;
        const bool changed = B.optimize_edge(v1, v2, i_opt, k_opt, eps_opt);
        std::copy(B.adj_.begin(), B.adj_.end(), adj);
        return changed ? 1 : 0;
    } catch (const std::exception&) {
        return -2;
    }
}

extern "C" int32_t oracle_check_graph(const int32_t* adj, int64_t n, int32_t degree, int64_t bridge_max_n) {
    int32_t bad = 0;
    if (degree < 4 || degree % 2) bad |= 32;
    for (int64_t u = 0; u < n; ++u)
        for (int32_t j = 0; j < degree; ++j) {
            const int32_t v = adj[u * degree + j];
            if (v < 0 || v >= n) { bad |= 1; continue; }
            if (v == u) bad |= 2;
            for (int32_t i = 0; i < j; ++i)
                if (adj[u * degree + i] == v) bad |= 4;
            bool back = false;
            for (int32_t i = 0; i < degree; ++i) back |= (adj[(int64_t)v * degree + i] == u);
            if (!back) bad |= 8;
        }
    if (bad & 1) return bad;
    // Connectivity by BFS from vertex 0, optionally with one edge (ru, rv) ignored.
    auto connected = [&](int64_t ru, int64_t rv) {
        std::vector<char> seen(n, 0);
        std::queue<int64_t> q;
        q.push(0);
        seen[0] = 1;
        int64_t cnt = 1;
        while (!q.empty()) {
            const int64_t u = q.front();
            q.pop();
            for (int32_t j = 0; j < degree; ++j) {
                const int64_t v = adj[u * degree + j];
                if ((u == ru && v == rv) || (u == rv && v == ru)) continue;
                if (!seen[v]) { seen[v] = 1; ++cnt; q.push(v); }
            }
        }
        return cnt == n;
    };
    if (!connected(-1, -1)) bad |= 16;
    if (n <= bridge_max_n && !(bad & (4 | 8 | 16))) {
        for (int64_t u = 0; u < n && !(bad & 64); ++u)
            for (int32_t j = 0; j < degree; ++j) {
                const int64_t v = adj[u * degree + j];
                if (v > u && !connected(u, v)) { bad |= 64; break; }
            }
    }
    return bad;
}

extern "C" double oracle_average_neighbor_distance(const float* base, int64_t n, int32_t dim,
                                                   const int32_t* adj, int32_t degree) {
    // Eq. 4 with U = V.
    double total = 0.0;
    for (int64_t u = 0; u < n; ++u) {
        double s = 0.0;
        for (int32_t j = 0; j < degree; ++j)
            s += distance(base + u * dim, base + (int64_t)adj[u * degree + j] * dim, dim);
        total += s / degree;
    }
    return total / (double)n;
}

extern "C" double oracle_graph_quality(const int32_t* adj, const int32_t* knn, int64_t n, int32_t degree) {
    // Eq. 3: mean over v of |N(G,v) intersect KNN(V,v)| / |N(G,v)|.
    double total = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        int hit = 0;
        for (int32_t j = 0; j < degree; ++j)
            for (int32_t i = 0; i < degree; ++i) hit += (adj[v * degree + j] == knn[v * degree + i]);
        total += (double)hit / degree;
    }
    return total / (double)n;
}
