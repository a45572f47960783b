// Native DEG construction for the library (host C++, FP32): the graph the GPU search runs on.
//
// Implements Sec. 5.2-5.3 of the paper: vertices are inserted in id order into the complete
// graph K_{d+1} on ids 0..d; each insertion runs ExtendGraph (Alg. 3: a range search for the
// new vertex, then scheme C -- replace the longest edge (b, n) of the best result b by (v, b),
// (v, n) -- with the checkMRNG test of Alg. 2 in a first pass and without it in a second), then
// optimizeEdge (Alg. 4, scheme-D gain) on each new edge to a vertex the search did not return.
// Optional rounds of dynamicEdgeOptimization (Alg. 5) follow.
//
// Same readings of the paper as the rest of the library: the checkMRNG of a vertex being
// inserted treats its tentative neighbour set U as N(v); skip b already in U; case b of Alg. 4
// requires v1 and v4 not adjacent; case a adds (v1, v5), (v1, v6); the case-b path exists iff v1
// is in S1 or v4 is in S4; i_opt bounds iterations; ties go to the lower id.
//
// Engineering: flat [n][d] adjacency + float weights, epoch-stamped visited marks (no clearing),
// binary heaps for the candidate and result sets, squared FP32 distances in the search.
#include "deg_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <unordered_set>
#include <stdexcept>
#include <vector>

namespace deg {
namespace {

struct Item {
    float d;
    int32_t id;
};
struct MinFirst {  // priority_queue comparator: smallest (d, id) on top
    bool operator()(const Item& a, const Item& b) const { return a.d > b.d || (a.d == b.d && a.id > b.id); }
};
struct MaxFirst {  // largest (d, id) on top
    bool operator()(const Item& a, const Item& b) const { return a.d < b.d || (a.d == b.d && a.id < b.id); }
};

struct Change {
    int32_t u, v, su, sv;
    float w;
    bool added;
};

class GraphBuilder {
  public:
    GraphBuilder(const float* x, int64_t n, int dim, int d)
        : x_(x), n_(n), dim_(dim), d_(d), nb_((size_t)n * d, -1), w_((size_t)n * d, 0.f), mark_(n, 0) {}

    const float* x_;
    int64_t n_;
    int dim_, d_;
    std::vector<int32_t> nb_;
    std::vector<float> w_;
    std::vector<uint32_t> mark_;
    uint32_t epoch_ = 0;

    float sq(int32_t a, int32_t b) const {
        // Eight independent partial sums so the compiler can vectorise without reassociating.
        const float* p = x_ + (size_t)a * dim_;
        const float* q = x_ + (size_t)b * dim_;
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int i = 0;
        for (; i + 8 <= dim_; i += 8)
            for (int j = 0; j < 8; ++j) {
                const float t = p[i + j] - q[i + j];
                acc[j] += t * t;
            }
        float s = 0.f;
        for (; i < dim_; ++i) {
            const float t = p[i] - q[i];
            s += t * t;
        }
        return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7])) + s;
    }
    float dist(int32_t a, int32_t b) const { return std::sqrt(sq(a, b)); }

    int32_t* row(int32_t u) { return nb_.data() + (size_t)u * d_; }
    const int32_t* row(int32_t u) const { return nb_.data() + (size_t)u * d_; }
    int find(int32_t u, int32_t v) const {
        const int32_t* r = row(u);
        for (int j = 0; j < d_; ++j)
            if (r[j] == v) return j;
        return -1;
    }
    bool linked(int32_t u, int32_t v) const { return find(u, v) >= 0; }
    float wgt(int32_t u, int32_t v) const { return w_[(size_t)u * d_ + find(u, v)]; }

    Change link(int32_t u, int32_t v, float w) {
        const int su = find(u, -1), sv = find(v, -1);
        if (su < 0 || sv < 0 || u == v || linked(u, v)) throw std::runtime_error("builder: link");
        row(u)[su] = v; w_[(size_t)u * d_ + su] = w;
        row(v)[sv] = u; w_[(size_t)v * d_ + sv] = w;
        return {u, v, su, sv, w, true};
    }
    Change unlink(int32_t u, int32_t v) {
        const int su = find(u, v), sv = find(v, u);
        if (su < 0 || sv < 0) throw std::runtime_error("builder: unlink");
        const float w = w_[(size_t)u * d_ + su];
        row(u)[su] = -1;
        row(v)[sv] = -1;
        return {u, v, su, sv, w, false};
    }
    void rollback(const Change& c) {
        if (c.added) {
            row(c.u)[c.su] = -1;
            row(c.v)[c.sv] = -1;
        } else {
            row(c.u)[c.su] = c.v; w_[(size_t)c.u * d_ + c.su] = c.w;
            row(c.v)[c.sv] = c.u; w_[(size_t)c.v * d_ + c.sv] = c.w;
        }
    }

    // Range search (Alg. 1) for the vector of vertex `qv`, over squared distances; returns the
    // result list sorted ascending by (distance, id) with true (not squared) distances.
    std::vector<Item> search(const int32_t* seeds, int nseeds, int32_t qv, int k, float eps) {
        if (++epoch_ == 0) { std::fill(mark_.begin(), mark_.end(), 0u); epoch_ = 1; }
        const float f = (1.f + eps) * (1.f + eps);
        std::priority_queue<Item, std::vector<Item>, MinFirst> S;
        std::priority_queue<Item, std::vector<Item>, MaxFirst> R;
        float r2 = INFINITY;
        for (int i = 0; i < nseeds; ++i) {
            const int32_t s = seeds[i];
            if (mark_[s] == epoch_) continue;
            mark_[s] = epoch_;
            const Item it{sq(s, qv), s};
            S.push(it);
            R.push(it);
        }
        while ((int)R.size() > k) { R.pop(); r2 = R.top().d; }
        while (!S.empty()) {
            const Item s = S.top();
            S.pop();
            if (s.d > r2 * f) break;
            const int32_t* r = row(s.id);
            for (int j = 0; j < d_; ++j) {
                const int32_t c = r[j];
                if (c < 0 || mark_[c] == epoch_) continue;
                mark_[c] = epoch_;
                const float dc = sq(c, qv);
                if (dc <= r2 * f) {
                    S.push({dc, c});
                    if (dc <= r2) {
                        R.push({dc, c});
                        if ((int)R.size() > k) { R.pop(); r2 = R.top().d; }
                    }
                }
            }
        }
        std::vector<Item> out(R.size());
        for (size_t i = out.size(); i-- > 0;) { out[i] = R.top(); out[i].d = std::sqrt(out[i].d); R.pop(); }
        return out;
    }

    bool mrng_ok_existing(int32_t v1, int32_t v2) const {
        const float w12 = wgt(v1, v2);
        const int32_t* r = row(v1);
        for (int j = 0; j < d_; ++j) {
            const int32_t u = r[j];
            if (u < 0 || !linked(v2, u)) continue;
            if (w12 > std::max(w_[(size_t)v1 * d_ + j], wgt(v2, u))) return false;
        }
        return true;
    }

    bool optimize(int32_t v1, int32_t v2, int i_opt, int k_opt, float eps_opt) {
        if (!linked(v1, v2)) return false;
        std::vector<Change> hist;
        float gain = wgt(v1, v2);
        hist.push_back(unlink(v1, v2));
        int32_t v3 = v1, v4 = v1;
        for (int it = 0; it < i_opt; ++it) {
            float best = gain;
            int32_t bs = -1, bn = -1;
            const int32_t seeds[2] = {v3, v4};
            for (const Item& c : search(seeds, v3 == v4 ? 1 : 2, v2, k_opt, eps_opt)) {
                const int32_t s = c.id;
                if (s == v1 || s == v2 || linked(v2, s)) continue;
                const int32_t* r = row(s);
                for (int j = 0; j < d_; ++j) {
                    const int32_t m = r[j];
                    if (m < 0 || m == v2) continue;
                    const float g = gain - c.d + w_[(size_t)s * d_ + j];
                    if (best < g) { best = g; bs = s; bn = m; }
                }
            }
            if (bs < 0) break;
            v3 = bs;
            v4 = bn;
            gain = best;
            hist.push_back(unlink(v3, v4));
            hist.push_back(link(v2, v3, dist(v2, v3)));
            if (v1 == v4) {
                float b2 = 0.f;
                int32_t v5 = -1, v6 = -1;
                const int32_t sd[2] = {v2, v3};
                for (const Item& c : search(sd, 2, v1, k_opt, eps_opt)) {
                    const int32_t s = c.id;
                    if (s == v1 || linked(v1, s)) continue;
                    const int32_t* r = row(s);
                    for (int j = 0; j < d_; ++j) {
                        const int32_t m = r[j];
                        if (m < 0 || m == v1 || linked(v1, m)) continue;
                        const float g = gain + w_[(size_t)s * d_ + j] - c.d - dist(m, v1);
                        if (b2 < g) { b2 = g; v5 = s; v6 = m; }
                    }
                }
                if (b2 > 0.f) {
                    unlink(v5, v6);
                    link(v1, v5, dist(v1, v5));
                    link(v1, v6, dist(v1, v6));
                    return true;
                }
            } else if (!linked(v1, v4) && 0.f < gain - dist(v1, v4)) {
                const int32_t sd[2] = {v2, v3};
                bool path = false;
                for (const Item& c : search(sd, 2, v1, k_opt, eps_opt)) path |= (c.id == v1);
                if (!path)
                    for (const Item& c : search(sd, 2, v4, k_opt, eps_opt)) path |= (c.id == v4);
                if (path) {
                    link(v1, v4, dist(v1, v4));
                    return true;
                }
            }
            const int32_t t = v4;
            v4 = v3;
            v3 = v2;
            v2 = t;
        }
        for (size_t i = hist.size(); i-- > 0;) rollback(hist[i]);
        return false;
    }

    void insert(int32_t v, int k_ext, float eps_ext, int i_opt, int k_opt, float eps_opt) {
        int kk = k_ext;
        const int32_t seed0 = 0;
        std::vector<Item> S = search(&seed0, 1, v, kk, eps_ext);
        std::vector<int32_t> U;
        U.reserve(d_);
        auto inU = [&](int32_t c) { return std::find(U.begin(), U.end(), c) != U.end(); };
        for (int pass = 0; (int)U.size() < d_; ++pass) {
            const bool rng_check = pass == 0;
            for (size_t i = 0; i < S.size() && (int)U.size() < d_; ++i) {
                const int32_t b = S[i].id;
                if (inU(b)) continue;
                if (rng_check) {   // checkMRNG(G, v, b) with N(v) := U
                    bool ok = true;
                    for (int32_t u : U) {
                        if (!linked(b, u)) continue;
                        if (S[i].d > std::max(dist(v, u), wgt(b, u))) { ok = false; break; }
                    }
                    if (!ok) continue;
                }
                int32_t n = -1;
                float wn = -1.f;
                const int32_t* r = row(b);
                for (int j = 0; j < d_; ++j) {
                    const int32_t c = r[j];
                    if (c < 0 || inU(c)) continue;
                    const float w = w_[(size_t)b * d_ + j];
                    if (w > wn || (w == wn && c < n)) { wn = w; n = c; }
                }
                if (n < 0) continue;
                U.push_back(n);
                U.push_back(b);
                unlink(n, b);
            }
            if (pass >= 1 && (int)U.size() < d_) {
                if (kk > 4 * n_) throw std::runtime_error("builder: no candidates left");
                kk *= 2;
                S = search(&seed0, 1, v, kk, eps_ext);
            }
        }
        for (int32_t e : U) link(v, e, dist(v, e));
        for (int32_t u : U) {
            bool inS = false;
            for (const Item& c : S) inS |= (c.id == u);
            if (!inS && linked(v, u)) optimize(v, u, i_opt, k_opt, eps_opt);
        }
    }
};

uint64_t mix64(uint64_t& s) {  // SplitMix64 (Steele, Lea, Flood 2014)
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

int build_graph(const float* x, int64_t n, int32_t dim, const deg_build_params& p,
                int32_t* adj_out, volatile int64_t* progress) {
    GraphBuilder g(x, n, dim, p.degree);
    for (int32_t u = 0; u <= p.degree; ++u)
        for (int32_t v = u + 1; v <= p.degree; ++v) g.link(u, v, g.dist(u, v));
    for (int64_t v = p.degree + 1; v < n; ++v) {
        g.insert((int32_t)v, p.k_ext, p.eps_ext, p.i_opt, p.k_opt, p.eps_opt);
        if (progress && (v & 1023) == 0) *progress = v;
    }
    uint64_t s = p.seed;
    for (int32_t r = 0; r < p.refine_rounds; ++r) {
        const int32_t v1 = (int32_t)(mix64(s) % (uint64_t)n);
        int32_t snap[256];
        const int dd = std::min(p.degree, 256);
        std::memcpy(snap, g.row(v1), sizeof(int32_t) * dd);
        for (int j = 0; j < dd; ++j)
            if (snap[j] >= 0 && g.linked(v1, snap[j]) && !g.mrng_ok_existing(v1, snap[j]))
                g.optimize(v1, snap[j], p.i_opt, p.k_opt, p.eps_opt);
        int32_t far = -1;
        float wf = -1.f;
        for (int j = 0; j < p.degree; ++j) {
            const int32_t c = g.row(v1)[j];
            if (c < 0) continue;
            const float w = g.w_[(size_t)v1 * p.degree + j];
            if (w > wf || (w == wf && c < far)) { wf = w; far = c; }
        }
        if (far >= 0) g.optimize(v1, far, p.i_opt, p.k_opt, p.eps_opt);
    }
    if (progress) *progress = n;
    std::memcpy(adj_out, g.nb_.data(), sizeof(int32_t) * (size_t)n * p.degree);
    return 0;
}

}  // namespace deg

// ---- removing a vertex (not in the paper) -----------------------------------------------------
// The paper builds and refines the graph but leaves removal open. A removal that keeps every
// invariant: drop v's d edges; its former neighbours, each one edge short, are paired by new
// edges (closest non-adjacent pairs first); a pair left adjacent is joined through a nearby edge
// (x, y), replaced by (a, x) and (b, y). If all former neighbours reach each other afterwards, the
// graph is connected (every vertex reached v through one of them); otherwise every change is
// undone and the removal refused. Finally the last vertex takes v's id, so ids stay 0 .. n-2.
// Work per removal: O(d^3) distances for the reconnection and a search that ends once the former
// neighbours have met (a few hops in a DEG), so removals cost the same on any graph size.
namespace deg {
namespace {

float dist_rows(const float* x, int dim, int32_t a, int32_t b) {
    double s = 0.0;
    for (int i = 0; i < dim; ++i) {
        const double t = (double)x[(size_t)a * dim + i] - (double)x[(size_t)b * dim + i];
        s += t * t;
    }
    return (float)std::sqrt(s);
}

}  // namespace

int remove_vertex(std::vector<float>& x, std::vector<int32_t>& adj, int64_t& n, int32_t dim, int32_t d, int32_t v,
                  int32_t* moved_from, std::vector<int32_t>* touched, std::string* why) {
    if (v < 0 || v >= n) return *why = "vertex out of range", 1;
    if (n <= d + 1) return *why = "the graph would have fewer than degree + 1 vertices", 1;
    auto row = [&](int32_t u) { return adj.data() + (size_t)u * d; };
    auto slot = [&](int32_t a, int32_t b) {
        const int32_t* r = row(a);
        for (int j = 0; j < d; ++j)
            if (r[j] == b) return j;
        return -1;
    };
    auto linked = [&](int32_t a, int32_t b) { return slot(a, b) >= 0; };
    std::vector<std::pair<size_t, int32_t>> undo;                 // (adjacency slot, old value)
    auto set = [&](int32_t a, int j, int32_t value) {
        undo.emplace_back((size_t)a * d + j, row(a)[j]);
        row(a)[j] = value;
    };
    auto rollback = [&] {
        for (size_t i = undo.size(); i-- > 0;) adj[undo[i].first] = undo[i].second;
    };
    auto link = [&](int32_t a, int32_t b) {
        set(a, slot(a, -1), b);
        set(b, slot(b, -1), a);
    };
    auto unlink = [&](int32_t a, int32_t b) {
        set(a, slot(a, b), -1);
        set(b, slot(b, a), -1);
    };
    const std::vector<int32_t> nb(row(v), row(v) + d);
    for (int32_t u : nb) unlink(v, u);                            // each neighbour: one free slot
    // closest non-adjacent pairs first (ties by the pair's slots in v's row)
    struct Pair {
        float w;
        int i, j;
    };
    std::vector<Pair> pairs;
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j)
            if (!linked(nb[i], nb[j])) pairs.push_back({dist_rows(x.data(), dim, nb[i], nb[j]), i, j});
    std::sort(pairs.begin(), pairs.end(), [&](const Pair& p, const Pair& q) {
        if (p.w != q.w) return p.w < q.w;
        if (nb[p.i] != nb[q.i]) return nb[p.i] < nb[q.i];
        return nb[p.j] < nb[q.j];
    });
    std::vector<char> done(d, 0);
    for (const Pair& p : pairs) {
        if (done[p.i] || done[p.j]) continue;
        link(nb[p.i], nb[p.j]);
        done[p.i] = done[p.j] = 1;
    }
    // the rest, two at a time (each pair adjacent): replace a nearby edge (x, y) by (a, x), (b, y),
    // x a neighbour of a neighbour of a, minimising |a-x| + |b-y| - |x-y|
    std::vector<int32_t> left;
    for (int i = 0; i < d; ++i)
        if (!done[i]) left.push_back(nb[i]);
    for (size_t i = 0; i + 1 < left.size(); i += 2) {
        const int32_t a = left[i], b = left[i + 1];
        float best = INFINITY;
        int32_t bx = -1, by = -1;
        for (int j = 0; j < d; ++j) {
            const int32_t m = row(a)[j];
            if (m < 0) continue;
            for (int jj = 0; jj < d; ++jj) {
                const int32_t xx = row(m)[jj];
                if (xx < 0 || xx == a || xx == b || linked(a, xx)) continue;
                const float ax = dist_rows(x.data(), dim, a, xx);
                for (int k = 0; k < d; ++k) {
                    const int32_t yy = row(xx)[k];
                    if (yy < 0 || yy == a || yy == b || linked(b, yy)) continue;
                    const float c = ax + dist_rows(x.data(), dim, b, yy) - dist_rows(x.data(), dim, xx, yy);
                    if (c < best) {
                        best = c;
                        bx = xx;
                        by = yy;
                    }
                }
            }
        }
        if (bx < 0) {
            rollback();
            return *why = "no edge to reconnect the removed vertex's neighbours", 1;
        }
        unlink(bx, by);
        link(a, bx);
        link(b, by);
    }
    // connected iff the former neighbours reach each other; the search stops once all have met
    {
        std::vector<int32_t> queue{nb[0]};
        std::unordered_set<int32_t> seen{nb[0]};
        const std::unordered_set<int32_t> want(nb.begin(), nb.end());
        int found = 1;
        for (size_t h = 0; h < queue.size() && found < d; ++h) {
            const int32_t* r = row(queue[h]);
            for (int j = 0; j < d; ++j) {
                const int32_t w = r[j];
                if (w < 0 || !seen.insert(w).second) continue;
                found += (int)want.count(w);
                queue.push_back(w);
            }
        }
        if (found < d) {
            rollback();
            return *why = "removing this vertex would disconnect the graph", 1;
        }
    }
    // the last vertex takes v's id
    const int32_t last = (int32_t)(n - 1);
    if (moved_from) *moved_from = v == last ? -1 : last;
    if (v != last) {
        for (int j = 0; j < d; ++j) {
            const int32_t u = row(last)[j];
            row(u)[slot(u, last)] = v;
            row(v)[j] = u;
        }
        std::copy(x.begin() + (size_t)last * dim, x.begin() + (size_t)(last + 1) * dim, x.begin() + (size_t)v * dim);
    }
    if (touched) {
        touched->clear();
        for (const auto& e : undo) {
            const int32_t u = (int32_t)(e.first / d);
            touched->push_back(u == last ? v : u);
        }
        if (v != last)
            for (int j = 0; j < d; ++j) touched->push_back(row(v)[j]);
        std::sort(touched->begin(), touched->end());
        touched->erase(std::unique(touched->begin(), touched->end()), touched->end());
        if (v == last) touched->erase(std::remove(touched->begin(), touched->end(), v), touched->end());
    }
    --n;
    adj.resize((size_t)n * d);
    x.resize((size_t)n * dim);
    return 0;
}

}  // namespace deg
