// CPU oracle (test infrastructure only): exact kNN (Eq. 1), RangeSearch (Alg. 1) and the fixed
// entry vertex (Sec. 5.4), all in FP64. Deliberately plain: std::set for the candidate and
// result sets, std::unordered_set for the checked set, no blocking, no fusion.
#include "deg_oracle.h"
#include "oracle_common.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <set>
#include <thread>
#include <unordered_set>
#include <vector>

namespace oracle {

double distance(const float* a, const float* b, int dim) {
    // delta(x, q): Euclidean distance (Sec. 2.1; the datasets are L2), accumulated in double.
    double s = 0.0;
    for (int i = 0; i < dim; ++i) {
        const double t = (double)a[i] - (double)b[i];
        s += t * t;
    }
    return std::sqrt(s);
}

void parallel_for(int64_t count, int nthreads, const std::function<void(int64_t)>& body) {
    if (nthreads <= 1 || count < 2) {
        for (int64_t i = 0; i < count; ++i) body(i);
        return;
    }
    std::vector<std::thread> pool;
    const int64_t per = (count + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        const int64_t lo = t * per, hi = std::min<int64_t>(count, lo + per);
        if (lo >= hi) break;
        pool.emplace_back([lo, hi, &body] { for (int64_t i = lo; i < hi; ++i) body(i); });
    }
    for (auto& th : pool) th.join();
}

// Alg. 1 RangeSearch(G, S, q, k, eps), with the readings:
//  * C starts as the seed set (seeds count as checked);
//  * plain search: R starts as the seeds; exploration: seeds are searched from but never
//    returned (the paper avoids showing a user the item they came from, Sec. 6.7);
//  * r stays +inf until R first exceeds k and is trimmed; r is only updated on a trim;
//  * argmin over S and argmax over R order by the key (distance, id), lower id first.
std::vector<Cand> range_search(const Graph& g,
                               const std::function<double(int32_t)>& dist_to_q,
                               const std::vector<int32_t>& seeds, int k, double eps,
                               bool seeds_in_result, SearchTrace* trace) {
    std::unordered_set<int32_t> C;                // checked vertices
    std::set<Cand> S;                             // candidate set, ordered by (d, id)
    std::set<Cand> R;                             // result list, ordered by (d, id)
    double r = std::numeric_limits<double>::infinity();
    int64_t hops = 0, evals = 0, max_s = 0;

    for (int32_t s : seeds) {
        if (!C.insert(s).second) continue;
        const double ds = dist_to_q(s);
        ++evals;
        S.insert({ds, s});
        if (seeds_in_result) R.insert({ds, s});
    }
    while ((int64_t)R.size() > k) {               // more seeds than k: trim at once
        R.erase(std::prev(R.end()));
        r = std::prev(R.end())->d;
    }
    max_s = (int64_t)S.size();

    while (!S.empty()) {
        const Cand s = *S.begin();                // s = argmin_{x in S} delta(x, q)
        S.erase(S.begin());
        if (s.d > r * (1.0 + eps)) break;         // too far away: return R
        ++hops;
        std::vector<int32_t> N;                   // N(G, s) \ C
        for (int32_t j = 0; j < g.degree; ++j) {
            const int32_t nb = g.adj[(int64_t)s.id * g.degree + j];
            if (nb >= 0 && !C.count(nb)) N.push_back(nb);
        }
        for (int32_t nb : N) {
            const double dn = dist_to_q(nb);
            ++evals;
            if (dn <= r * (1.0 + eps)) {          // close enough to expand later
                S.insert({dn, nb});
                if (dn <= r) {                    // close enough for the result list
                    R.insert({dn, nb});
                    if ((int64_t)R.size() > k) {  // keep the k best
                        R.erase(std::prev(R.end()));
                        r = std::prev(R.end())->d;
                    }
                }
            }
        }
        for (int32_t nb : N) C.insert(nb);        // C <- C u N
        max_s = std::max<int64_t>(max_s, (int64_t)S.size());
    }
    if (trace) {
        trace->hops = hops;
        trace->evals = evals;
        trace->max_s = max_s;
        trace->checked = (int64_t)C.size();
    }
    return std::vector<Cand>(R.begin(), R.end());
}

}  // namespace oracle

using namespace oracle;

extern "C" int oracle_knn_bruteforce(const float* base, int64_t n, int32_t dim,
                                     const float* queries, int64_t nq, int32_t k,
                                     const int32_t* exclude, int32_t* ids, double* dists,
                                     int32_t nthreads) {
    if (!base || !queries || !ids || !dists || n <= 0 || dim <= 0 || k <= 0) return -1;
    parallel_for(nq, nthreads, [&](int64_t q) {
        // Eq. 1: the k points with the smallest delta to q (ties by lower id).
        std::vector<Cand> all;
        all.reserve(n);
        const int32_t ex = exclude ? exclude[q] : -1;
        for (int64_t i = 0; i < n; ++i) {
            if (i == ex) continue;
            all.push_back({distance(base + i * dim, queries + q * dim, dim), (int32_t)i});
        }
        const int64_t kk = std::min<int64_t>(k, (int64_t)all.size());
        std::partial_sort(all.begin(), all.begin() + kk, all.end());
        for (int64_t j = 0; j < k; ++j) {
            ids[q * k + j] = j < kk ? all[j].id : -1;
            dists[q * k + j] = j < kk ? all[j].d : std::numeric_limits<double>::infinity();
        }
    });
    return 0;
}

extern "C" int oracle_range_search(const float* base, int64_t n, int32_t dim,
                                   const int32_t* adj, int32_t degree,
                                   const float* queries, const int32_t* seeds, int64_t nq,
                                   int32_t explore, int32_t k, double eps,
                                   int32_t* ids, double* dists, int64_t* trace,
                                   int32_t nthreads) {
    if (!base || !adj || !seeds || !ids || !dists || n <= 0 || dim <= 0 || degree <= 0 || k <= 0)
        return -1;
    if (!(eps >= 0.0)) return -1;
    if (!explore && !queries) return -1;
    for (int64_t q = 0; q < nq; ++q)
        if (seeds[q] < 0 || seeds[q] >= n) return -1;
    Graph g{n, degree, adj};
    parallel_for(nq, nthreads, [&](int64_t q) {
        const float* qv = explore ? base + (int64_t)seeds[q] * dim : queries + q * dim;
        auto dq = [&](int32_t v) { return distance(base + (int64_t)v * dim, qv, dim); };
        SearchTrace tr{};
        std::vector<Cand> R = range_search(g, dq, {seeds[q]}, k, eps, !explore, &tr);
        for (int32_t j = 0; j < k; ++j) {
            ids[q * k + j] = j < (int32_t)R.size() ? R[j].id : -1;
            dists[q * k + j] = j < (int32_t)R.size() ? R[j].d : std::numeric_limits<double>::infinity();
        }
        if (trace) {
            trace[q * 4 + 0] = tr.hops;
            trace[q * 4 + 1] = tr.evals;
            trace[q * 4 + 2] = tr.max_s;
            trace[q * 4 + 3] = tr.checked;
        }
    });
    return 0;
}

extern "C" int32_t oracle_median_vertex(const float* base, int64_t n, int32_t dim) {
    // Sec. 5.4 seeds the search at the graph's median vertex without defining that vertex.
    // Reading: per coordinate take the lower median (the element of rank floor((n-1)/2) in
    // ascending order), then return the base row nearest to that vector (tie -> lower id).
    if (!base || n <= 0 || dim <= 0) return -1;
    std::vector<double> med(dim);
    std::vector<float> col(n);
    for (int32_t j = 0; j < dim; ++j) {
        for (int64_t i = 0; i < n; ++i) col[i] = base[i * dim + j];
        std::sort(col.begin(), col.end());
        med[j] = col[(n - 1) / 2];
    }
    int32_t best = 0;
    double best_d = std::numeric_limits<double>::infinity();
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t j = 0; j < dim; ++j) {
            const double t = (double)base[i * dim + j] - med[j];
            s += t * t;
        }
        const double d = std::sqrt(s);
        if (d < best_d) { best_d = d; best = (int32_t)i; }
    }
    return best;
}
