// Internal declarations shared by the oracle's own translation units (test infrastructure).
#ifndef DEG_ORACLE_COMMON_H
#define DEG_ORACLE_COMMON_H
#include <cstdint>
#include <functional>
#include <vector>

namespace oracle {

struct Cand {
    double d;
    int32_t id;
    bool operator<(const Cand& o) const { return d < o.d || (d == o.d && id < o.id); }
};

struct Graph {            // read-only view of a fixed-degree adjacency [n][degree], -1 = empty slot
    int64_t n;
    int32_t degree;
    const int32_t* adj;
};

struct SearchTrace {
    int64_t hops, evals, max_s, checked;
};

double distance(const float* a, const float* b, int dim);
void parallel_for(int64_t count, int nthreads, const std::function<void(int64_t)>& body);
std::vector<Cand> range_search(const Graph& g,
                               const std::function<double(int32_t)>& dist_to_q,
                               const std::vector<int32_t>& seeds, int k, double eps,
                               bool seeds_in_result, SearchTrace* trace);

}  // namespace oracle
#endif
