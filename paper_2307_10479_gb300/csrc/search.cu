// Host side of the batched search and the serving loop: device-memory scratch, entry routing, and
// the launch of the per-format kernels (search_impl.cuh holds the kernels and the method).
#include "search_impl.cuh"

namespace deg {
using namespace sk;

namespace {

int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

int workspace_reserve(Workspace& ws, const DeviceIndex& ix, int64_t nq, std::string* why) {
    cudaError_t e;
    if (!ws.counters) {
        if ((e = cudaMalloc(&ws.counters, 4 * sizeof(int32_t))) != cudaSuccess) return *why = "counters", (int)e;
    }
    if (ws.cap_q < nq) {
        cudaFree(ws.overflow);
        ws.overflow = nullptr;
        ws.cap_q = 0;
        cudaFree(ws.route);
        ws.route = nullptr;
        if ((e = cudaMalloc(&ws.overflow, sizeof(int32_t) * nq)) != cudaSuccess ||
            (e = cudaMalloc(&ws.route, sizeof(int32_t) * (4 * nq + 2))) != cudaSuccess)
            return *why = "overflow list", (int)e;
        ws.cap_q = nq;
    }
    if (!ws.bitmaps) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t words = (ix.n + 127) / 128 * 4;
        // main kernel: one slot (bitmap + back pool) per resident warp, within about 2.5 GiB
        const int64_t per = words * 4 + 8ll * kBackPool + 4ll * kTouchCap;
        int64_t slots = std::min<int64_t>((int64_t)sms * kBlocksPerSM * kWarpsPerBlock, (5ll << 29) / per);
        slots = std::max<int64_t>(kWarpsPerBlock, slots / kWarpsPerBlock * kWarpsPerBlock);
        // second kernel: room for all n vertices per slot, within about 1 GiB
        const int64_t pper = words * 4 + 8 * (ix.n + 1);
        int64_t pslots = std::max<int64_t>(kWarpsPerBlock, std::min<int64_t>(64, (1ll << 30) / pper));
        pslots = pslots / kWarpsPerBlock * kWarpsPerBlock;
        if ((e = cudaMalloc(&ws.bitmaps, sizeof(uint32_t) * words * slots)) != cudaSuccess ||
            (e = cudaMalloc(&ws.backs, sizeof(uint64_t) * kBackPool * slots)) != cudaSuccess ||
            (e = cudaMalloc(&ws.touched, sizeof(int32_t) * kTouchCap * slots)) != cudaSuccess ||
            (e = cudaMemset(ws.bitmaps, 0, sizeof(uint32_t) * words * slots)) != cudaSuccess ||
            (e = cudaMalloc(&ws.pbitmaps, sizeof(uint32_t) * words * pslots)) != cudaSuccess ||
            (e = cudaMalloc(&ws.pbacks, sizeof(uint64_t) * (ix.n + 1) * pslots)) != cudaSuccess) {
            workspace_free(ws);
            return *why = "device-memory search state", (int)e;
        }
        ws.words = words;
        ws.slots = (int32_t)slots;
        ws.bcap = kBackPool;
        ws.pslots = (int32_t)pslots;
    }
    return 0;
}

void workspace_free(Workspace& ws) {
    cudaFree(ws.counters);
    cudaFree(ws.overflow);
    cudaFree(ws.route);
    cudaFree(ws.bitmaps);
    cudaFree(ws.backs);
    cudaFree(ws.touched);
    cudaFree(ws.pbitmaps);
    cudaFree(ws.pbacks);
    cudaFree(ws.dq);
    cudaFree(ws.did);
    cudaFree(ws.dd);
    ws = Workspace{};
}

int launch_search(const SearchArgs& a, Workspace& ws, deg_stream_t stream, std::string* why) {
    const DeviceIndex& ix = *a.ix;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (ix.degree > kMaxDegree) return *why = "degree above 128", (int)cudaErrorInvalidValue;
    Params P{};
    P.x32 = ix.x32;
    P.dim_pad = ix.dim_pad;
    P.adj = reinterpret_cast<const int2*>(ix.adj);
    P.degree = ix.degree;
    P.deg_pad = ix.deg_pad;
    P.n = ix.n;
    P.entry = ix.entry_internal;
    P.entry_caller = ix.entry;
    P.old2new = ix.old2new;
    P.new2old = ix.new2old;
    P.queries = a.queries;
    P.dim = ix.dim;
    P.seeds = a.seeds;
    P.seeds2 = a.seeds2;
    P.explore = a.explore;
    if (a.entry_mode >= 1 && !a.explore && !a.seeds) {
        // route every query to its nearest pivot first; those become internal seeds
        const int e = route_to_pivots(ix, a.queries, a.nq, ws.route, ws.route + ws.cap_q,
                                      reinterpret_cast<float*>(ws.route + 2 * ws.cap_q), ws.route + 3 * ws.cap_q,
                                      ws.route + 4 * ws.cap_q, a.entry_mode == 2, stream, why);
        if (e != 0) return e;
        P.seeds = ws.route + ws.cap_q;
        P.order = ws.route + 3 * ws.cap_q;
        P.seeds_internal = 1;
    }
    P.nq = (int32_t)a.nq;
    P.k = a.k;
    const bool reduced = a.precision != DEG_F32;
    P.ks = reduced && a.rerank > 0 ? std::max(a.rerank, a.k) : a.k;
    // long walks keep the front of S sorted: from the fixed entry vertex (~1,500 hops), or with
    // many results kept or a wide eps (hundreds of pops); short routed, seeded and exploration
    // walks keep it unsorted
    P.sorted_front = sorted_front_for(!P.seeds && !P.explore, P.ks, a.eps) ? 1 : 0;
    P.kcap = std::max(32, pow2_at_least(P.ks));
    P.rerank = reduced && a.rerank >= 0 ? 1 : 0;             // -1: the reduced-precision distances as computed
    const float2 fe = eps_factor(a.eps);
    P.f = fe.x;
    P.f_lo = fe.y;
    P.max_hops = a.max_hops;
    P.learned = a.learned_stop ? 1 : 0;
    P.stop_w = reinterpret_cast<const __nv_bfloat16*>(ix.stop_w);
    P.stop_logit = ix.stop_logit;
    if (P.learned && !P.stop_w) return *why = "no stop model set for this index", (int)cudaErrorInvalidValue;
    P.rec_feats = a.rec_feats;
    P.rec_labels = a.rec_labels;
    P.rec_counts = a.rec_counts;
    P.rec_cap = a.rec_cap;
    P.ids = a.ids;
    P.dists = a.dists;
    P.status = a.status;
    P.trace = a.trace;
    P.counters = ws.counters;
    P.overflow = ws.overflow;
    P.words = ws.words;
    P.bitmaps = ws.bitmaps;
    P.touched = ws.touched;
    P.backs = ws.backs;
    P.slots = ws.slots;
    P.bstride = ws.bcap;
    // queue_cap bounds the back pool of the main kernel (a small value sends queries to the
    // second kernel)
    P.bcap = a.queue_cap ? std::min(a.queue_cap, ws.bcap) : ws.bcap;
    P.pbitmaps = ws.pbitmaps;
    P.pbacks = ws.pbacks;
    P.pslots = ws.pslots;
    if (a.precision == DEG_F32) {
        P.rows = reinterpret_cast<const uint8_t*>(ix.x32);
        P.row_bytes = 4ll * ix.dim_pad;
        P.nchunk = ix.dim_pad / 4;
        return dispatch_search_f32(P, st, a.timer_start, a.timer_end, why);
    }
    if (a.precision == DEG_BF16) {
        P.rows = reinterpret_cast<const uint8_t*>(ix.xbf);
        P.row_bytes = 2ll * ix.dim_pad16;
        P.nchunk = ix.dim_pad16 / 8;
        return dispatch_search_bf16(P, st, a.timer_start, a.timer_end, why);
    }
    P.rows = ix.x8;
    P.row_bytes = ix.dim_pad8;
    P.nchunk = ix.dim_pad8 / 16;
    P.norm8 = reinterpret_cast<const float2*>(ix.norm8);
    return dispatch_search_fp8(P, st, a.timer_start, a.timer_end, why);
}

}  // namespace deg

namespace deg {
using namespace sk;

int launch_serving(const ServeArgs& a, Workspace& ws, deg_stream_t stream, int* warps, std::string* why) {
    const DeviceIndex& ix = *a.ix;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (ix.degree > kMaxDegree) return *why = "degree above 128", (int)cudaErrorInvalidValue;
    Params P{};
    P.x32 = ix.x32;
    P.dim_pad = ix.dim_pad;
    P.adj = reinterpret_cast<const int2*>(ix.adj);
    P.degree = ix.degree;
    P.deg_pad = ix.deg_pad;
    P.n = ix.n;
    P.entry = ix.entry_internal;
    P.entry_caller = ix.entry;
    P.old2new = ix.old2new;
    P.new2old = ix.new2old;
    P.dim = ix.dim;
    const bool reduced = a.precision != DEG_F32;
    P.ks = reduced && a.rerank ? a.rerank : 0;
    P.kcap = std::max(32, pow2_at_least(std::max(a.kmax, P.ks)));
    P.rerank = reduced ? 1 : 0;
    P.learned = a.learned_stop ? 1 : 0;
    P.stop_w = reinterpret_cast<const __nv_bfloat16*>(ix.stop_w);
    P.stop_logit = ix.stop_logit;
    if (P.learned && !P.stop_w) return *why = "no stop model set for this index", (int)cudaErrorInvalidValue;
    P.words = ws.words;
    P.bitmaps = ws.bitmaps;
    P.touched = ws.touched;
    P.backs = ws.backs;
    P.slots = ws.slots;
    P.bstride = ws.bcap;
    P.bcap = ws.bcap;
    const int32_t* piv = a.entry_mode == 2 ? ix.lpivots : ix.pivots;
    const int32_t npiv = a.entry_mode == 2 ? ix.lnpivots : ix.npivots;
    if (a.entry_mode == 2 && !piv) return *why = "no learned entry points (deg_train_entry)", (int)cudaErrorInvalidValue;
    ServeRing S{a.vecs, reinterpret_cast<const int4*>(a.meta), a.ids, a.dists, a.status, a.trace, a.done, a.times, a.tail,
                a.stop, a.kstatus, a.claim, a.cap, a.kmax, a.entry_mode, a.idle_ns, a.max_blocks};
    if (a.precision == DEG_F32) {
        P.rows = reinterpret_cast<const uint8_t*>(ix.x32);
        P.row_bytes = 4ll * ix.dim_pad;
        P.nchunk = ix.dim_pad / 4;
        return dispatch_serve_f32(P, S, piv, npiv, st, warps, why);
    }
    if (a.precision == DEG_BF16) {
        P.rows = reinterpret_cast<const uint8_t*>(ix.xbf);
        P.row_bytes = 2ll * ix.dim_pad16;
        P.nchunk = ix.dim_pad16 / 8;
        return dispatch_serve_bf16(P, S, piv, npiv, st, warps, why);
    }
    P.rows = ix.x8;
    P.row_bytes = ix.dim_pad8;
    P.nchunk = ix.dim_pad8 / 16;
    P.norm8 = reinterpret_cast<const float2*>(ix.norm8);
    return dispatch_serve_fp8(P, S, piv, npiv, st, warps, why);
}

}  // namespace deg
