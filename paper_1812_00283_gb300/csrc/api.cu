// C-ABI entry points of libbfc (declared in include/bfc.h).
#include <algorithm>
#include <cstdio>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {

int gather_vertices(Graph *g, cudaStream_t s, uint64_t *per_u, uint64_t *per_l);
int gather_edges(Graph *g, cudaStream_t s, uint64_t *per_edge);

namespace {
thread_local std::string g_last_error;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[64] = {};
}  // namespace

void set_last_error(const std::string &msg) { g_last_error = msg; }

namespace {
std::atomic<long long> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return BFC_ERR_OUT_OF_MEMORY;
    return BFC_ERR_CUDA;
}

static cudaError_t get_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t thr = ~0ull;   // keep freed blocks cached for reuse
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool;
    cudaError_t e = get_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void pool_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

cudaError_t pool_usage(int64_t *current, int64_t *high, bool reset_high) {
    cudaMemPool_t pool;
    cudaError_t e = get_pool(&pool);
    if (e != cudaSuccess) return e;
    if (reset_high) {
        uint64_t zero = 0;   // the high-water mark can only be reset to zero
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
        if (e != cudaSuccess) return e;
    }
    uint64_t cur = 0, hi = 0;
    e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &cur);
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &hi);
    if (current) *current = (int64_t)cur;
    if (high) *high = (int64_t)hi;
    return e;
}

}  // namespace bfc

using bfc::Graph;

struct bfc_graph {
    Graph g;
};

namespace bfc {
// the graph behind a handle, for entry points defined in other files
const Graph *graph_of_handle(const bfc_graph *h) { return &h->g; }
}  // namespace bfc

// Bin bounds chosen by bfc_autotune, per size class, for the rest of the
// process: key = (orientation, batch or single graph, floor(log2) of the edge
// count, floor(log2) of the vertex count).
namespace {
struct TunedKey {
    int orient, batch, le, ln;
    bool operator==(const TunedKey &o) const {
        return orient == o.orient && batch == o.batch && le == o.le && ln == o.ln;
    }
};
struct Tuned { TunedKey k; int32_t w, t, h; };
std::mutex g_tuned_mutex;
std::vector<Tuned> g_tuned;

TunedKey tuned_key(int orient, bool batch, int64_t m, int64_t n) {
    return TunedKey{orient, batch ? 1 : 0, bfc::bits_for((uint64_t)m), bfc::bits_for((uint64_t)n)};
}
void tuned_store(const TunedKey &k, int32_t w, int32_t t, int32_t h) {
    std::lock_guard<std::mutex> lk(g_tuned_mutex);
    for (auto &e : g_tuned)
        if (e.k == k) { e.w = w; e.t = t; e.h = h; return; }
    g_tuned.push_back(Tuned{k, w, t, h});
}
// applies a stored choice to *o when use_tuned asks for it
void tuned_apply(bfc_options *o, bool batch, int64_t m, int64_t n) {
    if (!o->use_tuned) return;
    const TunedKey k = tuned_key(o->orientation, batch, m, n);
    std::lock_guard<std::mutex> lk(g_tuned_mutex);
    for (const auto &e : g_tuned)
        if (e.k == k) { o->warp_max_work = e.w; o->team_max_work = e.t; o->hash_max_work = e.h; return; }
}
}  // namespace

static int check_options(const bfc_options *o) {
    if (o->warp_max_work < 0 || o->warp_max_work > bfc::kWarpMaxWork) {
        bfc::set_last_error("warp_max_work must lie in [0, " + std::to_string(bfc::kWarpMaxWork) + "]");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if ((o->hash_max_work < o->warp_max_work && !(o->orientation == 1 && o->hash_max_work == 0)) ||
        o->hash_max_work > bfc::kHashMaxWork || o->hash_max_work < 0) {
        bfc::set_last_error("hash_max_work must lie in [warp_max_work, " + std::to_string(bfc::kHashMaxWork) + "]");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (o->team_max_work < -1 || o->team_max_work > bfc::kTeamMaxWork) {
        bfc::set_last_error("team_max_work must be -1 (default) or lie in [0, " + std::to_string(bfc::kTeamMaxWork) + "]");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (o->num_ctas < 0) {
        bfc::set_last_error("num_ctas must be >= 0");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (o->wide_positions != 0 && o->wide_positions != 1) {
        bfc::set_last_error("wide_positions must be 0 or 1");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (o->orientation != 0 && o->orientation != 1) {
        bfc::set_last_error("orientation must be 0 (Algorithm 2) or 1 (Algorithm 3)");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (o->core_vertices < -1) {
        bfc::set_last_error("core_vertices must be -1 (automatic), 0 (off) or a core size");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (o->use_tuned != 0 && o->use_tuned != 1) {
        bfc::set_last_error("use_tuned must be 0 or 1");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    for (int i = 0; i < 7; ++i)
        if (o->reserved[i] != 0) {
            bfc::set_last_error("reserved option fields must be zero");
            return BFC_ERR_INVALID_ARGUMENT;
        }
    return BFC_OK;
}

namespace bfc {
namespace {

// Host <-> device copies done by the SMs: each thread moves T-sized words
// over the host link.  Measured on this GPU, copies by the copy engines slow
// down five- to eightfold while a large prepared graph is held in device
// memory, and copies by the SMs do not.
template <typename T>
__global__ void k_copy_words(const T *__restrict__ src, T *__restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// The device address of a page-locked host range (cudaHostAlloc or
// cudaHostRegister, both ends checked), or null for any other memory.
const void *locked_host_range(const void *p, size_t bytes) {
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a, b;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        cudaPointerGetAttributes(&b, static_cast<const char *>(p) + bytes - 1) != cudaSuccess) {
        cudaGetLastError();   // an unknown pointer is not an error here
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

// Copies `bytes` between host memory and device memory on s: by the SMs when
// the host side is page-locked, else by cudaMemcpyAsync.
int copy_host(void *dst, const void *src, size_t bytes, bool to_device, cudaStream_t s) {
    if (bytes == 0) return BFC_OK;
    const void *hp = locked_host_range(to_device ? src : dst, bytes);
    if (!hp) {
        BFC_CUDA(cudaMemcpyAsync(dst, src, bytes, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, s));
        return BFC_OK;
    }
    const void *from = to_device ? hp : src;
    void *to = to_device ? dst : const_cast<void *>(hp);
    const uintptr_t al = reinterpret_cast<uintptr_t>(from) | reinterpret_cast<uintptr_t>(to) | bytes;
    const unsigned grid = 152 * 8;
    if (al % 16 == 0)
        k_copy_words<uint4><<<grid, 512, 0, s>>>(static_cast<const uint4 *>(from), static_cast<uint4 *>(to),
                                                 (int64_t)(bytes / 16));
    else if (al % 8 == 0)
        k_copy_words<uint64_t><<<grid, 512, 0, s>>>(static_cast<const uint64_t *>(from),
                                                    static_cast<uint64_t *>(to), (int64_t)(bytes / 8));
    else if (al % 4 == 0)
        k_copy_words<uint32_t><<<grid, 512, 0, s>>>(static_cast<const uint32_t *>(from),
                                                    static_cast<uint32_t *>(to), (int64_t)(bytes / 4));
    else
        k_copy_words<uint8_t><<<grid, 512, 0, s>>>(static_cast<const uint8_t *>(from), static_cast<uint8_t *>(to),
                                                   (int64_t)bytes);
    note_launch();
    BFC_CUDA(cudaGetLastError());
    return BFC_OK;
}

}  // namespace
}  // namespace bfc

extern "C" {

void bfc_options_init(bfc_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->validate = 1;
    opt->warp_max_work = bfc::kWarpMaxWork;
    opt->hash_max_work = bfc::kHashMaxWork;
    opt->team_max_work = -1;
    opt->num_ctas = 0;
    opt->core_vertices = -1;
}

int bfc_prepare(const bfc_csr *csr, const bfc_options *opt_in, void *stream, bfc_graph **out) {
    bfc::set_last_error("");
    if (!csr || !out) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    *out = nullptr;
    bfc_options opt;
    if (opt_in) opt = *opt_in; else bfc_options_init(&opt);
    int rc = check_options(&opt);
    if (rc) return rc;
    if (csr->num_u < 0 || csr->num_l < 0 || csr->num_edges < 0) {
        bfc::set_last_error("negative size"); return BFC_ERR_INVALID_ARGUMENT;
    }
    if (csr->num_edges > 2147483647LL) {
        bfc::set_last_error("num_edges exceeds 2^31 - 1"); return BFC_ERR_INVALID_ARGUMENT;
    }
    if ((int64_t)csr->num_u + (int64_t)csr->num_l > 2147483646LL) {
        bfc::set_last_error("num_u + num_l exceeds 2^31 - 2"); return BFC_ERR_INVALID_ARGUMENT;
    }
    if (!csr->off_u || (csr->num_edges > 0 && !csr->adj_u)) {
        bfc::set_last_error("null CSR pointer"); return BFC_ERR_INVALID_ARGUMENT;
    }
    if (csr->num_edges > 0 && csr->num_l == 0) {
        bfc::set_last_error("edges with an empty L layer"); return BFC_ERR_INVALID_GRAPH;
    }
    tuned_apply(&opt, false, csr->num_edges, (int64_t)csr->num_u + csr->num_l);
    bfc_graph *h = new (std::nothrow) bfc_graph();
    if (!h) { bfc::set_last_error("host allocation failed"); return BFC_ERR_OUT_OF_MEMORY; }
    Graph *g = &h->g;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) { delete h; return bfc::cuda_fail(e, "cudaGetDevice"); }
    e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) { delete h; return bfc::cuda_fail(e, "cudaDeviceGetAttribute"); }
    int smem_optin = 0;
    e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);
    if (e != cudaSuccess) { delete h; return bfc::cuda_fail(e, "cudaDeviceGetAttribute"); }
    if (smem_optin < bfc::kCounterBytes + 32 * 1024 / bfc::kCountCtasPerSm) {
        delete h;
        bfc::set_last_error("device has too little shared memory per block");
        return BFC_ERR_CUDA;
    }
    g->grid = opt.num_ctas > 0 ? opt.num_ctas : g->num_sms * bfc::kCountCtasPerSm;
    rc = bfc::prepare_graph(csr, &opt, static_cast<cudaStream_t>(stream), g);
    if (rc != BFC_OK) {
        g->mem.release();
        cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        delete h;
        return rc;
    }
    *out = h;
    return BFC_OK;
}

static int count_common(bfc_graph *h, void *stream, int mode, uint64_t *per_a, uint64_t *per_b,
                        uint64_t *total_dev, uint64_t *per_edge = nullptr) {
    bfc::set_last_error("");
    if (!h) { bfc::set_last_error("null graph"); return BFC_ERR_INVALID_ARGUMENT; }
    Graph *g = &h->g;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->stream = s;
    unsigned long long *pv = nullptr, *pe = nullptr;
    if (bfc::wants_vertices(mode)) {
        pv = g->pv;
        BFC_CUDA(cudaMemsetAsync(pv, 0, sizeof(unsigned long long) * (size_t)(g->n > 0 ? g->n : 1), s));
    }
    if (bfc::wants_edges(mode)) {
        // the walks sum per G* slot (two per edge); the slot array is taken
        // from the pool on the first per-edge count (stream-ordered) and kept
        if (!g->pe_slot) {
            g->mem.stream = s;
            BFC_CUDA(g->mem.get(&g->pe_slot, (size_t)(2 * g->m > 0 ? 2 * g->m : 1)));
        }
        pe = g->pe_slot;
        if (g->m > 0) BFC_CUDA(cudaMemsetAsync(pe, 0, sizeof(uint64_t) * (size_t)(2 * g->m), s));
    }
    int rc = bfc::launch_count(g, s, mode, pv, pe);
    if (rc) return rc;
    if (bfc::wants_vertices(mode)) {
        rc = bfc::gather_vertices(g, s, per_a, per_b);
        if (rc) return rc;
    }
    if (bfc::wants_edges(mode)) {
        rc = bfc::gather_edges(g, s, mode == bfc::kModeEdges ? per_a : per_edge);
        if (rc) return rc;
    }
    if (total_dev)
        BFC_CUDA(cudaMemcpyAsync(total_dev, g->acc, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    return BFC_OK;
}

int bfc_prepare_batch(const bfc_csr *csr, const bfc_batch *batch, const bfc_options *opt_in,
                      void *stream, bfc_graph **out) {
    bfc::set_last_error("");
    if (!csr || !batch || !out) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    *out = nullptr;
    if (batch->num_graphs < 1 || !batch->graph_u_start || !batch->graph_l_start) {
        bfc::set_last_error("a batch needs num_graphs >= 1 and both start arrays");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    bfc_options opt;
    if (opt_in) opt = *opt_in; else bfc_options_init(&opt);
    int rc = check_options(&opt);
    if (rc) return rc;
    if (csr->num_u < 0 || csr->num_l < 0 || csr->num_edges < 0 || csr->num_edges > 2147483647LL ||
        (int64_t)csr->num_u + (int64_t)csr->num_l > 2147483646LL || !csr->off_u ||
        (csr->num_edges > 0 && !csr->adj_u)) {
        bfc::set_last_error("invalid union CSR arguments");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    tuned_apply(&opt, true, csr->num_edges, (int64_t)csr->num_u + csr->num_l);
    bfc_graph *h = new (std::nothrow) bfc_graph();
    if (!h) { bfc::set_last_error("host allocation failed"); return BFC_ERR_OUT_OF_MEMORY; }
    Graph *g = &h->g;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) { delete h; return bfc::cuda_fail(e, "cudaGetDevice"); }
    g->grid = opt.num_ctas > 0 ? opt.num_ctas : g->num_sms * bfc::kCountCtasPerSm;
    rc = bfc::prepare_graph(csr, &opt, static_cast<cudaStream_t>(stream), g, batch->num_graphs,
                            batch->graph_u_start, batch->graph_l_start);
    if (rc != BFC_OK) {
        g->mem.release();
        cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        delete h;
        return rc;
    }
    *out = h;
    return BFC_OK;
}

int bfc_count_batch(bfc_graph *h, void *stream, uint64_t *totals_dev, uint64_t *total_dev) {
    bfc::set_last_error("");
    if (!h || !totals_dev) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    Graph *g = &h->g;
    if (g->num_graphs < 1) { bfc::set_last_error("graph was not prepared as a batch"); return BFC_ERR_INVALID_ARGUMENT; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->stream = s;
    unsigned long long *gt = reinterpret_cast<unsigned long long *>(totals_dev);
    BFC_CUDA(cudaMemsetAsync(gt, 0, sizeof(uint64_t) * (size_t)g->num_graphs, s));
    int rc = bfc::launch_count(g, s, bfc::kModeBatch, nullptr, nullptr, gt);
    if (rc) return rc;
    if (total_dev)
        BFC_CUDA(cudaMemcpyAsync(total_dev, g->acc, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    return BFC_OK;
}

int bfc_batch_wedges(const bfc_graph *h, void *stream, uint64_t *wedges_dev) {
    if (!h || !wedges_dev) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    const Graph *g = &h->g;
    if (g->num_graphs < 1) { bfc::set_last_error("graph was not prepared as a batch"); return BFC_ERR_INVALID_ARGUMENT; }
    BFC_CUDA(cudaMemcpyAsync(wedges_dev, g->gwork, sizeof(uint64_t) * (size_t)g->num_graphs,
                             cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
    return BFC_OK;
}

struct bfc_batch_plan {
    bfc::BatchPlan p;
};

int bfc_batch_plan_create(const bfc_batch_shape *shape, const bfc_options *opt_in, void *stream,
                          bfc_batch_plan **out) {
    bfc::set_last_error("");
    if (!shape || !out) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    *out = nullptr;
    bfc_options opt;
    if (opt_in) opt = *opt_in; else bfc_options_init(&opt);
    int rc = check_options(&opt);
    if (rc) return rc;
    bool reserved_zero = true;
    for (int i = 0; i < 6; ++i) reserved_zero = reserved_zero && shape->reserved[i] == 0;
    if (shape->num_u < 0 || shape->num_l < 0 || shape->num_edges < 0 || shape->num_edges > 2147483647LL ||
        (int64_t)shape->num_u + shape->num_l > 2147483646LL || shape->num_graphs < 1 ||
        shape->max_layer < 1 || shape->max_layer > 65535 || !reserved_zero) {
        bfc::set_last_error("batch shape outside its ranges (max_layer in [1, 65535], num_graphs >= 1, "
                            "reserved fields zero)");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (opt.orientation != 0 || opt.team_max_work > bfc::kTeamFitWork) {
        bfc::set_last_error("a batch plan counts with Algorithm 2 and team_max_work <= 3072");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    bfc_batch_plan *h = new (std::nothrow) bfc_batch_plan();
    if (!h) { bfc::set_last_error("host allocation failed"); return BFC_ERR_OUT_OF_MEMORY; }
    bfc::BatchPlan &pl = h->p;
    Graph *g = &pl.g;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) { delete h; return bfc::cuda_fail(e, "cudaGetDevice"); }
    g->grid = opt.num_ctas > 0 ? opt.num_ctas : g->num_sms * bfc::kCountCtasPerSm;
    opt.core_vertices = 0;
    g->opt = opt;
    pl.r = shape->num_u; pl.l = shape->num_l; pl.m = shape->num_edges;
    pl.num_graphs = shape->num_graphs; pl.max_layer = shape->max_layer;
    // the team bin as schedule_graph sets it for Algorithm 2
    const uint64_t team_req = opt.team_max_work >= 0 ? (uint64_t)opt.team_max_work : (uint64_t)bfc::kTeamFitWork;
    pl.team_max = std::min<uint64_t>(std::max<uint64_t>(team_req, (uint64_t)opt.warp_max_work),
                                     (uint64_t)opt.hash_max_work);
    g->team_max = (int32_t)pl.team_max;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = bfc::batch_plan_create(&pl, s);
    if (rc) {
        g->mem.release();
        cudaStreamSynchronize(s);
        delete h;
        return rc;
    }
    *out = h;
    return BFC_OK;
}

int bfc_batch_plan_run(bfc_batch_plan *h, const int32_t *off_u, const int32_t *adj_u, const int32_t *gu,
                       const int32_t *gl, void *stream, uint64_t *totals_dev, int32_t *status_dev) {
    bfc::set_last_error("");
    if (!h || !off_u || (h->p.m > 0 && !adj_u) || !gu || !gl || !totals_dev) {
        bfc::set_last_error("null argument");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    return bfc::batch_plan_run(&h->p, off_u, adj_u, gu, gl, static_cast<cudaStream_t>(stream),
                               reinterpret_cast<unsigned long long *>(totals_dev), status_dev);
}

void bfc_batch_plan_destroy(bfc_batch_plan *h) {
    if (!h) return;
    Graph *g = &h->p.g;
    g->mem.stream = g->stream;
    g->mem.release();
    cudaStreamSynchronize(g->stream);
    delete h;
}

int bfc_autotune(bfc_graph *h, void *stream, int iters, bfc_options *chosen) {
    bfc::set_last_error("");
    if (!h) { bfc::set_last_error("null graph"); return BFC_ERR_INVALID_ARGUMENT; }
    if (iters < 1) iters = 1;
    Graph *g = &h->g;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->stream = s;
    // candidate (warp, team, hash) bounds; Algorithm 3 ignores the hash bound
    struct Cand { int32_t w, t, h; };
    Cand cands[12];
    int nc = 0;
    for (int32_t wmax : {32, 128, bfc::kWarpMaxWork}) {
        if (g->opt.orientation == 1) {
            for (int32_t tmax : {2048, bfc::kTeamMaxWork}) cands[nc++] = {wmax, tmax, bfc::kHashMaxWork};
        } else {
            for (int32_t tmax : {512, bfc::kTeamFitWork})
                for (int32_t hmax : {4096, bfc::kHashMaxWork}) cands[nc++] = {wmax, tmax, hmax};
        }
    }
    cudaEvent_t e0, e1;
    BFC_CUDA(cudaEventCreate(&e0));
    BFC_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int32_t bw = g->opt.warp_max_work, bt = g->opt.team_max_work, bh = g->opt.hash_max_work;
    int rc = BFC_OK;
    for (int c = 0; c < nc; ++c) {
        rc = bfc::rebin_graph(g, s, cands[c].w, cands[c].t, cands[c].h);
        if (rc) break;
        rc = bfc::launch_count(g, s, bfc::kModeTotal, nullptr, nullptr);   // warm-up
        if (rc) break;
        cudaEventRecord(e0, s);
        for (int i = 0; i < iters && rc == BFC_OK; ++i)
            rc = bfc::launch_count(g, s, bfc::kModeTotal, nullptr, nullptr);
        cudaEventRecord(e1, s);
        if (rc) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { rc = bfc::cuda_fail(e, "cudaEventSynchronize"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bw = cands[c].w; bt = cands[c].t; bh = cands[c].h; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = bfc::rebin_graph(g, s, bw, bt, bh);
    if (rc) return rc;
    tuned_store(tuned_key(g->opt.orientation, g->num_graphs > 0, g->m, (int64_t)g->n), bw, bt, bh);
    if (chosen) *chosen = g->opt;
    return BFC_OK;
}

int bfc_count(bfc_graph *g, void *stream, uint64_t *total_dev) {
    if (!total_dev) { bfc::set_last_error("null total_dev"); return BFC_ERR_INVALID_ARGUMENT; }
    return count_common(g, stream, bfc::kModeTotal, nullptr, nullptr, total_dev);
}

int bfc_count_vertices(bfc_graph *g, void *stream, uint64_t *per_u_dev, uint64_t *per_l_dev,
                       uint64_t *total_dev) {
    return count_common(g, stream, bfc::kModeVertices, per_u_dev, per_l_dev, total_dev);
}

int bfc_count_edges(bfc_graph *g, void *stream, uint64_t *per_edge_dev, uint64_t *total_dev) {
    if (!g) { bfc::set_last_error("null graph"); return BFC_ERR_INVALID_ARGUMENT; }
    if (!per_edge_dev && g->g.m > 0) {
        bfc::set_last_error("null per_edge_dev"); return BFC_ERR_INVALID_ARGUMENT;
    }
    return count_common(g, stream, bfc::kModeEdges, per_edge_dev, nullptr, total_dev);
}

int bfc_count_all(bfc_graph *g, void *stream, uint64_t *per_u_dev, uint64_t *per_l_dev,
                  uint64_t *per_edge_dev, uint64_t *total_dev) {
    if (!g) { bfc::set_last_error("null graph"); return BFC_ERR_INVALID_ARGUMENT; }
    if (!per_edge_dev && g->g.m > 0) {
        bfc::set_last_error("null per_edge_dev"); return BFC_ERR_INVALID_ARGUMENT;
    }
    return count_common(g, stream, bfc::kModeAll, per_u_dev, per_l_dev, total_dev, per_edge_dev);
}

int bfc_sync(bfc_graph *h, void *stream) {
    bfc::set_last_error("");
    if (!h) { bfc::set_last_error("null graph"); return BFC_ERR_INVALID_ARGUMENT; }
    Graph *g = &h->g;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int herr = 0;
    BFC_CUDA(cudaMemcpyAsync(&herr, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BFC_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        BFC_CUDA(cudaMemsetAsync(g->err, 0, sizeof(int), s));
        BFC_CUDA(cudaStreamSynchronize(s));
        char buf[96];
        if (herr & bfc::kErrTimeout) {
            snprintf(buf, sizeof(buf), "a bounded device wait gave up (flags 0x%x)", herr);
            bfc::set_last_error(buf);
            return BFC_ERR_TIMEOUT;
        }
        snprintf(buf, sizeof(buf), "kernel consistency check fired (flags 0x%x)", herr);
        bfc::set_last_error(buf);
        return BFC_ERR_INTERNAL;
    }
    return BFC_OK;
}

int bfc_graph_info(const bfc_graph *h, bfc_info *out) {
    if (!h || !out) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    *out = h->g.info;
    return BFC_OK;
}

int bfc_export(const bfc_graph *h, int which, void *dst, void *stream) {
    if (!h || !dst) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    const Graph *g = &h->g;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const void *src = nullptr;
    size_t bytes = 0;
    switch (which) {
        case BFC_RANK_U: src = g->rank_u; bytes = 4 * (size_t)g->r; break;
        case BFC_RANK_L: src = g->rank_l; bytes = 4 * (size_t)g->l; break;
        case BFC_PROJ_OFF: src = g->off; bytes = 8 * ((size_t)g->n + 1); break;
        case BFC_PROJ_ADJ: src = g->adj; bytes = 4 * (size_t)(2 * g->m); break;
        case BFC_PROJ_EID: src = g->eid; bytes = 4 * (size_t)(2 * g->m); break;
        case BFC_CUT: src = g->cut; bytes = 4 * (size_t)g->n; break;
        case BFC_WORK: src = g->work; bytes = 8 * (size_t)g->n; break;
        case BFC_RETRIES: src = g->cursors + 2; bytes = 4; break;
        case BFC_CORE_PRODUCT_U:
        case BFC_CORE_PRODUCT_L: {
            // rows of the padded product, core_u (core_l) columns each
            const bool u = which == BFC_CORE_PRODUCT_U;
            const int32_t k = u ? g->core_u : g->core_l;
            if (k > 0)
                BFC_CUDA(cudaMemcpy2DAsync(dst, 2 * (size_t)k, u ? g->core_au : g->core_al,
                                           2 * (size_t)(u ? g->core_ld_u : g->core_ld_l), 2 * (size_t)k,
                                           (size_t)k, cudaMemcpyDeviceToDevice, s));
            return BFC_OK;
        }
        default: bfc::set_last_error("unknown array"); return BFC_ERR_INVALID_ARGUMENT;
    }
    if (bytes) BFC_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    return BFC_OK;
}

int bfc_count_all_host(int32_t num_u, int32_t num_l, int64_t num_edges, const int32_t *off_u_host,
                       const int32_t *adj_u_host, const bfc_options *opt, void *stream,
                       uint64_t *per_u_host, uint64_t *per_l_host, uint64_t *per_edge_host,
                       uint64_t *total_host, uint64_t *wedges_host) {
    bfc::set_last_error("");
    if (!off_u_host || (num_edges > 0 && (!adj_u_host || !per_edge_host)) || !total_host || num_u < 0 ||
        num_l < 0 || num_edges < 0 || num_edges > 2147483647LL) {
        bfc::set_last_error("invalid host CSR or output arguments");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bfc::Allocs in;
    in.stream = s;
    struct Guard { bfc::Allocs *a; cudaStream_t s; ~Guard() { a->release(); cudaStreamSynchronize(s); } } guard{&in, s};
    int32_t *off = nullptr, *adj = nullptr;
    uint64_t *pu = nullptr, *pl = nullptr, *pe = nullptr, *tot = nullptr;
    if (in.get(&off, (size_t)num_u + 1) || in.get(&adj, (size_t)std::max<int64_t>(num_edges, 1)) ||
        in.get(&pu, (size_t)std::max(num_u, 1)) || in.get(&pl, (size_t)std::max(num_l, 1)) ||
        in.get(&pe, (size_t)std::max<int64_t>(num_edges, 1)) || in.get(&tot, 1)) {
        bfc::set_last_error("device allocation failed");
        return BFC_ERR_OUT_OF_MEMORY;
    }
    int rc = bfc::copy_host(off, off_u_host, sizeof(int32_t) * ((size_t)num_u + 1), true, s);
    if (rc == BFC_OK) rc = bfc::copy_host(adj, adj_u_host, sizeof(int32_t) * (size_t)num_edges, true, s);
    bfc_graph *g = nullptr;
    if (rc == BFC_OK) {
        bfc_csr csr{num_u, num_l, num_edges, off, adj};
        rc = bfc_prepare(&csr, opt, stream, &g);
    }
    if (rc == BFC_OK)
        rc = count_common(g, stream, bfc::kModeAll, per_u_host ? pu : nullptr, per_l_host ? pl : nullptr,
                          tot, pe);
    // the graph's memory goes back to the pool before the outputs travel
    if (rc == BFC_OK) rc = bfc_sync(g, stream);
    if (rc == BFC_OK && wedges_host) *wedges_host = g->g.info.wedges;
    if (g) bfc_release(g);
    if (rc == BFC_OK && per_u_host) rc = bfc::copy_host(per_u_host, pu, sizeof(uint64_t) * (size_t)num_u, false, s);
    if (rc == BFC_OK && per_l_host) rc = bfc::copy_host(per_l_host, pl, sizeof(uint64_t) * (size_t)num_l, false, s);
    if (rc == BFC_OK) rc = bfc::copy_host(per_edge_host, pe, sizeof(uint64_t) * (size_t)num_edges, false, s);
    if (rc == BFC_OK) {
        cudaError_t e = cudaMemcpyAsync(total_host, tot, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = bfc::cuda_fail(e, "copy of the results to the host");
    }
    return rc;
}

int bfc_count_host(int32_t num_u, int32_t num_l, int64_t num_edges, const int32_t *off_u_host,
                   const int32_t *adj_u_host, const bfc_options *opt, void *stream,
                   uint64_t *total_host, uint64_t *wedges_host) {
    bfc::set_last_error("");
    if (!off_u_host || (num_edges > 0 && !adj_u_host) || !total_host || num_u < 0 ||
        num_edges < 0 || num_edges > 2147483647LL) {
        bfc::set_last_error("invalid host CSR arguments");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bfc::Allocs in;
    in.stream = s;
    int32_t *off = nullptr, *adj = nullptr;
    if (in.get(&off, (size_t)num_u + 1) != cudaSuccess ||
        in.get(&adj, (size_t)(num_edges > 0 ? num_edges : 1)) != cudaSuccess) {
        in.release();
        bfc::set_last_error("device allocation failed");
        return BFC_ERR_OUT_OF_MEMORY;
    }
    int rc = bfc::copy_host(off, off_u_host, sizeof(int32_t) * ((size_t)num_u + 1), true, s);
    if (rc == BFC_OK) rc = bfc::copy_host(adj, adj_u_host, sizeof(int32_t) * (size_t)num_edges, true, s);
    cudaError_t e = cudaSuccess;
    bfc_graph *g = nullptr;
    if (rc == BFC_OK) {
        bfc_csr csr{num_u, num_l, num_edges, off, adj};
        rc = bfc_prepare(&csr, opt, stream, &g);
    }
    if (rc == BFC_OK) rc = count_common(g, stream, bfc::kModeTotal, nullptr, nullptr, nullptr);
    if (rc == BFC_OK) {
        e = cudaMemcpyAsync(total_host, g->g.acc, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = bfc::cuda_fail(e, "cudaMemcpyAsync(D2H)");
    }
    if (rc == BFC_OK) rc = bfc_sync(g, stream);
    if (rc == BFC_OK && wedges_host) *wedges_host = g->g.info.wedges;
    if (g) bfc_release(g);
    in.release();
    cudaStreamSynchronize(s);
    return rc;
}

void bfc_release(bfc_graph *h) {
    if (!h) return;
    h->g.mem.stream = h->g.stream;
    h->g.mem.release();
    delete h;
}

const char *bfc_status_string(int status) {
    switch (status) {
        case BFC_OK: return "BFC_OK";
        case BFC_ERR_INVALID_ARGUMENT: return "BFC_ERR_INVALID_ARGUMENT";
        case BFC_ERR_INVALID_GRAPH: return "BFC_ERR_INVALID_GRAPH";
        case BFC_ERR_OUT_OF_MEMORY: return "BFC_ERR_OUT_OF_MEMORY";
        case BFC_ERR_CUDA: return "BFC_ERR_CUDA";
        case BFC_ERR_TIMEOUT: return "BFC_ERR_TIMEOUT";
        case BFC_ERR_INTERNAL: return "BFC_ERR_INTERNAL";
        default: return "BFC_ERR_UNKNOWN";
    }
}

const char *bfc_last_error(void) { return bfc::g_last_error.c_str(); }

int bfc_version(void) { return 100; }

long long bfc_kernel_launches(void) { return bfc::g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
