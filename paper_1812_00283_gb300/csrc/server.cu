// A continuous-batching request server for butterfly counts.
//
// Requests (one graph each, U-side CSR in host memory) arrive at any time.
// Worker threads, each with its own CUDA stream, repeatedly take the oldest
// waiting requests that fit the device-memory budget, copy them into one
// disjoint-union batch on the device, prepare the batch and count it in one
// persistent launch (bfc_prepare_batch / bfc_count_batch), and complete the
// requests with their per-graph totals.  While one worker's batch is on the
// GPU, the next worker admits the requests that arrived meanwhile, so batches
// overlap on the device and memory freed by a finished batch is reused at
// once.  The method itself is untouched: the totals are exactly the counts of
// each graph alone (butterflies never span graphs of a disjoint union).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {
namespace {

// device footprint estimate of a batch (arena, prepare temporaries, union CSR)
int64_t batch_bytes(int64_t r, int64_t l, int64_t m) {
    return 112 * m + 64 * (r + l) + (4 << 20);
}

// The graph contract's cheap host-side part, checked at submission so that a
// malformed request fails alone instead of failing the batch it would join:
// off_u is a CSR of num_edges entries and every id lies in [0, num_l).
bool host_csr_ok(int32_t r, int32_t l, int64_t m, const int32_t *off, const int32_t *adj) {
    if (off[0] != 0 || (int64_t)off[r] != m) return false;
    for (int32_t u = 0; u < r; ++u)
        if (off[u + 1] < off[u]) return false;
    for (int64_t k = 0; k < m; ++k)
        if (adj[k] < 0 || adj[k] >= l) return false;
    return true;
}

// a union of graphs keeps its vertex ids and its CSR offsets in int32
constexpr int64_t kUnionMax = 0x7fffffffll;

// offsets and ids of each graph shifted into the union's id space
__global__ void k_union_fixup(int32_t *off, int32_t *adj, const int64_t *__restrict__ e_start,
                              const int32_t *__restrict__ u_start,
                              const int32_t *__restrict__ l_start, int32_t num_graphs,
                              int64_t total_u, int64_t total_m) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total_m; i += stride) {
        int32_t lo = 0, hi = num_graphs;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (e_start[mid] <= i) lo = mid; else hi = mid;
        }
        adj[i] += l_start[lo];
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total_u; i += stride) {
        int32_t lo = 0, hi = num_graphs;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (u_start[mid] <= i) lo = mid; else hi = mid;
        }
        off[i] += (int32_t)e_start[lo];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[total_u] = (int32_t)total_m;
}

struct Request {
    uint64_t id;
    int32_t r, l;
    int64_t m;
    const int32_t *off;
    const int32_t *adj;
    int64_t bytes;
    std::chrono::steady_clock::time_point t_submit, t_done;
    int status = -1;        // -1 pending, else a bfc_status
    uint64_t total = 0;
};

}  // namespace
}  // namespace bfc

struct bfc_server {
    bfc_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<bfc::Request *> waiting;
    std::unordered_map<uint64_t, bfc::Request *> all;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;   // one per worker, created before any worker starts
    uint64_t next_id = 1;
    int64_t bytes_in_use = 0;
    bool stop = false;
    bfc_server_stats stats{};
};

namespace bfc {
namespace {

void complete(bfc_server *sv, std::vector<Request *> &batch, const std::vector<int> &status,
              const std::vector<uint64_t> &totals) {
    const auto now = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    for (size_t i = 0; i < batch.size(); ++i) {
        const int st = status[i];
        batch[i]->status = st;
        batch[i]->total = (st == BFC_OK && i < totals.size()) ? totals[i] : 0;
        batch[i]->t_done = now;
        if (st == BFC_OK) sv->stats.completed += 1; else sv->stats.failed += 1;
    }
    sv->cv_done.notify_all();
}

// Counts one batch on stream s; returns a bfc_status.
int run_batch(bfc_server *sv, std::vector<Request *> &batch, cudaStream_t s,
              std::vector<uint64_t> &totals) {
    const int32_t G = (int32_t)batch.size();
    std::vector<int64_t> us64(G + 1, 0), ls64(G + 1, 0), es(G + 1, 0);
    for (int32_t g = 0; g < G; ++g) {
        us64[g + 1] = us64[g] + batch[g]->r;
        ls64[g + 1] = ls64[g] + batch[g]->l;
        es[g + 1] = es[g] + batch[g]->m;
    }
    // admission keeps a batch inside int32 ids and slots (kUnionMax)
    if (us64[G] + ls64[G] > kUnionMax || es[G] > kUnionMax) {
        set_last_error("batch exceeds the int32 range of a union");
        return BFC_ERR_INTERNAL;
    }
    std::vector<int32_t> us(G + 1), ls(G + 1);
    for (int32_t g = 0; g <= G; ++g) { us[g] = (int32_t)us64[g]; ls[g] = (int32_t)ls64[g]; }
    Allocs in;
    in.stream = s;
    struct Guard { Allocs *a; ~Guard() { a->release(); } } guard{&in};
    int32_t *off = nullptr, *adj = nullptr, *dus = nullptr, *dls = nullptr;
    int64_t *des = nullptr;
    unsigned long long *dtot = nullptr;
    if (in.get(&off, (size_t)us[G] + 1) || in.get(&adj, (size_t)std::max<int64_t>(es[G], 1)) ||
        in.get(&dus, (size_t)G + 1) || in.get(&dls, (size_t)G + 1) || in.get(&des, (size_t)G + 1) ||
        in.get(&dtot, (size_t)G))
        return BFC_ERR_OUT_OF_MEMORY;
    for (int32_t g = 0; g < G; ++g) {
        BFC_CUDA(cudaMemcpyAsync(off + us[g], batch[g]->off, sizeof(int32_t) * batch[g]->r,
                                 cudaMemcpyHostToDevice, s));
        if (batch[g]->m > 0)
            BFC_CUDA(cudaMemcpyAsync(adj + es[g], batch[g]->adj, sizeof(int32_t) * batch[g]->m,
                                     cudaMemcpyHostToDevice, s));
    }
    BFC_CUDA(cudaMemcpyAsync(dus, us.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, s));
    BFC_CUDA(cudaMemcpyAsync(dls, ls.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, s));
    BFC_CUDA(cudaMemcpyAsync(des, es.data(), sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice, s));
    {
        int64_t work = std::max<int64_t>(es[G], us[G]);
        int blocks = (int)std::min<int64_t>((work + 255) / 256, 152 * 32);
        if (blocks < 1) blocks = 1;
        k_union_fixup<<<blocks, 256, 0, s>>>(off, adj, des, dus, dls, G, us[G], es[G]);
        note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    bfc_csr csr{us[G], ls[G], es[G], off, adj};
    bfc_batch b{G, dus, dls};
    bfc_options opt;
    bfc_options_init(&opt);
    opt.warp_max_work = sv->cfg.warp_max_work > 0 ? sv->cfg.warp_max_work : opt.warp_max_work;
    opt.hash_max_work = sv->cfg.hash_max_work > 0 ? sv->cfg.hash_max_work : opt.hash_max_work;
    opt.team_max_work = sv->cfg.team_max_work > 0 ? sv->cfg.team_max_work : opt.team_max_work;
    bfc_graph *h = nullptr;
    int rc = bfc_prepare_batch(&csr, &b, &opt, s, &h);
    if (rc) return rc;
    rc = bfc_count_batch(h, s, reinterpret_cast<uint64_t *>(dtot), nullptr);
    if (rc == BFC_OK) {
        totals.assign(G, 0);
        cudaError_t e = cudaMemcpyAsync(totals.data(), dtot, sizeof(uint64_t) * G,
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(D2H totals)");
    }
    if (rc == BFC_OK) rc = bfc_sync(h, s);
    bfc_release(h);
    cudaStreamSynchronize(s);
    return rc;
}

// A batch that failed as a whole because one graph broke the contract (a
// duplicate edge, found by prepare's validation) is counted again graph by
// graph, so that only the offending request fails.
int run_batch_or_each(bfc_server *sv, std::vector<Request *> &batch, cudaStream_t s,
                      std::vector<uint64_t> &totals, std::vector<int> &status) {
    int rc = run_batch(sv, batch, s, totals);
    status.assign(batch.size(), rc);
    if (rc != BFC_ERR_INVALID_GRAPH || batch.size() < 2) return rc;
    totals.assign(batch.size(), 0);
    std::vector<uint64_t> one;
    for (size_t i = 0; i < batch.size(); ++i) {
        std::vector<Request *> single{batch[i]};
        status[i] = run_batch(sv, single, s, one);
        if (status[i] == BFC_OK) totals[i] = one[0];
    }
    return BFC_OK;
}

void worker_main(bfc_server *sv, cudaStream_t s) {
    cudaSetDevice(sv->device);
    std::vector<uint64_t> totals;
    std::vector<int> status;
    for (;;) {
        std::vector<Request *> batch;
        int64_t bytes = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            // admit the oldest waiting requests that fit the budget and the batch limits
            for (;;) {
                if (sv->stop) break;
                if (!sv->waiting.empty() &&
                    sv->bytes_in_use + sv->waiting.front()->bytes <= sv->cfg.memory_budget_bytes)
                    break;
                sv->cv_work.wait(lk);
            }
            if (sv->stop && sv->waiting.empty()) break;
            if (sv->stop && sv->bytes_in_use + sv->waiting.front()->bytes > sv->cfg.memory_budget_bytes) break;
            int64_t edges = 0, verts = 0;
            while (!sv->waiting.empty() && (int32_t)batch.size() < sv->cfg.max_batch_graphs) {
                Request *q = sv->waiting.front();
                if (sv->bytes_in_use + bytes + q->bytes > sv->cfg.memory_budget_bytes) break;
                if (!batch.empty() && edges + q->m > sv->cfg.max_batch_edges) break;
                // the union's ids and CSR offsets stay in int32 (each request alone does)
                if (!batch.empty() && (verts + q->r + q->l > kUnionMax || edges + q->m > kUnionMax))
                    break;
                sv->waiting.pop_front();
                batch.push_back(q);
                bytes += q->bytes;
                edges += q->m;
                verts += q->r + q->l;
            }
            sv->bytes_in_use += bytes;
            if (sv->bytes_in_use > sv->stats.peak_bytes_in_use) sv->stats.peak_bytes_in_use = sv->bytes_in_use;
            sv->stats.batches += 1;
            if ((int64_t)batch.size() > sv->stats.max_batch_graphs) sv->stats.max_batch_graphs = (int64_t)batch.size();
        }
        run_batch_or_each(sv, batch, s, totals, status);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->bytes_in_use -= bytes;
        }
        sv->cv_work.notify_all();
        complete(sv, batch, status, totals);
    }
}

}  // namespace
}  // namespace bfc

extern "C" {

void bfc_server_config_init(bfc_server_config *c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->memory_budget_bytes = 120ll << 30;
    c->workers = 2;
    c->max_batch_graphs = 1024;
    c->max_batch_edges = 64ll << 20;
}

int bfc_server_create(const bfc_server_config *cfg, bfc_server **out) {
    bfc::set_last_error("");
    if (!out) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    *out = nullptr;
    bfc_server_config c;
    if (cfg) c = *cfg; else bfc_server_config_init(&c);
    if (c.workers < 1 || c.workers > 16 || c.max_batch_graphs < 1 || c.memory_budget_bytes <= 0 ||
        c.max_batch_edges < 1 || c.max_batch_edges > bfc::kUnionMax) {
        bfc::set_last_error("invalid server configuration");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    bfc_server *sv = new (std::nothrow) bfc_server();
    if (!sv) { bfc::set_last_error("host allocation failed"); return BFC_ERR_OUT_OF_MEMORY; }
    sv->cfg = c;
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e != cudaSuccess) { delete sv; return bfc::cuda_fail(e, "cudaGetDevice"); }
    int rc = bfc::count_smem_setup(sv->device);   // before any worker launches
    if (rc) { delete sv; return rc; }
    // every worker's stream exists before any worker starts: a server that
    // could not start all its workers is not created, so no request can wait
    // for a worker that is not there
    for (int i = 0; i < c.workers; ++i) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
            delete sv;
            return bfc::cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        sv->streams.push_back(st);
    }
    // the pool's real high-water mark is tracked from here (stats)
    int64_t cur = 0;
    e = bfc::pool_usage(&cur, nullptr, true);
    if (e != cudaSuccess) {
        for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
        delete sv;
        return bfc::cuda_fail(e, "cudaMemPoolSetAttribute(UsedMemHigh)");
    }
    sv->stats.pool_bytes_at_create = cur;
    for (int i = 0; i < c.workers; ++i) sv->workers.emplace_back(bfc::worker_main, sv, sv->streams[i]);
    *out = sv;
    return BFC_OK;
}

int bfc_server_submit(bfc_server *sv, int32_t num_u, int32_t num_l, int64_t num_edges,
                      const int32_t *off_u_host, const int32_t *adj_u_host, uint64_t *request_id) {
    bfc::set_last_error("");
    if (!sv || !off_u_host || (num_edges > 0 && !adj_u_host) || !request_id || num_u < 0 ||
        num_l < 0 || num_edges < 0 || num_edges > 2147483647LL) {
        bfc::set_last_error("invalid request");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (!bfc::host_csr_ok(num_u, num_l, num_edges, off_u_host, adj_u_host)) {
        bfc::set_last_error("request is not a CSR of num_edges entries with ids in [0, num_l)");
        return BFC_ERR_INVALID_GRAPH;
    }
    if ((int64_t)num_u + num_l > bfc::kUnionMax) {
        bfc::set_last_error("request too large for int32 vertex ids");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    bfc::Request *q = new (std::nothrow) bfc::Request();
    if (!q) { bfc::set_last_error("host allocation failed"); return BFC_ERR_OUT_OF_MEMORY; }
    q->r = num_u; q->l = num_l; q->m = num_edges; q->off = off_u_host; q->adj = adj_u_host;
    q->bytes = bfc::batch_bytes(num_u, num_l, num_edges);
    q->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (q->bytes > sv->cfg.memory_budget_bytes) {
        delete q;
        bfc::set_last_error("request exceeds the server's memory budget on its own");
        return BFC_ERR_OUT_OF_MEMORY;
    }
    q->id = sv->next_id++;
    sv->all[q->id] = q;
    sv->waiting.push_back(q);
    sv->stats.submitted += 1;
    *request_id = q->id;
    sv->cv_work.notify_one();
    return BFC_OK;
}

int bfc_server_poll(bfc_server *sv, uint64_t request_id, int wait, uint64_t *total, int *status,
                    double *latency_s) {
    if (!sv || !status) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(request_id);
    if (it == sv->all.end()) { bfc::set_last_error("unknown request id"); return BFC_ERR_INVALID_ARGUMENT; }
    bfc::Request *q = it->second;
    if (wait) sv->cv_done.wait(lk, [q] { return q->status >= 0; });
    *status = q->status;
    if (q->status >= 0) {
        if (total) *total = q->total;
        if (latency_s)
            *latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
        sv->all.erase(it);
        delete q;
    }
    return BFC_OK;
}

int bfc_server_get_stats(bfc_server *sv, bfc_server_stats *out) {
    if (!sv || !out) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    int64_t cur = 0, high = 0;
    cudaError_t e = bfc::pool_usage(&cur, &high, false);
    if (e != cudaSuccess) return bfc::cuda_fail(e, "cudaMemPoolGetAttribute");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->bytes_in_use = sv->bytes_in_use;
    out->waiting = (int64_t)sv->waiting.size();
    out->pool_bytes_high = high;
    return BFC_OK;
}

void bfc_server_destroy(bfc_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers) t.join();
    for (cudaStream_t x : sv->streams) cudaStreamDestroy(x);
    {
        // requests never admitted are cancelled
        std::lock_guard<std::mutex> lk(sv->mu);
        for (bfc::Request *q : sv->waiting) {
            q->status = BFC_ERR_INTERNAL;
            sv->stats.failed += 1;
        }
        sv->waiting.clear();
        sv->cv_done.notify_all();
    }
    for (auto &kv : sv->all) delete kv.second;
    delete sv;
}

}  // extern "C"
