// Derived statistics of Section 1's applications, computed on the prepared
// graph G*: the caterpillars (three-paths) of the bipartite clustering
// coefficient 4·⋈_G / caterpillars.  A three-path a-b-c-d is fixed by its
// middle edge (b, c) and one more neighbour at each end, so the count is
// Σ over edges (deg b − 1)(deg c − 1); G* keeps every degree as a list length.
#include "bfc_internal.cuh"

#include <algorithm>

namespace bfc {
const Graph *graph_of_handle(const bfc_graph *h);   // api.cu

namespace {

// one warp per U vertex x of G* (ids l..n-1): its list holds each edge once
__global__ void k_caterpillars(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                               int32_t l, int32_t n, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long sum = 0;
    for (int64_t x = l + w0; x < n; x += nw) {
        const int64_t b = off[x], e = off[x + 1];
        const unsigned long long dx1 = (unsigned long long)(e - b) - 1ull;
        for (int64_t k = b + lane; k < e; k += 32) {
            const int32_t v = adj[k];
            sum += dx1 * (unsigned long long)(off[v + 1] - off[v] - 1);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (lane == 0 && sum) atomicAdd(out, sum);
}

// coefficient = 4·⋈_G / caterpillars, 0 when the graph has no three-path
__global__ void k_clustering(const unsigned long long *butterflies,
                             const unsigned long long *caterpillars, double *coefficient) {
    const unsigned long long c = *caterpillars;
    *coefficient = c ? 4.0 * (double)*butterflies / (double)c : 0.0;
}

}  // namespace
}  // namespace bfc

extern "C" int bfc_clustering_coefficient(bfc_graph *h, void *stream, const uint64_t *butterflies_dev,
                                          uint64_t *caterpillars_dev, double *coefficient_dev) {
    if (!h || !butterflies_dev || !caterpillars_dev || !coefficient_dev) {
        bfc::set_last_error("null argument");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    const int rc = bfc_caterpillars(h, stream, caterpillars_dev);
    if (rc) return rc;
    bfc::k_clustering<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const unsigned long long *>(butterflies_dev),
        reinterpret_cast<const unsigned long long *>(caterpillars_dev), coefficient_dev);
    bfc::note_launch();
    BFC_CUDA(cudaGetLastError());
    return BFC_OK;
}

extern "C" int bfc_caterpillars(bfc_graph *h, void *stream, uint64_t *caterpillars_dev) {
    bfc::set_last_error("");
    if (!h || !caterpillars_dev) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    const bfc::Graph *g = bfc::graph_of_handle(h);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BFC_CUDA(cudaMemsetAsync(caterpillars_dev, 0, sizeof(uint64_t), s));
    if (g->m > 0) {
        const int64_t warps = std::min<int64_t>(g->r, 152 * 64);
        bfc::k_caterpillars<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(
            g->off, g->adj, g->l, g->n, reinterpret_cast<unsigned long long *>(caterpillars_dev));
        bfc::note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    return BFC_OK;
}
