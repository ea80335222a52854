// The pair formulation of Section 6.3 (the external-memory algorithm's
// wedge pairs, run in device memory), a second exact way to the total.
//
// Every wedge (x, v, w) that the prepared orientation processes (Algorithm
// 2: x highest; Algorithm 3: w highest) becomes the 64-bit key (x, w).  A
// radix sort brings equal keys together; a run of c equal keys is the pair
// (x, w) with count_wedge = c, which holds C(c, 2) butterflies (Lemma 1), and
// by Lemma 4 / Theorem 1 every butterfly is counted by exactly one pair.
// With the run start s(i) of position i (a max-scan of the run heads),
// Σ_i (i - s(i)) = Σ_runs (0 + 1 + ... + c - 1) = Σ_runs C(c, 2).
//
// The counter walk of count.cu reads each end once; this path writes and
// sorts 8·W bytes of keys, so it is the slower exact path (kept as a check of
// the walk and for its own sake).
#include <algorithm>

#include "bfc_internal.cuh"

namespace bfc {
const Graph *graph_of_handle(const bfc_graph *h);   // api.cu

namespace {

constexpr int kT = 256;

unsigned blocks(int64_t n) {
    return (unsigned)std::min<int64_t>(std::max<int64_t>((n + kT - 1) / kT, 1), 152 * 64);
}

__global__ void k_pair_counts(const int32_t *__restrict__ plen, int64_t slots, int64_t *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < slots;
         e += (int64_t)gridDim.x * blockDim.x)
        cnt[e] = plen[e];
}

// one warp per start x: for each of its middle slots, the slot's run of ends
// becomes keys (x, w) at the slot's offset
__global__ void k_pair_emit(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                            const int32_t *__restrict__ cut, const int32_t *__restrict__ plen,
                            const int64_t *__restrict__ sbeg, const int64_t *__restrict__ out_off,
                            int32_t n, int orient, int bn, uint64_t *keys, int32_t *vals) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = w0; x < n; x += nw) {
        const int64_t e0 = off[x];
        const int64_t nmid = orient ? off[x + 1] - e0 : (int64_t)cut[x];
        const uint64_t hi = (uint64_t)x << bn;
        for (int64_t e = e0; e < e0 + nmid; ++e) {
            const int32_t len = plen[e];
            const int64_t src = sbeg[e], dst = out_off[e];
            for (int32_t i = lane; i < len; i += 32) {
                keys[dst + i] = hi | (uint64_t)(uint32_t)adj[src + i];
                vals[dst + i] = 0;
            }
        }
    }
}

// run heads: position i where a new key starts (else 0, below every head)
__global__ void k_pair_heads(const uint64_t *__restrict__ keys, int64_t n, int64_t *heads) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        heads[i] = (i == 0 || keys[i] != keys[i - 1]) ? i : 0;
}

// Σ_i (i - s(i)): each run of c keys adds 0 + 1 + ... + (c - 1) = C(c, 2)
__global__ void k_pair_sum(const int64_t *__restrict__ start, int64_t n, unsigned long long *total) {
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += (unsigned long long)(i - start[i]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

}  // namespace
}  // namespace bfc

extern "C" int bfc_count_pairs(bfc_graph *h, void *stream, uint64_t *total_dev) {
    bfc::set_last_error("");
    if (!h || !total_dev) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    const bfc::Graph *g = bfc::graph_of_handle(h);
    if (g->num_graphs > 0) { bfc::set_last_error("a batch: use bfc_count_batch"); return BFC_ERR_INVALID_ARGUMENT; }
    const uint64_t W = g->info.wedges;
    if (W >= 0xFFFFFFFFull) {
        bfc::set_last_error("the pair formulation sorts at most 2^32 - 1 pairs");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *tot = reinterpret_cast<unsigned long long *>(total_dev);
    BFC_CUDA(cudaMemsetAsync(tot, 0, sizeof(unsigned long long), s));
    if (W < 2) return BFC_OK;
    const int64_t slots = 2 * g->m, n = (int64_t)W;
    const int bn = bfc::bits_for((uint64_t)(g->n - 1));
    bfc::Allocs a;
    a.stream = s;
    struct Guard { bfc::Allocs *a; ~Guard() { a->release(); } } guard{&a};
    uint64_t *k0, *k1;
    int32_t *v0, *v1;
    uint32_t *hist, *hist_tmp;
    int64_t *cnt, *out_off, *scan_tmp, *mtmp;
    if (a.get(&k0, n) || a.get(&k1, n) || a.get(&v0, n) || a.get(&v1, n) ||
        a.get(&hist, bfc::radix_hist_elems(n)) ||
        a.get(&hist_tmp, bfc::scan_tmp_elems<uint32_t>((int64_t)bfc::radix_hist_elems(n))) ||
        a.get(&cnt, slots + 1) || a.get(&out_off, slots + 1) ||
        a.get(&scan_tmp, bfc::scan_tmp_elems<int64_t>(slots + 1)) ||
        a.get(&mtmp, bfc::max_scan_i64_tmp_elems(n))) {
        bfc::set_last_error("device allocation failed: pair keys (24 bytes per wedge)");
        return BFC_ERR_OUT_OF_MEMORY;
    }
    // each middle slot's output offset: exclusive scan of the run lengths
    bfc::k_pair_counts<<<bfc::blocks(slots), bfc::kT, 0, s>>>(g->plen, slots, cnt);
    bfc::note_launch();
    BFC_CUDA(cudaGetLastError());
    BFC_CUDA(bfc::scan_exclusive<int64_t>(cnt, out_off, slots, scan_tmp, s));
    bfc::k_pair_emit<<<bfc::blocks((int64_t)g->n * 32), bfc::kT, 0, s>>>(
        g->off, g->adj, g->cut, g->plen, g->sbeg, out_off, g->n, g->opt.orientation, bn, k0, v0);
    bfc::note_launch();
    BFC_CUDA(cudaGetLastError());
    int which = 0;
    BFC_CUDA(bfc::radix_sort_pairs(k0, v0, k1, v1, n, 0, 2 * bn, hist, hist_tmp, s, &which));
    const uint64_t *keys = which ? k1 : k0;
    // the other key buffer holds the run heads and then the run starts
    int64_t *heads = reinterpret_cast<int64_t *>(which ? k0 : k1);
    bfc::k_pair_heads<<<bfc::blocks(n), bfc::kT, 0, s>>>(keys, n, heads);
    bfc::note_launch();
    BFC_CUDA(cudaGetLastError());
    BFC_CUDA(bfc::max_scan_inclusive_i64(heads, heads, n, mtmp, s));
    bfc::k_pair_sum<<<bfc::blocks(n), bfc::kT, 0, s>>>(heads, n, tot);
    bfc::note_launch();
    BFC_CUDA(cudaGetLastError());
    return BFC_OK;
}
