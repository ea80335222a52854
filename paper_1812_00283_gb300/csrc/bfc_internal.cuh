// Internal declarations of libbfc (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "bfc.h"

namespace bfc {

// ---------------------------------------------------------------------------
// Sizes
// ---------------------------------------------------------------------------
constexpr int kCountCtasPerSm = 1;                        // persistent count CTAs per SM
constexpr int kCountThreads = 1024 / kCountCtasPerSm;     // 32 warps per SM
constexpr int kCountWarps = kCountThreads / 32;
constexpr int kCounterBytes = 192 * 1024 / kCountCtasPerSm;  // dynamic shared memory for counters
constexpr int kDense16 = kCounterBytes / 2;               // 98,304 packed 16-bit counters
constexpr int kDense32 = kCounterBytes / 4;               // 49,152 32-bit counters
constexpr int kHashMaxSlots = 32768 / kCountCtasPerSm;    // CTA hash: 128 KB keys + 64 KB counts
constexpr int kHashMaxWork = kHashMaxSlots / 4 * 3;       // 24,576 wedges: at most 3/4 of the slots fill
constexpr int kWarpRegion = kCounterBytes / kCountWarps;  // 6 KB of counters per warp
constexpr int kWarpSlots = 512;                           // warp hash: 2 KB keys + 2 KB counts
constexpr int kWarpMaxWork = kWarpSlots / 4 * 3;          // 384 wedges: at most 3/4 of the slots fill
constexpr int kTeamThreads = 256;                         // a team: 8 warps with a named barrier
constexpr int kTeams = kCountThreads / kTeamThreads;      // 4 teams per CTA
constexpr int kTeamRegion = kCounterBytes / kTeams;       // 48 KB of shared memory per team
constexpr int kTeamSlots = 4096;                          // team hash: 16 KB keys + 8 KB counts
constexpr int kTeamFitWork = kTeamSlots / 4 * 3;          // 3,072: a start this light always fits a team table
constexpr int kTeamMaxWork = 16384;                       // upper limit of team_max_work
constexpr uint32_t kNarrowMaxCut = 65535;                 // counts fit 16 bits when cut <= this
constexpr int kDense8 = kCounterBytes;                    // 196,608 packed 8-bit counters
constexpr uint32_t kByteMaxCut = 255;                     // counts fit 8 bits when cut <= this
constexpr int kDense4 = kCounterBytes * 2;                // 393,216 packed 4-bit counters
constexpr uint32_t kNibbleMax = 15;                       // counts fit 4 bits when at most this
constexpr int kChunkUnit = kDense32;                      // end-range chunk unit of the boundary table
static_assert(kDense16 % kChunkUnit == 0, "narrow chunks must be whole table units");
static_assert(kDense8 % kChunkUnit == 0, "byte chunks must be whole table units");
static_assert(kDense4 % kChunkUnit == 0, "nibble chunks must be whole table units");
// the end-range chunk of a dense start whose counts are at most `bound` (its
// middles): 32-bit, 16-bit or 8-bit counters in the same shared memory
__host__ __device__ constexpr int32_t dense_chunk_span(int64_t bound) {
    return bound > (int64_t)kNarrowMaxCut ? kDense32 : (bound > (int64_t)kByteMaxCut ? kDense16 : kDense8);
}
// Algorithm 2's dense chunk of start x that begins at end offset lo (a
// multiple of kChunkUnit) of its end range [lb, lb + R) in G*: the widest span
// whose counters hold every count in it.  count_wedge(x, w) is at most
// min(cut[x], deg(w)), and within a layer G* orders vertices by Definition 3's
// priority, so degrees do not decrease with the id and the chunk's last end
// bounds every count of the chunk.  Returns the chunk's end; *bits = 4, 8, 16
// or 32.  `off` is G*'s offset array.
__device__ __forceinline__ int32_t dense_chunk_end(int32_t lo, int32_t R, int64_t cut, const int64_t *off,
                                                   int32_t lb, int *bits) {
    int32_t hi = (int32_t)((int64_t)lo + kDense4 < R ? lo + kDense4 : R);
    int64_t top = off[lb + hi] - off[lb + hi - 1];
    if ((cut < top ? cut : top) <= (int64_t)kNibbleMax) { *bits = 4; return hi; }
    hi = (int32_t)((int64_t)lo + kDense8 < R ? lo + kDense8 : R);
    top = off[lb + hi] - off[lb + hi - 1];
    if ((cut < top ? cut : top) <= (int64_t)kByteMaxCut) { *bits = 8; return hi; }
    hi = (int32_t)((int64_t)lo + kDense16 < R ? lo + kDense16 : R);
    top = off[lb + hi] - off[lb + hi - 1];
    if ((cut < top ? cut : top) <= (int64_t)kNarrowMaxCut) { *bits = 16; return hi; }
    *bits = 32;
    return (int32_t)((int64_t)lo + kDense32 < R ? lo + kDense32 : R);
}
constexpr int64_t kChunkTableMaxEntries = 1ll << 29;      // 2 GB of int32 at most

// device error bits (graph-owned error word)
constexpr int kErrBadOffsets = 1;
constexpr int kErrBadId = 2;
constexpr int kErrDuplicate = 4;
constexpr int kErrHashFull = 8;
constexpr int kErrBounds = 16;
constexpr int kErrTimeout = 32;   // a bounded device wait gave up

// ---------------------------------------------------------------------------
// Host-side error reporting
// ---------------------------------------------------------------------------
void set_last_error(const std::string &msg);
// Counts kernel launches made by the library (reported by bfc_kernel_launches).
void note_launch();
int cuda_fail(cudaError_t e, const char *what);

#define BFC_CUDA(call)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return ::bfc::cuda_fail(e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// Stream-ordered allocations from the library's pool
// ---------------------------------------------------------------------------
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);
// Bytes of the current device's pool in use now and its high-water mark
// (reset to zero first when reset_high).
cudaError_t pool_usage(int64_t *current, int64_t *high, bool reset_high);

// A list of pool allocations released together.
struct Allocs {
    static constexpr int kMax = 64;
    void *ptr[kMax];
    size_t bytes[kMax];
    int n = 0;
    size_t total = 0;
    cudaStream_t stream = nullptr;
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        if (n >= kMax) return cudaErrorMemoryAllocation;
        size_t b = count * sizeof(T);
        if (b == 0) b = 16;
        b = (b + 255) & ~size_t(255);
        void *q = nullptr;
        cudaError_t e = pool_alloc(&q, b, stream);
        if (e != cudaSuccess) return e;
        ptr[n] = q;
        bytes[n] = b;
        ++n;
        total += b;
        *p = static_cast<T *>(q);
        return cudaSuccess;
    }
    // frees one allocation of the list (no-op for null or unknown pointers)
    void drop(void *p) {
        if (!p) return;
        for (int i = 0; i < n; ++i)
            if (ptr[i] == p) {
                pool_free(p, stream);
                total -= bytes[i];
                for (int j = i + 1; j < n; ++j) { ptr[j - 1] = ptr[j]; bytes[j - 1] = bytes[j]; }
                --n;
                return;
            }
    }
    void release() {
        for (int i = n - 1; i >= 0; --i) pool_free(ptr[i], stream);
        n = 0;
        total = 0;
    }
};

// ---------------------------------------------------------------------------
// The prepared graph
// ---------------------------------------------------------------------------
struct Graph {
    int32_t r = 0, l = 0, n = 0;
    int64_t m = 0;
    bfc_options opt{};
    bfc_info info{};
    cudaStream_t stream = nullptr;   // stream of the last call (for stream-ordered release)
    int device = 0;
    int num_sms = 0;
    int grid = 0;

    Allocs mem;          // everything below lives in `mem`
    int32_t *rank_u = nullptr, *rank_l = nullptr;  // original id -> rank in layer
    int64_t *off = nullptr;   // [n+1] CSR of G*
    int32_t *adj = nullptr;   // [2m]
    int32_t *eid = nullptr;   // [2m]
    int32_t *plen = nullptr;  // [2m] wedges through each middle slot (0 if not a middle slot)
    int32_t *cut = nullptr;   // [n]
    uint64_t *work = nullptr; // [n]
    int2 *cta_items = nullptr;    // (start, chunk) / (start, -1 = hash)
    int32_t *team_items = nullptr;
    int32_t *warp_items = nullptr;
    int64_t n_cta_items = 0, n_team_items = 0, n_warp_items = 0;
    int32_t team_max = 0;          // effective team bound of the current schedule
    bool may_retry = false;        // the schedule can re-queue starts (retry pass launched)
    int *cursors = nullptr;        // [8] work-queue cursors of the count kernels
    unsigned long long *acc = nullptr;  // [1] device accumulator for ⋈_G
    unsigned long long *pv = nullptr;   // [n] per-vertex scratch in G* ids (allocated on demand? no: in prepare)
    int *err = nullptr;            // device error word
    // chunk-boundary table: for vertex v of G*, entry c is the position in
    // N(v) of the first neighbour whose rank in its layer is >= c * kChunkUnit
    int32_t *coff = nullptr;
    int64_t *coff_start = nullptr;   // a batch's table while it is built: first entry of each vertex
    int32_t *ctb = nullptr;          // a batch's table: first entry of each slot's middle (-1: none)
    int32_t coff_u1 = 0;   // entries per L vertex (its neighbours are U vertices)
    int32_t coff_l1 = 0;   // entries per U vertex
    // batch of graphs prepared as one disjoint union
    int32_t num_graphs = 0;
    int32_t *gstar = nullptr;             // [n] graph of each vertex of G*
    int32_t *vbase = nullptr;             // [n] first G* id of x's graph in x's layer
    int32_t *vend = nullptr;              // [n] one past the last G* id of x's graph in x's layer
    // per middle slot e = (x, v), the run of N(v) holding the ends starts at
    // sbeg[e] and has plen[e] entries: the prefix below x (Algorithm 2) or the
    // suffix above both x and v (Algorithm 3)
    int64_t *sbeg = nullptr;
    // starts re-queued for the retry pass: x (its team table filled up: try a
    // CTA table) or -(x+1) (count with dense chunks)
    int32_t *retry = nullptr;
    int64_t retry_static = 0;             // of which assigned there by prepare
    int64_t retry_cap = 0;
    unsigned long long *gwork = nullptr;  // [num_graphs] wedges per graph
    // per-edge sums by G* slot [2m], taken from the pool by the first
    // per-edge count and kept until release
    unsigned long long *pe_slot = nullptr;
    // dense high-priority core counted by a product (total counts only):
    // core_u / core_l vertices at the top of each layer's ids, starting at
    // core_lo_u / core_lo_l; ccut[x] = neighbours of core vertex x outside the
    // other layer's core; B and Bm of both cores (bf16 bits, padded to
    // core_ld_* = multiples of 128); the products a(u, w) as uint16; per row
    // tile the contraction length in 64-column blocks; TMA maps of Bm and B
    int32_t core_u = 0, core_l = 0, core_lo_u = 0, core_lo_l = 0, core_ld_u = 0, core_ld_l = 0;
    int32_t *ccut = nullptr;
    uint16_t *core_bu = nullptr, *core_bum = nullptr, *core_bl = nullptr, *core_blm = nullptr;
    uint16_t *core_au = nullptr, *core_al = nullptr;
    int32_t *core_kb_u = nullptr, *core_kb_l = nullptr;
    alignas(64) unsigned char core_map_bytes[4][128];
    // batch plan: the bin sizes in device memory ([0] dense, [1] hash,
    // [2] team, [3] warp starts; null for graphs prepared by prepare_graph)
    unsigned long long *item_counts = nullptr;
};

// ---------------------------------------------------------------------------
// Primitives (scan_sort.cu)
// ---------------------------------------------------------------------------
// Exclusive prefix sum of n elements; writes n+1 outputs (out[n] = total).
// `tmp` must hold scan_tmp_elems(n) elements of T.
template <typename T>
size_t scan_tmp_elems(int64_t n);
template <typename T>
cudaError_t scan_exclusive(const T *in, T *out, int64_t n, T *tmp, cudaStream_t s);
// Inclusive running maximum (int32).
size_t max_scan_tmp_elems(int64_t n);
cudaError_t max_scan_inclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp,
                               cudaStream_t s);

// The same for int64 (pairs formulation: run starts of up to 2^32 keys).
size_t max_scan_i64_tmp_elems(int64_t n);
cudaError_t max_scan_inclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp,
                                   cudaStream_t s);

// Stable LSD radix sort of (uint64 key, int32 value) pairs on key bits
// [begin_bit, end_bit).  Ping-pongs between (k0, v0) and (k1, v1); returns
// 0 if the result is in (k0, v0), 1 if in (k1, v1).  `hist` needs
// radix_hist_elems(n) uint32 and `scan_tmp` scan_tmp_elems<uint32_t>(..).
size_t radix_hist_elems(int64_t n);
cudaError_t radix_sort_pairs(uint64_t *k0, int32_t *v0, uint64_t *k1, int32_t *v1, int64_t n,
                             int begin_bit, int end_bit, uint32_t *hist, uint32_t *scan_tmp,
                             cudaStream_t s, int *which);

// Device-wide max / sum reductions into one element (result in device memory).
cudaError_t reduce_max_i32(const int32_t *in, int64_t n, int32_t *out, cudaStream_t s);
cudaError_t reduce_max_u64(const uint64_t *in, int64_t n, unsigned long long *out, cudaStream_t s);

// ---------------------------------------------------------------------------
// Prepare and count (prepare.cu, count.cu)
// ---------------------------------------------------------------------------
int prepare_graph(const bfc_csr *csr, const bfc_options *opt, cudaStream_t s, Graph *g,
                  int32_t num_graphs = 0, const int32_t *graph_u_start = nullptr,
                  const int32_t *graph_l_start = nullptr);
// kModeBatch = total plus per-graph totals for a batch prepared as a disjoint union;
// kModeAll = per-vertex and per-edge counts from one first walk and one second walk
enum CountMode { kModeTotal = 0, kModeVertices = 1, kModeEdges = 2, kModeBatch = 3, kModeAll = 4 };
__host__ __device__ constexpr bool wants_vertices(int mode) { return mode == kModeVertices || mode == kModeAll; }
__host__ __device__ constexpr bool wants_edges(int mode) { return mode == kModeEdges || mode == kModeAll; }
__host__ __device__ constexpr bool has_second_walk(int mode) { return wants_vertices(mode) || wants_edges(mode); }
int launch_count(Graph *g, cudaStream_t s, int mode, unsigned long long *pv_proj,
                 unsigned long long *pe, unsigned long long *gtot = nullptr);
int rebin_graph(Graph *g, cudaStream_t s, int32_t warp_max_work, int32_t team_max_work,
                int32_t hash_max_work);
int count_smem_setup(int device);

// A batch of a fixed shape prepared and counted without host synchronisation
// or allocation (prepare.cu): every array is allocated by batch_plan_create.
struct BatchPlan {
    Graph g;                       // the prepared arrays, rewritten by every run
    int32_t r = 0, l = 0, num_graphs = 0, max_layer = 0;
    int64_t m = 0;
    uint64_t team_max = 0;         // team bin bound (at most 3,072: no retry pass)
    uint64_t *k0 = nullptr, *k1 = nullptr;
    int32_t *v0 = nullptr, *v1 = nullptr, *deg_u = nullptr, *deg_l = nullptr, *deg_star = nullptr;
    int32_t *rows = nullptr, *heads = nullptr, *rows_star = nullptr, *tier_rows = nullptr, *tier_n = nullptr;
    uint32_t *hist = nullptr, *hist_tmp = nullptr;
    int64_t *scan64_tmp = nullptr, *deg64 = nullptr;
    unsigned long long *red = nullptr;   // [0] W, [4..8) bin sizes
};
int batch_plan_create(BatchPlan *pl, cudaStream_t s);
int batch_plan_run(BatchPlan *pl, const int32_t *off_u, const int32_t *adj_u, const int32_t *gu,
                   const int32_t *gl, cudaStream_t s, unsigned long long *totals, int32_t *status);
// the dense-core hybrid (core.cu): core choice and matrices in prepare, the
// masked products before a total count
int core_prepare(Graph *g, cudaStream_t s, const int32_t *deg_star, int32_t core_vertices,
                 bool automatic);
// the automatic core size is at most this many vertices (the product grows as
// K^3), and is used only when each layer holds at least kCoreAutoMinLayer
constexpr int32_t kCoreAutoMax = 8192;
constexpr int32_t kCoreAutoMinLayer = 1024;
int core_product(Graph *g, cudaStream_t s);

// small helpers
inline int bits_for(uint64_t x) {  // bits needed to represent x (0 for x = 0)
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

}  // namespace bfc
