// Steps a1-a5 of the hot path: degrees, priority ranks, the projection
// graph G* with priority-sorted neighbour lists, the per-start orientation
// cut and exact wedge work, and the degree-binned schedule.
//
// Paper: Definition 3 (priority), Definition 4 (projection, Section 5.2),
// Section 4 (neighbour lists sorted by priority, early termination; the bin
// sort of Theorem 2's proof), Section 6.2 (workload of a start vertex and
// heaviest-first dynamic scheduling, Eq. 5).
#include <algorithm>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {

namespace {

constexpr int kT = 256;

inline unsigned blocks_for(int64_t n, int t = kT) {
    int64_t b = (n + t - 1) / t;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// A prepared batch run without host synchronisation (the batch plan) checks
// the caller's CSR on the device; every later kernel of that run is given
// the error word and returns at once when the CSR failed the checks, so no
// kernel indexes with unchecked input.  Elsewhere the word is null.
__device__ __forceinline__ bool aborted(const int *guard) {
    return guard && (*(volatile const int *)guard & (kErrBadOffsets | kErrBadId));
}

// ----- validation (always on: every later index depends on it) -------------
__global__ void k_check_offsets(const int32_t *__restrict__ off, int32_t r, int64_t m, int *err) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > r) return;
    if (u == 0 && off[0] != 0) atomicOr(err, kErrBadOffsets);
    if (u < r && off[u + 1] < off[u]) atomicOr(err, kErrBadOffsets);
    if (u == r && (int64_t)off[r] != m) atomicOr(err, kErrBadOffsets);
}

__global__ void k_check_ids(const int32_t *__restrict__ adj, int64_t m, int32_t l, int *err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = adj[k];
        if (v < 0 || v >= l) atomicOr(err, kErrBadId);
    }
}

// ----- a1: degrees -----------------------------------------------------------
__global__ void k_deg_u(const int32_t *__restrict__ off, int32_t r, int32_t *deg_u,
                        int32_t *heads,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= r) return;
    int32_t d = off[u + 1] - off[u];
    deg_u[u] = d;
    if (heads && d > 0) heads[off[u]] = (int32_t)u;   // row owning slot off[u]; rows via max-scan
}

__global__ void k_deg_l(const int32_t *__restrict__ adj, int64_t m, int32_t *deg_l,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg_l[adj[k]], 1);
}

// ----- a2: priority ranks ----------------------------------------------------
// keys = degree, values = vertex id (ascending), so a stable sort by degree
// orders each layer by (deg, id): Definition 3 restricted to one layer.
__global__ void k_iota_keys(const int32_t *__restrict__ deg, int32_t n, uint64_t *keys,
                            int32_t *vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = (uint64_t)(uint32_t)deg[i];
    vals[i] = (int32_t)i;
}

// batch of graphs: rank graph-major (graph id above the degree bits), so each
// graph's vertices keep Definition 3's order among themselves and occupy the
// contiguous rank range [start[g], start[g+1]) of their layer
__global__ void k_iota_keys_batch(const int32_t *__restrict__ deg, int32_t n,
                                  const int32_t *__restrict__ start, int32_t num_graphs, int bdeg,
                                  uint64_t *keys, int32_t *vals,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t lo = 0, hi = num_graphs;
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (start[mid] <= (int32_t)i) lo = mid; else hi = mid;
    }
    keys[i] = ((uint64_t)lo << bdeg) | (uint64_t)(uint32_t)deg[i];
    vals[i] = (int32_t)i;
}

// rank[order[i]] = i; degree of G* vertex (base + i) = sorted key
__global__ void k_ranks(const uint64_t *__restrict__ sorted_deg, const int32_t *__restrict__ order,
                        int32_t n, int32_t *rank, int32_t *deg_star, int32_t base, uint64_t deg_mask,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rank[order[i]] = (int32_t)i;
    deg_star[base + i] = (int32_t)(sorted_deg[i] & deg_mask);   // low bits: the degree
}

// ----- a3: projection + sorted adjacency -------------------------------------
// ---- U side row by row.  Row u of the caller's CSR becomes G* row l + rank_u[u]
// (its slots start at off_star[l + rank_u[u]]); inside the row the neighbours
// go in ascending L rank.  The ranks of a row are distinct (E is a set), so
// any ordering method gives the same layout.  Three tiers by degree:
//   d <= 32            one warp, each lane's position = the lanes below it;
//   32 < d <= 256      one warp, bitonic sort of (rank, slot) in its shared memory;
//   256 < d <= 4,096   one CTA, bitonic sort of (rank, slot) in shared memory;
//   d > 4,096          (a few hundred rows) one radix sort of their edges.
// Each tier also writes the swapped key (rank_l, rank_u) at the U-side
// position; U-side order is ascending in rank_u, so the stable sort of those
// keys on the rank_l bits yields the L side.
constexpr int kRowWarpMax = 32;
constexpr int kRowWarpSortMax = 256;
constexpr int kRowCtaMax = 4096;
constexpr int kRowCtaThreads = 256;

struct URowOut {
    int64_t m;
    int32_t l;
    int bu;
    const int64_t *off_star;
    int32_t *adj_star, *eid_star, *rows_star;
    uint64_t *keys2;
    int32_t *vals2;
    int *err;
    int check_dup;   // flag duplicate edges (validate)
    __device__ __forceinline__ void put(int32_t ru, int64_t pos, int32_t rl, int32_t slot) const {
        const int64_t k = off_star[l + ru] - m + pos;   // U-side position
        adj_star[m + k] = rl;
        eid_star[m + k] = slot;
        rows_star[m + k] = l + ru;
        keys2[k] = ((uint64_t)(uint32_t)rl << bu) | (uint64_t)(uint32_t)ru;
        vals2[k] = slot;
    }
};

__global__ void k_u_rows_warp(const int32_t *__restrict__ off_u, const int32_t *__restrict__ adj_u,
                              const int32_t *__restrict__ rank_u, const int32_t *__restrict__ rank_l,
                              int32_t r, URowOut o,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = w0; u < r; u += nw) {
        const int32_t b = off_u[u], d = off_u[u + 1] - b;
        if (d == 0 || d > kRowWarpMax) continue;   // warp-uniform
        const int32_t rl = lane < d ? rank_l[adj_u[b + lane]] : 0x7fffffff;
        int pos = 0;
        bool dup = false;
        for (int k = 0; k < d; ++k) {
            const int32_t ok = __shfl_sync(0xffffffffu, rl, k);
            // ties (duplicate edges) are broken by lane, so positions stay distinct
            pos += (ok < rl || (ok == rl && k < lane)) ? 1 : 0;
            dup |= ok == rl && k != lane;
        }
        if (lane < d) {
            if (dup && o.check_dup) atomicOr(o.err, kErrDuplicate);
            o.put(rank_u[u], pos, rl, b + lane);
        }
    }
}

// ascending bitonic sort of np (a power of two) values by the calling warp
__device__ __forceinline__ void warp_bitonic(uint64_t *buf, int np, int lane) {
    for (int k = 2; k <= np; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < np; i += 32) {
                const int ij = i ^ j;
                if (ij > i) {
                    const uint64_t a = buf[i], c = buf[ij];
                    if ((a > c) == ((i & k) == 0)) { buf[i] = c; buf[ij] = a; }
                }
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(kRowCtaThreads) k_u_rows_warp_sort(
    const int32_t *__restrict__ off_u, const int32_t *__restrict__ adj_u,
    const int32_t *__restrict__ rank_u, const int32_t *__restrict__ rank_l,
    const int32_t *__restrict__ rows, int32_t nrows, URowOut o,
    const int *guard = nullptr, const int32_t *nrows_dev = nullptr) {
    if (aborted(guard)) return;
    if (nrows_dev) nrows = *nrows_dev;
    __shared__ uint64_t buf[kRowCtaThreads / 32][kRowWarpSortMax];
    const int lane = threadIdx.x & 31;
    uint64_t *wb = buf[threadIdx.x >> 5];
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i0 = w0; i0 < nrows; i0 += nw) {
        const int32_t u = rows[i0];
        const int32_t b = off_u[u], d = off_u[u + 1] - b;
        int np = 64;
        while (np < d) np <<= 1;
        for (int i = lane; i < np; i += 32)
            wb[i] = i < d ? ((uint64_t)(uint32_t)rank_l[adj_u[b + i]] << 32) | (uint32_t)(b + i) : ~0ull;
        __syncwarp();
        warp_bitonic(wb, np, lane);
        const int32_t ru = rank_u[u];
        for (int i = lane; i < d; i += 32) {
            const uint64_t vv = wb[i];
            const int32_t rl = (int32_t)(vv >> 32);
            if (o.check_dup && i > 0 && (int32_t)(wb[i - 1] >> 32) == rl) atomicOr(o.err, kErrDuplicate);
            o.put(ru, i, rl, (int32_t)(uint32_t)vv);
        }
        __syncwarp();   // the buffer is reused by the warp's next row
    }
}

__global__ void __launch_bounds__(kRowCtaThreads) k_u_rows_cta(
    const int32_t *__restrict__ off_u, const int32_t *__restrict__ adj_u,
    const int32_t *__restrict__ rank_u, const int32_t *__restrict__ rank_l,
    const int32_t *__restrict__ rows, int32_t nrows, URowOut o,
    const int *guard = nullptr, const int32_t *nrows_dev = nullptr) {
    if (aborted(guard)) return;
    if (nrows_dev) nrows = *nrows_dev;
    __shared__ uint64_t buf[kRowCtaMax];
    for (int64_t i0 = blockIdx.x; i0 < nrows; i0 += gridDim.x) {
        const int32_t u = rows[i0];
        const int32_t b = off_u[u], d = off_u[u + 1] - b;
        int np = 64;
        while (np < d) np <<= 1;
        // (rank, slot): slots are distinct, so the sort has no ties
        for (int i = threadIdx.x; i < np; i += kRowCtaThreads)
            buf[i] = i < d ? ((uint64_t)(uint32_t)rank_l[adj_u[b + i]] << 32) | (uint32_t)(b + i) : ~0ull;
        __syncthreads();
        for (int k = 2; k <= np; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < np; i += kRowCtaThreads) {
                    const int ij = i ^ j;
                    if (ij > i) {
                        const uint64_t a = buf[i], c = buf[ij];
                        if ((a > c) == ((i & k) == 0)) { buf[i] = c; buf[ij] = a; }
                    }
                }
                __syncthreads();
            }
        }
        const int32_t ru = rank_u[u];
        for (int i = threadIdx.x; i < d; i += kRowCtaThreads) {
            const uint64_t vv = buf[i];
            const int32_t rl = (int32_t)(vv >> 32);
            if (o.check_dup && i > 0 && (int32_t)(buf[i - 1] >> 32) == rl) atomicOr(o.err, kErrDuplicate);
            o.put(ru, i, rl, (int32_t)(uint32_t)vv);
        }
        __syncthreads();   // buf is reused by the next row
    }
}

// lists of the rows of the CTA tier and of the largest rows (any order: every
// row is written to its own slots); one atomic per warp and list
__global__ void k_row_tiers(const int32_t *__restrict__ off_u, int32_t r, int32_t *lists,
                            int32_t *counts,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    // lists[t * r ...]: rows of tier t (0: warp sort, 1: CTA sort, 2: radix)
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    for (int64_t u0 = (int64_t)blockIdx.x * blockDim.x; u0 < r; u0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = u0 + threadIdx.x;
        const int32_t d = u < r ? off_u[u + 1] - off_u[u] : 0;
        const int tier = d <= kRowWarpMax ? -1 : d <= kRowWarpSortMax ? 0 : d <= kRowCtaMax ? 1 : 2;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const uint32_t bm = __ballot_sync(0xffffffffu, tier == t);
            int32_t o = 0;
            if (lane == 0 && bm) o = atomicAdd(counts + t, __popc(bm));
            o = __shfl_sync(0xffffffffu, o, 0);
            if (tier == t) lists[(int64_t)t * r + o + __popc(bm & lt)] = (int32_t)u;
        }
    }
}

__global__ void k_large_deg(const int32_t *__restrict__ off_u, const int32_t *__restrict__ large,
                            int32_t nlarge, int64_t *ldeg) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nlarge) return;
    ldeg[i] = off_u[large[i] + 1] - off_u[large[i]];
}

// one CTA per large row copies its edges with composite keys (rank_u, rank_l)
__global__ void k_large_keys(const int32_t *__restrict__ off_u, const int32_t *__restrict__ adj_u,
                             const int32_t *__restrict__ rank_u, const int32_t *__restrict__ rank_l,
                             const int32_t *__restrict__ large, const int64_t *__restrict__ loff,
                             int32_t nlarge, int bl, uint64_t *keys, int32_t *vals) {
    for (int64_t i0 = blockIdx.x; i0 < nlarge; i0 += gridDim.x) {
        const int32_t u = large[i0];
        const int64_t o = loff[i0], d = loff[i0 + 1] - o;
        const int32_t b = off_u[u];
        const uint64_t hi = (uint64_t)(uint32_t)rank_u[u] << bl;
        for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
            keys[o + i] = hi | (uint64_t)(uint32_t)rank_l[adj_u[b + i]];
            vals[o + i] = b + (int32_t)i;
        }
    }
}

__global__ void k_large_heads(const uint64_t *__restrict__ keys, int64_t n, int bl, int32_t *heads) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        heads[i] = (i == 0 || (keys[i] >> bl) != (keys[i - 1] >> bl)) ? (int32_t)i : 0;
}

__global__ void k_large_emit(const uint64_t *__restrict__ keys, const int32_t *__restrict__ vals,
                             const int32_t *__restrict__ row_first, int64_t n, int bl, URowOut o) {
    const uint64_t mask_l = (1ull << bl) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[i];
        if (o.check_dup && i > 0 && keys[i - 1] == key) atomicOr(o.err, kErrDuplicate);
        o.put((int32_t)(key >> bl), i - row_first[i], (int32_t)(key & mask_l), vals[i]);
    }
}

__global__ void k_emit_l_side(const uint64_t *__restrict__ keys2, const int32_t *__restrict__ vals2,
                              int64_t m, int bu, int32_t l, int32_t *adj_star, int32_t *eid_star,
                              int32_t *rows_star,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    const uint64_t mask_u = (1ull << bu) - 1ull;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = keys2[k];
        adj_star[k] = l + (int32_t)(key & mask_u);
        eid_star[k] = vals2[k];
        rows_star[k] = (int32_t)(key >> bu);
    }
}

__global__ void k_deg_to_i64(const int32_t *__restrict__ d, int32_t n, int64_t *out,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = d[i];
}

// ----- a4: orientation cut and per-start work ---------------------------------
// cut[x] = |{y in N(x): p(y) < p(x)}|.  Lists are ascending in priority and
// the degree of G* ids is non-decreasing inside a layer, so the cut is a
// lower bound on degree: for x in L a U neighbour of equal degree has higher
// priority (U ids > L ids); for x in U an L neighbour of equal degree is lower.
__global__ void k_cut(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                      const int32_t *__restrict__ deg_star, int32_t n, int32_t l, int32_t *cut,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int64_t b = off[x];
    int64_t lo = 0, hi = off[x + 1] - b;
    const int32_t dx = deg_star[x];
    const bool in_u = x >= l;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        int32_t dy = deg_star[adj[b + mid]];
        bool lower = in_u ? (dy <= dx) : (dy < dx);
        if (lower) lo = mid + 1; else hi = mid;
    }
    cut[x] = (int32_t)lo;
}

// plen[e] for a middle slot e = (x, v): the number of ends w in N(v) with
// p(w) < p(x), i.e. the prefix of v's ascending list below x; sbeg[e] = the
// position where that prefix starts (off[v]), so the count kernel reads it
// with the slot instead of after the slot's neighbour id.
__global__ void k_plen(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                       const int32_t *__restrict__ rows, const int32_t *__restrict__ cut,
                       int64_t slots, int32_t *plen, int64_t *sbeg,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < slots;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = rows[e];
        int32_t out = 0;
        int64_t b = 0;
        if (e - off[x] < cut[x]) {
            const int32_t v = adj[e];
            b = off[v];
            int64_t lo = 0, hi = off[v + 1] - b;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (adj[b + mid] < x) lo = mid + 1; else hi = mid;
            }
            out = (int32_t)lo;
        }
        plen[e] = out;
        sbeg[e] = b;
    }
}

// Algorithm 3: for slot e = (x, v) the ends are the w in N(v) with
// p(w) > p(x) and p(w) > p(v).  N(v) ascends in priority, so they form the
// suffix that starts after both x (x is in N(v)) and v's cut.
__global__ void k_slen(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                       const int32_t *__restrict__ rows, const int32_t *__restrict__ cut,
                       int64_t slots, int32_t *slen, int64_t *sbeg) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < slots;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = rows[e];
        const int32_t v = adj[e];
        const int64_t b = off[v], d = off[v + 1] - b;
        int64_t lo = 0, hi = d;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (adj[b + mid] <= x) lo = mid + 1; else hi = mid;
        }
        const int64_t a = lo > cut[v] ? lo : (int64_t)cut[v];
        slen[e] = (int32_t)(d - a);
        sbeg[e] = b + a;
    }
}

// work[x] = Σ plen over x's middle slots (the first cut[x] slots for
// Algorithm 2, every slot for Algorithm 3); one warp per start.
__global__ void k_work(const int64_t *__restrict__ off, const int32_t *__restrict__ cut,
                       const int32_t *__restrict__ plen, int32_t n, int all_slots, uint64_t *work,
                       unsigned long long *total,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long tot = 0;
    for (int64_t x = warp; x < n; x += nwarps) {
        const int64_t b = off[x];
        const int64_t c = all_slots ? off[x + 1] - b : (int64_t)cut[x];
        unsigned long long s = 0;
        for (int64_t j = lane; j < c; j += 32) s += (unsigned)plen[b + j];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) work[x] = s;
        tot += s;
    }
    if (lane == 0 && tot) atomicAdd(total, tot);
}

// ----- a5: bins and schedule ---------------------------------------------------
// A core start (dense-core hybrid) with wedges is always a dense item: only
// dense items skip the core wedges and add the core pairs after the walk.
__device__ __forceinline__ bool forced_dense(int32_t x, int32_t l, int32_t core_lo_u, int32_t core_lo_l,
                                             uint64_t w) {
    return w > 0 && (x >= l ? x >= core_lo_u : x >= core_lo_l);
}

__global__ void k_sched_keys(const uint64_t *__restrict__ work, int32_t n, uint64_t maxw,
                             int32_t l, int32_t core_lo_u, int32_t core_lo_l, uint64_t *keys,
                             int32_t *vals,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    // ascending key = descending work; zero work last; forced dense starts first
    keys[x] = forced_dense((int32_t)x, l, core_lo_u, core_lo_l, work[x]) ? 0 : maxw - work[x];
    vals[x] = (int32_t)x;
}

// starts with more than `bound` wedges (the dense bin's size before any core)
__global__ void k_count_heavy(const uint64_t *__restrict__ work, int32_t n, uint64_t bound,
                              unsigned long long *count) {
    unsigned long long c = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        c += work[x] > bound ? 1 : 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// counts[0] = dense starts, [1] = hash starts, [2] = warp starts
// Bins of a6: [0] dense (work > hash_max), [1] CTA hash (team_max < work <=
// hash_max), [2] team (warp_max < work <= team_max), [3] warp (0 < work <= warp_max).
__global__ void k_classify(const uint64_t *__restrict__ work, int32_t n, uint64_t warp_max,
                           uint64_t team_max, uint64_t hash_max, int32_t l, int32_t core_lo_u,
                           int32_t core_lo_l, unsigned long long *counts,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    unsigned long long c[4] = {0, 0, 0, 0};
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        uint64_t w = work[x];
        if (w > hash_max || forced_dense((int32_t)x, l, core_lo_u, core_lo_l, w)) ++c[0];
        else if (w > team_max) ++c[1];
        else if (w > warp_max) ++c[2];
        else if (w > 0) ++c[3];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) c[k] += __shfl_xor_sync(0xffffffffu, c[k], d);
        if ((threadIdx.x & 31) == 0 && c[k]) atomicAdd(&counts[k], c[k]);
    }
}

// the dense chunks of start x (dense_chunk_end from offset 0 up); with `out`,
// each chunk's item (x, first end offset) is written there
__device__ __forceinline__ int32_t dense_chunks(int32_t x, int32_t l, int32_t cut, const int64_t *off,
                                                const int32_t *vbase, int2 *out = nullptr) {
    const int32_t lb = vbase ? vbase[x] : (x >= l ? l : 0);
    const int32_t R = x - lb;
    int32_t k = 0;
    for (int32_t lo = 0; lo < R; ++k) {
        int bits;
        const int32_t hi = dense_chunk_end(lo, R, cut, off, lb, &bits);
        if (out) out[k] = make_int2(x, lo);
        lo = hi;
    }
    return k;
}

__global__ void k_chunk_counts(const int32_t *__restrict__ order, int64_t n_dense, int32_t l,
                               const int32_t *__restrict__ cut, const int64_t *__restrict__ off,
                               const int32_t *__restrict__ vbase, int64_t *nch) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_dense) return;
    int32_t x = order[i];
    nch[i] = dense_chunks(x, l, cut[x], off, vbase);
}

// starts in descending work order: dense (chunked), CTA hash, team, warp
__global__ void k_emit_items(const int32_t *__restrict__ order, int64_t n_dense, int64_t n_hash,
                             int64_t n_team, int64_t n_warp, const int64_t *__restrict__ nch_scan,
                             int32_t l, const int32_t *__restrict__ cut, const int64_t *__restrict__ off,
                             const int32_t *__restrict__ vbase, int2 *cta_items,
                             int32_t *team_items, int32_t *warp_items) {
    const int64_t total_dense = nch_scan[n_dense];
    const int64_t all = n_dense + n_hash + n_team + n_warp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < all;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = order[i];
        if (i < n_dense) {
            dense_chunks(x, l, cut[x], off, vbase, cta_items + nch_scan[i]);
        } else if (i < n_dense + n_hash) {
            cta_items[total_dense + (i - n_dense)] = make_int2(x, -1);
        } else if (i < n_dense + n_hash + n_team) {
            team_items[i - n_dense - n_hash] = x;
        } else {
            warp_items[i - n_dense - n_hash - n_team] = x;
        }
    }
}

// retry entries -(x+1): counted with dense chunks
__global__ void k_items_to_dense_retries(const int2 *__restrict__ items, int64_t n, int32_t *starts) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) starts[i] = -(items[i].x + 1);
}

// ----- chunk-boundary table for the dense bin ----------------------------------
__device__ __forceinline__ int64_t coff_base(int32_t v, int32_t l, int32_t u1, int32_t l1) {
    return v < l ? (int64_t)v * u1 : (int64_t)l * u1 + (int64_t)(v - l) * l1;
}

__global__ void k_coff_fill(const int64_t *__restrict__ off, int32_t l, int32_t u1, int32_t l1,
                            int64_t entries, int32_t *coff) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < entries;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t split = (int64_t)l * u1;
        const int32_t v = i < split ? (int32_t)(i / u1) : l + (int32_t)((i - split) / l1);
        coff[i] = (int32_t)(off[v + 1] - off[v]);
    }
}

// entry c of v = first position in N(v) whose neighbour rank is >= c * unit
__global__ void k_coff_slots(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                             const int32_t *__restrict__ rows, int64_t slots, int32_t l,
                             int32_t u1, int32_t l1, int32_t *coff) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < slots;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = rows[p];
        const int32_t lbe = v < l ? l : 0;
        const int64_t b = off[v];
        const int32_t cp = (adj[p] - lbe) / kChunkUnit;
        const int32_t cprev = p == b ? -1 : (adj[p - 1] - lbe) / kChunkUnit;
        const int64_t tb = coff_base(v, l, u1, l1);
        for (int32_t c = cprev + 1; c <= cp; ++c) coff[tb + c] = (int32_t)(p - b);
    }
}

// A batch's table.  The middles of every dense start with several chunks
// (one warp per start: its cut[x] lower-priority neighbours).
__global__ void k_coff_mark(const int32_t *__restrict__ order, int64_t n_dense, const int64_t *__restrict__ nch,
                            const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                            const int32_t *__restrict__ cut, int32_t *mark) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n_dense; i += nw) {
        if (nch[i] <= 1) continue;
        const int32_t x = order[i];
        const int64_t e0 = off[x];
        for (int64_t e = e0 + lane; e < e0 + cut[x]; e += 32) mark[adj[e]] = 1;
    }
}

// entries of a marked v: the chunks of its graph's neighbour layer, plus one
// (the neighbours' layer range is that of any neighbour w: vend[w] - vbase[w])
__global__ void k_coff_sizes(const int32_t *__restrict__ mark, const int64_t *__restrict__ off,
                             const int32_t *__restrict__ adj, const int32_t *__restrict__ vbase,
                             const int32_t *__restrict__ vend, int32_t n, int64_t *cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0;
        if (mark[v] && off[v + 1] > off[v]) {
            const int32_t w = adj[off[v]];
            c = (int64_t)(vend[w] - vbase[w] + kChunkUnit - 1) / kChunkUnit + 1;
        }
        cnt[v] = c;
    }
}

// every entry of v starts at "past the end of N(v)"
__global__ void k_coff_fill_var(const int64_t *__restrict__ off, const int64_t *__restrict__ cstart, int32_t n,
                                int32_t *coff) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = (int32_t)(off[v + 1] - off[v]);
        for (int64_t c = cstart[v]; c < cstart[v + 1]; ++c) coff[c] = d;
    }
}

// entry c of a marked v = first position in N(v) whose neighbour id is at
// least (first id of the neighbours' graph range) + c * unit
__global__ void k_coff_slots_var(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                                 const int32_t *__restrict__ rows, int64_t slots,
                                 const int32_t *__restrict__ vbase, const int64_t *__restrict__ cstart,
                                 int32_t *coff) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < slots;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = rows[p];
        const int64_t tb = cstart[v], te = cstart[v + 1];
        if (te == tb) continue;
        const int64_t b = off[v];
        const int32_t lbe = vbase[adj[b]];
        const int32_t cp = (adj[p] - lbe) / kChunkUnit;
        const int32_t cprev = p == b ? -1 : (adj[p - 1] - lbe) / kChunkUnit;
        for (int32_t c = cprev + 1; c <= cp && tb + c < te; ++c) coff[tb + c] = (int32_t)(p - b);
    }
}

// the first entry of each middle of those starts, at the middle's slot
__global__ void k_coff_slot_bases(const int32_t *__restrict__ order, int64_t n_dense,
                                  const int64_t *__restrict__ nch, const int64_t *__restrict__ off,
                                  const int32_t *__restrict__ adj, const int32_t *__restrict__ cut,
                                  const int64_t *__restrict__ cstart, int32_t *ctb) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n_dense; i += nw) {
        if (nch[i] <= 1) continue;
        const int32_t x = order[i];
        const int64_t e0 = off[x];
        for (int64_t e = e0 + lane; e < e0 + cut[x]; e += 32) ctb[e] = (int32_t)cstart[adj[e]];
    }
}

unsigned grid_stride_blocks(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// ----- batches prepared as one disjoint union ------------------------------------
__device__ __forceinline__ int32_t graph_of(const int32_t *start, int32_t num_graphs, int32_t id) {
    int32_t lo = 0, hi = num_graphs;   // last g with start[g] <= id
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (start[mid] <= id) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_check_starts(const int32_t *__restrict__ start, int32_t num_graphs,
                               int32_t total, int *err, int32_t max_len = 0x7fffffff) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= num_graphs;
         g += (int64_t)gridDim.x * blockDim.x) {
        if (g == 0 && start[0] != 0) atomicOr(err, kErrBadOffsets);
        if (g < num_graphs && (start[g + 1] < start[g] || start[g + 1] - start[g] > max_len))
            atomicOr(err, kErrBadOffsets);
        if (g == num_graphs && start[g] != total) atomicOr(err, kErrBadOffsets);
    }
}

// every edge must join a U and an L vertex of the same graph
__global__ void k_check_batch_edges(const int32_t *__restrict__ rows, const int32_t *__restrict__ adj,
                                    int64_t m, const int32_t *__restrict__ gu,
                                    const int32_t *__restrict__ gl, int32_t num_graphs, int *err,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x)
        if (graph_of(gu, num_graphs, rows[k]) != graph_of(gl, num_graphs, adj[k]))
            atomicOr(err, kErrBadId);
}

// graph-major ranks: vertex x of G* belongs to the graph whose rank range
// holds it; vbase[x] = the first G* id of that graph in x's layer
__global__ void k_graph_star(int32_t r, int32_t l, const int32_t *__restrict__ gu,
                             const int32_t *__restrict__ gl, int32_t num_graphs, int32_t *gstar,
                             int32_t *vbase, int32_t *vend,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < (int64_t)r + l;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (x < l) {
            const int32_t gg = graph_of(gl, num_graphs, (int32_t)x);
            gstar[x] = gg;
            vbase[x] = gl[gg];
            vend[x] = gl[gg + 1];
        } else {
            const int32_t gg = graph_of(gu, num_graphs, (int32_t)(x - l));
            gstar[x] = gg;
            vbase[x] = l + gu[gg];
            vend[x] = l + gu[gg + 1];
        }
    }
}

__global__ void k_graph_work(const uint64_t *__restrict__ work, const int32_t *__restrict__ gstar,
                             int32_t n, unsigned long long *gwork,
    const int *guard = nullptr) {
    if (aborted(guard)) return;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        if (work[x]) atomicAdd(gwork + gstar[x], (unsigned long long)work[x]);
}

// slot -> owning vertex of G*, one warp per vertex
__global__ void k_rows_from_off(const int64_t *__restrict__ off, int32_t n, int32_t *rows) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = w; x < n; x += nw)
        for (int64_t p = off[x] + lane; p < off[x + 1]; p += 32) rows[p] = (int32_t)x;
}

}  // namespace

// Step a5: order the starts by descending exact work and split them into the
// warp, CTA-hash and CTA-dense bins (dense starts into end-range chunks);
// builds the chunk-boundary table when a dense start has several chunks.
// `rows_star` (slot -> vertex of G*) may be null; it is rebuilt when needed.
static int schedule_graph(Graph *g, cudaStream_t s, int32_t warp_max_work, int32_t team_max_work,
                          int32_t hash_max_work, const int32_t *rows_star) {
    const int32_t r = g->r, l = g->l, n = g->n;
    const int64_t m = g->m;
    const bool vpp = g->opt.orientation == 1;
    Allocs tmp;
    tmp.stream = s;
    struct TmpGuard { Allocs *a; ~TmpGuard() { a->release(); } } guard{&tmp};
#define GET(allocs, ptr, cnt)                                                         \
    do {                                                                              \
        cudaError_t e_ = (allocs).get(&(ptr), (size_t)(cnt));                         \
        if (e_ != cudaSuccess) {                                                      \
            set_last_error(std::string("device allocation failed: ") + #ptr);         \
            return BFC_ERR_OUT_OF_MEMORY;                                             \
        }                                                                             \
    } while (0)
    const uint64_t warp_max = (uint64_t)warp_max_work;
    // Algorithm 3: ends concentrate on few high-priority vertices, so no start
    // gets dense counters up front; every start beyond the warp bin gets a
    // team or CTA hash table and one whose table fills up is re-queued
    const uint64_t hash_max = vpp ? ~0ull : (uint64_t)hash_max_work;
    const int32_t team_req = team_max_work >= 0 ? team_max_work : (vpp ? kTeamMaxWork : kTeamFitWork);
    uint64_t team_max = std::max<uint64_t>((uint64_t)team_req, warp_max);
    if (!vpp) team_max = std::min<uint64_t>(team_max, hash_max);
    if (vpp && hash_max_work == 0) team_max = warp_max;   // all of them to the dense pass
    const uint64_t maxw = g->info.max_start_work;
    int64_t n_dense = 0, n_hash = 0, n_team = 0, n_warp = 0, n_items = 0, h_dense_items = 0;
    if (n > 0 && g->info.wedges > 0) {
        const int64_t nn = (int64_t)n + 1;
        uint64_t *k0, *k1;
        int32_t *v0, *v1;
        uint32_t *hist, *hist_tmp;
        int64_t *scan64_tmp, *nch;
        unsigned long long *red;
        GET(tmp, k0, nn); GET(tmp, k1, nn); GET(tmp, v0, nn); GET(tmp, v1, nn);
        GET(tmp, hist, radix_hist_elems(n));
        GET(tmp, hist_tmp, scan_tmp_elems<uint32_t>((int64_t)radix_hist_elems(n)));
        GET(tmp, scan64_tmp, scan_tmp_elems<int64_t>(nn));
        GET(tmp, nch, nn);
        GET(tmp, red, 4);
        BFC_CUDA(cudaMemsetAsync(red, 0, 4 * sizeof(unsigned long long), s));
        int which = 0;
        // without a core the bounds lie past every id
        const int32_t clo_u = g->core_u > 0 ? g->core_lo_u : n, clo_l = g->core_l > 0 ? g->core_lo_l : n;
        k_sched_keys<<<blocks_for(n), kT, 0, s>>>(g->work, n, maxw, l, clo_u, clo_l, k0, v0); note_launch();
        BFC_CUDA(cudaGetLastError());
        BFC_CUDA(radix_sort_pairs(k0, v0, k1, v1, n, 0, bits_for(maxw), hist, hist_tmp, s, &which));
        const int32_t *order = which ? v1 : v0;
        k_classify<<<grid_stride_blocks(n), kT, 0, s>>>(g->work, n, warp_max, team_max, hash_max, l, clo_u,
                                                        clo_l, red); note_launch();
        BFC_CUDA(cudaGetLastError());
        unsigned long long hc[4];
        BFC_CUDA(cudaMemcpyAsync(hc, red, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        BFC_CUDA(cudaStreamSynchronize(s));
        n_dense = (int64_t)hc[0]; n_hash = (int64_t)hc[1]; n_team = (int64_t)hc[2]; n_warp = (int64_t)hc[3];
        if (n_dense > 0) {
            k_chunk_counts<<<blocks_for(n_dense), kT, 0, s>>>(order, n_dense, l, g->cut, g->off, g->vbase, nch); note_launch();
            BFC_CUDA(cudaGetLastError());
        }
        // the sorted keys are no longer needed; the other key buffer holds the scan
        int64_t *nch_scan = reinterpret_cast<int64_t *>(which ? k0 : k1);
        BFC_CUDA(scan_exclusive<int64_t>(nch, nch_scan, n_dense, scan64_tmp, s));
        BFC_CUDA(cudaMemcpyAsync(&h_dense_items, nch_scan + n_dense, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
        BFC_CUDA(cudaStreamSynchronize(s));
        n_items = h_dense_items + n_hash;
        GET(g->mem, g->cta_items, std::max<int64_t>(n_items, 1));
        GET(g->mem, g->team_items, std::max<int64_t>(n_team, 1));
        GET(g->mem, g->warp_items, std::max<int64_t>(n_warp, 1));
        if (n_dense + n_hash + n_team + n_warp > 0) {
            k_emit_items<<<grid_stride_blocks(n_dense + n_hash + n_team + n_warp), kT, 0, s>>>(
                order, n_dense, n_hash, n_team, n_warp, nch_scan, l, g->cut, g->off, g->vbase, g->cta_items,
                g->team_items, g->warp_items); note_launch();
            BFC_CUDA(cudaGetLastError());
        }
        // chunk boundaries of every list, so dense items read them instead of searching
        const int32_t u1 = (int32_t)((r + kChunkUnit - 1) / kChunkUnit) + 1;
        const int32_t l1 = (int32_t)((l + kChunkUnit - 1) / kChunkUnit) + 1;
        const int64_t entries = (int64_t)l * u1 + (int64_t)r * l1;
        if (!g->coff && g->num_graphs > 0 && h_dense_items > n_dense) {
            // a batch: entries only for the middles of starts with several
            // chunks, as many as the chunks of their graph's neighbour layer
            // (+1), found through a per-vertex start array
            int32_t *mark;
            int64_t *ecnt;
            GET(tmp, mark, n);
            GET(tmp, ecnt, (int64_t)n + 1);
            GET(g->mem, g->coff_start, (int64_t)n + 1);
            BFC_CUDA(cudaMemsetAsync(mark, 0, sizeof(int32_t) * (size_t)n, s));
            k_coff_mark<<<grid_stride_blocks(n_dense * 32), kT, 0, s>>>(order, n_dense, nch, g->off, g->adj,
                                                                         g->cut, mark); note_launch();
            k_coff_sizes<<<grid_stride_blocks(n), kT, 0, s>>>(mark, g->off, g->adj, g->vbase, g->vend, n, ecnt); note_launch();
            BFC_CUDA(cudaGetLastError());
            BFC_CUDA(scan_exclusive<int64_t>(ecnt, g->coff_start, n, scan64_tmp, s));
            int64_t ventries = 0;
            BFC_CUDA(cudaMemcpyAsync(&ventries, g->coff_start + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            BFC_CUDA(cudaStreamSynchronize(s));
            if (ventries <= kChunkTableMaxEntries) {   // else searches
                if (!rows_star) {
                    int32_t *rs;
                    GET(tmp, rs, 2 * m);
                    k_rows_from_off<<<grid_stride_blocks((int64_t)n * 32), kT, 0, s>>>(g->off, n, rs); note_launch();
                    BFC_CUDA(cudaGetLastError());
                    rows_star = rs;
                }
                GET(g->mem, g->coff, std::max<int64_t>(ventries, 1));
                k_coff_fill_var<<<grid_stride_blocks(n), kT, 0, s>>>(g->off, g->coff_start, n, g->coff); note_launch();
                BFC_CUDA(cudaGetLastError());
                k_coff_slots_var<<<grid_stride_blocks(2 * m), kT, 0, s>>>(g->off, g->adj, rows_star, 2 * m,
                                                                          g->vbase, g->coff_start, g->coff); note_launch();
                BFC_CUDA(cudaGetLastError());
                // each middle slot of those starts holds its middle's first
                // entry (-1 elsewhere), read with the slot's other arrays
                GET(g->mem, g->ctb, 2 * m);
                BFC_CUDA(cudaMemsetAsync(g->ctb, 0xff, sizeof(int32_t) * (size_t)(2 * m), s));
                k_coff_slot_bases<<<grid_stride_blocks(n_dense * 32), kT, 0, s>>>(order, n_dense, nch, g->off, g->adj,
                                                                                   g->cut, g->coff_start, g->ctb); note_launch();
                BFC_CUDA(cudaGetLastError());
            }
            g->mem.drop(g->coff_start);
            g->coff_start = nullptr;
        }
        if (!g->coff && g->num_graphs == 0 && h_dense_items > n_dense && entries <= kChunkTableMaxEntries) {
            if (!rows_star) {
                int32_t *rs;
                GET(tmp, rs, 2 * m);
                k_rows_from_off<<<grid_stride_blocks((int64_t)n * 32), kT, 0, s>>>(g->off, n, rs); note_launch();
                BFC_CUDA(cudaGetLastError());
                rows_star = rs;
            }
            GET(g->mem, g->coff, entries);
            g->coff_u1 = u1;
            g->coff_l1 = l1;
            k_coff_fill<<<grid_stride_blocks(entries), kT, 0, s>>>(g->off, l, u1, l1, entries, g->coff); note_launch();
            BFC_CUDA(cudaGetLastError());
            k_coff_slots<<<grid_stride_blocks(2 * m), kT, 0, s>>>(g->off, g->adj, rows_star, 2 * m, l, u1, l1,
                                                                  g->coff); note_launch();
            BFC_CUDA(cudaGetLastError());
        }
    } else {
        GET(g->mem, g->cta_items, 1);
        GET(g->mem, g->team_items, 1);
        GET(g->mem, g->warp_items, 1);
    }
    g->n_cta_items = n_items;
    g->n_team_items = n_team;
    g->n_warp_items = n_warp;
    g->team_max = (int32_t)std::min<uint64_t>(team_max, (uint64_t)kTeamMaxWork);
    // each hash start is re-queued at most once per launch
    g->mem.drop(g->retry);
    g->retry = nullptr;
    g->retry_static = 0;
    g->retry_cap = std::max<int64_t>(n_hash + n_team, 1);
    GET(g->mem, g->retry, g->retry_cap);
    if (vpp && hash_max_work == 0 && n_hash > 0) {
        // every start beyond the warp bin goes to the dense pass directly
        k_items_to_dense_retries<<<blocks_for(n_hash), kT, 0, s>>>(g->cta_items, n_hash, g->retry); note_launch();
        BFC_CUDA(cudaGetLastError());
        g->retry_static = n_hash;
        g->n_cta_items = 0;
    }
    // Algorithm 2's tables always fit when a team start has at most 3,072
    // wedges (4,096 slots) and a CTA start at most 24,576 (32,768 slots)
    g->may_retry = vpp ? (n_hash + n_team > 0) : (n_team > 0 && team_max > (uint64_t)kTeamFitWork);
    g->info.dense_items = h_dense_items;
    g->info.starts_with_work = n_dense + n_hash + n_team + n_warp;
    g->info.dense_starts = n_dense;
    g->info.hash_starts = n_hash;
    g->info.team_starts = n_team;
    g->info.warp_starts = n_warp;
    g->opt.warp_max_work = warp_max_work;
    g->opt.team_max_work = team_max_work;
    g->opt.hash_max_work = hash_max_work;
    BFC_CUDA(cudaStreamSynchronize(s));
#undef GET
    return BFC_OK;
}

int rebin_graph(Graph *g, cudaStream_t s, int32_t warp_max_work, int32_t team_max_work,
                int32_t hash_max_work) {
    g->mem.stream = s;
    g->mem.drop(g->cta_items);
    g->mem.drop(g->team_items);
    g->mem.drop(g->warp_items);
    g->cta_items = nullptr;
    g->team_items = nullptr;
    g->warp_items = nullptr;
    int rc = schedule_graph(g, s, warp_max_work, team_max_work, hash_max_work, nullptr);
    g->info.device_bytes = (int64_t)g->mem.total;
    return rc;
}

int prepare_graph(const bfc_csr *csr, const bfc_options *opt, cudaStream_t s, Graph *g,
                  int32_t num_graphs, const int32_t *graph_u_start, const int32_t *graph_l_start) {
    const int32_t r = csr->num_u, l = csr->num_l;
    const int64_t m = csr->num_edges;
    const int32_t n = r + l;
    g->r = r; g->l = l; g->n = n; g->m = m;
    g->opt = *opt;
    g->stream = s;
    g->mem.stream = s;

    Allocs tmp;
    tmp.stream = s;
    struct TmpGuard { Allocs *a; ~TmpGuard() { a->release(); } } guard{&tmp};

#define GET(allocs, ptr, cnt)                                                         \
    do {                                                                              \
        cudaError_t e_ = (allocs).get(&(ptr), (size_t)(cnt));                         \
        if (e_ != cudaSuccess) {                                                      \
            set_last_error(std::string("device allocation failed: ") + #ptr);         \
            return BFC_ERR_OUT_OF_MEMORY;                                             \
        }                                                                             \
    } while (0)

    // ---- kept arrays
    GET(g->mem, g->err, 4);
    GET(g->mem, g->rank_u, r);
    GET(g->mem, g->rank_l, l);
    GET(g->mem, g->off, (int64_t)n + 1);
    GET(g->mem, g->adj, 2 * m);
    GET(g->mem, g->eid, 2 * m);
    GET(g->mem, g->plen, 2 * m);
    GET(g->mem, g->cut, n);
    GET(g->mem, g->work, n);
    GET(g->mem, g->cursors, 8);
    GET(g->mem, g->acc, 2);
    GET(g->mem, g->pv, n);
    BFC_CUDA(cudaMemsetAsync(g->err, 0, 4 * sizeof(int), s));

    // ---- validation of the caller's CSR (memory safety of everything below)
    k_check_offsets<<<blocks_for((int64_t)r + 1), kT, 0, s>>>(csr->off_u, r, m, g->err); note_launch();
    BFC_CUDA(cudaGetLastError());
    int herr = 0;
    BFC_CUDA(cudaMemcpyAsync(&herr, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BFC_CUDA(cudaStreamSynchronize(s));
    if (herr) { set_last_error("off_u is not a CSR offset array of num_edges entries"); return BFC_ERR_INVALID_GRAPH; }
    if (m > 0) {
        k_check_ids<<<grid_stride_blocks(m), kT, 0, s>>>(csr->adj_u, m, l, g->err); note_launch();
        BFC_CUDA(cudaGetLastError());
        BFC_CUDA(cudaMemcpyAsync(&herr, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
        BFC_CUDA(cudaStreamSynchronize(s));
        if (herr) { set_last_error("adj_u holds an id outside [0, num_l)"); return BFC_ERR_INVALID_GRAPH; }
    }

    if (num_graphs > 0) {
        k_check_starts<<<blocks_for((int64_t)num_graphs + 1), kT, 0, s>>>(graph_u_start, num_graphs, r, g->err); note_launch();
        k_check_starts<<<blocks_for((int64_t)num_graphs + 1), kT, 0, s>>>(graph_l_start, num_graphs, l, g->err); note_launch();
        BFC_CUDA(cudaGetLastError());
        BFC_CUDA(cudaMemcpyAsync(&herr, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
        BFC_CUDA(cudaStreamSynchronize(s));
        if (herr) { set_last_error("graph start arrays are not prefix sums of the layer sizes"); return BFC_ERR_INVALID_GRAPH; }
        g->num_graphs = num_graphs;
        GET(g->mem, g->gstar, std::max<int64_t>(n, 1));
        GET(g->mem, g->vbase, std::max<int64_t>(n, 1));
        GET(g->mem, g->vend, std::max<int64_t>(n, 1));
        GET(g->mem, g->gwork, num_graphs);
        BFC_CUDA(cudaMemsetAsync(g->gwork, 0, sizeof(unsigned long long) * num_graphs, s));
    }

    // ---- temporaries
    const int64_t nsort = std::max<int64_t>({(int64_t)r, (int64_t)l, m, (int64_t)n, 1});
    uint64_t *k0, *k1;
    int32_t *v0, *v1, *deg_u, *deg_l, *deg_star, *rows, *rows_star, *heads, *order_u, *order_l;
    uint32_t *hist, *hist_tmp;
    int64_t *scan64_tmp, *deg64;
    int32_t *maxdeg;
    unsigned long long *red;
    GET(tmp, k0, nsort + 1); GET(tmp, k1, nsort + 1);
    GET(tmp, v0, nsort); GET(tmp, v1, nsort);
    GET(tmp, deg_u, r); GET(tmp, deg_l, l); GET(tmp, deg_star, n);
    GET(tmp, rows, m); GET(tmp, heads, m); GET(tmp, rows_star, 2 * m);
    GET(tmp, order_u, r); GET(tmp, order_l, l);
    GET(tmp, hist, radix_hist_elems(nsort));
    GET(tmp, hist_tmp, scan_tmp_elems<uint32_t>((int64_t)radix_hist_elems(nsort)));
    GET(tmp, scan64_tmp, std::max(scan_tmp_elems<int64_t>((int64_t)n + 1),
                                  max_scan_tmp_elems(m)));
    GET(tmp, deg64, (int64_t)n + 1);
    GET(tmp, maxdeg, 4);
    GET(tmp, red, 8);

    // ---- a1: degrees (and the head of each U row for the slot -> row map)
    BFC_CUDA(cudaMemsetAsync(deg_l, 0, sizeof(int32_t) * std::max<int64_t>(l, 1), s));
    // the row of every input slot is only needed to check a batch's edges
    if (num_graphs > 0) BFC_CUDA(cudaMemsetAsync(heads, 0, sizeof(int32_t) * std::max<int64_t>(m, 1), s));
    if (r > 0) {
        k_deg_u<<<blocks_for(r), kT, 0, s>>>(csr->off_u, r, deg_u, num_graphs > 0 ? heads : nullptr); note_launch();
    }
    if (m > 0) { k_deg_l<<<grid_stride_blocks(m), kT, 0, s>>>(csr->adj_u, m, deg_l); note_launch(); }
    BFC_CUDA(cudaGetLastError());
    BFC_CUDA(reduce_max_i32(deg_u, r, maxdeg, s));
    BFC_CUDA(reduce_max_i32(deg_l, l, maxdeg + 1, s));
    int32_t hmax[2] = {0, 0};
    BFC_CUDA(cudaMemcpyAsync(hmax, maxdeg, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BFC_CUDA(cudaStreamSynchronize(s));
    g->info.max_deg_u = hmax[0];
    g->info.max_deg_l = hmax[1];

    // ---- a2: per-layer priority ranks by a stable sort on degree
    int which = 0;
    if (r > 0) {
        int bkey = bits_for((uint64_t)hmax[0]);
        if (num_graphs > 0) {
            k_iota_keys_batch<<<blocks_for(r), kT, 0, s>>>(deg_u, r, graph_u_start, num_graphs, bkey, k0, v0); note_launch();
            bkey += bits_for((uint64_t)(num_graphs - 1));
        } else {
            k_iota_keys<<<blocks_for(r), kT, 0, s>>>(deg_u, r, k0, v0); note_launch();
        }
        BFC_CUDA(cudaGetLastError());
        BFC_CUDA(radix_sort_pairs(k0, v0, k1, v1, r, 0, bkey, hist,
                                  hist_tmp, s, &which));
        const uint64_t *ks = which ? k1 : k0;
        const int32_t *vs = which ? v1 : v0;
        BFC_CUDA(cudaMemcpyAsync(order_u, vs, sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, s));
        k_ranks<<<blocks_for(r), kT, 0, s>>>(ks, vs, r, g->rank_u, deg_star, l, (1ull << bits_for((uint64_t)hmax[0])) - 1); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    if (l > 0) {
        int bkey = bits_for((uint64_t)hmax[1]);
        if (num_graphs > 0) {
            k_iota_keys_batch<<<blocks_for(l), kT, 0, s>>>(deg_l, l, graph_l_start, num_graphs, bkey, k0, v0); note_launch();
            bkey += bits_for((uint64_t)(num_graphs - 1));
        } else {
            k_iota_keys<<<blocks_for(l), kT, 0, s>>>(deg_l, l, k0, v0); note_launch();
        }
        BFC_CUDA(cudaGetLastError());
        BFC_CUDA(radix_sort_pairs(k0, v0, k1, v1, l, 0, bkey, hist,
                                  hist_tmp, s, &which));
        const uint64_t *ks = which ? k1 : k0;
        const int32_t *vs = which ? v1 : v0;
        BFC_CUDA(cudaMemcpyAsync(order_l, vs, sizeof(int32_t) * l, cudaMemcpyDeviceToDevice, s));
        k_ranks<<<blocks_for(l), kT, 0, s>>>(ks, vs, l, g->rank_l, deg_star, 0, (1ull << bits_for((uint64_t)hmax[1])) - 1); note_launch();
        BFC_CUDA(cudaGetLastError());
    }

    if (num_graphs > 0 && n > 0) {
        k_graph_star<<<grid_stride_blocks(n), kT, 0, s>>>(r, l, graph_u_start, graph_l_start,
                                                         num_graphs, g->gstar, g->vbase, g->vend); note_launch();
        BFC_CUDA(cudaGetLastError());
    }

    // ---- a3: G* offsets and priority-sorted lists
    if (n > 0) {
        k_deg_to_i64<<<blocks_for(n), kT, 0, s>>>(deg_star, n, deg64); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    BFC_CUDA(scan_exclusive<int64_t>(deg64, g->off, n, scan64_tmp, s));
    const int bu = bits_for(r > 0 ? (uint64_t)(r - 1) : 0);
    const int bl = bits_for(l > 0 ? (uint64_t)(l - 1) : 0);
    if (m > 0) {
        if (num_graphs > 0) {
            BFC_CUDA(max_scan_inclusive(heads, rows, m, (int32_t *)scan64_tmp, s));
            k_check_batch_edges<<<grid_stride_blocks(m), kT, 0, s>>>(rows, csr->adj_u, m, graph_u_start,
                                                                     graph_l_start, num_graphs, g->err); note_launch();
            BFC_CUDA(cudaGetLastError());
            BFC_CUDA(cudaMemcpyAsync(&herr, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
            BFC_CUDA(cudaStreamSynchronize(s));
            if (herr) { set_last_error("an edge joins vertices of two different graphs of the batch"); return BFC_ERR_INVALID_GRAPH; }
        }
        // U side row by row (warp / CTA tiers, radix sort for the largest rows);
        // the swapped keys for the L side land in (k1, v1)
        const URowOut uo{m, l, bu, g->off, g->adj, g->eid, rows_star, k1, v1, g->err, opt->validate};
        k_u_rows_warp<<<grid_stride_blocks((int64_t)r * 32), kT, 0, s>>>(csr->off_u, csr->adj_u, g->rank_u,
                                                                         g->rank_l, r, uo); note_launch();
        BFC_CUDA(cudaGetLastError());
        {
            int32_t *tier_rows, *tier_n;
            GET(tmp, tier_rows, 3 * std::max<int64_t>(r, 1));
            GET(tmp, tier_n, 4);
            BFC_CUDA(cudaMemsetAsync(tier_n, 0, 4 * sizeof(int32_t), s));
            k_row_tiers<<<grid_stride_blocks(r), kT, 0, s>>>(csr->off_u, r, tier_rows, tier_n); note_launch();
            BFC_CUDA(cudaGetLastError());
            int32_t hn[3] = {0, 0, 0};
            BFC_CUDA(cudaMemcpyAsync(hn, tier_n, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            BFC_CUDA(cudaStreamSynchronize(s));
            if (hn[0] > 0) {
                const int64_t warps = std::min<int64_t>(hn[0], 152 * 64);
                k_u_rows_warp_sort<<<(unsigned)((warps * 32 + kRowCtaThreads - 1) / kRowCtaThreads), kRowCtaThreads, 0, s>>>(
                    csr->off_u, csr->adj_u, g->rank_u, g->rank_l, tier_rows, hn[0], uo); note_launch();
                BFC_CUDA(cudaGetLastError());
            }
            if (hn[1] > 0) {
                k_u_rows_cta<<<(unsigned)std::min<int32_t>(hn[1], 152 * 16), kRowCtaThreads, 0, s>>>(
                    csr->off_u, csr->adj_u, g->rank_u, g->rank_l, tier_rows + r, hn[1], uo); note_launch();
                BFC_CUDA(cudaGetLastError());
            }
            const int32_t *large_rows = tier_rows + 2 * (int64_t)r;
            const int32_t nl = hn[2];
            int64_t *ldeg, *loff;
            GET(tmp, ldeg, (int64_t)nl + 1);
            GET(tmp, loff, (int64_t)nl + 1);
            int64_t nlarge = 0;
            if (nl > 0) {
                k_large_deg<<<blocks_for(nl), kT, 0, s>>>(csr->off_u, large_rows, nl, ldeg); note_launch();
                BFC_CUDA(cudaGetLastError());
                BFC_CUDA(scan_exclusive<int64_t>(ldeg, loff, nl, scan64_tmp, s));
                BFC_CUDA(cudaMemcpyAsync(&nlarge, loff + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                BFC_CUDA(cudaStreamSynchronize(s));
            }
            if (nlarge > 0) {
                uint64_t *ka;
                int32_t *va, *rowf;
                GET(tmp, ka, nlarge); GET(tmp, va, nlarge); GET(tmp, rowf, nlarge);
                k_large_keys<<<(unsigned)std::min<int32_t>(nl, 1024), kT, 0, s>>>(csr->off_u, csr->adj_u, g->rank_u,
                                                                                   g->rank_l, large_rows, loff, nl, bl,
                                                                                   k0, v0); note_launch();
                BFC_CUDA(cudaGetLastError());
                int wl = 0;
                BFC_CUDA(radix_sort_pairs(k0, v0, ka, va, nlarge, 0, bu + bl, hist, hist_tmp, s, &wl));
                const uint64_t *kl = wl ? ka : k0;
                const int32_t *vl = wl ? va : v0;
                k_large_heads<<<grid_stride_blocks(nlarge), kT, 0, s>>>(kl, nlarge, bl, heads); note_launch();
                BFC_CUDA(cudaGetLastError());
                BFC_CUDA(max_scan_inclusive(heads, rowf, nlarge, (int32_t *)scan64_tmp, s));
                k_large_emit<<<grid_stride_blocks(nlarge), kT, 0, s>>>(kl, vl, rowf, nlarge, bl, uo); note_launch();
                BFC_CUDA(cudaGetLastError());
            }
        }
        uint64_t *ks = k0;
        int32_t *vs = v0;
        uint64_t *ko = k1;
        int32_t *vo = v1;
        // stable sort of the (rank_l, rank_u) keys on the rank_l bits only:
        // the input is already ascending in rank_u within each rank_l
        int which2 = 0;
        BFC_CUDA(radix_sort_pairs(ko, vo, ks, vs, m, bu, bu + bl, hist, hist_tmp, s, &which2));
        const uint64_t *k2 = which2 ? ks : ko;
        const int32_t *v2 = which2 ? vs : vo;
        k_emit_l_side<<<grid_stride_blocks(m), kT, 0, s>>>(k2, v2, m, bu, l, g->adj, g->eid,
                                                            rows_star); note_launch();
        BFC_CUDA(cudaGetLastError());
        if (opt->validate) {
            BFC_CUDA(cudaMemcpyAsync(&herr, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
            BFC_CUDA(cudaStreamSynchronize(s));
            if (herr & kErrDuplicate) { set_last_error("duplicate edge"); return BFC_ERR_INVALID_GRAPH; }
        }
    }

    // ---- a4: cut, per-middle prefix lengths, per-start work, W
    BFC_CUDA(cudaMemsetAsync(red, 0, 8 * sizeof(unsigned long long), s));
    if (n > 0) {
        k_cut<<<blocks_for(n), kT, 0, s>>>(g->off, g->adj, deg_star, n, l, g->cut); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    GET(g->mem, g->sbeg, std::max<int64_t>(2 * m, 1));
    if (m > 0 && opt->orientation == 0) {
        k_plen<<<grid_stride_blocks(2 * m), kT, 0, s>>>(g->off, g->adj, rows_star, g->cut, 2 * m,
                                                         g->plen, g->sbeg); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    if (m > 0 && opt->orientation == 1) {
        k_slen<<<grid_stride_blocks(2 * m), kT, 0, s>>>(g->off, g->adj, rows_star, g->cut, 2 * m,
                                                         g->plen, g->sbeg); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    if (n > 0) {
        k_work<<<grid_stride_blocks((int64_t)n * 32), kT, 0, s>>>(g->off, g->cut, g->plen, n,
                                                                   opt->orientation, g->work, red); note_launch();
        BFC_CUDA(cudaGetLastError());
        BFC_CUDA(reduce_max_u64(g->work, n, red + 1, s));
    }
    if (num_graphs > 0 && n > 0) {
        k_graph_work<<<grid_stride_blocks(n), kT, 0, s>>>(g->work, g->gstar, n, g->gwork); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    const bool core_auto = opt->core_vertices < 0 && opt->orientation == 0 && num_graphs == 0;
    if (core_auto && n > 0) {
        k_count_heavy<<<grid_stride_blocks(n), kT, 0, s>>>(g->work, n, (uint64_t)opt->hash_max_work, red + 2); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    unsigned long long hred[3] = {0, 0, 0};
    BFC_CUDA(cudaMemcpyAsync(hred, red, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    BFC_CUDA(cudaStreamSynchronize(s));
    g->info.wedges = hred[0];
    g->info.max_start_work = hred[1];

    // ---- dense-core hybrid (Algorithm 2 single graphs): the requested core
    // size, or (core_vertices = -1) as many vertices as starts heavier than
    // the CTA-hash bin, at most kCoreAutoMax
    // (an automatic core below 2 x kCoreAutoMinLayer vertices cannot hold
    // both layers: nothing is launched for it)
    if (opt->core_vertices != 0 && opt->orientation == 0 && num_graphs == 0 &&
        !(core_auto && hred[2] < 2ull * kCoreAutoMinLayer)) {
        const int32_t k = core_auto ? (int32_t)std::min<unsigned long long>(hred[2], (unsigned long long)kCoreAutoMax)
                                    : opt->core_vertices;
        int rc = core_prepare(g, s, deg_star, k, core_auto);
        if (rc) return rc;
    }
    g->info.core_u = g->core_u;
    g->info.core_l = g->core_l;

    // ---- a5: heaviest-first order and bins
    {
        int rc = schedule_graph(g, s, opt->warp_max_work, opt->team_max_work, opt->hash_max_work, rows_star);
        if (rc) return rc;
    }
    g->info.num_u = r; g->info.num_l = l; g->info.num_edges = m;
    g->info.device_bytes = (int64_t)g->mem.total;
    BFC_CUDA(cudaStreamSynchronize(s));
#undef GET
    return BFC_OK;
}

// ----------------------------------------------------------------------------
// Batch plan: a batch of a fixed shape prepared and counted with no host
// synchronisation and no allocation, so the whole step can be captured in a
// CUDA graph and replayed on new contents.  Sizes that prepare_graph reads
// back to the host come from the shape instead: the degree bits of the rank
// keys from the largest layer of one graph, the row tiers and the bin sizes
// from counts in device memory that the kernels read themselves, and every
// dense start is one end-range chunk (a graph's layer holds at most 65,535
// vertices, so counts fit 16 bits and the end range one chunk).
// ----------------------------------------------------------------------------
namespace {

constexpr int32_t kPlanMaxLayer = 65535;
constexpr int kBitmapWords = (kPlanMaxLayer + 1) / 32;   // 2,048 words, 8 KB

// U rows of more than 4,096 neighbours, one CTA per row.  The row's L ranks
// are distinct and lie in its graph's L rank range, so a bitmap of that range
// gives every neighbour its position: the number of set bits below its rank.
// A bit that is already set is a duplicate edge.
__global__ void __launch_bounds__(kRowCtaThreads) k_u_rows_bitmap(
    const int32_t *__restrict__ off_u, const int32_t *__restrict__ adj_u,
    const int32_t *__restrict__ rank_u, const int32_t *__restrict__ rank_l,
    const int32_t *__restrict__ rows, const int32_t *__restrict__ nrows_dev,
    const int32_t *__restrict__ gl, const int32_t *__restrict__ gu, int32_t num_graphs, URowOut o,
    const int *guard) {
    if (aborted(guard)) return;
    __shared__ uint32_t bits[kBitmapWords];
    __shared__ int32_t wpre[kBitmapWords];
    __shared__ int32_t part[kRowCtaThreads / 32];
    constexpr int kPerThread = kBitmapWords / kRowCtaThreads;   // 8 words
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t nrows = *nrows_dev;
    for (int64_t i0 = blockIdx.x; i0 < nrows; i0 += gridDim.x) {
        const int32_t u = rows[i0];
        const int32_t b = off_u[u], d = off_u[u + 1] - b;
        const int32_t g = graph_of(gu, num_graphs, u);
        const int32_t base = gl[g];   // the graph's L ranks: [gl[g], gl[g + 1])
        for (int i = tid; i < kBitmapWords; i += kRowCtaThreads) bits[i] = 0;
        __syncthreads();
        for (int32_t i = tid; i < d; i += kRowCtaThreads) {
            // every edge stays inside its graph (checked), so 0 <= k < 65,536
            const int32_t k = rank_l[adj_u[b + i]] - base;
            const uint32_t bit = 1u << (k & 31);
            const uint32_t old = atomicOr(&bits[k >> 5], bit);
            if ((old & bit) && o.check_dup) atomicOr(o.err, kErrDuplicate);
        }
        __syncthreads();
        // exclusive prefix of the words' popcounts: 8 words per thread
        int32_t loc[kPerThread], sum = 0;
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            loc[j] = sum;
            sum += __popc(bits[tid * kPerThread + j]);
        }
        int32_t incl = sum;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, incl, dd);
            if (lane >= dd) incl += t;
        }
        if (lane == 31) part[warp] = incl;
        __syncthreads();
        int32_t before = 0;
        for (int w = 0; w < warp; ++w) before += part[w];
        before += incl - sum;
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) wpre[tid * kPerThread + j] = before + loc[j];
        __syncthreads();
        const int32_t ru = rank_u[u];
        for (int32_t i = tid; i < d; i += kRowCtaThreads) {
            const int32_t rl = rank_l[adj_u[b + i]];
            const int32_t k = rl - base;
            const int32_t pos = wpre[k >> 5] + __popc(bits[k >> 5] & ((1u << (k & 31)) - 1u));
            o.put(ru, pos, rl, b + i);
        }
        __syncthreads();   // the bitmap is reused by the next row
    }
}

// heaviest first by exact work, 32 key bits (work saturated at 2^32 - 1)
__global__ void k_sched_keys_plan(const uint64_t *__restrict__ work, int32_t n, uint64_t *keys,
                                  int32_t *vals, const int *guard) {
    if (aborted(guard)) return;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint64_t w = work[x];
    keys[x] = 0xFFFFFFFFull - (w < 0xFFFFFFFFull ? w : 0xFFFFFFFFull);
    vals[x] = (int32_t)x;
}

// the item lists from the sorted order and the bin sizes on the device: a
// dense start is one chunk, so the lists follow the order directly
__global__ void k_emit_items_plan(const int32_t *__restrict__ order,
                                  const unsigned long long *__restrict__ counts, int2 *cta_items,
                                  int32_t *team_items, int32_t *warp_items, const int *guard) {
    if (aborted(guard)) return;
    const int64_t nd = (int64_t)counts[0], nh = (int64_t)counts[1], nt = (int64_t)counts[2],
                  nw = (int64_t)counts[3];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd + nh + nt + nw;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = order[i];
        if (i < nd) cta_items[i] = make_int2(x, 0);
        else if (i < nd + nh) cta_items[i] = make_int2(x, -1);
        else if (i < nd + nh + nt) team_items[i - nd - nh] = x;
        else warp_items[i - nd - nh - nt] = x;
    }
}

__global__ void k_plan_status(const int *__restrict__ err, int check_dup, int32_t *status) {
    const int e = *err;
    int32_t st = BFC_OK;
    if (e & (kErrBadOffsets | kErrBadId)) st = BFC_ERR_INVALID_GRAPH;
    else if ((e & kErrDuplicate) && check_dup) st = BFC_ERR_INVALID_GRAPH;
    else if (e & kErrTimeout) st = BFC_ERR_TIMEOUT;
    else if (e & (kErrHashFull | kErrBounds)) st = BFC_ERR_INTERNAL;
    *status = st;
}

}  // namespace

int batch_plan_create(BatchPlan *pl, cudaStream_t s) {
    Graph *g = &pl->g;
    const int32_t r = pl->r, l = pl->l, n = r + l, G = pl->num_graphs;
    const int64_t m = pl->m;
    g->r = r; g->l = l; g->n = n; g->m = m;
    g->num_graphs = G;
    g->stream = s;
    g->mem.stream = s;
#define GET(ptr, cnt)                                                                 \
    do {                                                                              \
        cudaError_t e_ = g->mem.get(&(ptr), (size_t)std::max<int64_t>((int64_t)(cnt), 1)); \
        if (e_ != cudaSuccess) {                                                      \
            set_last_error(std::string("device allocation failed: ") + #ptr);         \
            return BFC_ERR_OUT_OF_MEMORY;                                             \
        }                                                                             \
    } while (0)
    // kept arrays (those of prepare_graph for a batch)
    GET(g->err, 4); GET(g->rank_u, r); GET(g->rank_l, l); GET(g->off, (int64_t)n + 1);
    GET(g->adj, 2 * m); GET(g->eid, 2 * m); GET(g->plen, 2 * m); GET(g->cut, n); GET(g->work, n);
    GET(g->cursors, 8); GET(g->acc, 2); GET(g->pv, 1); GET(g->sbeg, 2 * m);
    GET(g->gstar, n); GET(g->vbase, n); GET(g->vend, n); GET(g->gwork, G);
    GET(g->cta_items, n); GET(g->team_items, n); GET(g->warp_items, n); GET(g->retry, 1);
    // temporaries, kept with the plan
    const int64_t nsort = std::max<int64_t>({(int64_t)r, (int64_t)l, m, (int64_t)n, 1});
    GET(pl->k0, nsort + 1); GET(pl->k1, nsort + 1); GET(pl->v0, nsort); GET(pl->v1, nsort);
    GET(pl->deg_u, r); GET(pl->deg_l, l); GET(pl->deg_star, n);
    GET(pl->rows, m); GET(pl->heads, m); GET(pl->rows_star, 2 * m);
    GET(pl->tier_rows, 3 * (int64_t)std::max(r, 1)); GET(pl->tier_n, 4);
    GET(pl->hist, radix_hist_elems(nsort));
    GET(pl->hist_tmp, scan_tmp_elems<uint32_t>((int64_t)radix_hist_elems(nsort)));
    GET(pl->scan64_tmp, std::max(scan_tmp_elems<int64_t>((int64_t)n + 1), max_scan_tmp_elems(m)));
    GET(pl->deg64, (int64_t)n + 1); GET(pl->red, 8);
#undef GET
    // every kept array starts zeroed: a run that stops at the checks leaves
    // arrays that later kernels can still index safely
    for (int i = 0; i < g->mem.n; ++i) BFC_CUDA(cudaMemsetAsync(g->mem.ptr[i], 0, g->mem.bytes[i], s));
    g->n_cta_items = 0; g->n_team_items = 0; g->n_warp_items = 0;
    g->retry_static = 0; g->retry_cap = 1; g->may_retry = false;
    g->info.num_u = r; g->info.num_l = l; g->info.num_edges = m;
    g->info.device_bytes = (int64_t)g->mem.total;
    // the radix sort's and the count's kernel attributes are set here, outside
    // any capture: a two-key sort and the count's per-device setup
    int which = 0;
    BFC_CUDA(radix_sort_pairs(pl->k0, pl->v0, pl->k1, pl->v1, 2, 0, 8, pl->hist, pl->hist_tmp, s, &which));
    int rc = count_smem_setup(g->device);
    if (rc) return rc;
    BFC_CUDA(cudaStreamSynchronize(s));
    return BFC_OK;
}

int batch_plan_run(BatchPlan *pl, const int32_t *off_u, const int32_t *adj_u, const int32_t *gu,
                   const int32_t *gl, cudaStream_t s, unsigned long long *totals, int32_t *status) {
    Graph *g = &pl->g;
    const int32_t r = pl->r, l = pl->l, n = r + l, G = pl->num_graphs;
    const int64_t m = pl->m;
    const int *guard = g->err;
    g->stream = s;
    const bfc_options *opt = &g->opt;
    BFC_CUDA(cudaMemsetAsync(g->err, 0, 4 * sizeof(int), s));
    // ---- checks: the CSR, the graph start arrays, edges inside their graph
    k_check_offsets<<<blocks_for((int64_t)r + 1), kT, 0, s>>>(off_u, r, m, g->err); note_launch();
    if (m > 0) { k_check_ids<<<grid_stride_blocks(m), kT, 0, s>>>(adj_u, m, l, g->err); note_launch(); }
    k_check_starts<<<blocks_for((int64_t)G + 1), kT, 0, s>>>(gu, G, r, g->err, pl->max_layer); note_launch();
    k_check_starts<<<blocks_for((int64_t)G + 1), kT, 0, s>>>(gl, G, l, g->err, pl->max_layer); note_launch();
    BFC_CUDA(cudaGetLastError());
    // ---- a1: degrees
    BFC_CUDA(cudaMemsetAsync(pl->deg_l, 0, sizeof(int32_t) * std::max<int64_t>(l, 1), s));
    BFC_CUDA(cudaMemsetAsync(pl->heads, 0, sizeof(int32_t) * std::max<int64_t>(m, 1), s));
    if (r > 0) { k_deg_u<<<blocks_for(r), kT, 0, s>>>(off_u, r, pl->deg_u, pl->heads, guard); note_launch(); }
    if (m > 0) { k_deg_l<<<grid_stride_blocks(m), kT, 0, s>>>(adj_u, m, pl->deg_l, guard); note_launch(); }
    BFC_CUDA(cudaGetLastError());
    // ---- a2: graph-major ranks; a degree is below 2^bdeg (at most the other layer)
    const int bdeg = bits_for((uint64_t)pl->max_layer);
    const int bkey = bdeg + bits_for((uint64_t)(G - 1));
    const uint64_t dmask = (1ull << bdeg) - 1;
    int which = 0;
    for (int side = 0; side < 2; ++side) {
        const int32_t cnt = side == 0 ? r : l;
        if (cnt == 0) continue;
        const int32_t *deg = side == 0 ? pl->deg_u : pl->deg_l;
        const int32_t *start = side == 0 ? gu : gl;
        k_iota_keys_batch<<<blocks_for(cnt), kT, 0, s>>>(deg, cnt, start, G, bdeg, pl->k0, pl->v0, guard); note_launch();
        BFC_CUDA(cudaGetLastError());
        BFC_CUDA(radix_sort_pairs(pl->k0, pl->v0, pl->k1, pl->v1, cnt, 0, bkey, pl->hist, pl->hist_tmp, s, &which));
        const uint64_t *ks = which ? pl->k1 : pl->k0;
        const int32_t *vs = which ? pl->v1 : pl->v0;
        k_ranks<<<blocks_for(cnt), kT, 0, s>>>(ks, vs, cnt, side == 0 ? g->rank_u : g->rank_l, pl->deg_star,
                                               side == 0 ? l : 0, dmask, guard); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    if (n > 0) {
        k_graph_star<<<grid_stride_blocks(n), kT, 0, s>>>(r, l, gu, gl, G, g->gstar, g->vbase, g->vend, guard); note_launch();
        k_deg_to_i64<<<blocks_for(n), kT, 0, s>>>(pl->deg_star, n, pl->deg64, guard); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    BFC_CUDA(scan_exclusive<int64_t>(pl->deg64, g->off, n, pl->scan64_tmp, s));
    // ---- a3: G*
    const int bu = bits_for(r > 0 ? (uint64_t)(r - 1) : 0);
    const int bl = bits_for(l > 0 ? (uint64_t)(l - 1) : 0);
    if (m > 0) {
        BFC_CUDA(max_scan_inclusive(pl->heads, pl->rows, m, (int32_t *)pl->scan64_tmp, s));
        k_check_batch_edges<<<grid_stride_blocks(m), kT, 0, s>>>(pl->rows, adj_u, m, gu, gl, G, g->err, guard); note_launch();
        const URowOut uo{m, l, bu, g->off, g->adj, g->eid, pl->rows_star, pl->k1, pl->v1, g->err, opt->validate};
        k_u_rows_warp<<<grid_stride_blocks((int64_t)r * 32), kT, 0, s>>>(off_u, adj_u, g->rank_u, g->rank_l, r, uo,
                                                                         guard); note_launch();
        BFC_CUDA(cudaMemsetAsync(pl->tier_n, 0, 4 * sizeof(int32_t), s));
        k_row_tiers<<<grid_stride_blocks(r), kT, 0, s>>>(off_u, r, pl->tier_rows, pl->tier_n, guard); note_launch();
        k_u_rows_warp_sort<<<152 * 8, kRowCtaThreads, 0, s>>>(off_u, adj_u, g->rank_u, g->rank_l, pl->tier_rows, 0,
                                                              uo, guard, pl->tier_n); note_launch();
        k_u_rows_cta<<<152 * 16, kRowCtaThreads, 0, s>>>(off_u, adj_u, g->rank_u, g->rank_l, pl->tier_rows + r, 0,
                                                         uo, guard, pl->tier_n + 1); note_launch();
        k_u_rows_bitmap<<<152 * 4, kRowCtaThreads, 0, s>>>(off_u, adj_u, g->rank_u, g->rank_l,
                                                           pl->tier_rows + 2 * (int64_t)r, pl->tier_n + 2, gl, gu,
                                                           G, uo, guard); note_launch();
        BFC_CUDA(cudaGetLastError());
        // L side: stable sort of the swapped keys on their rank_l bits
        int which2 = 0;
        BFC_CUDA(radix_sort_pairs(pl->k1, pl->v1, pl->k0, pl->v0, m, bu, bu + bl, pl->hist, pl->hist_tmp, s, &which2));
        const uint64_t *k2 = which2 ? pl->k0 : pl->k1;
        const int32_t *v2 = which2 ? pl->v0 : pl->v1;
        k_emit_l_side<<<grid_stride_blocks(m), kT, 0, s>>>(k2, v2, m, bu, l, g->adj, g->eid, pl->rows_star,
                                                            guard); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    // ---- a4: cut, runs, work
    BFC_CUDA(cudaMemsetAsync(pl->red, 0, 8 * sizeof(unsigned long long), s));
    if (n > 0) { k_cut<<<blocks_for(n), kT, 0, s>>>(g->off, g->adj, pl->deg_star, n, l, g->cut, guard); note_launch(); }
    if (m > 0) {
        k_plen<<<grid_stride_blocks(2 * m), kT, 0, s>>>(g->off, g->adj, pl->rows_star, g->cut, 2 * m, g->plen,
                                                         g->sbeg, guard); note_launch();
    }
    if (n > 0) {
        k_work<<<grid_stride_blocks((int64_t)n * 32), kT, 0, s>>>(g->off, g->cut, g->plen, n, 0, g->work, pl->red,
                                                                   guard); note_launch();
        BFC_CUDA(cudaMemsetAsync(g->gwork, 0, sizeof(unsigned long long) * G, s));
        k_graph_work<<<grid_stride_blocks(n), kT, 0, s>>>(g->work, g->gstar, n, g->gwork, guard); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    // ---- a5: heaviest first, bins from device counts
    unsigned long long *bins = pl->red + 4;
    if (n > 0) {
        k_sched_keys_plan<<<blocks_for(n), kT, 0, s>>>(g->work, n, pl->k0, pl->v0, guard); note_launch();
        BFC_CUDA(cudaGetLastError());
        BFC_CUDA(radix_sort_pairs(pl->k0, pl->v0, pl->k1, pl->v1, n, 0, 32, pl->hist, pl->hist_tmp, s, &which));
        const int32_t *order = which ? pl->v1 : pl->v0;
        k_classify<<<grid_stride_blocks(n), kT, 0, s>>>(g->work, n, (uint64_t)opt->warp_max_work,
                                                        (uint64_t)pl->team_max, (uint64_t)opt->hash_max_work, l, n, n,
                                                        bins, guard); note_launch();
        k_emit_items_plan<<<grid_stride_blocks(n), kT, 0, s>>>(order, bins, g->cta_items, g->team_items,
                                                               g->warp_items, guard); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    // ---- a6-a7: one persistent count; per-graph totals
    BFC_CUDA(cudaMemsetAsync(totals, 0, sizeof(unsigned long long) * G, s));
    g->item_counts = bins;
    int rc = launch_count(g, s, kModeBatch, nullptr, nullptr, totals);
    if (rc) return rc;
    if (status) {
        k_plan_status<<<1, 1, 0, s>>>(g->err, opt->validate, status); note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    return BFC_OK;
}

}  // namespace bfc
