// Steps a6-a9: wedge enumeration with per-start aggregation (Algorithm 2),
// the reduction to ⋈_G, and the per-vertex / per-edge second walk
// (Algorithm 4 in the orientation of Algorithm 2).
//
// One persistent launch, one CTA of 1024 threads per SM.  Each CTA first
// takes CTA work items from a global queue (heaviest first, Section 6.2's
// dynamic scheduling with the exact per-start workload), then its 32 warps
// take single light starts from a second queue.
//
//   dense item (x, c): the wedges of start x whose end lies in the c-th
//       chunk of x's end range [0, rank(x)); count_wedge is a dense array in
//       shared memory (16-bit counts when cut[x] <= 65535, else 32-bit).
//       Chunks split the END range, so every pair (x, w) is aggregated by
//       exactly one item and C(count, 2) is never split.
//   hash item (x): a start with at most 16,384 wedges; count_wedge is an
//       open-addressing hash table in shared memory.
//   warp item (x): a start with at most 256 wedges, one warp, a per-warp
//       hash table.
//
// Aggregation uses the running form of Lemma 1: adding old = count_wedge(w)
// before each increment gives Σ_w C(count_wedge(w), 2) exactly.
#include "bfc_internal.cuh"

#ifndef BFC_CHECKED
#define BFC_CHECKED 1
#endif

namespace bfc {

namespace {

struct CountParams {
    const int64_t *__restrict__ off;
    const int32_t *__restrict__ adj;
    const int32_t *__restrict__ eid;
    const int32_t *__restrict__ plen;
    const int32_t *__restrict__ cut;
    const uint64_t *__restrict__ work;
    const int2 *__restrict__ cta_items;
    const int32_t *__restrict__ warp_items;
    int64_t n_cta;
    int64_t n_warp;
    int *cursors;
    unsigned long long *acc;
    unsigned long long *pv;   // [n] in G* ids
    unsigned long long *pe;   // [m] by edge id
    const int32_t *__restrict__ coff;  // chunk-boundary table (nullable)
    const int32_t *__restrict__ gstar; // graph of each G* vertex (batch mode)
    const int32_t *__restrict__ vbase; // first id of x's graph in x's layer (batch mode)
    const int32_t *__restrict__ vend;  // one past the last id of x's graph in x's layer (batch mode)
    const int64_t *__restrict__ sbeg;  // Algorithm 3: start of each slot's run of ends
    int32_t *retry;                    // Algorithm 3: starts left to the chunked retry pass
    int64_t retry_cap;
    int64_t retry_static;              // retry[0, retry_static) were assigned by prepare
    int32_t orient;                    // 0 = Algorithm 2, 1 = Algorithm 3
    int32_t n;
    unsigned long long *gtot;          // per-graph totals (batch mode)
    int32_t coff_u1, coff_l1;          // entries per L vertex / per U vertex
    int64_t adj_len;
    int32_t l;
    int *err;
};

// Middles per batch: two per thread when adjacency positions fit 32 bits,
// one otherwise (shared memory holds the compacted batch).
template <typename Pos>
struct Batch {
    static constexpr int kSize = sizeof(Pos) == 4 ? 2 * kCountThreads : kCountThreads;
    static constexpr int kPer = kSize / kCountThreads;
};

template <int MODE, typename Pos>
struct SharedCTA {
    static constexpr int kB = Batch<Pos>::kSize;
    int32_t start[kB + 1];              // compacted batch: exclusive prefix of run lengths (+ sentinel)
    Pos src[kB];                        // compacted batch: adjacency position of a run minus its prefix
    unsigned long long msum[has_second_walk(MODE) ? kB : 1];  // second walk: Σ δ per compacted middle
    long long wtot[32];
    unsigned long long red[32];
    int item;
    int overflow;   // Algorithm 3: this item's hash table filled up
    int inserts;    // Algorithm 3: distinct ends inserted so far
};

__device__ __forceinline__ unsigned long long c2(unsigned long long c) {
    return c < 2 ? 0ull : c * (c - 1) / 2;
}

__device__ __forceinline__ int lower_bound_g(const int32_t *a, int len, int32_t key) {
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Exclusive block scan of one int64 per thread (1024 threads).
template <class SH>
__device__ __forceinline__ long long block_excl_scan(long long v, SH &sh, long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long o = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += o;
    }
    if (lane == 31) sh.wtot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = sh.wtot[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            long long o = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += o;
        }
        sh.wtot[lane] = w;
    }
    __syncthreads();
    long long before = warp > 0 ? sh.wtot[warp - 1] : 0;
    *total = sh.wtot[31];
    return before + x - v;
}

template <class SH>
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, SH &sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    __syncthreads();
    if (lane == 0) sh.red[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (warp == 0) {
        t = sh.red[lane];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
    }
    return t;   // valid in warp 0
}

// largest j in [0, n) with a[j] <= k, given a[0] <= k and a ascending
__device__ __forceinline__ int last_le(const int32_t *a, int n, int32_t k) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= k) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t hash_slot(int32_t key, uint32_t mask) {
    return ((uint32_t)key * 0x9E3779B1u) & mask;
}

// Finds (inserting if absent) the slot of `key`.  Returns -1 if the table is
// full, which the slot sizing rules out.
__device__ __forceinline__ int hash_find(int32_t *keys, uint32_t mask, int32_t key, bool insert,
                                         int *inserted = nullptr) {
    uint32_t h = hash_slot(key, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        int32_t k = *((volatile int32_t *)(keys + h));
        if (k == key) return (int)h;
        if (k == -1) {
            if (!insert) return -1;
            int32_t prev = atomicCAS(keys + h, -1, key);
            if (prev == -1) {
                if (inserted) *inserted = 1;
                return (int)h;
            }
            if (prev == key) return (int)h;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// 16-bit counters packed two per 32-bit word
__device__ __forceinline__ uint32_t inc16(uint32_t *w32, int idx) {
    const uint32_t sh = (uint32_t)(idx & 1) << 4;
    uint32_t old = atomicAdd(w32 + (idx >> 1), 1u << sh);
    return (old >> sh) & 0xffffu;
}
__device__ __forceinline__ uint32_t get16(const uint32_t *w32, int idx) {
    const uint32_t sh = (uint32_t)(idx & 1) << 4;
    return (w32[idx >> 1] >> sh) & 0xffffu;
}

enum CounterKind { kDenseNarrow = 0, kDenseWide = 1, kHash = 2 };

// The counter operation for one wedge (x, middle, w) whose end id is w and
// whose end sits at adjacency slot pos.  First walk: increment count_wedge(w)
// and return the old value.  Second walk: read the final count and attribute
// δ = count − 1 to the edge (middle, w) and to the middle's batch sum.
template <int MODE, int KIND, bool kSecond, typename Pos>
__device__ __forceinline__ unsigned long long wedge_op(const CountParams &p, int32_t w,
                                                       Pos pos, int q, int32_t lb, int32_t lo,
                                                       int32_t span, uint32_t hmask,
                                                       unsigned char *ctr,
                                                       unsigned long long *msum, int *ovf,
                                                       int *ins) {
    uint32_t *w32 = reinterpret_cast<uint32_t *>(ctr);
    uint32_t c;
    if (KIND == kHash) {
        int32_t *hkeys = reinterpret_cast<int32_t *>(ctr);
        uint32_t *hcnt = reinterpret_cast<uint32_t *>(ctr + (size_t)(hmask + 1) * 4);
        int inserted = 0;
        const int slot = hash_find(hkeys, hmask, w - lb, !kSecond, &inserted);
        if (slot < 0) {
            // Algorithm 3 sizes tables by a guess: a full table sends the start
            // to the retry pass; Algorithm 2's sizing rules it out
            if (p.orient && !kSecond) *ovf = 1; else atomicOr(p.err, kErrHashFull);
            return 0;
        }
        if (!kSecond) {
            if (inserted && p.orient && atomicAdd(ins, 1) >= (int)((hmask + 1) / 4 * 3)) *ovf = 1;
            return inc16(hcnt, slot);
        }
        c = get16(hcnt, slot);
    } else {
        const int idx = w - lb - lo;
#if BFC_CHECKED
        if ((uint32_t)idx >= (uint32_t)span) { atomicOr(p.err, kErrBounds); return 0; }
#endif
        if (!kSecond) return (KIND == kDenseWide) ? atomicAdd(w32 + idx, 1u) : inc16(w32, idx);
        c = (KIND == kDenseWide) ? w32[idx] : get16(w32, idx);
    }
    const unsigned long long delta = (unsigned long long)c - 1ull;
    if (delta) {
        if (MODE == kModeEdges) atomicAdd(p.pe + __ldg(p.eid + pos), delta);
        atomicAdd(msum + q, delta);
    }
    return 0;
}

// One walk over the wedges of start x whose ends fall in [lb+lo, lb+hi).
// kSecond = false: count (returns Σ old, i.e. Σ C(count, 2)).
// kSecond = true : read the final counts and attribute δ = count − 1.
//
// The middles of x are taken a batch at a time (2048, or 1024 with 64-bit
// positions).  For each middle, the run of ends in range is [s0, s1) of its
// list (from the chunk-boundary table, or a binary search when there is
// none).  Non-empty runs are compacted and their concatenation is cut into
// windows of 32 wedges; each warp takes a contiguous range of windows.
// Inside a window the run of every lane is found from a 32-bit mask of run
// starts (reduce-or + popc), so no search is needed per wedge, and four
// windows are in flight per iteration so their end loads overlap.
template <int MODE, int KIND, bool kSecond, typename Pos, class SH>
__device__ unsigned long long cta_walk(const CountParams &p, int32_t x, int32_t lb, int32_t lo,
                                       int32_t hi, int flags, uint32_t hmask, unsigned char *ctr,
                                       SH &sh) {
    constexpr int kPer = Batch<Pos>::kPer;
    constexpr int kB = Batch<Pos>::kSize;
    constexpr int kU = 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e0 = p.off[x];
    // Algorithm 2: the middles are the cut[x] lower-priority neighbours;
    // Algorithm 3: every neighbour is a middle
    const int32_t nmid = p.orient ? (int32_t)(p.off[x + 1] - e0) : p.cut[x];
    const int32_t span = hi - lo;
    const uint32_t le_mask = 0xffffffffu >> (31 - lane);
    unsigned long long acc = 0;
    for (int32_t mb = 0; mb < nmid; mb += kB) {
        int32_t len[kPer], v[kPer];
        Pos src[kPer];
        int64_t e[kPer];
        long long packed_run = 0;
        long long pk[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int32_t j = mb + i * kCountThreads + tid;
            len[i] = 0; v[i] = 0; src[i] = 0; e[i] = 0;
            if (j < nmid) {
                e[i] = e0 + j;
                v[i] = __ldg(p.adj + e[i]);
                const int32_t pl = __ldg(p.plen + e[i]);
                // run of ends: prefix of N(v) below x (Algorithm 2) or the
                // suffix above both x and v (Algorithm 3)
                const int64_t b = p.orient ? __ldg(p.sbeg + e[i]) : __ldg(p.off + v[i]);
                int32_t s0 = 0, s1 = pl;
                if (KIND != kHash) {
                    if (p.coff) {
                        const int64_t tb = v[i] < p.l ? (int64_t)v[i] * p.coff_u1
                                                      : (int64_t)p.l * p.coff_u1 + (int64_t)(v[i] - p.l) * p.coff_l1;
                        if (flags & 1) s0 = __ldg(p.coff + tb + lo / kChunkUnit);
                        if (flags & 2) s1 = __ldg(p.coff + tb + hi / kChunkUnit);
                    } else {
                        if (flags & 1) s0 = lower_bound_g(p.adj + b, pl, lb + lo);
                        if (flags & 2) s1 = lower_bound_g(p.adj + b, pl, lb + hi);
                    }
                }
                len[i] = s1 - s0;
                src[i] = (Pos)(b + s0);
            }
            // run length in the high bits, "non-empty" in the low 20 bits:
            // one scan yields both the run offsets and the compacted slots
            pk[i] = ((long long)len[i] << 20) | (len[i] > 0 ? 1 : 0);
            packed_run += pk[i];
        }
        long long packed_total;
        long long packed = block_excl_scan(packed_run, sh, &packed_total);
        const int32_t total = (int32_t)(packed_total >> 20);
        const int nnz = (int)(packed_total & 0xfffff);
        int nzs[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int32_t excl = (int32_t)(packed >> 20);
            nzs[i] = (int)(packed & 0xfffff);
            if (len[i] > 0) {
                sh.start[nzs[i]] = excl;
                sh.src[nzs[i]] = src[i] - (Pos)excl;
                if (kSecond) sh.msum[nzs[i]] = 0;
            }
            packed += pk[i];
        }
        if (tid == 0) sh.start[nnz] = total;
        __syncthreads();
        const int32_t nwin = (total + 31) >> 5;
        int32_t wb = (int32_t)(((int64_t)warp * nwin) >> 5);
        const int32_t wend = (int32_t)(((int64_t)(warp + 1) * nwin) >> 5);
        if (wb < wend) {
            int32_t k0 = wb << 5;
            int q0 = last_le(sh.start, nnz, k0);
            for (; wb < wend; wb += kU) {
                int q[kU];
                Pos pos[kU];
                bool ok[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    q[u] = 0;
                    ok[u] = false;
                    pos[u] = 0;
                    if (wb + u < wend) {   // warp-uniform
                        const int32_t kw = k0 + 32 * u;
                        const int idx = q0 + 1 + lane;
                        const int32_t d = (idx <= nnz ? sh.start[idx] : 0x7fffffff) - kw;
                        const uint32_t m = __reduce_or_sync(0xffffffffu, d < 32 ? (1u << d) : 0u);
                        q[u] = q0 + __popc(m & le_mask);
                        q0 += __popc(__ballot_sync(0xffffffffu, d <= 32));
                        ok[u] = kw + lane < total;
                        if (ok[u]) pos[u] = sh.src[q[u]] + (Pos)(kw + lane);
                    }
                }
                int32_t w[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
#if BFC_CHECKED
                    if (ok[u] && (unsigned long long)pos[u] >= (unsigned long long)p.adj_len) {
                        atomicOr(p.err, kErrBounds);
                        ok[u] = false;
                    }
#endif
                    w[u] = ok[u] ? __ldg(p.adj + pos[u]) : 0;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (ok[u]) acc += wedge_op<MODE, KIND, kSecond, Pos>(p, w[u], pos[u], q[u], lb, lo, span, hmask, ctr, sh.msum, &sh.overflow, &sh.inserts);
                k0 += 32 * kU;
            }
        }
        __syncthreads();
        if (KIND == kHash && !kSecond && sh.overflow) break;   // uniform: read after the barrier
        if (kSecond) {
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                if (len[i] > 0) {
                    const unsigned long long dsum = sh.msum[nzs[i]];
                    if (dsum) {
                        if (MODE == kModeVertices) atomicAdd(p.pv + v[i], dsum);
                        if (MODE == kModeEdges) atomicAdd(p.pe + __ldg(p.eid + e[i]), dsum);
                    }
                }
            }
        }
    }
    return acc;
}

template <int MODE, int KIND, typename Pos, class SH>
__device__ unsigned long long cta_item_body(const CountParams &p, int32_t x, int32_t lb,
                                            int32_t lo, int32_t hi, int flags, uint32_t hmask,
                                            unsigned char *ctr, SH &sh) {
    unsigned long long acc = cta_walk<MODE, KIND, false, Pos>(p, x, lb, lo, hi, flags, hmask, ctr, sh);
    if (KIND == kHash && p.orient) {
        __syncthreads();
        if (sh.overflow) return 0;   // the caller re-queues x
    }
    if (has_second_walk(MODE)) {
        __syncthreads();
        if (MODE == kModeVertices) {
            // ends: each pair (x, w) adds C(count, 2) to ⋈_w
            if (KIND == kHash) {
                const int32_t *hkeys = reinterpret_cast<const int32_t *>(ctr);
                const uint32_t *hcnt = reinterpret_cast<const uint32_t *>(ctr + (size_t)(hmask + 1) * 4);
                for (uint32_t s = threadIdx.x; s <= hmask; s += kCountThreads) {
                    const int32_t k = hkeys[s];
                    if (k >= 0) {
                        const unsigned long long b = c2(get16(hcnt, (int)s));
                        if (b) atomicAdd(p.pv + lb + k, b);
                    }
                }
            } else {
                const uint32_t *w32 = reinterpret_cast<const uint32_t *>(ctr);
                for (int32_t i = threadIdx.x; i < hi - lo; i += kCountThreads) {
                    const uint32_t c = (KIND == kDenseWide) ? w32[i] : get16(w32, i);
                    if (c >= 2) atomicAdd(p.pv + lb + lo + i, c2(c));
                }
            }
        }
        cta_walk<MODE, KIND, true, Pos>(p, x, lb, lo, hi, flags, hmask, ctr, sh);
        if (MODE == kModeVertices) {
            const unsigned long long t = block_sum(acc, sh);
            if (threadIdx.x == 0 && t) atomicAdd(p.pv + x, t);
        }
    }
    return acc;
}

__device__ __forceinline__ void zero_smem(unsigned char *p, int bytes, uint32_t fill) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    const int n16 = (bytes + 15) >> 4;
    const uint4 f = make_uint4(fill, fill, fill, fill);
    for (int i = threadIdx.x; i < n16; i += kCountThreads) q[i] = f;
}

template <int MODE, typename Pos, class SH>
__device__ unsigned long long cta_item(const CountParams &p, int2 item, unsigned char *ctr,
                                       SH &sh) {
    const int32_t x = item.x;
    // ends lie in x's layer (in a batch: x's graph's part of it) from lb on
    const int32_t lb = p.vbase ? __ldg(p.vbase + x) : (x >= p.l ? p.l : 0);
    const int32_t R = x - lb;   // Algorithm 2: the ends are the R vertices below x
    unsigned long long acc;
    if (item.y >= 0) {          // dense items exist only for Algorithm 2
        const bool wide = (uint32_t)p.cut[x] > kNarrowMaxCut;
        const int32_t S = wide ? kDense32 : kDense16;
        const int32_t lo = item.y * S;
        const int32_t hi = min(R, lo + S);
        const int32_t span = hi - lo;
        const int flags = (lo > 0 ? 1 : 0) | (hi < R ? 2 : 0);
        zero_smem(ctr, wide ? span * 4 : ((span + 1) >> 1) * 4, 0u);
        __syncthreads();
        acc = wide ? cta_item_body<MODE, kDenseWide, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh)
                   : cta_item_body<MODE, kDenseNarrow, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh);
    } else {
        // how many distinct ends x can have: the vertices below it (Algorithm 2)
        // or above it (Algorithm 3), and at most one per wedge
        unsigned long long range = (unsigned long long)R;
        if (p.orient) {
            const int32_t hiend = p.vend ? __ldg(p.vend + x) : (x >= p.l ? p.n : p.l);
            range = (unsigned long long)(hiend - x - 1);
        }
        const unsigned long long w = p.work[x];
        const unsigned long long bound = w < range ? w : range;
        uint32_t cap = 64;
        while (cap < 2 * bound && cap < (uint32_t)kHashMaxSlots) cap <<= 1;
        // Algorithm 3: counts are bounded by deg(x), which must fit 16 bits here
        const bool too_wide = p.orient && (p.off[x + 1] - p.off[x]) > (int64_t)kNarrowMaxCut;
        if (threadIdx.x == 0) { sh.overflow = too_wide ? 1 : 0; sh.inserts = 0; }
        zero_smem(ctr, (int)cap * 4, 0xffffffffu);           // keys = -1
        zero_smem(ctr + (size_t)cap * 4, (int)cap * 2, 0u);  // packed 16-bit counts
        __syncthreads();
        acc = sh.overflow ? 0ull : cta_item_body<MODE, kHash, Pos>(p, x, lb, 0, 0, 0, cap - 1, ctr, sh);
        if (p.orient && sh.overflow) {
            // discard this attempt: the retry pass counts x with dense chunks
            if (threadIdx.x == 0) {
                const int64_t k = p.retry_static + atomicAdd(p.cursors + 2, 1);
                if (k < p.retry_cap) p.retry[k] = x; else atomicOr(p.err, kErrBounds);
            }
            __syncthreads();
            return 0;
        }
    }
    if (MODE == kModeBatch) {
        // the batch is a disjoint union: every butterfly of start x lies in x's graph
        const unsigned long long t = block_sum(acc, sh);
        if (threadIdx.x == 0 && t) atomicAdd(p.gtot + p.gstar[x], t);
    }
    __syncthreads();
    return acc;
}

// ---- warp items -------------------------------------------------------------
// The warp version of cta_walk for a light start: batches of 32 middles,
// compacted runs and the same window masks, with a per-warp hash table.
template <int MODE, bool kSecond>
__device__ unsigned long long warp_walk(const CountParams &p, int32_t x, int32_t lb, uint32_t mask,
                                        int32_t *keys, uint32_t *cnt, unsigned long long *msum,
                                        int32_t *wstart, long long *wsrc) {
    const int lane = threadIdx.x & 31;
    const int64_t e0 = p.off[x];
    const int32_t nmid = p.orient ? (int32_t)(p.off[x + 1] - e0) : p.cut[x];
    const uint32_t le_mask = 0xffffffffu >> (31 - lane);
    const uint32_t lt_mask = (1u << lane) - 1u;
    unsigned long long acc = 0;
    for (int32_t mb = 0; mb < nmid; mb += 32) {
        const int32_t j = mb + lane;
        int32_t len = 0, v = 0;
        long long src = 0;
        int64_t e = 0;
        if (j < nmid) {
            e = e0 + j;
            v = __ldg(p.adj + e);
            len = __ldg(p.plen + e);
            src = p.orient ? __ldg(p.sbeg + e) : __ldg(p.off + v);
        }
        int32_t incl = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const int32_t excl = incl - len;
        const uint32_t fm = __ballot_sync(0xffffffffu, len > 0);
        const int nz = __popc(fm & lt_mask), nnz = __popc(fm);
        if (len > 0) {
            wstart[nz] = excl;
            wsrc[nz] = src - excl;
            if (kSecond) msum[nz] = 0;
        }
        if (lane == 0) wstart[nnz] = total;
        __syncwarp();
        int q0 = 0;
        for (int32_t k0 = 0; k0 < total; k0 += 32) {
            const int idx = q0 + 1 + lane;
            const int32_t d = (idx <= nnz ? wstart[idx] : 0x7fffffff) - k0;
            const uint32_t m = __reduce_or_sync(0xffffffffu, d < 32 ? (1u << d) : 0u);
            const int q = q0 + __popc(m & le_mask);
            q0 += __popc(__ballot_sync(0xffffffffu, d <= 32));
            const int32_t k = k0 + lane;
            if (k < total) {
                const long long pos = wsrc[q] + k;
#if BFC_CHECKED
                if (pos < 0 || pos >= p.adj_len) { atomicOr(p.err, kErrBounds); continue; }
#endif
                const int32_t w = __ldg(p.adj + pos);
                const int slot = hash_find(keys, mask, w - lb, !kSecond);
                if (slot < 0) { atomicOr(p.err, kErrHashFull); continue; }
                if (!kSecond) {
                    acc += atomicAdd(cnt + slot, 1u);
                } else {
                    const unsigned long long delta = (unsigned long long)cnt[slot] - 1ull;
                    if (delta) {
                        if (MODE == kModeEdges) atomicAdd(p.pe + __ldg(p.eid + pos), delta);
                        atomicAdd(msum + q, delta);
                    }
                }
            }
        }
        __syncwarp();
        if (kSecond && len > 0) {
            const unsigned long long dsum = msum[nz];
            if (dsum) {
                if (MODE == kModeVertices) atomicAdd(p.pv + v, dsum);
                if (MODE == kModeEdges) atomicAdd(p.pe + __ldg(p.eid + e), dsum);
            }
        }
        __syncwarp();
    }
    return acc;
}

// per-warp region: keys[512] | counts[512] | msum[32] | src[32] | start[33]
constexpr int kWarpCntOff = kWarpSlots * 4;
constexpr int kWarpMsumOff = kWarpSlots * 8;
constexpr int kWarpSrcOff = kWarpMsumOff + 32 * 8;
constexpr int kWarpStartOff = kWarpSrcOff + 32 * 8;
static_assert(kWarpStartOff + 33 * 4 <= kWarpRegion, "per-warp region overflow");

template <int MODE>
__device__ unsigned long long warp_item(const CountParams &p, int32_t x, unsigned char *region) {
    const int lane = threadIdx.x & 31;
    // ends lie in x's layer (in a batch: x's graph's part of it) from lb on
    const int32_t lb = p.vbase ? __ldg(p.vbase + x) : (x >= p.l ? p.l : 0);
    unsigned long long range = (unsigned long long)(x - lb);
    if (p.orient) {
        const int32_t hiend = p.vend ? __ldg(p.vend + x) : (x >= p.l ? p.n : p.l);
        range = (unsigned long long)(hiend - x - 1);
    }
    const unsigned long long w = p.work[x];
    const unsigned long long bound = w < range ? w : range;
    uint32_t cap = 32;
    while (cap < 2 * bound && cap < (uint32_t)kWarpSlots) cap <<= 1;
    int32_t *keys = reinterpret_cast<int32_t *>(region);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(region + kWarpCntOff);
    unsigned long long *msum = reinterpret_cast<unsigned long long *>(region + kWarpMsumOff);
    long long *wsrc = reinterpret_cast<long long *>(region + kWarpSrcOff);
    int32_t *wstart = reinterpret_cast<int32_t *>(region + kWarpStartOff);
    for (uint32_t s = lane; s < cap; s += 32) { keys[s] = -1; cnt[s] = 0; }
    __syncwarp();
    unsigned long long acc = warp_walk<MODE, false>(p, x, lb, cap - 1, keys, cnt, msum, wstart, wsrc);
    if (has_second_walk(MODE)) {
        __syncwarp();
        if (MODE == kModeVertices) {
            for (uint32_t s = lane; s < cap; s += 32) {
                const int32_t k = keys[s];
                if (k >= 0 && cnt[s] >= 2) atomicAdd(p.pv + lb + k, c2(cnt[s]));
            }
        }
        warp_walk<MODE, true>(p, x, lb, cap - 1, keys, cnt, msum, wstart, wsrc);
        if (MODE == kModeVertices) {
            unsigned long long t = acc;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
            if (lane == 0 && t) atomicAdd(p.pv + x, t);
        }
    }
    if (MODE == kModeBatch) {
        unsigned long long t = acc;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
        if (lane == 0 && t) atomicAdd(p.gtot + p.gstar[x], t);
    }
    __syncwarp();
    return acc;
}

template <int MODE, typename Pos>
__global__ void __launch_bounds__(kCountThreads, 1) k_count(CountParams p) {
    extern __shared__ __align__(16) unsigned char ctr[];
    __shared__ SharedCTA<MODE, Pos> sh;
    unsigned long long acc = 0;
    // phase 1: CTA items, heaviest first
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(p.cursors, 1);
        __syncthreads();
        const int64_t it = sh.item;
        __syncthreads();
        if (it >= p.n_cta) break;
        acc += cta_item<MODE, Pos>(p, p.cta_items[it], ctr, sh);
    }
    // phase 2: warp items
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        unsigned char *region = ctr + (size_t)warp * kWarpRegion;
        for (;;) {
            int it = 0;
            if (lane == 0) it = atomicAdd(p.cursors + 1, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= p.n_warp) break;
            acc += warp_item<MODE>(p, p.warp_items[it], region);
        }
    }
    // a7: reduction of the per-thread partial sums
    const unsigned long long t = block_sum(acc, sh);
    if (threadIdx.x == 0 && t) atomicAdd(p.acc, t);
}

// Algorithm 3's retry pass: the starts whose hash table filled up (or whose
// counts could pass 16 bits) are counted with dense counters, one CTA per
// start, chunk after chunk of the end range (x, end of x's layer).
template <int MODE, typename Pos>
__global__ void __launch_bounds__(kCountThreads, 1) k_count_retry(CountParams p) {
    extern __shared__ __align__(16) unsigned char ctr[];
    __shared__ SharedCTA<MODE, Pos> sh;
    unsigned long long acc = 0;
    const int nretry = (int)min(p.retry_static + *((volatile int *)(p.cursors + 2)), p.retry_cap);
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(p.cursors + 3, 1);
        __syncthreads();
        const int it = sh.item;
        __syncthreads();
        if (it >= nretry) break;
        const int32_t x = p.retry[it];
        const int32_t lb = p.vbase ? __ldg(p.vbase + x) : (x >= p.l ? p.l : 0);
        const int32_t hiend = p.vend ? __ldg(p.vend + x) : (x >= p.l ? p.n : p.l);
        const bool wide = (p.off[x + 1] - p.off[x]) > (int64_t)kNarrowMaxCut;
        const int32_t S = wide ? kDense32 : kDense16;
        const int32_t first = x + 1 - lb, last = hiend - lb;   // ends in [lb + first, lb + last)
        unsigned long long item_acc = 0;
        for (int32_t c = first / S; c * S < last; ++c) {
            const int32_t lo = max(c * S, first), hi = min((c + 1) * S, last);
            const int32_t span = hi - lo;
            const int flags = (lo > first ? 1 : 0) | (hi < last ? 2 : 0);
            zero_smem(ctr, wide ? span * 4 : ((span + 1) >> 1) * 4, 0u);
            __syncthreads();
            item_acc += wide ? cta_item_body<MODE, kDenseWide, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh)
                             : cta_item_body<MODE, kDenseNarrow, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh);
            __syncthreads();
        }
        if (MODE == kModeBatch) {
            const unsigned long long t = block_sum(item_acc, sh);
            if (threadIdx.x == 0 && t) atomicAdd(p.gtot + p.gstar[x], t);
            __syncthreads();
        }
        acc += item_acc;
    }
    const unsigned long long t = block_sum(acc, sh);
    if (threadIdx.x == 0 && t) atomicAdd(p.acc, t);
}

__global__ void k_gather_vertices(const unsigned long long *__restrict__ pv,
                                  const int32_t *__restrict__ rank_u,
                                  const int32_t *__restrict__ rank_l, int32_t r, int32_t l,
                                  uint64_t *per_u, uint64_t *per_l) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < r && per_u) per_u[i] = pv[l + rank_u[i]];
    if (i < l && per_l) per_l[i] = pv[rank_l[i]];
}

template <int MODE, typename Pos>
cudaError_t setup_one() {
    cudaError_t e = cudaFuncSetAttribute(k_count<MODE, Pos>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kCounterBytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_count_retry<MODE, Pos>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kCounterBytes);
}

}  // namespace

int count_smem_setup(int device) {
    static bool done[64] = {false};
    if (device < 0 || device >= 64) return BFC_ERR_INVALID_ARGUMENT;
    if (done[device]) return BFC_OK;
    BFC_CUDA((setup_one<kModeTotal, int32_t>()));
    BFC_CUDA((setup_one<kModeVertices, int32_t>()));
    BFC_CUDA((setup_one<kModeEdges, int32_t>()));
    BFC_CUDA((setup_one<kModeTotal, long long>()));
    BFC_CUDA((setup_one<kModeBatch, int32_t>()));
    BFC_CUDA((setup_one<kModeBatch, long long>()));
    BFC_CUDA((setup_one<kModeVertices, long long>()));
    BFC_CUDA((setup_one<kModeEdges, long long>()));
    done[device] = true;
    return BFC_OK;
}

int launch_count(Graph *g, cudaStream_t s, int mode, unsigned long long *pv_proj,
                 unsigned long long *pe, unsigned long long *gtot) {
    int rc = count_smem_setup(g->device);
    if (rc) return rc;
    CountParams p;
    p.off = g->off; p.adj = g->adj; p.eid = g->eid; p.plen = g->plen; p.cut = g->cut;
    p.work = g->work; p.cta_items = g->cta_items; p.warp_items = g->warp_items;
    p.n_cta = g->n_cta_items; p.n_warp = g->n_warp_items;
    p.cursors = g->cursors; p.acc = g->acc; p.pv = pv_proj; p.pe = pe;
    p.adj_len = 2 * g->m; p.l = g->l; p.err = g->err;
    p.coff = g->coff; p.coff_u1 = g->coff_u1; p.coff_l1 = g->coff_l1;
    p.gstar = g->gstar; p.gtot = gtot; p.vbase = g->vbase;
    p.vend = g->vend; p.sbeg = g->sbeg; p.retry = g->retry; p.retry_cap = g->retry_cap;
    p.retry_static = g->retry_static;
    p.orient = g->opt.orientation; p.n = g->n;
    BFC_CUDA(cudaMemsetAsync(g->cursors, 0, 4 * sizeof(int), s));
    BFC_CUDA(cudaMemsetAsync(g->acc, 0, sizeof(unsigned long long), s));
    const int grid = g->grid;
    // 32-bit adjacency positions whenever G* has fewer than 2^31 slots
    if (2 * g->m <= 0x7fffffffll && !g->opt.wide_positions) {
        if (mode == kModeTotal) k_count<kModeTotal, int32_t><<<grid, kCountThreads, kCounterBytes, s>>>(p);
        else if (mode == kModeBatch) k_count<kModeBatch, int32_t><<<grid, kCountThreads, kCounterBytes, s>>>(p);
        else if (mode == kModeVertices) k_count<kModeVertices, int32_t><<<grid, kCountThreads, kCounterBytes, s>>>(p);
        else k_count<kModeEdges, int32_t><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    } else {
        if (mode == kModeTotal) k_count<kModeTotal, long long><<<grid, kCountThreads, kCounterBytes, s>>>(p);
        else if (mode == kModeBatch) k_count<kModeBatch, long long><<<grid, kCountThreads, kCounterBytes, s>>>(p);
        else if (mode == kModeVertices) k_count<kModeVertices, long long><<<grid, kCountThreads, kCounterBytes, s>>>(p);
        else k_count<kModeEdges, long long><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    }
    note_launch();
    BFC_CUDA(cudaGetLastError());
    if (g->opt.orientation == 1) {
        // the retry pass reads how many starts the first launch re-queued
        if (2 * g->m <= 0x7fffffffll && !g->opt.wide_positions) {
            if (mode == kModeTotal) k_count_retry<kModeTotal, int32_t><<<grid, kCountThreads, kCounterBytes, s>>>(p);
            else if (mode == kModeBatch) k_count_retry<kModeBatch, int32_t><<<grid, kCountThreads, kCounterBytes, s>>>(p);
            else if (mode == kModeVertices) k_count_retry<kModeVertices, int32_t><<<grid, kCountThreads, kCounterBytes, s>>>(p);
            else k_count_retry<kModeEdges, int32_t><<<grid, kCountThreads, kCounterBytes, s>>>(p);
        } else {
            if (mode == kModeTotal) k_count_retry<kModeTotal, long long><<<grid, kCountThreads, kCounterBytes, s>>>(p);
            else if (mode == kModeBatch) k_count_retry<kModeBatch, long long><<<grid, kCountThreads, kCounterBytes, s>>>(p);
            else if (mode == kModeVertices) k_count_retry<kModeVertices, long long><<<grid, kCountThreads, kCounterBytes, s>>>(p);
            else k_count_retry<kModeEdges, long long><<<grid, kCountThreads, kCounterBytes, s>>>(p);
        }
        note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    return BFC_OK;
}

int gather_vertices(Graph *g, cudaStream_t s, uint64_t *per_u, uint64_t *per_l) {
    const int64_t nmax = g->r > g->l ? g->r : g->l;
    if (nmax == 0) return BFC_OK;
    k_gather_vertices<<<(unsigned)((nmax + 255) / 256), 256, 0, s>>>(g->pv, g->rank_u, g->rank_l,
                                                                      g->r, g->l, per_u, per_l); note_launch();
    BFC_CUDA(cudaGetLastError());
    return BFC_OK;
}

}  // namespace bfc
