// Steps a6-a9: wedge enumeration with per-start aggregation, the reduction
// to ⋈_G, and the per-vertex / per-edge second walk (Algorithm 4).
//
// Two orientations of the same wedge set (Lemma 4):
//   Algorithm 2 (orient 0): start u highest; the middles v with p(v) < p(u)
//     are the first cut[u] entries of N(u); the ends w with p(w) < p(u) are
//     the prefix of N(v) below u.
//   Algorithm 3 (orient 1): end w highest; every neighbour v of the start u
//     is a middle; the ends are the suffix of N(v) above both u and v.
// Either way count_wedge(w) for the pair (u, w) is aggregated in one place and
// Lemma 1 gives C(count, 2) butterflies.  Adding old = count_wedge(w) before
// each increment gives Σ_w C(count_wedge(w), 2) exactly.
//
// One persistent launch, one CTA of 1024 threads per SM, 192 KB of dynamic
// shared memory.  Three phases, each fed by its own queue, heaviest first
// (Section 6.2's dynamic scheduling with the exact per-start work):
//   A. CTA items, the whole CTA on one item:
//      dense (u, lo) count_wedge is a dense array over the chunk of u's end
//                    range that starts at offset lo: 4-bit counts when
//                    every count of the chunk is at most 15, 8-bit when at
//                    most 255, 16-bit when at most 65,535, else 32-bit (the
//                    same shared memory holds 393,216, 196,608, 98,304 or
//                    49,152 of them; a count is at most min(cut[u], deg of
//                    the chunk's last end)).  Chunks
//                    split the END range, so every pair is aggregated by
//                    exactly one item and C(count, 2) is never split;
//      hash (u)      an open-addressing table of up to 32,768 slots.
//      Without a second walk the dense items are streamed: each item takes
//      the next from the queue and clears the counters inside its first
//      batch's scan, so warps that finish early start the next item's loads.
//   B. team items: four teams of 256 threads, each with a 48 KB region (a
//      4,096-slot table and its batch arrays), one start per team.
//   C. warp items: 32 warps, each with a 512-slot table, one light start each.
// A table sized from a bound that can be exceeded (Algorithm 3's ends, or a
// team bound above 3,072 wedges) detects when it fills up; the start is then
// re-queued and counted by k_count_retry, first with a CTA table, then if
// needed with dense chunks of its end range.
#include "bfc_internal.cuh"

#include <algorithm>
#include <type_traits>

namespace bfc {

namespace {

constexpr int kTeamTableBytes = kTeamSlots * 6;   // 32-bit keys + 16-bit counts
static_assert(kTeamRegion == (kCountWarps / kTeams) * kWarpRegion,
              "a team's region is exactly the regions of its warps");

struct CountParams {
    const int64_t *__restrict__ off;
    const int32_t *__restrict__ adj;
    const int32_t *__restrict__ eid;
    const int32_t *__restrict__ plen;
    const int32_t *__restrict__ cut;
    const uint64_t *__restrict__ work;
    const int2 *__restrict__ cta_items;
    const int32_t *__restrict__ team_items;
    const int32_t *__restrict__ warp_items;
    int64_t n_cta;
    int64_t n_team;
    int64_t n_warp;
    int *cursors;                      // [0] CTA, [1] warp, [2] retry pushes, [3] retry, [4] team
    unsigned long long *acc;
    unsigned long long *pv;            // [n] in G* ids
    unsigned long long *pe;            // [2m] by G* slot (each edge has two)
    const int32_t *__restrict__ coff;  // chunk-boundary table (nullable; Algorithm 2 only)
    const int32_t *__restrict__ ctb;   // a batch's table: first entry of each slot's middle, -1 if none (else null)
    const int32_t *__restrict__ gstar; // graph of each G* vertex (batch mode)
    const int32_t *__restrict__ vbase; // first id of x's graph in x's layer (batch mode)
    const int32_t *__restrict__ vend;  // one past the last id of x's graph in x's layer (batch mode)
    const int64_t *__restrict__ sbeg;  // start of each middle slot's run of ends
    unsigned long long *gtot;          // per-graph totals (batch mode)
    int32_t *retry;                    // re-queued starts: x (CTA table next) or -(x+1) (dense)
    int64_t retry_cap;
    int64_t retry_static;              // retry[0, retry_static) were assigned by prepare
    int32_t retry_on;                  // the retry pass runs after this launch
    int32_t coff_u1, coff_l1;          // entries per L vertex / per U vertex
    int32_t orient;                    // 0 = Algorithm 2, 1 = Algorithm 3
    int32_t n;
    int64_t adj_len;
    int32_t l;
    int *err;
    // dense-core hybrid (total counts): core starts skip core middles' core
    // ends and add a·b + C(a, 2) per core pair after their walk
    int32_t core_on;
    int32_t core_lo_u, core_lo_l;          // first core id of each layer (n when none)
    int32_t core_ld_u, core_ld_l;          // row pitch of the products
    const int32_t *__restrict__ ccut;      // neighbours outside the other layer's core
    const uint16_t *__restrict__ core_au;  // a(u, w) of the U core
    const uint16_t *__restrict__ core_al;  // a(v, x) of the L core
    // batch plan: bin sizes in device memory (dense, hash, team, warp
    // starts; a dense start is one item), and the error word whose check
    // failures stop the launch (null otherwise)
    const unsigned long long *__restrict__ item_counts;
    const int *guard;
};

// item queue lengths: from the host, or from a batch plan's device counts
__device__ __forceinline__ int64_t n_cta_items(const CountParams &p) {
    return p.item_counts ? (int64_t)(p.item_counts[0] + p.item_counts[1]) : p.n_cta;
}
__device__ __forceinline__ int64_t n_team_items(const CountParams &p) {
    return p.item_counts ? (int64_t)p.item_counts[2] : p.n_team;
}
__device__ __forceinline__ int64_t n_warp_items(const CountParams &p) {
    return p.item_counts ? (int64_t)p.item_counts[3] : p.n_warp;
}

// The threads that walk one start together: the whole CTA (barrier 0) or one
// of its four 256-thread teams (hardware barriers 1..4).
template <int kThreads>
struct Team {
    int tid;
    int bar;
    __device__ __forceinline__ void sync() const {
        if (kThreads == kCountThreads) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(kThreads) : "memory");
    }
};

// Middles per batch: two per thread when adjacency positions fit 32 bits.
template <typename Pos, int kThreads>
struct Batch {
    static constexpr int kPer = sizeof(Pos) == 4 ? 2 : 1;
    static constexpr int kSize = kPer * kThreads;
};

template <int MODE, typename Pos, int kThreads>
struct SharedTeam {
    static constexpr int kB = Batch<Pos, kThreads>::kSize;
    int32_t start[kB + 33];             // compacted batch: exclusive prefix of run lengths, then
                                        // the total and 32 sentinels (INT_MAX)
    Pos src[kB];                        // compacted batch: adjacency position of a run minus its prefix
    unsigned long long msum[has_second_walk(MODE) ? kB : 1];  // second walk: Σ δ per compacted middle
    long long wtot[kThreads / 32];
    unsigned long long red[kThreads / 32];
    int item;
    int overflow;   // this item's table filled up
    int inserts;    // distinct ends inserted so far
    int track;      // the item's bound lets its table pass 3/4 full: count inserts
    int64_t next[2];  // streamed dense items: the item after the current one, by parity
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

// Exclusive scan of one int64 per thread across the team.
template <int kThreads, class SH>
__device__ __forceinline__ long long team_excl_scan(long long v, SH &sh, const Team<kThreads> &t,
                                                    long long *total) {
    constexpr int kWarps = kThreads / 32;
    const int lane = t.tid & 31, warp = t.tid >> 5;
    long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long o = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += o;
    }
    if (lane == 31) sh.wtot[warp] = x;
    t.sync();
    if (warp == 0) {
        long long w = lane < kWarps ? sh.wtot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            long long o = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += o;
        }
        if (lane < kWarps) sh.wtot[lane] = w;
    }
    t.sync();
    long long before = warp > 0 ? sh.wtot[warp - 1] : 0;
    *total = sh.wtot[kWarps - 1];
    return before + x - v;
}

// Sum over the team; the result is valid in the team's first warp.
template <int kThreads, class SH>
__device__ __forceinline__ unsigned long long team_sum(unsigned long long v, SH &sh,
                                                       const Team<kThreads> &t) {
    constexpr int kWarps = kThreads / 32;
    const int lane = t.tid & 31, warp = t.tid >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    t.sync();
    if (lane == 0) sh.red[warp] = v;
    t.sync();
    unsigned long long r = 0;
    if (warp == 0) {
        r = lane < kWarps ? sh.red[lane] : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) r += __shfl_xor_sync(0xffffffffu, r, d);
    }
    return r;
}

template <int kThreads>
__device__ __forceinline__ void team_fill(unsigned char *p, int bytes, uint32_t fill,
                                          const Team<kThreads> &t) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    const int n16 = (bytes + 15) >> 4;
    const uint4 f = make_uint4(fill, fill, fill, fill);
    for (int i = t.tid; i < n16; i += kThreads) q[i] = f;
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
// full.  *inserted is set when this call claimed an empty slot.
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

// 8-bit counters packed four per 32-bit word (a start whose counts stay below 256)
__device__ __forceinline__ uint32_t inc8(uint32_t *w32, int idx) {
    const uint32_t sh = (uint32_t)(idx & 3) << 3;
    uint32_t old = atomicAdd(w32 + (idx >> 2), 1u << sh);
    return (old >> sh) & 0xffu;
}
__device__ __forceinline__ uint32_t get8(const uint32_t *w32, int idx) {
    const uint32_t sh = (uint32_t)(idx & 3) << 3;
    return (w32[idx >> 2] >> sh) & 0xffu;
}

// 4-bit counters packed eight per 32-bit word (a chunk whose counts stay below 16)
__device__ __forceinline__ uint32_t inc4(uint32_t *w32, int idx) {
    const uint32_t sh = (uint32_t)(idx & 7) << 2;
    uint32_t old = atomicAdd(w32 + (idx >> 3), 1u << sh);
    return (old >> sh) & 0xfu;
}
__device__ __forceinline__ uint32_t get4(const uint32_t *w32, int idx) {
    const uint32_t sh = (uint32_t)(idx & 7) << 2;
    return (w32[idx >> 3] >> sh) & 0xfu;
}

enum CounterKind { kDenseNarrow = 0, kDenseWide = 1, kHash = 2, kDenseByte = 3, kDenseNibble = 4 };

// the dense counter kind of a start with at most `bound` middles, its chunk
// span (dense_chunk_span) and the bytes to clear for `span` counters
__device__ __forceinline__ int dense_kind(int64_t bound) {
    return bound > (int64_t)kNarrowMaxCut ? kDenseWide : (bound > (int64_t)kByteMaxCut ? kDenseNarrow : kDenseByte);
}
__device__ __forceinline__ int dense_clear_bytes(int kind, int32_t span) {
    return kind == kDenseWide ? span * 4
         : kind == kDenseNarrow ? ((span + 1) >> 1) * 4
         : kind == kDenseByte ? ((span + 3) >> 2) * 4 : ((span + 7) >> 3) * 4;
}
__device__ __forceinline__ uint32_t dense_get(int kind, const uint32_t *w32, int idx) {
    return kind == kDenseWide ? w32[idx]
         : kind == kDenseNarrow ? get16(w32, idx) : (kind == kDenseByte ? get8(w32, idx) : get4(w32, idx));
}
__device__ __forceinline__ int kind_of_bits(int bits) {
    return bits == 32 ? kDenseWide : (bits == 16 ? kDenseNarrow : (bits == 8 ? kDenseByte : kDenseNibble));
}

// The counter operation for one wedge whose end id is w and whose end sits at
// adjacency slot pos.  First walk: increment count_wedge(w), return the old
// value.  Second walk: read the final count, attribute δ = count − 1 to the
// edge (middle, w) and return δ for the middle's batch sum.
template <int MODE, int KIND, bool kSecond, typename Pos>
__device__ __forceinline__ unsigned long long wedge_op(const CountParams &p, int32_t w, Pos pos,
                                                       int32_t lb, int32_t lo, int32_t span,
                                                       uint32_t hmask, unsigned char *ctr, int *ovf,
                                                       int *ins) {
    uint32_t *w32 = reinterpret_cast<uint32_t *>(ctr);
    uint32_t c;
    if (KIND == kHash) {
        int32_t *hkeys = reinterpret_cast<int32_t *>(ctr);
        uint32_t *hcnt = reinterpret_cast<uint32_t *>(ctr + (size_t)(hmask + 1) * 4);
        int inserted = 0;
        const int slot = hash_find(hkeys, hmask, w - lb, !kSecond, &inserted);
        if (slot < 0) {
            // the first walk re-queues a start whose table filled up; the
            // second walk only looks up ends the first walk inserted
            if (!kSecond) *ovf = 1; else atomicOr(p.err, kErrHashFull);
            return 0;
        }
        if (!kSecond) {
            // keep the load factor at most 3/4 so probes stay short
            // (ins is null when the start cannot reach that load)
            if (inserted && ins && atomicAdd(ins, 1) >= (int)((hmask + 1) / 4 * 3)) *ovf = 1;
            return inc16(hcnt, slot);
        }
        c = get16(hcnt, slot);
    } else {
        const int idx = w - lb - lo;
        if ((uint32_t)idx >= (uint32_t)span) { atomicOr(p.err, kErrBounds); return 0; }
        if (!kSecond)
            return (KIND == kDenseWide) ? atomicAdd(w32 + idx, 1u)
                 : (KIND == kDenseByte) ? inc8(w32, idx) : (KIND == kDenseNibble ? inc4(w32, idx) : inc16(w32, idx));
        c = (KIND == kDenseWide) ? w32[idx]
          : (KIND == kDenseByte) ? get8(w32, idx) : (KIND == kDenseNibble ? get4(w32, idx) : get16(w32, idx));
    }
    // δ = count − 1 for the edge (middle, w); the caller sums it per middle
    const unsigned long long delta = (unsigned long long)c - 1ull;
    // per-edge sums are kept by G* slot: the ends of one run are consecutive
    // slots, so a window's atomics fall on a few consecutive sectors
    if (wants_edges(MODE) && delta) atomicAdd(p.pe + pos, delta);
    return delta;
}

// Adds each lane's x to msum[q], where equal q occupy consecutive lanes (the
// runs of a window are contiguous): the last lane of each run takes the
// difference of an inclusive warp scan at its lane and at the previous run's
// last lane (found from a ballot of run ends), and makes the one shared atomic.
template <typename T>
__device__ __forceinline__ void run_add(unsigned long long *msum, int q, T x, int lane) {
    T sc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, sc, o);
        if (lane >= o) sc += t;
    }
    const int qn = __shfl_down_sync(0xffffffffu, q, 1);
    const bool last = lane == 31 || qn != q;
    const uint32_t below = __ballot_sync(0xffffffffu, last) & ((1u << lane) - 1u);
    const T prev = __shfl_sync(0xffffffffu, sc, below ? 31 - __clz(below) : 0);
    const T sum = below ? sc - prev : sc;
    if (last && sum) atomicAdd(msum + q, (unsigned long long)sum);
}

// The per-thread state of one batch of middles that the second walk needs
// after the windows: each middle's run length, id, slot and compacted index.
template <typename Pos, int kThreads>
struct BatchSlots {
    static constexpr int kPer = Batch<Pos, kThreads>::kPer;
    int32_t len[kPer], v[kPer];
    int64_t e[kPer];
    int nzs[kPer];
};

// The per-middle sums of a second-walk batch: Σ δ over each middle's ends
// goes to the middle (per-vertex) and to the edge (x, v) at its slot.
template <int MODE, typename Pos, int kThreads, class SH>
__device__ __forceinline__ void middle_sums(const CountParams &p, const BatchSlots<Pos, kThreads> &bs,
                                            const SH &sh) {
#pragma unroll
    for (int i = 0; i < Batch<Pos, kThreads>::kPer; ++i) {
        if (bs.len[i] > 0) {
            const unsigned long long dsum = sh.msum[bs.nzs[i]];
            if (dsum) {
                if (wants_vertices(MODE)) atomicAdd(p.pv + bs.v[i], dsum);
                if (wants_edges(MODE)) atomicAdd(p.pe + bs.e[i], dsum);
            }
        }
    }
}

// Sets up one batch of the middles of x (those with index mb .. mb+kB-1):
// the run of ends in range for each middle comes from the slot arrays (plus
// the chunk-boundary table or a binary search for dense chunks); non-empty
// runs are compacted into sh.start / sh.src by one team scan of packed
// (length, non-empty) values.  The scan's first barrier is the point after
// which every thread of the team has finished the previous windows, so
// `zero_bytes` > 0 clears that many bytes of counters there.  Returns the
// batch's wedge count in *total and its non-empty runs in *nnz; the entries
// are visible to the team after its next barrier.
template <bool kDense, bool kSecond, typename Pos, int kThreads, class SH>
__device__ __forceinline__ void batch_runs(const CountParams &p, int64_t e0, int32_t nmid, int32_t mb,
                                           int32_t lb, int32_t lo, int32_t hi, int flags,
                                           unsigned char *ctr, int zero_bytes, SH &sh,
                                           const Team<kThreads> &t, BatchSlots<Pos, kThreads> &bs,
                                           int32_t *total_out, int *nnz_out,
                                           int32_t core_lo_v = 0x7fffffff) {
    constexpr int kPer = Batch<Pos, kThreads>::kPer;
    const int tid = t.tid;
    int32_t pl[kPer], ct[kPer];
    Pos src[kPer];
    int64_t b[kPer];
    bool has[kPer];
    // the slot loads of all of this thread's middles first, then the
    // chunk-boundary loads that depend on them: two rounds of latency
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int32_t j = mb + i * kThreads + tid;
        has[i] = j < nmid;
        bs.e[i] = has[i] ? e0 + j : e0;
        bs.v[i] = has[i] ? __ldg(p.adj + bs.e[i]) : 0;
        pl[i] = has[i] ? __ldg(p.plen + bs.e[i]) : 0;
        // run of ends: prefix of N(v) below x (Algorithm 2) or the
        // suffix above both x and v (Algorithm 3)
        b[i] = has[i] ? __ldg(p.sbeg + bs.e[i]) : 0;
        ct[i] = (kDense && has[i] && p.ctb) ? __ldg(p.ctb + bs.e[i]) : -1;
    }
    // a core start: a core middle's run stops before its core ends (they are
    // the top of the run, and the product counts those wedges)
    if (core_lo_v != 0x7fffffff) {
#pragma unroll
        for (int i = 0; i < kPer; ++i)
            if (has[i] && bs.v[i] >= core_lo_v) pl[i] = min(pl[i], __ldg(p.ccut + bs.v[i]));
    }
    int32_t s0[kPer], s1[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        s0[i] = 0;
        s1[i] = pl[i];
        if (kDense && has[i] && pl[i] > 0) {
            const int32_t v = bs.v[i];
            int64_t tb = -1;
            if (p.coff) {
                if (p.ctb) {   // a batch: entries only for the middles of its chunked dense starts
                    tb = ct[i];
                } else {
                    tb = v < p.l ? (int64_t)v * p.coff_u1
                                 : (int64_t)p.l * p.coff_u1 + (int64_t)(v - p.l) * p.coff_l1;
                }
            }
            if (tb >= 0) {
                if (flags & 1) s0[i] = __ldg(p.coff + tb + lo / kChunkUnit);
                if (flags & 2) s1[i] = __ldg(p.coff + tb + hi / kChunkUnit);
                if (core_lo_v != 0x7fffffff) {   // chunk bounds past a shortened run
                    s1[i] = min(s1[i], pl[i]);
                    s0[i] = min(s0[i], s1[i]);
                }
            } else {
                if (flags & 1) s0[i] = lower_bound_g(p.adj + b[i], pl[i], lb + lo);
                if (flags & 2) s1[i] = lower_bound_g(p.adj + b[i], pl[i], lb + hi);
            }
        }
    }
    long long packed_run = 0;
    long long pk[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        int32_t len = s1[i] - s0[i];
        src[i] = (Pos)(b[i] + s0[i]);
        // every wedge of a run reads a slot in [b + s0, b + s1): checking
        // the run here covers the slot of each of its wedges
        if (len > 0 && (b[i] + s0[i] < 0 || b[i] + s1[i] > p.adj_len)) {
            atomicOr(p.err, kErrBounds);
            len = 0;
        }
        if (len < 0) len = 0;
        bs.len[i] = len;
        // run length in the high bits, "non-empty" in the low 20 bits:
        // one scan yields both the run offsets and the compacted slots
        pk[i] = ((long long)len << 20) | (len > 0 ? 1 : 0);
        packed_run += pk[i];
    }
    long long packed_total;
    long long packed = team_excl_scan(packed_run, sh, t, &packed_total);
    if (zero_bytes > 0) team_fill(ctr, zero_bytes, 0u, t);
    const int32_t total = (int32_t)(packed_total >> 20);
    const int nnz = (int)(packed_total & 0xfffff);
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int32_t excl = (int32_t)(packed >> 20);
        bs.nzs[i] = (int)(packed & 0xfffff);
        if (bs.len[i] > 0) {
            sh.start[bs.nzs[i]] = excl;
            sh.src[bs.nzs[i]] = src[i] - (Pos)excl;
            if (kSecond) sh.msum[bs.nzs[i]] = 0;
        }
        packed += pk[i];
    }
    if (tid <= 32) sh.start[nnz + tid] = tid == 0 ? total : 0x7fffffff;
    *total_out = total;
    *nnz_out = nnz;
}

// The windows of one compacted batch.  The concatenated runs are cut into
// windows of 32 wedges and each warp takes a contiguous range of windows.
// Inside a window the run of every lane is found from a 32-bit mask of run
// starts (reduce-or + popc), so no search is needed per wedge, and four
// windows are in flight per iteration so their end loads overlap.
// kSecond = false: count (returns Σ old, i.e. Σ C(count, 2)).
// kSecond = true : read the final counts and attribute δ = count − 1.
template <int MODE, int KIND, bool kSecond, typename Pos, int kThreads, class SH>
__device__ __forceinline__ unsigned long long batch_windows(const CountParams &p, int32_t lb, int32_t lo,
                                                            int32_t span, uint32_t hmask,
                                                            unsigned char *ctr, int32_t total, int nnz,
                                                            int *ins, SH &sh, const Team<kThreads> &t) {
    constexpr int kWarps = kThreads / 32;
    constexpr int kU = 4;
    const int lane = t.tid & 31, warp = t.tid >> 5;
    const uint32_t le_mask = 0xffffffffu >> (31 - lane);
    unsigned long long acc = 0;
    const int32_t nwin = (total + 31) >> 5;
    int32_t wb = (int32_t)(((int64_t)warp * nwin) / kWarps);
    const int32_t wend = (int32_t)(((int64_t)(warp + 1) * nwin) / kWarps);
    if (wb < wend) {
        int32_t k0 = wb << 5;
        int q0 = last_le(sh.start, nnz, k0);
        // Fast path: the next N windows lie inside run q0 (most wedges do, as
        // runs of heavy starts are long), so the slots are consecutive, no
        // run lookup is needed and N loads are in flight per lane.
        auto fast = [&](auto n_windows, int32_t next_run) {
            constexpr int N = decltype(n_windows)::value;
            const Pos base = sh.src[q0] + (Pos)(k0 + lane);
            int32_t w[N];
#pragma unroll
            for (int u = 0; u < N; ++u) w[u] = __ldg(p.adj + base + (Pos)(32 * u));
            uint32_t sum32 = 0;   // N olds (or δ) of 16-bit counts stay below 2^20
            unsigned long long sum64 = 0;
#pragma unroll
            for (int u = 0; u < N; ++u) {
                const unsigned long long r = wedge_op<MODE, KIND, kSecond, Pos>(
                    p, w[u], base + (Pos)(32 * u), lb, lo, span, hmask, ctr, &sh.overflow, ins);
                if (KIND == kDenseWide) sum64 += r; else sum32 += (uint32_t)r;
            }
            if (!kSecond) {
                acc += (KIND == kDenseWide) ? sum64 : (unsigned long long)sum32;
            } else if (KIND == kDenseWide) {
                run_add<unsigned long long>(sh.msum, q0, sum64, lane);
            } else {
                // one run: the warp's δ sum goes to middle q0
                const uint32_t tot = __reduce_add_sync(0xffffffffu, sum32);
                if (lane == 0 && tot) atomicAdd(sh.msum + q0, (unsigned long long)tot);
            }
            if (next_run == k0 + 32 * N) ++q0;   // the next window starts run q0 + 1
            k0 += 32 * N;
            wb += N;
        };
        while (wb < wend) {
            const int32_t next_run = sh.start[q0 + 1];   // warp-uniform
            if (wb + 2 * kU <= wend && next_run >= k0 + 64 * kU) {
                fast(std::integral_constant<int, 2 * kU>(), next_run);
                continue;
            }
            if (wb + kU <= wend && next_run >= k0 + 32 * kU) {
                fast(std::integral_constant<int, kU>(), next_run);
                continue;
            }
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
                    // run starts after this window's first wedge: 1 <= d, and
                    // the sentinels keep the index below nnz + 33
                    const int32_t d = sh.start[q0 + 1 + lane] - kw;
                    uint32_t bit;   // 1 << d, 0 once d >= 32 (PTX clamps the shift)
                    asm("shl.b32 %0, %1, %2;" : "=r"(bit) : "r"(1u), "r"(d));
                    const uint32_t m = __reduce_or_sync(0xffffffffu, bit);
                    q[u] = q0 + __popc(m & le_mask);
                    q0 += __popc(__ballot_sync(0xffffffffu, d <= 32));
                    ok[u] = kw + lane < total;
                    if (ok[u]) pos[u] = sh.src[q[u]] + (Pos)(kw + lane);
                }
            }
            int32_t w[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) w[u] = ok[u] ? __ldg(p.adj + pos[u]) : 0;
            // counts below 2^16 keep four olds far below 2^32
            uint32_t acc32 = 0;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if (!kSecond) {
                    if (ok[u]) {
                        const unsigned long long old =
                            wedge_op<MODE, KIND, false, Pos>(p, w[u], pos[u], lb, lo, span, hmask,
                                                             ctr, &sh.overflow, ins);
                        if (KIND == kDenseWide) acc += old; else acc32 += (uint32_t)old;
                    }
                } else if (wb + u < wend) {   // warp-uniform: all lanes take part in run_add
                    const unsigned long long d =
                        ok[u] ? wedge_op<MODE, KIND, true, Pos>(p, w[u], pos[u], lb, lo, span, hmask,
                                                                ctr, &sh.overflow, ins)
                              : 0ull;
                    // 16-bit counts keep a window's δ sum below 2^21
                    if (KIND == kDenseWide) run_add<unsigned long long>(sh.msum, q[u], d, lane);
                    else run_add<uint32_t>(sh.msum, q[u], (uint32_t)d, lane);
                }
            }
            if (KIND != kDenseWide) acc += acc32;
            k0 += 32 * kU;
            wb += kU;
        }
    }
    return acc;
}

// One walk over the wedges of start x whose ends fall in [lb+lo, lb+hi).
// kSecond = false: count (returns Σ old, i.e. Σ C(count, 2)).
// kSecond = true : read the final counts and attribute δ = count − 1.
// flags: bit 0 = cut the runs below lb+lo, bit 1 = cut them at lb+hi.
// The middles of x are taken a batch at a time (two per thread, or one with
// 64-bit positions): batch_runs, a barrier, batch_windows.
template <int MODE, int KIND, bool kSecond, typename Pos, int kThreads, class SH>
__device__ unsigned long long team_walk(const CountParams &p, int32_t x, int32_t lb, int32_t lo,
                                        int32_t hi, int flags, uint32_t hmask, unsigned char *ctr,
                                        SH &sh, const Team<kThreads> &t) {
    constexpr int kPer = Batch<Pos, kThreads>::kPer;
    constexpr int kB = Batch<Pos, kThreads>::kSize;
    const int64_t e0 = p.off[x];
    // Algorithm 2: the middles are the cut[x] lower-priority neighbours;
    // Algorithm 3: every neighbour is a middle
    const int32_t nmid = p.orient ? (int32_t)(p.off[x + 1] - e0) : p.cut[x];
    const int32_t span = hi - lo;
    int *const ins = (KIND == kHash && !kSecond && sh.track) ? &sh.inserts : nullptr;
    unsigned long long acc = 0;
    for (int32_t mb = 0; mb < nmid; mb += kB) {
        BatchSlots<Pos, kThreads> bs;
        int32_t total;
        int nnz;
        batch_runs<KIND != kHash, kSecond, Pos>(p, e0, nmid, mb, lb, lo, hi, flags, ctr, 0, sh, t, bs,
                                                 &total, &nnz);
        t.sync();
        acc += batch_windows<MODE, KIND, kSecond, Pos>(p, lb, lo, span, hmask, ctr, total, nnz, ins, sh, t);
        // Dense counting needs no join here: the next batch's scan barriers
        // come before its compaction overwrites the run arrays, so warps that
        // finish their windows early already load the next batch's slots.
        if (KIND == kHash || kSecond) t.sync();
        if (KIND == kHash && !kSecond && sh.overflow) break;   // uniform: read after the barrier
        if (kSecond) middle_sums<MODE, Pos>(p, bs, sh);
    }
    return acc;
}

// First walk, then (per-vertex / per-edge) the end contributions and the
// second walk.  Returns Σ C(count, 2) over the pairs of this item, or 0 with
// sh.overflow set when a hash table filled up (nothing is attributed then).
// The per-vertex end contributions of one item: each pair (x, w) of the
// item adds C(count, 2) to ⋈_w.  Called after the first walk, with its
// counters final.
template <int MODE, int KIND, int kThreads>
__device__ __forceinline__ void end_contributions(const CountParams &p, int32_t lb, int32_t lo,
                                                  int32_t hi, uint32_t hmask, const unsigned char *ctr,
                                                  const Team<kThreads> &t);

template <int MODE, int KIND, typename Pos, int kThreads, class SH>
__device__ unsigned long long item_body(const CountParams &p, int32_t x, int32_t lb, int32_t lo,
                                        int32_t hi, int flags, uint32_t hmask, unsigned char *ctr,
                                        SH &sh, const Team<kThreads> &t) {
    constexpr int kB = Batch<Pos, kThreads>::kSize;
    if (has_second_walk(MODE)) {
        const int32_t nmid = p.orient ? (int32_t)(p.off[x + 1] - p.off[x]) : p.cut[x];
        if (nmid <= kB) {
            // One batch of middles: the second walk reuses the first walk's
            // compacted runs (shared arrays and each thread's slots), so the
            // slot loads and the scan happen once.
            BatchSlots<Pos, kThreads> bs;
            int32_t total;
            int nnz;
            batch_runs<KIND != kHash, false, Pos>(p, p.off[x], nmid, 0, lb, lo, hi, flags, ctr, 0, sh, t, bs,
                                                  &total, &nnz);
            t.sync();
            int *const ins = (KIND == kHash && sh.track) ? &sh.inserts : nullptr;
            const int32_t span = hi - lo;
            const unsigned long long acc =
                batch_windows<MODE, KIND, false, Pos>(p, lb, lo, span, hmask, ctr, total, nnz, ins, sh, t);
            t.sync();   // counters final
            if (KIND == kHash && sh.overflow) return 0;   // the caller re-queues x
            if (wants_vertices(MODE)) end_contributions<MODE, KIND>(p, lb, lo, hi, hmask, ctr, t);
#pragma unroll
            for (int i = 0; i < Batch<Pos, kThreads>::kPer; ++i)
                if (bs.len[i] > 0) sh.msum[bs.nzs[i]] = 0;
            t.sync();
            batch_windows<MODE, KIND, true, Pos>(p, lb, lo, span, hmask, ctr, total, nnz, nullptr, sh, t);
            t.sync();
            middle_sums<MODE, Pos>(p, bs, sh);
            if (wants_vertices(MODE)) {
                const unsigned long long s = team_sum(acc, sh, t);
                if (t.tid == 0 && s) atomicAdd(p.pv + x, s);
            }
            return acc;
        }
    }
    unsigned long long acc = team_walk<MODE, KIND, false, Pos>(p, x, lb, lo, hi, flags, hmask, ctr, sh, t);
    if (KIND == kHash) {
        t.sync();
        if (sh.overflow) return 0;   // the caller re-queues x
    }
    if (has_second_walk(MODE)) {
        t.sync();
        if (wants_vertices(MODE)) end_contributions<MODE, KIND>(p, lb, lo, hi, hmask, ctr, t);
        team_walk<MODE, KIND, true, Pos>(p, x, lb, lo, hi, flags, hmask, ctr, sh, t);
        if (wants_vertices(MODE)) {
            const unsigned long long s = team_sum(acc, sh, t);
            if (t.tid == 0 && s) atomicAdd(p.pv + x, s);
        }
    }
    return acc;
}

template <int MODE, int KIND, int kThreads>
__device__ __forceinline__ void end_contributions(const CountParams &p, int32_t lb, int32_t lo,
                                                  int32_t hi, uint32_t hmask, const unsigned char *ctr,
                                                  const Team<kThreads> &t) {
    if (KIND == kHash) {
        const int32_t *hkeys = reinterpret_cast<const int32_t *>(ctr);
        const uint32_t *hcnt = reinterpret_cast<const uint32_t *>(ctr + (size_t)(hmask + 1) * 4);
        for (uint32_t s = t.tid; s <= hmask; s += kThreads) {
            const int32_t k = hkeys[s];
            if (k >= 0) {
                const unsigned long long b = c2(get16(hcnt, (int)s));
                if (b) atomicAdd(p.pv + lb + k, b);
            }
        }
    } else {
        // 16 bytes per thread and step (32 nibble, 16 byte, 8 narrow or 4 wide counters);
        // a word whose counts are all below 2 adds nothing.  The
        // clear before the walk covered whole 16-byte words.
        const uint4 *q4 = reinterpret_cast<const uint4 *>(ctr);
        constexpr int kPerQ = (KIND == kDenseWide) ? 4 : (KIND == kDenseByte ? 16 : (KIND == kDenseNibble ? 32 : 8));
        constexpr uint32_t kAtLeast2 = (KIND == kDenseWide) ? 0xFFFFFFFEu
                                     : (KIND == kDenseByte) ? 0xFEFEFEFEu
                                     : (KIND == kDenseNibble) ? 0xEEEEEEEEu : 0xFFFEFFFEu;
        const int32_t span = hi - lo;
        unsigned long long *pvb = p.pv + lb + lo;
        for (int32_t j = t.tid; j * kPerQ < span; j += kThreads) {
            const uint4 q = q4[j];
            if (((q.x | q.y | q.z | q.w) & kAtLeast2) == 0) continue;
            const uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (KIND == kDenseWide) {
                    const int32_t i = j * 4 + k;
                    if (wv[k] >= 2 && i < span) atomicAdd(pvb + i, c2(wv[k]));
                } else if (KIND == kDenseByte) {
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        const int32_t i = j * 16 + 4 * k + bb;
                        const uint32_t c = (wv[k] >> (8 * bb)) & 0xFFu;
                        if (c >= 2 && i < span) atomicAdd(pvb + i, c2(c));
                    }
                } else if (KIND == kDenseNibble) {
                    if ((wv[k] & kAtLeast2) == 0) continue;
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) {
                        const int32_t i = j * 32 + 8 * k + bb;
                        const uint32_t c = (wv[k] >> (4 * bb)) & 0xFu;
                        if (c >= 2 && i < span) atomicAdd(pvb + i, c2(c));
                    }
                } else {
                    const int32_t i = j * 8 + 2 * k;
                    const uint32_t c0 = wv[k] & 0xFFFFu, c1 = wv[k] >> 16;
                    if (c0 >= 2 && i < span) atomicAdd(pvb + i, c2(c0));
                    if (c1 >= 2 && i + 1 < span) atomicAdd(pvb + i + 1, c2(c1));
                }
            }
        }
    }
}

// first id of x's part of its layer, and one past its last
__device__ __forceinline__ int32_t range_lo(const CountParams &p, int32_t x) {
    return p.vbase ? __ldg(p.vbase + x) : (x >= p.l ? p.l : 0);
}
__device__ __forceinline__ int32_t range_hi(const CountParams &p, int32_t x) {
    return p.vend ? __ldg(p.vend + x) : (x >= p.l ? p.n : p.l);
}

// How many distinct ends x can have: the vertices below it (Algorithm 2) or
// above it (Algorithm 3) in its part of its layer, and at most one per wedge.
__device__ __forceinline__ unsigned long long end_bound(const CountParams &p, int32_t x,
                                                        int32_t lb) {
    const unsigned long long range = p.orient ? (unsigned long long)(range_hi(p, x) - x - 1)
                                              : (unsigned long long)(x - lb);
    const unsigned long long w = p.work[x];
    return w < range ? w : range;
}

// A count_wedge is at most the number of middles: cut[x] (Algorithm 2) or
// deg(x) (Algorithm 3).
__device__ __forceinline__ int64_t middles(const CountParams &p, int32_t x) {
    return p.orient ? p.off[x + 1] - p.off[x] : (int64_t)p.cut[x];
}

// A start counted by the team with one hash table of at most `max_slots`
// slots.  Returns its Σ C(count, 2), or sets sh.overflow.
template <int MODE, typename Pos, int kThreads, class SH>
__device__ unsigned long long hash_item(const CountParams &p, int32_t x, unsigned char *ctr,
                                        int max_slots, SH &sh, const Team<kThreads> &t) {
    const int32_t lb = range_lo(p, x);
    const unsigned long long bound = end_bound(p, x, lb);
    uint32_t cap = 64;
    while (cap < 2 * bound && cap < (uint32_t)max_slots) cap <<= 1;
    // hash tables hold 16-bit counts; a count is at most min(middles, work)
    const bool wide = middles(p, x) > (int64_t)kNarrowMaxCut && p.work[x] > (uint64_t)kNarrowMaxCut;
    if (t.tid == 0) {
        sh.overflow = wide ? 1 : 0;
        sh.inserts = 0;
        sh.track = bound > (unsigned long long)(cap / 4 * 3) ? 1 : 0;
    }
    team_fill(ctr, (int)cap * 4, 0xffffffffu, t);           // keys = -1
    team_fill(ctr + (size_t)cap * 4, (int)cap * 2, 0u, t);  // packed 16-bit counts
    t.sync();
    if (sh.overflow) return 0;
    return item_body<MODE, kHash, Pos>(p, x, lb, 0, 0, 0, cap - 1, ctr, sh, t);
}

// A start counted by the CTA with dense counters, chunk after chunk of its
// end range: [0, x - lb) for Algorithm 2, (x, end of x's part) for Algorithm 3.
template <int MODE, typename Pos, class SH>
__device__ unsigned long long dense_all_chunks(const CountParams &p, int32_t x, unsigned char *ctr,
                                               SH &sh, const Team<kCountThreads> &t) {
    const int32_t lb = range_lo(p, x);
    const int kind = dense_kind(middles(p, x));
    const int32_t S = dense_chunk_span(middles(p, x));
    const int32_t first = p.orient ? x + 1 - lb : 0;
    const int32_t last = p.orient ? range_hi(p, x) - lb : x - lb;   // ends in [lb + first, lb + last)
    unsigned long long acc = 0;
    for (int32_t c = first / S; c * S < last; ++c) {
        const int32_t lo = max(c * S, first), hi = min((c + 1) * S, last);
        const int32_t span = hi - lo;
        const int flags = (lo > first ? 1 : 0) | (hi < last ? 2 : 0);
        team_fill(ctr, dense_clear_bytes(kind, span), 0u, t);
        t.sync();
        acc += kind == kDenseWide ? item_body<MODE, kDenseWide, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh, t)
             : kind == kDenseNarrow ? item_body<MODE, kDenseNarrow, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh, t)
                                    : item_body<MODE, kDenseByte, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh, t);
        t.sync();
    }
    return acc;
}

template <int kThreads, class SH>
__device__ __forceinline__ void add_to_graph(const CountParams &p, int32_t x, unsigned long long acc,
                                             SH &sh, const Team<kThreads> &t) {
    // a batch is a disjoint union: every butterfly of start x lies in x's graph
    const unsigned long long s = team_sum(acc, sh, t);
    if (t.tid == 0 && s) atomicAdd(p.gtot + p.gstar[x], s);
}

__device__ __forceinline__ void push_retry(const CountParams &p, int32_t entry) {
    // without a retry pass the schedule's bounds rule overflow out; a count
    // that lost a start this way fails loudly
    if (!p.retry_on) { atomicOr(p.err, kErrHashFull); return; }
    const int64_t k = p.retry_static + atomicAdd(p.cursors + 2, 1);
    if (k < p.retry_cap) p.retry[k] = entry; else atomicOr(p.err, kErrBounds);
}

// ---- phase A: CTA items ---------------------------------------------------------
template <int MODE, typename Pos, class SH>
__device__ unsigned long long cta_item(const CountParams &p, int2 item, unsigned char *ctr, SH &sh,
                                       const Team<kCountThreads> &t) {
    const int32_t x = item.x;
    unsigned long long acc;
    if (item.y >= 0) {          // dense items exist only for Algorithm 2
        const int32_t lb = range_lo(p, x);
        const int32_t R = x - lb;   // the ends are the R vertices below x
        const int32_t lo = item.y;   // the chunk's first end offset
        int bits;
        const int32_t hi = dense_chunk_end(lo, R, p.cut[x], p.off, lb, &bits);
        const int kind = kind_of_bits(bits);
        const int32_t span = hi - lo;
        const int flags = (lo > 0 ? 1 : 0) | (hi < R ? 2 : 0);
        team_fill(ctr, dense_clear_bytes(kind, span), 0u, t);
        t.sync();
        acc = kind == kDenseWide ? item_body<MODE, kDenseWide, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh, t)
            : kind == kDenseNarrow ? item_body<MODE, kDenseNarrow, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh, t)
            : kind == kDenseByte ? item_body<MODE, kDenseByte, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh, t)
                                 : item_body<MODE, kDenseNibble, Pos>(p, x, lb, lo, hi, flags, 0, ctr, sh, t);
    } else {
        acc = hash_item<MODE, Pos>(p, x, ctr, kHashMaxSlots, sh, t);
        if (sh.overflow) {
            // the CTA table was too small: dense chunks next
            if (t.tid == 0) push_retry(p, -(x + 1));
            t.sync();
            return 0;
        }
    }
    if (MODE == kModeBatch) add_to_graph(p, x, acc, sh, t);
    t.sync();
    return acc;
}

// Phase A's dense items when there is no second walk, streamed: the first
// batch of each item takes the next item from the queue and clears the
// counters after its scan's first barrier (by then every warp has left the
// previous item's windows), so a warp that finishes its windows early goes
// straight on to the next item's slot loads, and an item of one batch costs
// three barriers.  `it` is the current item (dense, the same in every thread);
// on return it is the first item that is not dense, or past the queue.  The
// caller joins before it reuses the counters' memory.
template <int MODE, typename Pos, class SH>
__device__ unsigned long long dense_stream(const CountParams &p, int64_t &it, unsigned char *ctr,
                                           SH &sh, const Team<kCountThreads> &t) {
    constexpr int kB = Batch<Pos, kCountThreads>::kSize;
    unsigned long long acc = 0;
    int par = 0;
    int2 item = p.cta_items[it];
    for (;;) {
        const int32_t x = item.x;
        const int32_t lb = range_lo(p, x);
        const int32_t R = x - lb;   // the ends are the R vertices below x
        const int32_t lo = item.y;   // the chunk's first end offset
        int bits;
        const int32_t hi = dense_chunk_end(lo, R, p.cut[x], p.off, lb, &bits);
        const int kind = kind_of_bits(bits);
        const int32_t span = hi - lo;
        const int flags = (lo > 0 ? 1 : 0) | (hi < R ? 2 : 0);
        const int64_t e0 = p.off[x];
        const int32_t nmid = p.cut[x];
        // dense-core hybrid: x in its layer's core (uniform over the item).  Only
        // dense items split: a core start in a hash bin walks all its wedges
        // and its row of the product is not used.
        const int32_t clo_x = x >= p.l ? p.core_lo_u : p.core_lo_l;
        const bool core_x = p.core_on && x >= clo_x;
        const int32_t core_lo_v = core_x ? (x >= p.l ? p.core_lo_l : p.core_lo_u) : 0x7fffffff;
        unsigned long long item_acc = 0;
        int32_t mb = 0;
        do {
            // sh.next[par] is written before this batch's barriers and read at
            // the end of the item; the next write to it comes two items later,
            // after every warp has passed the next item's barriers
            if (mb == 0 && t.tid == 0) sh.next[par] = atomicAdd(p.cursors, 1);
            BatchSlots<Pos, kCountThreads> bs;
            int32_t total;
            int nnz;
            const int zero_bytes = mb > 0 ? 0 : dense_clear_bytes(kind, span);
            batch_runs<true, false, Pos>(p, e0, nmid, mb, lb, lo, hi, flags, ctr, zero_bytes, sh, t, bs,
                                         &total, &nnz, core_lo_v);
            t.sync();
            item_acc += kind == kDenseWide
                            ? batch_windows<MODE, kDenseWide, false, Pos>(p, lb, lo, span, 0, ctr, total, nnz,
                                                                          nullptr, sh, t)
                        : kind == kDenseNarrow
                            ? batch_windows<MODE, kDenseNarrow, false, Pos>(p, lb, lo, span, 0, ctr, total, nnz,
                                                                            nullptr, sh, t)
                        : kind == kDenseByte
                            ? batch_windows<MODE, kDenseByte, false, Pos>(p, lb, lo, span, 0, ctr, total, nnz,
                                                                          nullptr, sh, t)
                            : batch_windows<MODE, kDenseNibble, false, Pos>(p, lb, lo, span, 0, ctr, total, nnz,
                                                                            nullptr, sh, t);
            mb += kB;
        } while (mb < nmid);
        if (core_x) {
            // every core end w of this chunk: count_wedge(w) = b (the walk's
            // middles outside the core) + a (the product's core middles), and
            // C(a + b, 2) - C(b, 2) = a·b + C(a, 2) (Lemma 1).  The next
            // item's scan clears the counters after its first barrier, so
            // the reads below come before it.
            t.sync();
            const bool in_u = x >= p.l;
            const uint16_t *arow = (in_u ? p.core_au : p.core_al) +
                                   (int64_t)(x - clo_x) * (in_u ? p.core_ld_u : p.core_ld_l);
            const uint32_t *w32 = reinterpret_cast<const uint32_t *>(ctr);
            const int32_t w_hi = lb + hi;
            unsigned long long e = 0;
            for (int32_t w = max(lb + lo, clo_x) + t.tid; w < w_hi; w += kCountThreads) {
                const unsigned long long a = __ldg(arow + (w - clo_x));
                const int idx = w - lb - lo;
                const unsigned long long b = dense_get(kind, w32, idx);
                e += a * b + (a * (a - 1)) / 2;   // a = 0 gives 0
            }
            item_acc += e;
        }
        if (MODE == kModeBatch) {
            // this warp's share of x's butterflies goes to x's graph
            unsigned long long w = item_acc;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
            if ((t.tid & 31) == 0 && w) atomicAdd(p.gtot + p.gstar[x], w);
        }
        acc += item_acc;
        it = sh.next[par];
        par ^= 1;
        if (it >= n_cta_items(p)) return acc;
        item = p.cta_items[it];
        if (item.y < 0) return acc;
    }
}

// ---- phase B: team items ----------------------------------------------------------
template <int MODE, typename Pos, class SH>
__device__ unsigned long long team_item(const CountParams &p, int32_t x, unsigned char *table,
                                        SH &sh, const Team<kTeamThreads> &t) {
    unsigned long long acc = hash_item<MODE, Pos>(p, x, table, kTeamSlots, sh, t);
    if (sh.overflow) {
        // a CTA table next
        if (t.tid == 0) push_retry(p, x);
        t.sync();
        return 0;
    }
    if (MODE == kModeBatch) add_to_graph(p, x, acc, sh, t);
    t.sync();
    return acc;
}

// ---- phase C: warp items ----------------------------------------------------------
// The warp version of team_walk for a light start: batches of 32 middles,
// compacted runs and the same window masks, with a per-warp hash table that
// always fits (at most 384 wedges, 512 slots).
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
            src = __ldg(p.sbeg + e);
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
            uint32_t delta = 0;
            if (k < total) {
                const long long pos = wsrc[q] + k;
                bool good = true;
                if (pos < 0 || pos >= p.adj_len) { atomicOr(p.err, kErrBounds); good = false; }
                const int32_t w = good ? __ldg(p.adj + pos) : 0;
                const int slot = good ? hash_find(keys, mask, w - lb, !kSecond) : -1;
                if (good && slot < 0) atomicOr(p.err, kErrHashFull);
                if (slot >= 0) {
                    if (!kSecond) {
                        acc += atomicAdd(cnt + slot, 1u);
                    } else {
                        delta = cnt[slot] - 1u;   // below 384
                        if (wants_edges(MODE) && delta) atomicAdd(p.pe + pos, (unsigned long long)delta);
                    }
                }
            }
            if (kSecond) run_add<uint32_t>(msum, q, delta, lane);
        }
        __syncwarp();
        if (kSecond && len > 0) {
            const unsigned long long dsum = msum[nz];
            if (dsum) {
                if (wants_vertices(MODE)) atomicAdd(p.pv + v, dsum);
                if (wants_edges(MODE)) atomicAdd(p.pe + e, dsum);
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
    const int32_t lb = range_lo(p, x);
    const unsigned long long bound = end_bound(p, x, lb);
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
        if (wants_vertices(MODE)) {
            for (uint32_t s = lane; s < cap; s += 32) {
                const int32_t k = keys[s];
                if (k >= 0 && cnt[s] >= 2) atomicAdd(p.pv + lb + k, c2(cnt[s]));
            }
        }
        warp_walk<MODE, true>(p, x, lb, cap - 1, keys, cnt, msum, wstart, wsrc);
        if (wants_vertices(MODE)) {
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
__global__ void __launch_bounds__(kCountThreads, kCountCtasPerSm) k_count(CountParams p) {
    extern __shared__ __align__(16) unsigned char ctr[];
    __shared__ SharedTeam<MODE, Pos, kCountThreads> sh;
    const Team<kCountThreads> cta{(int)threadIdx.x, 0};
    // a batch plan whose input failed the checks counts nothing (uniform)
    if (p.guard && (*(volatile const int *)p.guard & (kErrBadOffsets | kErrBadId))) return;
    unsigned long long acc = 0;
    // phase A: CTA items, heaviest first (the dense items, then the hash items)
    if (threadIdx.x == 0) sh.item = atomicAdd(p.cursors, 1);
    __syncthreads();
    int64_t it = sh.item;
    __syncthreads();
    const int64_t n_cta = n_cta_items(p);
    while (it < n_cta) {
        if (!has_second_walk(MODE) && p.cta_items[it].y >= 0) {
            acc += dense_stream<MODE, Pos>(p, it, ctr, sh, cta);
            __syncthreads();   // join: the last item's slowest warps
            continue;
        }
        acc += cta_item<MODE, Pos>(p, p.cta_items[it], ctr, sh, cta);
        if (threadIdx.x == 0) sh.item = atomicAdd(p.cursors, 1);
        __syncthreads();
        it = sh.item;
        __syncthreads();
    }
    // phase B: team items.  Team k owns warps 8k..8k+7 and the 48 KB of shared
    // memory that are their warp regions; its table is followed by its batch
    // arrays.  A team leaves together (its item index is read before its
    // barrier), so none of its warps is still using the region when the
    // first one starts phase C in its own part of it.
    const int64_t n_team = n_team_items(p);
    if (n_team > 0) {
        typedef SharedTeam<MODE, Pos, kTeamThreads> TS;
        static_assert(kTeamTableBytes + sizeof(TS) <= kTeamRegion, "team region overflow");
        const int k = threadIdx.x / kTeamThreads;
        const Team<kTeamThreads> team{(int)(threadIdx.x % kTeamThreads), 1 + k};
        unsigned char *table = ctr + (size_t)k * kTeamRegion;
        TS &tsh = *reinterpret_cast<TS *>(table + kTeamTableBytes);
        for (;;) {
            if (team.tid == 0) tsh.item = atomicAdd(p.cursors + 4, 1);
            team.sync();
            const int64_t it = tsh.item;
            team.sync();
            if (it >= n_team) break;
            acc += team_item<MODE, Pos>(p, p.team_items[it], table, tsh, team);
        }
    }
    // phase C: warp items
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        unsigned char *region = ctr + (size_t)warp * kWarpRegion;
        const int64_t n_warp = n_warp_items(p);
        for (;;) {
            int it = 0;
            if (lane == 0) it = atomicAdd(p.cursors + 1, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= n_warp) break;
            acc += warp_item<MODE>(p, p.warp_items[it], region);
        }
    }
    // a7: reduction of the per-thread partial sums
    const unsigned long long t = team_sum(acc, sh, cta);
    if (threadIdx.x == 0 && t) atomicAdd(p.acc, t);
}

// The retry pass over the starts the first launch (or prepare) re-queued.
// Entry x >= 0: its team table filled up, so try a CTA table; entry -(x+1),
// or a CTA table that fills up too: dense counters over the chunks of x's
// end range.
template <int MODE, typename Pos>
__global__ void __launch_bounds__(kCountThreads, kCountCtasPerSm) k_count_retry(CountParams p) {
    extern __shared__ __align__(16) unsigned char ctr[];
    __shared__ SharedTeam<MODE, Pos, kCountThreads> sh;
    const Team<kCountThreads> cta{(int)threadIdx.x, 0};
    unsigned long long acc = 0;
    const int nretry = (int)min(p.retry_static + *((volatile int *)(p.cursors + 2)), p.retry_cap);
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(p.cursors + 3, 1);
        __syncthreads();
        const int it = sh.item;
        __syncthreads();
        if (it >= nretry) break;
        const int32_t entry = p.retry[it];
        const int32_t x = entry >= 0 ? entry : -(entry + 1);
        unsigned long long item_acc = 0;
        bool done = false;
        if (entry >= 0) {
            item_acc = hash_item<MODE, Pos>(p, x, ctr, kHashMaxSlots, sh, cta);
            done = !sh.overflow;
            __syncthreads();
        }
        if (!done) item_acc = dense_all_chunks<MODE, Pos>(p, x, ctr, sh, cta);
        if (MODE == kModeBatch) add_to_graph(p, x, item_acc, sh, cta);
        __syncthreads();
        acc += item_acc;
    }
    const unsigned long long t = team_sum(acc, sh, cta);
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

// ⋈_e from the two G* slots of every edge: the U-side slots [m, 2m) hold
// each edge once, in rows that are permutations of the caller's rows (so
// the stores stay inside one row), then the L-side slots [0, m) add theirs,
// at edge ids in no useful order.  Every edge id occurs once per side, so the
// second pass needs no atomicity; it adds with reductions anyway, which the
// L2 carries out without returning the old value to the SM, so no thread
// waits on the scattered reads.  The second runs after the first on the same
// stream.
__global__ void k_edges_from_slots_u(const unsigned long long *__restrict__ pe_slot,
                                     const int32_t *__restrict__ eid, int64_t m, uint64_t *per_edge) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        per_edge[__ldg(eid + m + i)] = pe_slot[m + i];
}
__global__ void k_edges_from_slots_l(const unsigned long long *__restrict__ pe_slot,
                                     const int32_t *__restrict__ eid, int64_t m, uint64_t *per_edge) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const unsigned long long x = pe_slot[i];
        if (x) atomicAdd(reinterpret_cast<unsigned long long *>(per_edge) + __ldg(eid + i), x);
    }
}

template <int MODE, typename Pos>
cudaError_t setup_one() {
    cudaError_t e = cudaFuncSetAttribute(k_count<MODE, Pos>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kCounterBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_count<MODE, Pos>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_count_retry<MODE, Pos>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kCounterBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_count_retry<MODE, Pos>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

template <typename Pos>
void launch_main(int mode, int grid, cudaStream_t s, const CountParams &p) {
    if (mode == kModeTotal) k_count<kModeTotal, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    else if (mode == kModeBatch) k_count<kModeBatch, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    else if (mode == kModeVertices) k_count<kModeVertices, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    else if (mode == kModeAll) k_count<kModeAll, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    else k_count<kModeEdges, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
}

template <typename Pos>
void launch_retry(int mode, int grid, cudaStream_t s, const CountParams &p) {
    if (mode == kModeTotal) k_count_retry<kModeTotal, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    else if (mode == kModeBatch) k_count_retry<kModeBatch, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    else if (mode == kModeVertices) k_count_retry<kModeVertices, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    else if (mode == kModeAll) k_count_retry<kModeAll, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
    else k_count_retry<kModeEdges, Pos><<<grid, kCountThreads, kCounterBytes, s>>>(p);
}

}  // namespace

int count_smem_setup(int device) {
    static bool done[64] = {false};
    if (device < 0 || device >= 64) return BFC_ERR_INVALID_ARGUMENT;
    if (done[device]) return BFC_OK;
    BFC_CUDA((setup_one<kModeTotal, int32_t>()));
    BFC_CUDA((setup_one<kModeVertices, int32_t>()));
    BFC_CUDA((setup_one<kModeEdges, int32_t>()));
    BFC_CUDA((setup_one<kModeBatch, int32_t>()));
    BFC_CUDA((setup_one<kModeTotal, long long>()));
    BFC_CUDA((setup_one<kModeVertices, long long>()));
    BFC_CUDA((setup_one<kModeEdges, long long>()));
    BFC_CUDA((setup_one<kModeBatch, long long>()));
    BFC_CUDA((setup_one<kModeAll, int32_t>()));
    BFC_CUDA((setup_one<kModeAll, long long>()));
    done[device] = true;
    return BFC_OK;
}

int launch_count(Graph *g, cudaStream_t s, int mode, unsigned long long *pv_proj,
                 unsigned long long *pe, unsigned long long *gtot) {
    int rc = count_smem_setup(g->device);
    if (rc) return rc;
    CountParams p;
    p.off = g->off; p.adj = g->adj; p.eid = g->eid; p.plen = g->plen; p.cut = g->cut;
    p.work = g->work; p.cta_items = g->cta_items; p.team_items = g->team_items;
    p.warp_items = g->warp_items;
    p.n_cta = g->n_cta_items; p.n_team = g->n_team_items; p.n_warp = g->n_warp_items;
    p.cursors = g->cursors; p.acc = g->acc; p.pv = pv_proj; p.pe = pe;
    // the chunk-boundary table is relative to the start of each list, which
    // is where Algorithm 2's runs start
    p.coff = g->opt.orientation == 0 ? g->coff : nullptr;
    p.coff_u1 = g->coff_u1; p.coff_l1 = g->coff_l1;
    p.ctb = g->ctb;
    p.gstar = g->gstar; p.vbase = g->vbase; p.vend = g->vend; p.sbeg = g->sbeg; p.gtot = gtot;
    p.retry = g->retry; p.retry_cap = g->retry_cap; p.retry_static = g->retry_static;
    p.retry_on = g->may_retry ? 1 : 0;
    p.orient = g->opt.orientation; p.n = g->n;
    p.adj_len = 2 * g->m; p.l = g->l; p.err = g->err;
    p.core_on = (mode == kModeTotal && g->core_u + g->core_l > 0) ? 1 : 0;
    p.core_lo_u = g->core_u > 0 ? g->core_lo_u : g->n;
    p.core_lo_l = g->core_l > 0 ? g->core_lo_l : g->n;
    p.core_ld_u = g->core_ld_u; p.core_ld_l = g->core_ld_l;
    p.ccut = g->ccut; p.core_au = g->core_au; p.core_al = g->core_al;
    p.item_counts = g->item_counts;
    p.guard = g->item_counts ? g->err : nullptr;
    if (p.core_on) {
        // the core pairs' a(u, w), on the same stream before the walk
        int rc2 = core_product(g, s);
        if (rc2) return rc2;
    }
    BFC_CUDA(cudaMemsetAsync(g->cursors, 0, 8 * sizeof(int), s));
    BFC_CUDA(cudaMemsetAsync(g->acc, 0, sizeof(unsigned long long), s));
    const int grid = g->grid;
    // 32-bit adjacency positions whenever G* has fewer than 2^31 slots
    const bool narrow_pos = 2 * g->m <= 0x7fffffffll && !g->opt.wide_positions;
    if (narrow_pos) launch_main<int32_t>(mode, grid, s, p);
    else launch_main<long long>(mode, grid, s, p);
    note_launch();
    BFC_CUDA(cudaGetLastError());
    if (g->may_retry) {
        // the retry pass reads how many starts the first launch re-queued
        if (narrow_pos) launch_retry<int32_t>(mode, grid, s, p);
        else launch_retry<long long>(mode, grid, s, p);
        note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    return BFC_OK;
}

int gather_edges(Graph *g, cudaStream_t s, uint64_t *per_edge) {
    if (g->m == 0) return BFC_OK;
    const unsigned blocks = (unsigned)std::min<int64_t>((g->m + 255) / 256, (int64_t)g->num_sms * 16);
    k_edges_from_slots_u<<<blocks, 256, 0, s>>>(g->pe_slot, g->eid, g->m, per_edge);
    note_launch();
    BFC_CUDA(cudaGetLastError());
    k_edges_from_slots_l<<<blocks, 256, 0, s>>>(g->pe_slot, g->eid, g->m, per_edge);
    note_launch();
    BFC_CUDA(cudaGetLastError());
    return BFC_OK;
}

int gather_vertices(Graph *g, cudaStream_t s, uint64_t *per_u, uint64_t *per_l) {
    const int64_t nmax = g->r > g->l ? g->r : g->l;
    if (nmax == 0) return BFC_OK;
    k_gather_vertices<<<(unsigned)((nmax + 255) / 256), 256, 0, s>>>(g->pv, g->rank_u, g->rank_l,
                                                                      g->r, g->l, per_u, per_l);
    note_launch();
    BFC_CUDA(cudaGetLastError());
    return BFC_OK;
}

}  // namespace bfc
