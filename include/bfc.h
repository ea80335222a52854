/*
 * libbfc — exact butterfly counting in bipartite graphs on one GB300 GPU.
 *
 * The method is the vertex-priority counting of Wang, Lin, Qin, Zhang and
 * Zhang, "Efficient Butterfly Counting for Large Bipartite Networks":
 *   - priority p(x) of Definition 3 (higher degree first, ties broken by id,
 *     with every U id above every L id as Section 2 assumes);
 *   - the projection of Definition 4 (vertices renumbered by per-layer
 *     priority rank, L first, U offset by |L|) with neighbour lists sorted by
 *     priority;
 *   - Algorithm 2's wedge processing: for a start u, every middle v with
 *     p(v) < p(u) and every end w with p(w) < p(u); the butterflies of the
 *     pair (u, w) number C(count_wedge(w), 2) (Lemma 1);
 *   - per-edge counts by the second wedge walk of Algorithm 4 (Eq. 7), and
 *     per-vertex counts by the same walk (Eq. 1 / Eq. 2).
 * All counts are exact unsigned 64-bit integers.
 *
 * Memory and streams
 *   Every pointer whose name ends in _dev is device memory owned by the
 *   caller; the library never frees it.  `stream` is a cudaStream_t passed
 *   as void* (NULL = the legacy default stream).  The library allocates its
 *   own working memory (the renumbered graph and schedule) from a
 *   stream-ordered pool that it owns; bfc_release() returns it.
 *
 * Errors
 *   Every int-returning call returns a bfc_status.  Nothing crosses the ABI
 *   as an exception.  Outputs are defined only when the call returned
 *   BFC_OK (and, for asynchronous calls, once bfc_sync() on the same graph
 *   and stream returned BFC_OK).  bfc_last_error() gives a one-line message
 *   for the calling thread's last failure.
 *
 * Graph contract
 *   A simple bipartite graph G(U, L, E) with E ⊆ U × L (Section 2): no
 *   duplicate edges.  It is given by its U-side CSR: off_u[num_u + 1]
 *   (non-decreasing, off_u[0] = 0, off_u[num_u] = num_edges) and
 *   adj_u[num_edges] (L ids in [0, num_l), any order within a list).  The
 *   edge stored at slot k of adj_u has edge id k; per-edge outputs use it.
 *   Isolated vertices are allowed.  Limits: num_edges <= 2^31 - 1,
 *   num_u + num_l <= 2^31 - 2.
 */
#ifndef BFC_H
#define BFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bfc_status {
    BFC_OK = 0,
    BFC_ERR_INVALID_ARGUMENT = 1, /* null pointer, negative or oversized sizes */
    BFC_ERR_INVALID_GRAPH = 2,    /* offsets not a CSR, id out of range, duplicate edge */
    BFC_ERR_OUT_OF_MEMORY = 3,    /* device or host allocation failed */
    BFC_ERR_CUDA = 4,             /* a CUDA runtime call failed */
    BFC_ERR_TIMEOUT = 5,          /* reserved: a bounded device wait gave up */
    BFC_ERR_INTERNAL = 6          /* a kernel's own consistency check fired */
} bfc_status;

/* Opaque handle of a prepared graph; owned by the library. */
typedef struct bfc_graph bfc_graph;

/* U-side CSR in device memory (see "Graph contract"). */
typedef struct bfc_csr {
    int32_t num_u;          /* r = |U| */
    int32_t num_l;          /* l = |L| */
    int64_t num_edges;      /* m = |E| */
    const int32_t *off_u;   /* device, [num_u + 1] */
    const int32_t *adj_u;   /* device, [num_edges] */
} bfc_csr;

/* Tuning and checking knobs.  Call bfc_options_init() first; a NULL
 * options pointer means the defaults. */
typedef struct bfc_options {
    int32_t validate;       /* 1 (default): reject duplicate edges.  Offsets and
                               id ranges are always checked. */
    int32_t warp_max_work;  /* starts with at most this many wedges are counted
                               by one warp with a 512-slot shared-memory hash
                               table (default 384, range [0, 384]; a table is at
                               most 3/4 full) */
    int32_t hash_max_work;  /* Algorithm 2: starts with at most this many
                               wedges (and more than team_max_work) are counted
                               by one CTA with a shared-memory hash table of up
                               to 32,768 slots, at most 3/4 full (default
                               24576, range [warp_max_work, 24576]); heavier
                               starts get dense
                               shared-memory counters over chunks of their end
                               range.  Algorithm 3: ignored, except that 0 sends
                               every start beyond the warp bin to the dense pass */
    int32_t num_ctas;       /* persistent grid size; 0 (default) = one CTA per SM */
    int32_t wide_positions; /* 1: count with 64-bit adjacency positions even when
                               32 bits suffice (they are used automatically when
                               the graph has 2^30 edges or more); default 0 */
    int32_t orientation;    /* which wedges are enumerated (same W by Lemma 4):
                               0 (default) = Algorithm 2: start u highest,
                               p(v) < p(u), p(w) < p(u);
                               1 = Algorithm 3 (BFC-VP++): end w highest,
                               p(w) > p(u), p(w) > p(v).  With 1, every start
                               beyond the warp bin gets a team or CTA hash table
                               and a start whose table fills up is counted again
                               by a retry pass (a CTA table, then dense chunks). */
    int32_t team_max_work;  /* starts with more than warp_max_work and at most
                               this many wedges are counted by a 256-thread team
                               (four per CTA) with a 4,096-slot hash table.
                               -1 (default) = 3072 for Algorithm 2 (its tables
                               then always fit) and 16384 for Algorithm 3;
                               otherwise in [0, 16384], and a value <=
                               warp_max_work leaves the team bin empty.
                               Algorithm 2 caps it at hash_max_work; above 3072
                               a start whose team table fills up goes to the
                               retry pass. */
    int32_t core_vertices;  /* Algorithm 2 total counts (bfc_count) of single
                               graphs only: the K vertices of highest priority
                               (Definition 3) form a core whose pairs are
                               counted by a masked 0/1 matrix product on the
                               tensor cores (the walk of every core start skips
                               the wedges with middle and end in the core too
                               and adds a·b + C(a, 2) per core pair, Lemma 1;
                               core starts are always counted with dense
                               counters).  -1 (default) = automatic: K = the
                               number of starts with more than hash_max_work
                               wedges, at most 8,192, and no core unless each
                               layer holds at least 1,024 of its vertices;
                               0 = off; K > 0: that many (at most 65,535 core
                               vertices per layer, else
                               BFC_ERR_INVALID_ARGUMENT).  Per-vertex and
                               per-edge counts of the same graph walk every
                               wedge as usual.  Costs 8·K_U·K_L bytes of bf16
                               operands and 2·(K_U² + K_L²) bytes of products. */
    int32_t use_tuned;      /* 1: if bfc_autotune has tuned a graph of the same
                               size class in this process (same orientation,
                               single graph or batch, and the same
                               floor(log2) of the edge count and of the vertex
                               count), prepare with the bin bounds it chose
                               instead of warp/team/hash_max_work; 0 (default):
                               use the bounds given here */
    int32_t reserved[7];    /* must be zero */
} bfc_options;

/* Figures of a prepared graph (host values). */
typedef struct bfc_info {
    int32_t num_u, num_l;
    int64_t num_edges;
    uint64_t wedges;          /* W: wedges Algorithm 2 processes (Section 4) */
    uint64_t max_start_work;  /* largest per-start wedge count */
    int64_t starts_with_work; /* starts u with at least one wedge */
    int64_t warp_starts;      /* starts in the warp/hash bin */
    int64_t hash_starts;      /* starts in the CTA/hash bin (Algorithm 3 with
                                 hash_max_work 0: starts sent to the dense pass) */
    int64_t dense_starts;     /* starts in the CTA/dense bin */
    int64_t dense_items;      /* (start, end-range chunk) work items of the dense bin */
    int64_t device_bytes;     /* library-owned device memory held by the graph */
    int32_t max_deg_u, max_deg_l;
    int64_t team_starts;      /* starts in the team/hash bin */
    int32_t core_u, core_l;   /* core vertices per layer (core_vertices option; 0 = no core) */
} bfc_info;

/* What bfc_export() can copy out (for parity tests; layouts as stated). */
typedef enum bfc_array {
    BFC_RANK_U = 0,   /* int32[num_u]: per-layer priority rank of each U vertex (Definition 4) */
    BFC_RANK_L = 1,   /* int32[num_l] */
    BFC_PROJ_OFF = 2, /* int64[n + 1]: CSR offsets of the projection graph G*, n = num_u + num_l;
                         ids of G*: L vertex v -> rank_l[v], U vertex u -> num_l + rank_u[u] */
    BFC_PROJ_ADJ = 3, /* int32[2m]: neighbour ids in G*, each list ascending */
    BFC_PROJ_EID = 4, /* int32[2m]: edge id (U-side slot) of each entry */
    BFC_CUT = 5,      /* int32[n]: |{y in N(x) : p(y) < p(x)}| per vertex of G* */
    BFC_WORK = 6,     /* uint64[n]: wedges Algorithm 2 processes from each start x of G* */
    BFC_RETRIES = 7,  /* int32[1]: starts whose hash table filled up in the last
                         count's first launch and went to the retry pass */
    BFC_CORE_PRODUCT_U = 8, /* uint16[core_u * core_u] (bfc_info), row-major: for core U
                         vertices u, w (G* ids num_l + num_u - core_u + i), entry
                         (i_u, i_w) with i_w < i_u = the core middles v with p(v) < p(u)
                         adjacent to both (the a of Lemma 1's split); entries with
                         i_w >= i_u are unspecified.  Written by the last bfc_count
                         of a graph prepared with core_vertices > 0 */
    BFC_CORE_PRODUCT_L = 9  /* uint16[core_l * core_l]: the same for the L core (G* ids
                         num_l - core_l + i) */
} bfc_array;

/* Fills *opt with the defaults listed above (NULL is ignored).  Library
 * plumbing with no counterpart in the paper. */
void bfc_options_init(bfc_options *opt);

/* Steps a1-a5 of the hot path: degrees, priority ranks (Definition 3),
 * the projection G* with priority-sorted lists (Definition 4, Section 4's
 * neighbour sort), the per-start orientation cut and exact wedge work, and
 * the degree-binned, heaviest-first schedule (Section 6.2's dynamic
 * scheduling).  Reads the caller's CSR on `stream`; the caller may free it
 * once this call returns.  Synchronises `stream` (it needs sizes on the
 * host).  On success *out owns library memory until bfc_release(). */
int bfc_prepare(const bfc_csr *csr, const bfc_options *opt, void *stream, bfc_graph **out);

/* Steps a6-a7: wedge enumeration with per-start aggregation (Algorithm 2)
 * and the reduction to ⋈_G.  Writes one uint64 to total_dev.  Asynchronous
 * on `stream`; no host synchronisation, no allocation. */
int bfc_count(bfc_graph *g, void *stream, uint64_t *total_dev);

/* Step a8: per-vertex counts ⋈_x (Eq. 1) in ORIGINAL ids: per_u_dev[num_u],
 * per_l_dev[num_l] (either may be NULL), and the total if total_dev != NULL.
 * Asynchronous; no allocation. */
int bfc_count_vertices(bfc_graph *g, void *stream, uint64_t *per_u_dev, uint64_t *per_l_dev,
                       uint64_t *total_dev);

/* Step a9: per-edge counts ⋈_e (Eq. 7, Algorithm 4) indexed by edge id
 * (U-side slot): per_edge_dev[num_edges]; plus the total if total_dev !=
 * NULL.  Asynchronous; no host synchronisation.  The walks sum per slot of
 * G* (two per edge): the first per-edge call on a graph takes that array,
 * 16·num_edges bytes, from the library's pool (stream-ordered) and keeps it
 * until bfc_release (BFC_ERR_OUT_OF_MEMORY if the pool cannot grow). */
int bfc_count_edges(bfc_graph *g, void *stream, uint64_t *per_edge_dev, uint64_t *total_dev);

/* ⋈_G by the pair formulation of Section 6.3 (Algorithm 6's wedge pairs,
 * run in device memory instead of on disk): every wedge (x, v, w) of the
 * prepared orientation becomes the key (x, w); a radix sort groups equal
 * keys, and a run of c equal keys adds C(c, 2) (Lemma 1; each butterfly is
 * counted by one pair, Lemma 4).  A second exact path beside the counter
 * walk of bfc_count (which reads each end once, where this one writes and
 * sorts 8·W bytes of keys).  Writes one uint64 to total_dev.  Takes 24·W
 * bytes plus the sort's histograms from the library's pool and frees them,
 * stream-ordered; no host synchronisation.  BFC_ERR_INVALID_ARGUMENT for a
 * batch or for W >= 2^32 - 1 (the sort's offsets are 32-bit),
 * BFC_ERR_OUT_OF_MEMORY if the pool cannot grow. */
int bfc_count_pairs(bfc_graph *g, void *stream, uint64_t *total_dev);

/* Steps a8 and a9 together: the outputs of bfc_count_vertices and
 * bfc_count_edges from ONE first walk and ONE second walk (Algorithm 4's
 * pass attributes to vertices and edges at once).  per_u_dev / per_l_dev may
 * be NULL; per_edge_dev may be NULL only when num_edges is 0.  Asynchronous;
 * memory as bfc_count_edges. */
int bfc_count_all(bfc_graph *g, void *stream, uint64_t *per_u_dev, uint64_t *per_l_dev,
                  uint64_t *per_edge_dev, uint64_t *total_dev);

/* A batch of independent graphs given as one disjoint union: the union's
 * U-side CSR (bfc_csr; L ids global) plus, per graph g, its U vertices
 * [graph_u_start[g], graph_u_start[g+1]) and L vertices
 * [graph_l_start[g], graph_l_start[g+1]).  Every edge must join a U and an L
 * vertex of the same graph. */
typedef struct bfc_batch {
    int32_t num_graphs;
    const int32_t *graph_u_start;   /* device, [num_graphs + 1], prefix sums of |U_g| */
    const int32_t *graph_l_start;   /* device, [num_graphs + 1], prefix sums of |L_g| */
} bfc_batch;

/* Steps a1-a5 for a whole batch at once: one set of segmented sorts and
 * scans over the union (Theorem 1: any total order counts every component
 * exactly, so the union's priority order serves all graphs).  Rejects edges
 * that cross graphs (BFC_ERR_INVALID_GRAPH).  Synchronises `stream`. */
int bfc_prepare_batch(const bfc_csr *union_csr, const bfc_batch *batch, const bfc_options *opt,
                      void *stream, bfc_graph **out);

/* Steps a6-a7 for a batch in ONE persistent launch (Algorithm 2 for every
 * start of every graph, scheduled together as Section 6.2's dynamic
 * scheduling): totals_dev[g] = ⋈ of graph g (uint64[num_graphs], device);
 * total_dev (nullable) = their sum.  BFC_ERR_INVALID_ARGUMENT if g was not
 * prepared by bfc_prepare_batch.
 * Asynchronous, no allocation, no host synchronisation: it can be captured
 * in a CUDA graph once a first call has been made outside capture. */
int bfc_count_batch(bfc_graph *g, void *stream, uint64_t *totals_dev, uint64_t *total_dev);

/* Processed wedges W of every graph of a batch (the wedges Algorithm 2
 * visits, equal to Algorithm 3's by Lemma 4): uint64[num_graphs], device,
 * caller-owned.  Asynchronous. */
int bfc_batch_wedges(const bfc_graph *g, void *stream, uint64_t *wedges_dev);

/* Autotuner for the bin thresholds of step a5: re-bins the prepared graph for
 * each candidate (Algorithm 2: warp_max_work in {32, 128, 384} x
 * team_max_work in {512, 3072} x hash_max_work in {4096, 24576}; Algorithm 3:
 * warp_max_work in {32, 128, 384} x team_max_work in {2048, 16384}), times
 * `iters` count launches of each with CUDA events on `stream`, keeps the
 * fastest and writes it to *chosen (nullable).  The choice is also kept for
 * the graph's size class for the rest of the process (see use_tuned; a later
 * tuning of the same class replaces it).  The CTA shape of the count (1,024
 * threads per SM, four 256-thread teams, 2,048 middles per batch) is fixed
 * at compile time.  Synchronises `stream`; allocates only the schedule
 * arrays. */
int bfc_autotune(bfc_graph *g, void *stream, int iters, bfc_options *chosen);

/* ---- Batches of a fixed shape, counted with no host synchronisation -------
 * A batch plan prepares and counts batches (bfc_batch) whose union always has
 * the same shape, with every step on the stream and every array allocated
 * once: steps a1-a5 (Definition 3's ranks of every graph, Definition 4's
 * projection, the cut and exact work of Section 4 / Eq. 5, Section 6.2's
 * heaviest-first bins) and a6-a7 (Algorithm 2 for every start of every
 * graph in one persistent launch).  No call of bfc_batch_plan_run
 * synchronises or allocates, so a caller can record a whole step in a CUDA
 * graph and replay it after writing new contents of the same shape into the
 * same input buffers.  The library has no counterpart in the paper for this
 * plumbing; the counts are those of bfc_prepare_batch + bfc_count_batch. */
typedef struct bfc_batch_plan bfc_batch_plan;
typedef struct bfc_batch_shape {
    int32_t num_u, num_l;   /* layer sizes of the union (all graphs together) */
    int64_t num_edges;      /* edges of the union, at most 2^31 - 1 */
    int32_t num_graphs;     /* graphs per batch, at least 1 */
    int32_t max_layer;      /* the largest layer of any one graph, 1 .. 65,535: a
                               degree stays below 2^16, and each dense start's
                               end range is one chunk of counters */
    int32_t reserved[6];    /* must be zero */
} bfc_batch_shape;

/* Allocates a plan for batches of this shape on the current device (library
 * pool) and sets up the kernels it uses, on `stream`; synchronises it.  The
 * options must choose Algorithm 2 (orientation 0) and a team bound of at most
 * 3,072 wedges (team_max_work -1 or <= 3072: every team table fits, so no
 * retry pass is needed); core_vertices is ignored (batches have no core).
 * BFC_ERR_INVALID_ARGUMENT for a shape or options outside these ranges,
 * BFC_ERR_OUT_OF_MEMORY if the pool cannot hold the plan.  Create the plan
 * before any stream capture. */
int bfc_batch_plan_create(const bfc_batch_shape *shape, const bfc_options *opt, void *stream,
                          bfc_batch_plan **out);

/* One batch of the plan's shape: off_u_dev[num_u + 1] / adj_u_dev[num_edges]
 * (the union's U-side CSR, L ids global) and graph_u_start_dev /
 * graph_l_start_dev [num_graphs + 1] (as in bfc_batch), all device memory
 * that the caller owns.  Writes totals_dev[g] = ⋈ of graph g (uint64
 * [num_graphs], device) and, if status_dev is not NULL, one int32 status
 * (device): BFC_OK; BFC_ERR_INVALID_GRAPH for offsets that are not a CSR, an
 * id out of range, start arrays that are not prefix sums of the layer sizes,
 * an edge across graphs, a graph layer above max_layer, or (validate) a
 * duplicate edge; BFC_ERR_INTERNAL for a failed consistency check.  The
 * totals are defined only when the status is BFC_OK (they are 0 when the
 * input failed its checks: no kernel after the checks indexes with it).
 * Asynchronous on `stream`: no host synchronisation, no allocation; the
 * return value reports launch errors only.  Runs of one plan share its
 * arrays: issue them on one stream. */
int bfc_batch_plan_run(bfc_batch_plan *plan, const int32_t *off_u_dev, const int32_t *adj_u_dev,
                       const int32_t *graph_u_start_dev, const int32_t *graph_l_start_dev,
                       void *stream, uint64_t *totals_dev, int32_t *status_dev);

/* Frees the plan (stream-ordered on the stream of its last run, then waits
 * for it).  NULL is ignored. */
void bfc_batch_plan_destroy(bfc_batch_plan *plan);

/* ---- Approximate counting by edge sparsification --------------------------
 * Section 7 uses the exact counter as the inner block of a sampling
 * estimator: each sample is a graph in which every edge of G is kept
 * independently with probability p, and is counted exactly.  A butterfly
 * survives a sample iff its four edges do, so E[⋈(G_j)] = p^4 · ⋈(G) and
 *     estimate = Σ_j ⋈(G_j) / (num_samples · p^4).
 * Keep rule: sample j (0 <= j < num_samples) keeps the edge at U-side slot e
 * iff the (j·num_edges + e + 1)-th output of SplitMix64 (Steele, Lea and
 * Flood, OOPSLA 2014) seeded with `seed` is below floor(p · 2^64); p = 1
 * keeps every edge.  The counts of the samples are exact (uint64); the
 * number of samples an (ε, δ) guarantee needs is the caller's choice.
 *
 * bfc_prepare_sparsified draws the samples from the U-side CSR
 * (off_u_dev[num_u + 1], adj_u_dev[num_edges], device, int32, read only)
 * and prepares them as ONE batch (bfc_prepare_batch) of num_samples
 * disjoint graphs: sample j has U vertices [j·num_u, (j+1)·num_u) and L
 * vertices [j·num_l, (j+1)·num_l) of the prepared union.  Count it with
 * bfc_count_batch (totals_dev[j] = ⋈(G_j)); bfc_batch_wedges and
 * bfc_graph_info describe the samples.  sample_edges_dev (nullable, device,
 * uint64[num_samples]) receives the edges each sample kept.
 * Requires 0 < p <= 1, num_samples >= 1, num_samples · (num_u + num_l) below
 * 2^31 - 1 and at most 2^31 - 1 kept edges over all samples
 * (BFC_ERR_INVALID_ARGUMENT otherwise); offsets that are not a CSR of
 * num_edges slots, or L ids outside [0, num_l), give BFC_ERR_INVALID_GRAPH
 * before any sample is written.  Synchronises `stream`; the sampled union is
 * transient (freed in stream order once prepared). */
int bfc_prepare_sparsified(int32_t num_u, int32_t num_l, int64_t num_edges, const int32_t *off_u_dev,
                           const int32_t *adj_u_dev, double p, uint64_t seed, int32_t num_samples,
                           const bfc_options *opt, void *stream, uint64_t *sample_edges_dev,
                           bfc_graph **out);

/* The estimator from the samples' exact counts (sample_counts_dev,
 * uint64[num_samples], device): estimate_dev[0] = Σ c_j / (num_samples ·
 * p^4), estimate_dev[1] = its standard error, the sample standard deviation
 * of c_j / p^4 over sqrt(num_samples) (NaN for one sample).  estimate_dev is
 * double[2], device, caller-owned.  Asynchronous (one kernel on `stream`). */
int bfc_sparsified_estimate(const uint64_t *sample_counts_dev, int32_t num_samples, double p,
                            void *stream, double *estimate_dev);

/* All of it in one call: bfc_prepare_sparsified, bfc_count_batch into
 * sample_counts_dev (uint64[num_samples], device, caller-owned),
 * bfc_sparsified_estimate into estimate_dev (double[2], device, nullable),
 * then the prepared samples are released.  Synchronises `stream`. */
int bfc_estimate_sparsified(int32_t num_u, int32_t num_l, int64_t num_edges, const int32_t *off_u_dev,
                            const int32_t *adj_u_dev, double p, uint64_t seed, int32_t num_samples,
                            const bfc_options *opt, void *stream, uint64_t *sample_counts_dev,
                            double *estimate_dev);

/* ---- Serving: continuous batching of counting requests -------------------
 * Requests (one graph each, U-side CSR in HOST memory) may arrive at any time
 * from any thread.  Worker threads (one CUDA stream each) take the oldest
 * waiting requests that fit the device-memory budget, count them as one
 * batch (bfc_prepare_batch + bfc_count_batch), and complete them; requests
 * that arrive while other batches are on the GPU are admitted as soon as a
 * worker and memory are free, so batches overlap on the device.  A request's
 * total is exactly its graph's count alone (no butterfly spans two graphs of
 * a batch).  The paper has no serving layer; this wraps steps a1-a9 only. */
typedef struct bfc_server bfc_server;

typedef struct bfc_server_config {
    int64_t memory_budget_bytes; /* device bytes admitted batches may hold at once (default 120 GiB) */
    int32_t workers;             /* worker threads / streams (default 2, range [1, 16]) */
    int32_t max_batch_graphs;    /* requests per batch at most (default 1024; 1 = one graph per launch) */
    int64_t max_batch_edges;     /* edges per batch at most, unless one request alone is larger (default 2^26) */
    int32_t warp_max_work;       /* bin thresholds passed to every batch (0 = library default) */
    int32_t hash_max_work;
    int32_t team_max_work;
    int32_t reserved[7];
} bfc_server_config;

typedef struct bfc_server_stats {
    int64_t submitted, completed, failed, batches;
    int64_t max_batch_graphs;    /* largest batch formed */
    int64_t peak_bytes_in_use;   /* largest admitted footprint (the admission estimate) */
    int64_t bytes_in_use;        /* admitted footprint now */
    int64_t waiting;             /* requests not yet admitted */
    int64_t pool_bytes_at_create; /* the library pool's bytes in use when the server was created */
    int64_t pool_bytes_high;     /* the pool's measured high-water mark since then (all users of the
                                    pool on this device, the server's batches included) */
} bfc_server_stats;

/* Fills *cfg with the defaults listed above (NULL is ignored). */
void bfc_server_config_init(bfc_server_config *cfg);

/* Starts the workers on the current device.  *out is owned by the caller
 * until bfc_server_destroy.  BFC_ERR_INVALID_ARGUMENT for a configuration
 * outside the ranges above (max_batch_edges at most 2^31 - 1, so a batch's
 * CSR offsets fit int32); BFC_ERR_CUDA if a worker's stream cannot be created
 * (no server is created then).  Resets the high-water mark of the library's
 * device memory pool (see bfc_server_stats). */
int bfc_server_create(const bfc_server_config *cfg, bfc_server **out);

/* Queues one request.  off_u_host[num_u + 1] / adj_u_host[num_edges] must stay
 * valid until bfc_server_poll reports the request complete.  A request whose
 * footprint alone exceeds the budget returns BFC_ERR_OUT_OF_MEMORY; offsets
 * that are not a CSR of num_edges entries, or an id outside [0, num_l),
 * return BFC_ERR_INVALID_GRAPH (checked on the host here, so a bad request
 * never joins a batch); |U| + |L| or num_edges above 2^31 - 1 return
 * BFC_ERR_INVALID_ARGUMENT.  A duplicate edge is found on the device: the
 * request completes with BFC_ERR_INVALID_GRAPH, and the other requests of its
 * batch are counted again one by one, so their results are unchanged. */
int bfc_server_submit(bfc_server *sv, int32_t num_u, int32_t num_l, int64_t num_edges,
                      const int32_t *off_u_host, const int32_t *adj_u_host, uint64_t *request_id);

/* *status = -1 while pending, else the request's bfc_status; when complete,
 * *total = ⋈ of its graph, *latency_s = seconds from submit to completion,
 * and the request id is retired (a later poll of it returns
 * BFC_ERR_INVALID_ARGUMENT).  wait != 0 blocks until completion.  Different
 * requests may be polled from different threads at once; one request must
 * not be polled by two threads at the same time. */
int bfc_server_poll(bfc_server *sv, uint64_t request_id, int wait, uint64_t *total, int *status,
                    double *latency_s);

/* A snapshot of the counters above (thread-safe). */
int bfc_server_get_stats(bfc_server *sv, bfc_server_stats *out);

/* Stops the server: the workers first count every request still waiting
 * (each fits the budget on its own, so the queue drains), then exit; a
 * request that could still not be admitted completes with
 * BFC_ERR_INTERNAL.  Frees every request, polled or not.  No thread may be
 * inside bfc_server_poll or bfc_server_submit. */
void bfc_server_destroy(bfc_server *sv);

/* Waits for `stream` and reports any error a kernel of this graph flagged
 * since the last bfc_sync (BFC_ERR_INTERNAL), then clears the flag; a CUDA
 * failure returns BFC_ERR_CUDA.  Library plumbing (no paper counterpart). */
int bfc_sync(bfc_graph *g, void *stream);

/* Host figures of a prepared graph (sizes, W of Section 4, bin sizes; see
 * bfc_info).  Does not touch the GPU. */
int bfc_graph_info(const bfc_graph *g, bfc_info *out);

/* Copies one internal array (see bfc_array: Definition 3's ranks,
 * Definition 4's G*, Section 4's cut, Eq. 5's per-start work) to
 * caller-owned device memory dst_dev (size as listed), asynchronously on
 * `stream`.  BFC_ERR_INVALID_ARGUMENT for an unknown `which`. */
int bfc_export(const bfc_graph *g, int which, void *dst_dev, void *stream);

/* Steps a1-a7 (Algorithm 2, or 3 with opt->orientation = 1) end to end from
 * HOST memory: copies the CSR to the device, prepares, counts, copies ⋈_G
 * back to *total_host (and W to *wedges_host, nullable) and frees everything
 * it took.  Errors as bfc_prepare and bfc_count.
 * Synchronous.  off_u_host/adj_u_host may be pinned or pageable; page-locked
 * buffers are copied by the SMs, as in bfc_count_all_host. */
int bfc_count_host(int32_t num_u, int32_t num_l, int64_t num_edges, const int32_t *off_u_host,
                   const int32_t *adj_u_host, const bfc_options *opt, void *stream,
                   uint64_t *total_host, uint64_t *wedges_host);

/* Steps a1-a9 end to end from HOST memory (Algorithm 2 with Algorithm 4's
 * attribution): copies the CSR to the device, prepares, counts ⋈_G with the
 * per-vertex (Eq. 1) and per-edge (Eq. 7) counts, and copies them back:
 * per_u_host[num_u] and per_l_host[num_l] in original ids (either may be
 * NULL), per_edge_host[num_edges] by U-side slot (NULL only when num_edges
 * is 0), *total_host, and W to *wedges_host (nullable).  Frees everything it
 * took; synchronous.  A page-locked host buffer (cudaHostAlloc or
 * cudaHostRegister over the whole range) is moved by the SMs over the host
 * link, any other by cudaMemcpyAsync: on a GB300 the copy engines ran five
 * to eight times slower while a large prepared graph was held in device
 * memory, the SMs did not.  Errors as bfc_prepare and bfc_count_all. */
int bfc_count_all_host(int32_t num_u, int32_t num_l, int64_t num_edges, const int32_t *off_u_host,
                       const int32_t *adj_u_host, const bfc_options *opt, void *stream,
                       uint64_t *per_u_host, uint64_t *per_l_host, uint64_t *per_edge_host,
                       uint64_t *total_host, uint64_t *wedges_host);

/* Allocation-free count for small graphs.  The paper has no counterpart: this
 * exists for callers that may not allocate device memory where they count:
 * code whose device memory is reserved up front by its own allocator (a
 * caching allocator that already holds the whole budget, where one more
 * cudaMalloc fails or fragments it), or latency-bound loops that must not
 * enter the driver's allocator (cudaMalloc and cudaFree can synchronise the
 * device).  bfc_prepare cannot serve them because it allocates the
 * renumbered graph.
 *
 * Computes ⋈_G of the U-side CSR (off_u_dev, adj_u_dev: device memory, the
 * graph contract above) into *total_dev (one uint64, device memory) and, if
 * status_dev is not NULL, BFC_OK or BFC_ERR_INVALID_GRAPH (offsets not a CSR
 * of num_edges entries, or an id out of range) into *status_dev (one int32,
 * device memory); *total_dev is 0 for an invalid graph.  Duplicate edges are
 * not detected.  Asynchronous on `stream`; one cooperative kernel launch.
 *
 * Limits: num_u <= 49,152, num_l <= 49,152, num_u + num_l <= 65,536,
 * num_edges <= 1,048,576; larger graphs return BFC_ERR_INVALID_ARGUMENT
 * before any GPU work.
 *
 * All working memory is one fixed array of about 4.8 MB that every GPU which
 * loads the library holds until the process exits; no call allocates.  The
 * first call on a device looks up that array's device address and sets the
 * kernel's attributes, so make one call per device before any stream capture.
 * Every call uses the same array, which keeps the previous call's contents
 * (the kernel clears what must start at zero): calls whose kernels can overlap
 * on the GPU (different streams, or several host threads) race and give wrong
 * results; issue them on one stream. */
int bfc_count_small_noalloc(int32_t num_u, int32_t num_l, int64_t num_edges,
                            const int32_t *off_u_dev, const int32_t *adj_u_dev, void *stream,
                            uint64_t *total_dev, int32_t *status_dev);

/* Frees the graph's library memory (stream-ordered on the stream of its
 * last call).  NULL is ignored.  Library plumbing (no paper counterpart). */
void bfc_release(bfc_graph *g);

/* Static text for a status code. */
const char *bfc_status_string(int status);

/* One-line description of the calling thread's last failure ("" if none). */
const char *bfc_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int bfc_version(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all devices, all threads). */
long long bfc_kernel_launches(void);

/* Caterpillars (three-paths) of the prepared graph, the denominator of the
 * bipartite clustering coefficient 4·⋈_G / caterpillars named among the
 * applications of Section 1: Σ over edges (u, v) of (deg u − 1)(deg v − 1),
 * written as one uint64 to caterpillars_dev (device).  Asynchronous on
 * `stream`; no allocation. */
int bfc_caterpillars(bfc_graph *g, void *stream, uint64_t *caterpillars_dev);

/* The bipartite clustering coefficient of Section 1's applications,
 * 4·⋈_G / caterpillars (0 for a graph without three-paths), as one double
 * in coefficient_dev (device).  butterflies_dev (device, one uint64) holds
 * ⋈_G of this graph, for example written by bfc_count on the same stream
 * before this call; the caterpillars are computed as by bfc_caterpillars
 * into caterpillars_dev (device, one uint64).  Asynchronous on `stream`; no
 * allocation.  BFC_ERR_INVALID_ARGUMENT for a null pointer. */
int bfc_clustering_coefficient(bfc_graph *g, void *stream, const uint64_t *butterflies_dev,
                               uint64_t *caterpillars_dev, double *coefficient_dev);

/* Measurement aid (no counterpart in the paper): the throughput of the
 * count kernel's counter operation on the current device -- a returning
 * 32-bit shared-memory atomicAdd on a 16-bit counter packed two per word, at
 * pseudo-random indexes, one 1024-thread CTA with 192 KB of shared memory
 * per SM, `iters` (>= 1) increments per thread.  Writes increments per
 * second to *increments_per_s and the timed launch's device time to *ms
 * (nullable).  Synchronises `stream`; allocates 256 bytes from the
 * library's pool for the duration of the call. */
int bfc_bench_smem_atomics(void *stream, int32_t iters, double *increments_per_s, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* BFC_H */
