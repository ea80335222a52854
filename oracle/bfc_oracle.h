/*
 * CPU oracle for exact butterfly counting (Wang, Lin, Qin, Zhang, Zhang,
 * "Efficient Butterfly Counting for Large Bipartite Networks").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline arm may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two meet only through the
 * seeded input generators.
 *
 * Every routine takes the U-side CSR of a simple bipartite graph:
 *   r = |U|, l = |L|, off[r+1] (int32, off[0] = 0, off[r] = m), adj[m]
 *   (int32 L-ids).  The edge at U-side slot k has edge id k.
 * Outputs are caller-owned host arrays.  Return 0 on success, -1 on a
 * malformed graph (bad offsets, ids out of range, duplicate edges), -2 on
 * allocation failure.
 *
 * Parity status: every function below is pinned by tests against closed
 * forms, the paper's worked examples, exhaustive enumeration on tiny graphs
 * or cross-agreement with an independent definition (see tests/).
 */
#ifndef BFC_ORACLE_H
#define BFC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Definition 2 + Lemma 1 (Eq. 1, Eq. 2): for every unordered pair {x, y} of
 * the chosen layer, c = |N(x) ∩ N(y)| by merging sorted lists; the total is
 * the sum of C(c,2).  pair_layer: 0 = pairs of U vertices, 1 = pairs of L.
 * O(|layer|^2 * d); for small graphs only. */
int orc_brute_total(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                    int pair_layer, uint64_t *total);

/* Eq. 1 for every vertex: ⋈_x = Σ_{y ≠ x in x's layer} C(|N(x) ∩ N(y)|, 2).
 * pv_u[r], pv_l[l]. */
int orc_brute_vertices(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                       uint64_t *pv_u, uint64_t *pv_l);

/* Eq. 7 for every edge e = (u, v): ⋈_e = Σ_{w ∈ N(v), w ≠ u} (|N(u) ∩ N(w)| − 1),
 * summed only over w that share at least one more neighbour with u (terms
 * with |N(u) ∩ N(w)| = 1 contribute 0).  pe[m] in U-side slot order. */
int orc_brute_edges(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                    uint64_t *pe);

/* Eq. 1 for the listed vertices only, for graphs too large for the loops
 * above: for x, every two-hop path x - v - y with y != x adds one to
 * c_y = |N(x) ∩ N(y)|, and ⋈_x = Σ_y C(c_y, 2).  layer 0: xs are U ids,
 * layer 1: L ids.  out[i] belongs to xs[i].  O(m + Σ two-hop paths). */
int orc_vertices_sampled(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                         int layer, const int32_t *xs, int64_t k, uint64_t *out);

/* Eq. 7 for the listed edges only (U-side slots es[i]): for e = (u, v),
 * ⋈_e = Σ_{w ∈ N(v), w ≠ u} (|N(u) ∩ N(w)| − 1), with N(u) marked once and
 * each |N(u) ∩ N(w)| counted over N(w).  out[i] belongs to es[i]. */
int orc_edges_sampled(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                      const int64_t *es, int64_t k, uint64_t *out);

/* Algorithm 1 (BFC-IBS, layer priority).  The start layer S is U unless
 * Σ_U deg² < Σ_L deg², in which case S = L; wedges (u, v, w) with
 * w.id > u.id are hashed per start; total = Σ C(count, 2).  *wedges = number
 * of wedges that pass the id filter.  *start_layer = 0 (U) or 1 (L). */
int orc_ibs(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
            uint64_t *total, uint64_t *wedges, int *start_layer);

/* Definition 3 (priority) with global ids gid(v ∈ L) = v, gid(u ∈ U) = l + u,
 * and Definition 4 (projection): rank_u[u] ∈ [0, r), rank_l[v] ∈ [0, l) are
 * the per-layer ranks of the priority, 0 = lowest.  prio[n] (optional, may be
 * NULL) receives p(x) ∈ [1, n] indexed by gid. */
int orc_priority(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                 int32_t *rank_u, int32_t *rank_l, int32_t *prio);

/* The projection graph G* (Definition 4) with every neighbour list sorted
 * ascending by priority, in the unified id space of G*: L vertex v has id
 * rank_l[v], U vertex u has id l + rank_u[u].  Outputs (n = r + l):
 *   poff[n+1] (int64), padj[2m], peid[2m] (U-side slot of each entry),
 *   cut[n]  = |{y ∈ N(x) : p(y) < p(x)}|,
 *   work[n] = |{(y, z) : y ∈ N(x), p(y) < p(x), z ∈ N(y), p(z) < p(x)}|,
 *             the wedges Algorithm 2 processes from start x. */
int orc_projection(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                   int64_t *poff, int32_t *padj, int32_t *peid, int32_t *cut,
                   uint64_t *work);

/* Algorithm 2 (BFC-VP), run in parallel as Algorithm 5 prescribes: starts in
 * non-ascending priority, handed dynamically to `threads` workers (OpenMP),
 * each with its own dense count_wedge array and partial sum.
 *   total  : ⋈_G
 *   wedges : processed wedges (may be NULL)
 *   pv_u/pv_l (may be NULL): per-vertex counts; pe (may be NULL): per-edge
 *            counts in U-side slot order.  These take a second walk over the
 *            same wedges, reading the final count_wedge of each end vertex.
 * threads <= 0 uses the OpenMP default. */
int orc_vp(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, int threads,
           uint64_t *total, uint64_t *wedges, uint64_t *pv_u, uint64_t *pv_l, uint64_t *pe);

/* Algorithm 3 (BFC-VP++): projection, neighbour lists in descending
 * priority, wedges whose end vertex has the highest priority, early break.
 * Single thread.  *wedges = processed wedges. */
int orc_vppp(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
             uint64_t *total, uint64_t *wedges);

/* Σ_{(u,v) ∈ E} min(deg u, deg v) (Lemma 3), Σ_U deg², Σ_L deg². */
int orc_degree_stats(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                     uint64_t *tc_new, uint64_t *sum_du2, uint64_t *sum_dl2);

/* Algorithm 2 with every start's END set cut into ranges of `chunk`
 * consecutive priorities, each range counted with its own counters (the
 * split of one heavy start over several workers that Section 6.2 leaves
 * open).  Every pair (u, w) falls in one range, so C(count, 2) is applied
 * to whole counts and the total equals Algorithm 2's.  Plain loops over
 * every range and every wedge: tiny graphs only. */
int orc_vp_chunked(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, int32_t chunk,
                   uint64_t *total);

/* Algorithm 2 with the top-K priority vertices (the "core", both layers)
 * split off, as a dense-core hybrid would count them.  For a start u and an
 * end w that are both in the core, c_uw = a_uw + b_uw with a_uw the middles
 * in the core and b_uw the others, and
 *     C(a + b, 2) = C(b, 2) + a·b + C(a, 2)          (Lemma 1 per pair).
 * The walk skips every wedge whose start, middle and end all lie in the core
 * (C(b, 2) and the other pairs by the running form); a_uw is counted apart
 * by its definition and the pair adds a·b + C(a, 2).  *total = ⋈_G for every
 * K; *core_wedges = the wedges skipped; *core_c2 = Σ C(a_uw, 2) (the part a
 * dense product over the core would give); *core_cross = Σ a_uw·b_uw.
 * Plain loops: small graphs. */
int orc_vp_core_split(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, int32_t K,
                      uint64_t *total, uint64_t *core_wedges, uint64_t *core_c2, uint64_t *core_cross);

/* Section 6.3's pair formulation (BFC-EM), in memory: for every middle v,
 * each wedge (u, v, w) with p(w) > p(v) and p(w) > p(u) is written as the
 * pair (w, u); the pairs are sorted and every run of c equal pairs gives
 * C(c, 2) butterflies (Lemma 1).  *pairs = pairs written (= W, Lemma 4).
 * Holds all pairs in memory: small graphs only. */
int orc_pairs_total(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                    uint64_t *total, uint64_t *pairs);

/* Caterpillars (three-paths) of Section 1's bipartite clustering coefficient
 * 4·⋈_G / caterpillars: a three-path a-b-c-d is fixed by its middle edge
 * (b, c) and a choice of a in N(b) \ {c} and d in N(c) \ {b}, so the count is
 * Σ_{(u,v) ∈ E} (deg u − 1)(deg v − 1). */
int orc_caterpillars(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                     uint64_t *caterpillars);

/* SplitMix64 (Steele, Lea and Flood, "Fast Splittable Pseudorandom Number
 * Generators", OOPSLA 2014): the k-th output (k >= 1) of the generator seeded
 * with `seed`, i.e. its mixing function applied to seed + k * 0x9E3779B97F4A7C15. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k);

/* Edge sparsification for approximate counting (Section 7: the exact counter
 * is the inner block of a sampling estimator; each sample is a graph in which
 * every edge is kept independently with probability p).  Sample j keeps the
 * edge at U-side slot e iff orc_splitmix64(seed, j*m + e + 1) < threshold,
 * threshold = floor(p * 2^64) given by the caller; keep_all = 1 keeps every
 * edge (p = 1).  Writes the kept edges as a CSR over the same vertex sets:
 * out_off[r+1], out_adj[m] (caller-owned; slots beyond *kept untouched),
 * *kept = edges kept. */
int orc_sparsify(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, uint64_t seed,
                 uint64_t j, uint64_t threshold, int keep_all, int32_t *out_off, int32_t *out_adj,
                 int64_t *kept);

#ifdef __cplusplus
}
#endif
#endif
