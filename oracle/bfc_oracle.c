/*
 * CPU oracle for exact butterfly counting — plain, slow, written to be read
 * against the paper (Wang et al., "Efficient Butterfly Counting for Large
 * Bipartite Networks").
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline arm, never by the product path.  It shares no code
 * with the CUDA library.
 *
 * Conventions (Section 2): G(U, L, E) is given by its U-side CSR.  Vertex
 * ids are 0-based per layer; where the paper needs one id space (the
 * tie-break of Definition 3) we use gid(v ∈ L) = v and gid(u ∈ U) = l + u,
 * so that every U id exceeds every L id as Section 2 assumes and as the
 * projection of Definition 4 lays them out.
 */
#include "bfc_oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static uint64_t choose2(uint64_t c) { return c < 2 ? 0 : c * (c - 1) / 2; }

/* ------------------------------------------------------------------------- */
/* Graph in the gid space: both layers, adjacency sorted by gid.            */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t r, l, n;
    int64_t m;
    int64_t *off;   /* [n+1] over gids */
    int32_t *adj;   /* [2m] neighbour gids, ascending */
    int64_t *eid;   /* [2m] U-side slot of the edge */
    int32_t *deg;   /* [n] */
} graph_t;

static void graph_free(graph_t *g) {
    free(g->off); free(g->adj); free(g->eid); free(g->deg);
    memset(g, 0, sizeof(*g));
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Build the gid-space graph; validates the input (offsets, ids, duplicates). */
static int graph_build(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, graph_t *g) {
    memset(g, 0, sizeof(*g));
    if (r < 0 || l < 0 || off == NULL) return -1;
    if (off[0] != 0) return -1;
    for (int32_t u = 0; u < r; ++u)
        if (off[u + 1] < off[u]) return -1;
    int64_t m = off[r];
    if (m > 0 && adj == NULL) return -1;
    for (int64_t k = 0; k < m; ++k)
        if (adj[k] < 0 || adj[k] >= l) return -1;
    g->r = r; g->l = l; g->n = r + l; g->m = m;
    int32_t n = g->n;
    g->off = calloc((size_t)n + 1, sizeof(int64_t));
    g->adj = malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->eid = malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    g->deg = calloc((size_t)n + 1, sizeof(int32_t));
    if (!g->off || !g->adj || !g->eid || !g->deg) { graph_free(g); return -2; }
    /* degrees: gid of L vertex v is v, of U vertex u is l + u */
    for (int32_t u = 0; u < r; ++u) g->deg[l + u] = off[u + 1] - off[u];
    for (int64_t k = 0; k < m; ++k) g->deg[adj[k]] += 1;
    for (int32_t x = 0; x < n; ++x) g->off[x + 1] = g->off[x] + g->deg[x];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!fill) { graph_free(g); return -2; }
    memcpy(fill, g->off, sizeof(int64_t) * (size_t)n);
    for (int32_t u = 0; u < r; ++u) {
        for (int64_t k = off[u]; k < off[u + 1]; ++k) {
            int32_t v = adj[k];
            int64_t a = fill[l + u]++;
            g->adj[a] = v; g->eid[a] = k;
            int64_t b = fill[v]++;
            g->adj[b] = l + u; g->eid[b] = k;
        }
    }
    free(fill);
    /* sort every list by gid (carry the edge id) and reject duplicates */
    int64_t maxd = 0;
    for (int32_t x = 0; x < n; ++x) if (g->deg[x] > maxd) maxd = g->deg[x];
    int64_t *tmp = malloc(sizeof(int64_t) * (size_t)(maxd + 1));
    if (!tmp) { graph_free(g); return -2; }
    for (int32_t x = 0; x < n; ++x) {
        int64_t b = g->off[x], d = g->deg[x];
        for (int64_t i = 0; i < d; ++i) tmp[i] = ((int64_t)g->adj[b + i] << 32) | (int64_t)g->eid[b + i];
        qsort(tmp, (size_t)d, sizeof(int64_t), cmp_i64);
        for (int64_t i = 0; i < d; ++i) {
            g->adj[b + i] = (int32_t)(tmp[i] >> 32);
            g->eid[b + i] = tmp[i] & 0xffffffffLL;
            if (i > 0 && g->adj[b + i] == g->adj[b + i - 1]) { free(tmp); graph_free(g); return -1; }
        }
    }
    free(tmp);
    return 0;
}

/* |N(x) ∩ N(y)| by merging two ascending lists. */
static uint64_t common(const graph_t *g, int32_t x, int32_t y) {
    int64_t i = g->off[x], ie = g->off[x + 1], j = g->off[y], je = g->off[y + 1];
    uint64_t c = 0;
    while (i < ie && j < je) {
        if (g->adj[i] < g->adj[j]) ++i;
        else if (g->adj[i] > g->adj[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

/* ------------------------------------------------------------------------- */
/* Definitions (Definition 2, Lemma 1, Eq. 7)                                */
/* ------------------------------------------------------------------------- */
int orc_brute_total(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                    int pair_layer, uint64_t *total) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    int32_t lo = pair_layer == 0 ? l : 0, hi = pair_layer == 0 ? l + r : l;
    uint64_t s = 0;
    for (int32_t x = lo; x < hi; ++x)
        for (int32_t y = x + 1; y < hi; ++y)
            s += choose2(common(&g, x, y));
    *total = s;
    graph_free(&g);
    return 0;
}

int orc_brute_vertices(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                       uint64_t *pv_u, uint64_t *pv_l) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    /* Eq. 1: ⋈_x = Σ_{y in x's layer, y != x} C(|N(x) ∩ N(y)|, 2) */
    for (int32_t u = 0; u < r; ++u) {
        uint64_t s = 0;
        for (int32_t w = 0; w < r; ++w)
            if (w != u) s += choose2(common(&g, l + u, l + w));
        pv_u[u] = s;
    }
    for (int32_t v = 0; v < l; ++v) {
        uint64_t s = 0;
        for (int32_t x = 0; x < l; ++x)
            if (x != v) s += choose2(common(&g, v, x));
        pv_l[v] = s;
    }
    graph_free(&g);
    return 0;
}

/* Checks of the U-side CSR and its transpose (L-side lists of U ids, in no
 * particular order) for the sampled counts. */
static int transpose_u_side(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                            int64_t **loff_out, int32_t **lu_out) {
    if (r < 0 || l < 0 || off == NULL || off[0] != 0) return -1;
    for (int32_t u = 0; u < r; ++u)
        if (off[u + 1] < off[u]) return -1;
    const int64_t m = off[r];
    if (m > 0 && adj == NULL) return -1;
    int64_t *loff = calloc((size_t)l + 1, sizeof(int64_t));
    int32_t *lu = malloc(sizeof(int32_t) * (size_t)(m + 1));
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)(l + 1));
    if (!loff || !lu || !fill) { free(loff); free(lu); free(fill); return -2; }
    for (int64_t e = 0; e < m; ++e) {
        if (adj[e] < 0 || adj[e] >= l) { free(loff); free(lu); free(fill); return -1; }
        loff[adj[e] + 1] += 1;
    }
    for (int32_t v = 0; v < l; ++v) loff[v + 1] += loff[v];
    memcpy(fill, loff, sizeof(int64_t) * (size_t)(l + 1));
    for (int32_t u = 0; u < r; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e) lu[fill[adj[e]]++] = u;
    free(fill);
    *loff_out = loff;
    *lu_out = lu;
    return 0;
}

int orc_vertices_sampled(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                         int layer, const int32_t *xs, int64_t k, uint64_t *out) {
    int64_t *loff;
    int32_t *lu;
    int rc = transpose_u_side(r, l, off, adj, &loff, &lu);
    if (rc) return rc;
    const int32_t nl = layer ? l : r;   /* size of x's layer */
    uint32_t *c = calloc((size_t)nl + 1, sizeof(uint32_t));
    int32_t *touched = malloc(sizeof(int32_t) * ((size_t)nl + 1));
    if (!c || !touched) { free(c); free(touched); free(loff); free(lu); return -2; }
    for (int64_t i = 0; i < k; ++i) {
        const int32_t x = xs[i];
        if (x < 0 || x >= nl) { rc = -1; break; }
        int32_t nt = 0;
        /* two-hop paths x - v - y: U side goes through off/adj then the
         * transpose, L side the other way round */
        const int64_t b = layer ? loff[x] : off[x], e = layer ? loff[x + 1] : off[x + 1];
        for (int64_t j = b; j < e; ++j) {
            const int32_t v = layer ? lu[j] : adj[j];
            const int64_t b2 = layer ? off[v] : loff[v], e2 = layer ? off[v + 1] : loff[v + 1];
            for (int64_t t = b2; t < e2; ++t) {
                const int32_t y = layer ? adj[t] : lu[t];
                if (y == x) continue;
                if (c[y]++ == 0) touched[nt++] = y;
            }
        }
        uint64_t sum = 0;
        for (int32_t t = 0; t < nt; ++t) { sum += choose2(c[touched[t]]); c[touched[t]] = 0; }
        out[i] = sum;
    }
    free(c); free(touched); free(loff); free(lu);
    return rc;
}

int orc_edges_sampled(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                      const int64_t *es, int64_t k, uint64_t *out) {
    int64_t *loff;
    int32_t *lu;
    int rc = transpose_u_side(r, l, off, adj, &loff, &lu);
    if (rc) return rc;
    const int64_t m = off[r];
    unsigned char *mark = calloc((size_t)l + 1, 1);
    if (!mark) { free(loff); free(lu); return -2; }
    for (int64_t i = 0; i < k; ++i) {
        const int64_t e = es[i];
        if (e < 0 || e >= m) { rc = -1; break; }
        /* owner u of slot e: the last u with off[u] <= e */
        int32_t lo = 0, hi = r;
        while (hi - lo > 1) {
            const int32_t mid = lo + (hi - lo) / 2;
            if (off[mid] <= e) lo = mid; else hi = mid;
        }
        const int32_t u = lo, v = adj[e];
        for (int64_t j = off[u]; j < off[u + 1]; ++j) mark[adj[j]] = 1;
        uint64_t sum = 0;
        for (int64_t j = loff[v]; j < loff[v + 1]; ++j) {
            const int32_t w = lu[j];
            if (w == u) continue;
            uint64_t cw = 0;   /* |N(u) ∩ N(w)|, at least 1 (v) */
            for (int64_t t = off[w]; t < off[w + 1]; ++t) cw += mark[adj[t]];
            sum += cw - 1;
        }
        for (int64_t j = off[u]; j < off[u + 1]; ++j) mark[adj[j]] = 0;
        out[i] = sum;
    }
    free(mark); free(loff); free(lu);
    return rc;
}

int orc_brute_edges(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, uint64_t *pe) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    /* Eq. 7: ⋈_(u,v) = Σ_{w ∈ N(v), w != u} (|N(u) ∩ N(w)| − 1) */
    for (int32_t u = 0; u < r; ++u) {
        for (int64_t k = off[u]; k < off[u + 1]; ++k) {
            int32_t v = adj[k];
            uint64_t s = 0;
            for (int64_t j = g.off[v]; j < g.off[v + 1]; ++j) {
                int32_t w = g.adj[j];
                if (w == l + u) continue;
                s += common(&g, l + u, w) - 1;
            }
            pe[k] = s;
        }
    }
    graph_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 (BFC-IBS)                                                     */
/* ------------------------------------------------------------------------- */
int orc_ibs(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
            uint64_t *total, uint64_t *wedges, int *start_layer) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    uint64_t su = 0, sl = 0;
    for (int32_t u = 0; u < r; ++u) su += (uint64_t)g.deg[l + u] * (uint64_t)g.deg[l + u];
    for (int32_t v = 0; v < l; ++v) sl += (uint64_t)g.deg[v] * (uint64_t)g.deg[v];
    /* S = U unless Σ_U deg² < Σ_L deg² */
    int layer = (su < sl) ? 1 : 0;
    int32_t lo = layer == 0 ? l : 0, hi = layer == 0 ? l + r : l;
    uint32_t *count_wedge = calloc((size_t)g.n + 1, sizeof(uint32_t));
    int32_t *touched = malloc(sizeof(int32_t) * ((size_t)g.n + 1));
    if (!count_wedge || !touched) { free(count_wedge); free(touched); graph_free(&g); return -2; }
    uint64_t btf = 0, wd = 0;
    for (int32_t u = lo; u < hi; ++u) {
        int64_t nt = 0;
        for (int64_t i = g.off[u]; i < g.off[u + 1]; ++i) {
            int32_t v = g.adj[i];
            for (int64_t j = g.off[v]; j < g.off[v + 1]; ++j) {
                int32_t w = g.adj[j];
                if (!(w > u)) continue;           /* w.id > u.id */
                if (count_wedge[w] == 0) touched[nt++] = w;
                count_wedge[w] += 1;
                ++wd;
            }
        }
        for (int64_t t = 0; t < nt; ++t) {
            int32_t w = touched[t];
            if (count_wedge[w] > 1) btf += choose2(count_wedge[w]);
            count_wedge[w] = 0;
        }
    }
    *total = btf;
    if (wedges) *wedges = wd;
    if (start_layer) *start_layer = layer;
    free(count_wedge); free(touched); graph_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Definition 3 (priority) and Definition 4 (projection)                     */
/* ------------------------------------------------------------------------- */

/* p[gid] ∈ [1, n]: sort gids by (deg, gid) ascending; position + 1. */
static int compute_priority(const graph_t *g, int32_t *p) {
    int32_t n = g->n;
    int64_t *key = malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!key) return -2;
    for (int32_t x = 0; x < n; ++x) key[x] = ((int64_t)g->deg[x] << 32) | (int64_t)x;
    qsort(key, (size_t)n, sizeof(int64_t), cmp_i64);
    for (int32_t i = 0; i < n; ++i) p[key[i] & 0xffffffffLL] = i + 1;
    free(key);
    return 0;
}

/* Per-layer rank of the priority (Definition 4): the number of vertices of
 * the same layer with lower priority. */
static void layer_ranks(const graph_t *g, const int32_t *p, int32_t *rank_u, int32_t *rank_l) {
    int32_t n = g->n, l = g->l;
    int32_t *by_p = malloc(sizeof(int32_t) * ((size_t)n + 2));
    for (int32_t x = 0; x < n; ++x) by_p[p[x]] = x;
    int32_t nu = 0, nl = 0;
    for (int32_t q = 1; q <= n; ++q) {
        int32_t x = by_p[q];
        if (x >= l) rank_u[x - l] = nu++;
        else rank_l[x] = nl++;
    }
    free(by_p);
}

int orc_priority(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                 int32_t *rank_u, int32_t *rank_l, int32_t *prio) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    int32_t *p = malloc(sizeof(int32_t) * ((size_t)g.n + 1));
    if (!p) { graph_free(&g); return -2; }
    compute_priority(&g, p);
    layer_ranks(&g, p, rank_u, rank_l);
    if (prio) memcpy(prio, p, sizeof(int32_t) * (size_t)g.n);
    free(p); graph_free(&g);
    return 0;
}

int orc_projection(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                   int64_t *poff, int32_t *padj, int32_t *peid, int32_t *cut, uint64_t *work) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    int32_t n = g.n;
    int32_t *p = malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *ru = malloc(sizeof(int32_t) * ((size_t)r + 1));
    int32_t *rl = malloc(sizeof(int32_t) * ((size_t)l + 1));
    int32_t *star = malloc(sizeof(int32_t) * ((size_t)n + 1)); /* gid -> id in G* */
    int32_t *inv = malloc(sizeof(int32_t) * ((size_t)n + 1));  /* id in G* -> gid */
    int64_t maxd = 1;
    for (int32_t x = 0; x < n; ++x) if (g.deg[x] > maxd) maxd = g.deg[x];
    int64_t *tmp = malloc(sizeof(int64_t) * (size_t)maxd);
    if (!p || !ru || !rl || !star || !inv || !tmp) { rc = -2; goto done; }
    compute_priority(&g, p);
    layer_ranks(&g, p, ru, rl);
    /* Definition 4: v* = rankL(v), u* = rankU(u) + l */
    for (int32_t v = 0; v < l; ++v) { star[v] = rl[v]; inv[rl[v]] = v; }
    for (int32_t u = 0; u < r; ++u) { star[l + u] = l + ru[u]; inv[l + ru[u]] = l + u; }
    poff[0] = 0;
    for (int32_t xs = 0; xs < n; ++xs) poff[xs + 1] = poff[xs] + g.deg[inv[xs]];
    for (int32_t xs = 0; xs < n; ++xs) {
        int32_t x = inv[xs];
        int64_t d = g.deg[x];
        /* neighbours of x sorted ascending by priority p */
        for (int64_t i = 0; i < d; ++i) {
            int32_t y = g.adj[g.off[x] + i];
            tmp[i] = ((int64_t)p[y] << 32) | (int64_t)i;
        }
        qsort(tmp, (size_t)d, sizeof(int64_t), cmp_i64);
        int32_t c = 0;
        for (int64_t i = 0; i < d; ++i) {
            int64_t src = g.off[x] + (tmp[i] & 0xffffffffLL);
            int32_t y = g.adj[src];
            padj[poff[xs] + i] = star[y];
            peid[poff[xs] + i] = (int32_t)g.eid[src];
            if (p[y] < p[x]) ++c;
        }
        cut[xs] = c;
    }
    /* work[x*] = wedges (x, y, z) with p(y) < p(x) and p(z) < p(x), counted directly */
    for (int32_t xs = 0; xs < n; ++xs) {
        int32_t x = inv[xs];
        uint64_t w = 0;
        for (int64_t i = g.off[x]; i < g.off[x + 1]; ++i) {
            int32_t y = g.adj[i];
            if (!(p[y] < p[x])) continue;
            for (int64_t j = g.off[y]; j < g.off[y + 1]; ++j)
                if (p[g.adj[j]] < p[x]) ++w;
        }
        work[xs] = w;
    }
done:
    free(p); free(ru); free(rl); free(star); free(inv); free(tmp); graph_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2 (BFC-VP), scheduled as Algorithm 5                            */
/* ------------------------------------------------------------------------- */
int orc_vp(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, int threads,
           uint64_t *total, uint64_t *wedges, uint64_t *pv_u, uint64_t *pv_l, uint64_t *pe) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    int32_t n = g.n;
    int32_t *p = malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *by_p = malloc(sizeof(int32_t) * ((size_t)n + 2));
    uint64_t *pv = (pv_u || pv_l) ? calloc((size_t)n + 1, sizeof(uint64_t)) : NULL;
    if (!p || !by_p || ((pv_u || pv_l) && !pv)) { free(p); free(by_p); free(pv); graph_free(&g); return -2; }
    compute_priority(&g, p);
    for (int32_t x = 0; x < n; ++x) by_p[p[x]] = x;
    /* sort N(x) ascending by priority (line 2 of Algorithm 2) */
    {
        int64_t maxd = 1;
        for (int32_t x = 0; x < n; ++x) if (g.deg[x] > maxd) maxd = g.deg[x];
        int64_t *tmp = malloc(sizeof(int64_t) * (size_t)maxd);
        int32_t *a2 = malloc(sizeof(int32_t) * (size_t)maxd);
        int64_t *e2 = malloc(sizeof(int64_t) * (size_t)maxd);
        for (int32_t x = 0; x < n; ++x) {
            int64_t b = g.off[x], d = g.deg[x];
            for (int64_t i = 0; i < d; ++i) tmp[i] = ((int64_t)p[g.adj[b + i]] << 32) | (int64_t)i;
            qsort(tmp, (size_t)d, sizeof(int64_t), cmp_i64);
            for (int64_t i = 0; i < d; ++i) {
                int64_t s = tmp[i] & 0xffffffffLL;
                a2[i] = g.adj[b + s]; e2[i] = g.eid[b + s];
            }
            memcpy(g.adj + b, a2, sizeof(int32_t) * (size_t)d);
            memcpy(g.eid + b, e2, sizeof(int64_t) * (size_t)d);
        }
        free(tmp); free(a2); free(e2);
    }
    const int need_walk2 = (pv != NULL) || (pe != NULL);
    if (pe) memset(pe, 0, sizeof(uint64_t) * (size_t)g.m);
    uint64_t btf = 0, wd = 0;
#ifdef _OPENMP
    if (threads <= 0) threads = omp_get_max_threads();
#else
    threads = 1;
#endif
#pragma omp parallel num_threads(threads) reduction(+ : btf, wd)
    {
        /* local_count_wedge of Algorithm 5: a dense array per thread */
        uint32_t *count_wedge = calloc((size_t)n + 1, sizeof(uint32_t));
        int32_t *touched = malloc(sizeof(int32_t) * ((size_t)n + 1));
#pragma omp for schedule(dynamic, 16)
        for (int32_t q = n; q >= 1; --q) {   /* non-ascending priority */
            int32_t u = by_p[q];
            int64_t nt = 0;
            for (int64_t i = g.off[u]; i < g.off[u + 1]; ++i) {
                int32_t v = g.adj[i];
                if (!(p[v] < p[u])) break;           /* sorted: the rest are higher */
                for (int64_t j = g.off[v]; j < g.off[v + 1]; ++j) {
                    int32_t w = g.adj[j];
                    if (!(p[w] < p[u])) break;
                    if (count_wedge[w] == 0) touched[nt++] = w;
                    count_wedge[w] += 1;
                    ++wd;
                }
            }
            uint64_t bu = 0;
            for (int64_t t = 0; t < nt; ++t) {
                int32_t w = touched[t];
                if (count_wedge[w] > 1) {
                    uint64_t c2 = choose2(count_wedge[w]);
                    bu += c2;
                    if (pv) {
#pragma omp atomic
                        pv[w] += c2;
                    }
                }
            }
            btf += bu;
            if (pv && bu) {
#pragma omp atomic
                pv[u] += bu;
            }
            if (need_walk2) {
                /* second walk (Algorithm 4 in the VP orientation): every wedge
                 * (u, v, w) lies in count_wedge(w) − 1 butterflies through the
                 * pair (u, w), which all contain the edges (u, v), (v, w) and
                 * the middle vertex v. */
                for (int64_t i = g.off[u]; i < g.off[u + 1]; ++i) {
                    int32_t v = g.adj[i];
                    if (!(p[v] < p[u])) break;
                    uint64_t sum = 0;
                    for (int64_t j = g.off[v]; j < g.off[v + 1]; ++j) {
                        int32_t w = g.adj[j];
                        if (!(p[w] < p[u])) break;
                        uint64_t delta = (uint64_t)count_wedge[w] - 1;
                        sum += delta;
                        if (pe && delta) {
#pragma omp atomic
                            pe[g.eid[j]] += delta;
                        }
                    }
                    if (sum) {
                        if (pe) {
#pragma omp atomic
                            pe[g.eid[i]] += sum;
                        }
                        if (pv) {
#pragma omp atomic
                            pv[v] += sum;
                        }
                    }
                }
            }
            for (int64_t t = 0; t < nt; ++t) count_wedge[touched[t]] = 0;
        }
        free(count_wedge); free(touched);
    }
    *total = btf;
    if (wedges) *wedges = wd;
    if (pv_u) for (int32_t u = 0; u < r; ++u) pv_u[u] = pv[l + u];
    if (pv_l) for (int32_t v = 0; v < l; ++v) pv_l[v] = pv[v];
    free(pv); free(p); free(by_p); graph_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 3 (BFC-VP++)                                                     */
/* ------------------------------------------------------------------------- */
int orc_vppp(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
             uint64_t *total, uint64_t *wedges) {
    int32_t n = r + l;
    int64_t m = off[r];
    int64_t *poff = malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *padj = malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int32_t *peid = malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int32_t *cut = malloc(sizeof(int32_t) * ((size_t)n + 1));
    uint64_t *work = malloc(sizeof(uint64_t) * ((size_t)n + 1));
    if (!poff || !padj || !peid || !cut || !work) { free(poff); free(padj); free(peid); free(cut); free(work); return -2; }
    /* line 2: G* = projection(G, f) */
    int rc = orc_projection(r, l, off, adj, poff, padj, peid, cut, work);
    if (rc) { free(poff); free(padj); free(peid); free(cut); free(work); return rc; }
    /* line 3: p on G* by Definition 3 (ids of G*: L first, then U) */
    graph_t gs;
    {
        /* degrees of G*, then priority by (deg, id*) */
        gs.n = n; gs.r = r; gs.l = l; gs.m = m;
        gs.deg = malloc(sizeof(int32_t) * ((size_t)n + 1));
        for (int32_t x = 0; x < n; ++x) gs.deg[x] = (int32_t)(poff[x + 1] - poff[x]);
        gs.off = poff; gs.adj = padj; gs.eid = NULL;
    }
    int32_t *p = malloc(sizeof(int32_t) * ((size_t)n + 1));
    compute_priority(&gs, p);
    /* line 4: N(x*) in descending priority (ascending lists reversed) */
    for (int32_t x = 0; x < n; ++x) {
        for (int64_t a = poff[x], b = poff[x + 1] - 1; a < b; ++a, --b) {
            int32_t t = padj[a]; padj[a] = padj[b]; padj[b] = t;
        }
    }
    uint32_t *count_wedge = calloc((size_t)n + 1, sizeof(uint32_t));
    int32_t *touched = malloc(sizeof(int32_t) * ((size_t)n + 1));
    uint64_t btf = 0, wd = 0;
    for (int32_t u = 0; u < n; ++u) {
        int64_t nt = 0;
        for (int64_t i = poff[u]; i < poff[u + 1]; ++i) {
            int32_t v = padj[i];
            for (int64_t j = poff[v]; j < poff[v + 1]; ++j) {
                int32_t w = padj[j];
                /* descending lists: stop at the first w with p(w) <= p(u) or
                 * p(w) <= p(v); all later w are lower still */
                if (!(p[w] > p[u]) || !(p[w] > p[v])) break;
                if (count_wedge[w] == 0) touched[nt++] = w;
                count_wedge[w] += 1;
                ++wd;
            }
        }
        for (int64_t t = 0; t < nt; ++t) {
            int32_t w = touched[t];
            if (count_wedge[w] > 1) btf += choose2(count_wedge[w]);
            count_wedge[w] = 0;
        }
    }
    *total = btf;
    if (wedges) *wedges = wd;
    free(count_wedge); free(touched); free(p); free(gs.deg);
    free(poff); free(padj); free(peid); free(cut); free(work);
    return 0;
}

int orc_degree_stats(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                     uint64_t *tc_new, uint64_t *sum_du2, uint64_t *sum_dl2) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    uint64_t tc = 0, su = 0, sl = 0;
    for (int32_t u = 0; u < r; ++u) {
        uint64_t du = (uint64_t)g.deg[l + u];
        su += du * du;
        for (int64_t k = off[u]; k < off[u + 1]; ++k) {
            uint64_t dv = (uint64_t)g.deg[adj[k]];
            tc += du < dv ? du : dv;
        }
    }
    for (int32_t v = 0; v < l; ++v) sl += (uint64_t)g.deg[v] * (uint64_t)g.deg[v];
    *tc_new = tc; *sum_du2 = su; *sum_dl2 = sl;
    graph_free(&g);
    return 0;
}

int orc_caterpillars(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                     uint64_t *caterpillars) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    uint64_t c = 0;
    for (int32_t u = 0; u < r; ++u) {
        const uint64_t du = (uint64_t)g.deg[l + u];
        for (int64_t k = off[u]; k < off[u + 1]; ++k) c += (du - 1) * ((uint64_t)g.deg[adj[k]] - 1);
    }
    *caterpillars = c;
    graph_free(&g);
    return 0;
}

static int cmp_u64(const void *a, const void *b) {
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

int orc_pairs_total(int32_t r, int32_t l, const int32_t *off, const int32_t *adj,
                    uint64_t *total, uint64_t *pairs) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    int32_t *p = malloc(sizeof(int32_t) * ((size_t)g.n + 1));
    if (!p) { graph_free(&g); return -2; }
    rc = compute_priority(&g, p);
    if (rc) { free(p); graph_free(&g); return rc; }
    /* first pass: how many pairs */
    uint64_t np = 0;
    for (int32_t v = 0; v < g.n; ++v)
        for (int64_t i = g.off[v]; i < g.off[v + 1]; ++i) {
            const int32_t w = g.adj[i];
            if (p[w] <= p[v]) continue;
            for (int64_t j = g.off[v]; j < g.off[v + 1]; ++j)
                if (p[g.adj[j]] < p[w]) ++np;
        }
    uint64_t *key = malloc(sizeof(uint64_t) * (size_t)(np + 1));
    if (!key) { free(p); graph_free(&g); return -2; }
    uint64_t k = 0;
    for (int32_t v = 0; v < g.n; ++v)
        for (int64_t i = g.off[v]; i < g.off[v + 1]; ++i) {
            const int32_t w = g.adj[i];
            if (p[w] <= p[v]) continue;
            for (int64_t j = g.off[v]; j < g.off[v + 1]; ++j) {
                const int32_t u = g.adj[j];
                if (p[u] < p[w]) key[k++] = ((uint64_t)(uint32_t)w << 32) | (uint32_t)u;
            }
        }
    qsort(key, (size_t)np, sizeof(uint64_t), cmp_u64);
    uint64_t t = 0, run = 0;
    for (uint64_t i = 0; i < np; ++i) {
        run = (i > 0 && key[i] == key[i - 1]) ? run + 1 : 1;
        t += run - 1;   /* Σ over a run of c pairs of 0 + 1 + ... + (c - 1) = C(c, 2) */
    }
    *total = t;
    *pairs = np;
    free(key); free(p); graph_free(&g);
    return 0;
}

int orc_vp_chunked(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, int32_t chunk,
                   uint64_t *total) {
    if (chunk < 1) return -1;
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    const int32_t n = g.n;
    int32_t *p = malloc(sizeof(int32_t) * ((size_t)n + 1));
    uint32_t *count_wedge = calloc((size_t)n + 1, sizeof(uint32_t));
    if (!p || !count_wedge) { free(p); free(count_wedge); graph_free(&g); return -2; }
    rc = compute_priority(&g, p);
    if (rc) { free(p); free(count_wedge); graph_free(&g); return rc; }
    uint64_t t = 0;
    for (int32_t u = 0; u < n; ++u) {
        /* ends of u have priorities 1 .. p(u) - 1: ranges [lo, lo + chunk) */
        for (int32_t lo = 1; lo < p[u]; lo += chunk) {
            const int32_t hi = lo + chunk;
            for (int64_t i = g.off[u]; i < g.off[u + 1]; ++i) {
                const int32_t v = g.adj[i];
                if (!(p[v] < p[u])) continue;
                for (int64_t j = g.off[v]; j < g.off[v + 1]; ++j) {
                    const int32_t w = g.adj[j];
                    if (p[w] < p[u] && p[w] >= lo && p[w] < hi) count_wedge[w] += 1;
                }
            }
            /* the range's pairs, then clear its counters */
            for (int32_t w = 0; w < n; ++w) {
                const uint64_t c = count_wedge[w];
                if (c > 1) t += c * (c - 1) / 2;
                count_wedge[w] = 0;
            }
        }
    }
    *total = t;
    free(p); free(count_wedge); graph_free(&g);
    return 0;
}

int orc_vp_core_split(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, int32_t K,
                      uint64_t *total, uint64_t *core_wedges, uint64_t *core_c2, uint64_t *core_cross) {
    if (K < 0) return -1;
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);
    if (rc) return rc;
    const int32_t n = g.n;
    int32_t *p = malloc(sizeof(int32_t) * ((size_t)n + 1));
    uint32_t *b = calloc((size_t)n + 1, sizeof(uint32_t));   /* count_wedge of the walk */
    uint32_t *a = calloc((size_t)n + 1, sizeof(uint32_t));   /* core middles per core end */
    if (!p || !a || !b) { free(p); free(a); free(b); graph_free(&g); return -2; }
    rc = compute_priority(&g, p);
    if (rc) { free(p); free(a); free(b); graph_free(&g); return rc; }
    uint64_t t = 0, skipped = 0, c2a = 0, cross = 0;
    for (int32_t u = 0; u < n; ++u) {
        const int cu = p[u] > n - K;
        for (int64_t i = g.off[u]; i < g.off[u + 1]; ++i) {
            const int32_t v = g.adj[i];
            if (!(p[v] < p[u])) continue;
            const int cv = p[v] > n - K;
            for (int64_t j = g.off[v]; j < g.off[v + 1]; ++j) {
                const int32_t w = g.adj[j];
                if (!(p[w] < p[u])) continue;
                if (cu && cv && p[w] > n - K) {
                    /* start, middle and end in the core: left to the core part */
                    ++skipped;
                    a[w] += 1;
                    continue;
                }
                t += b[w];       /* running form: Σ old = Σ C(b, 2) */
                b[w] += 1;
            }
        }
        /* the pairs (u, w) with both in the core: a·b + C(a, 2) */
        for (int32_t w = 0; w < n; ++w) {
            if (a[w]) {
                const uint64_t aw = a[w];
                t += aw * (uint64_t)b[w] + aw * (aw - 1) / 2;
                c2a += aw * (aw - 1) / 2;
                cross += aw * (uint64_t)b[w];
            }
            a[w] = 0;
            b[w] = 0;
        }
    }
    *total = t;
    *core_wedges = skipped;
    *core_c2 = c2a;
    *core_cross = cross;
    free(p); free(a); free(b); graph_free(&g);
    return 0;
}

uint64_t orc_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int orc_sparsify(int32_t r, int32_t l, const int32_t *off, const int32_t *adj, uint64_t seed,
                 uint64_t j, uint64_t threshold, int keep_all, int32_t *out_off, int32_t *out_adj,
                 int64_t *kept) {
    graph_t g;
    int rc = graph_build(r, l, off, adj, &g);   /* checks the CSR */
    if (rc) return rc;
    graph_free(&g);
    const uint64_t m = (uint64_t)off[r];
    int64_t k = 0;
    out_off[0] = 0;
    for (int32_t u = 0; u < r; ++u) {
        for (int32_t e = off[u]; e < off[u + 1]; ++e) {
            /* one draw per (sample, edge): the edge survives with probability p */
            if (keep_all || orc_splitmix64(seed, j * m + (uint64_t)e + 1) < threshold)
                out_adj[k++] = adj[e];
        }
        out_off[u + 1] = (int32_t)k;
    }
    *kept = k;
    return 0;
}
