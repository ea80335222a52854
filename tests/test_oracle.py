"""Pins for the CPU oracle: closed forms, the paper's worked examples,
exhaustive enumeration on tiny graphs, and the identities the paper states.

Nothing here touches a GPU.  Each pin is chosen so that a plausible slip in
the oracle (a dropped term, a wrong comparison, a transposed layer, a wrong
tie-break) makes at least one test fail.
"""
import hashlib
import json
import math
import os

import numpy as np
import pytest

import oracle
from bfc_inputs import generators as G

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def c2(x):
    return x * (x - 1) // 2


# ---------------------------------------------------------------------------
# the input generator itself
# ---------------------------------------------------------------------------

def test_splitmix64_published_vector():
    # SplitMix64 from state 0: first output 0xE220A8397B1DCDAF (Steele et al.)
    out = G.splitmix64_np(np.array([0], dtype=np.uint64), 0)
    assert int(out[0]) == 0xE220A8397B1DCDAF


def test_generators_numpy_torch_agree():
    torch = pytest.importorskip("torch")
    a = G.splitmix64_np(np.arange(4096, dtype=np.uint64), 99)
    b = G.splitmix64_torch(torch.arange(4096), 99).numpy().view(np.uint64)
    assert np.array_equal(a, b)
    g1 = G.chung_lu_bipartite(3000, 2000, 20000, 2.1, 1.9, 5)
    g2 = G.chung_lu_bipartite(3000, 2000, 20000, 2.1, 1.9, 5, device="cpu")
    assert np.array_equal(g1.off_u, g2.off_u) and np.array_equal(g1.adj_u, g2.adj_u)


def test_generator_shape_and_simplicity():
    g = G.uniform_small()
    assert (g.num_u, g.num_l, g.num_edges) == (2000, 3000, 20000)
    u, v = g.edges()
    assert np.unique(u * g.num_l + v).size == g.num_edges
    h = G.chung_lu_bipartite(5000, 3000, 40000, 2.1, 2.1, 3)
    assert h.num_edges == 40000
    u, v = h.edges()
    assert np.unique(u * h.num_l + v).size == h.num_edges
    assert v.max() < h.num_l and u.max() < h.num_u


def test_uniform_small_golden_graph():
    gold = json.load(open(os.path.join(GOLDEN, "uniform_small.json")))
    g = G.uniform_small()
    assert hashlib.sha256(g.adj_u.tobytes()).hexdigest() == gold["graph"]["adj_sha256"]
    assert hashlib.sha256(g.off_u.tobytes()).hexdigest() == gold["graph"]["off_sha256"]


# ---------------------------------------------------------------------------
# closed forms (Definition 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("a,b", [(2, 2), (3, 5), (5, 3), (4, 4), (1, 7), (6, 2), (7, 9)])
def test_complete_bipartite(a, b):
    g = G.complete_bipartite(a, b)
    tot = c2(a) * c2(b)
    r = oracle.vp(g, vertices=True, edges=True)
    assert r["total"] == tot
    assert oracle.brute_total(g, 0) == tot and oracle.brute_total(g, 1) == tot
    assert oracle.ibs(g)[0] == tot
    assert oracle.vppp(g)[0] == tot
    assert np.all(r["pv_u"] == (a - 1) * c2(b))
    assert np.all(r["pv_l"] == (b - 1) * c2(a))
    assert np.all(r["pe"] == (a - 1) * (b - 1))
    # processed wedges: the layer X holding the higher-priority vertices has
    # x vertices of degree y; W = y * C(x, 2).  U wins ties (U ids > L ids).
    if b >= a:     # U vertices have degree b >= a = degree of L vertices
        x, y = a, b
    else:
        x, y = b, a
    assert r["wedges"] == y * c2(x)
    assert oracle.vppp(g)[1] == y * c2(x)


@pytest.mark.parametrize("p,c,n", [(5, 13, 60), (7, 40, 300), (11, 100, 700), (13, 7, 90)])
def test_circulant_closed_form(p, c, n):
    # U vertex x is joined to L vertex x + s (mod n) for s in a shift set S.
    # Two U vertices at distance d share cnt(d) = #{(s, s') : s - s' = d mod n}
    # neighbours, so ⋈ = (n / 2) * sum_{d != 0} C(cnt(d), 2) (each unordered
    # pair is seen at d and at -d), and by rotation every vertex of either
    # layer lies in 2 ⋈ / n butterflies.
    g = G.shifted_sidon_circulant(p, c, n)
    t = [2 * p * k + (k * k) % p for k in range(p)]
    shifts = sorted({x % n for x in t} | {(x + c) % n for x in t})
    cnt = [0] * n
    for a in shifts:
        for b in shifts:
            cnt[(a - b) % n] += 1
    tot = n * sum(c2(k) for k in cnt[1:]) // 2
    r = oracle.vp(g, vertices=True, edges=True)
    assert r["total"] == tot and tot > 0
    assert np.all(r["pv_u"] == 2 * tot // n) and np.all(r["pv_l"] == 2 * tot // n)
    assert int(r["pe"].sum()) == 4 * tot
    assert oracle.vppp(g)[0] == tot


# ---------------------------------------------------------------------------
# Splitting one start over several workers: only the end set may be split
# ---------------------------------------------------------------------------

def _middle_split_total(g):
    """Algorithm 2 with each start's MIDDLES cut in two halves counted apart:
    a pair whose middles fall in both halves gets C(a, 2) + C(b, 2) instead
    of C(a + b, 2), so this undercounts (C is superadditive)."""
    pr = oracle.projection(g)
    off, adj, cut = pr["off"], pr["adj"], pr["cut"]
    t = 0
    for x in range(g.num_u + g.num_l):
        mids = adj[off[x]:off[x] + cut[x]]
        for half in (mids[:len(mids) // 2], mids[len(mids) // 2:]):
            cnt = {}
            for v in half:
                for w in adj[off[v]:off[v + 1]]:
                    if w < x:   # same layer as x: a lower G* id is a lower priority
                        cnt[w] = cnt.get(w, 0) + 1
            t += sum(c2(c) for c in cnt.values())
    return t


@pytest.mark.parametrize("gi", range(5))
def test_end_range_split_is_exact(gi):
    g = [G.complete_bipartite(3, 3), G.complete_bipartite(5, 7), G.chung_lu_bipartite(80, 60, 700, 2.1, 2.1, 9),
         G.uniform_bipartite(60, 40, 500, 3), G.random_tiny(9, 8, 3, 6, 17)][gi]
    ref = oracle.vp(g)["total"]
    n = g.num_u + g.num_l
    for chunk in (1, 2, 3, 7, n):
        assert oracle.vp_chunked(g, chunk) == ref
    # the other split (of the middles) is not exact wherever a pair has
    # middles in both halves, e.g. every pair of K_{3,3} and K_{5,7}
    wrong = _middle_split_total(g)
    assert wrong <= ref
    if gi < 2:
        assert wrong < ref


def test_chunked_rejects_bad_width():
    with pytest.raises(ValueError):
        oracle.vp_chunked(G.complete_bipartite(2, 2), 0)


# ---------------------------------------------------------------------------
# A dense core counted apart: the top-K priority vertices
# ---------------------------------------------------------------------------

def _core_blocks(g, K):
    """Per start layer X: the core's 0/1 adjacency A[i, j] (core vertices of X
    and of the other layer Y, each sorted by priority) and t[i] = the number
    of Y's core vertices below x_i, i.e. x_i's middles are y_j with j < t[i]
    (t is non-decreasing in i)."""
    _, _, p = oracle.priority(g)
    l, n = g.num_l, g.num_u + g.num_l
    core = p > n - K
    u = np.repeat(np.arange(g.num_u), np.diff(g.off_u.astype(np.int64))) + l
    v = g.adj_u.astype(np.int64)
    out = []
    for xs_layer, ys_layer in ((np.arange(l, n), np.arange(0, l)), (np.arange(0, l), np.arange(l, n))):
        xs = xs_layer[core[xs_layer]]
        ys = ys_layer[core[ys_layer]]
        if xs.size == 0 or ys.size == 0:
            continue
        xs = xs[np.argsort(p[xs])]
        ys = ys[np.argsort(p[ys])]
        xi = np.full(n, -1); xi[xs] = np.arange(xs.size)
        yi = np.full(n, -1); yi[ys] = np.arange(ys.size)
        A = np.zeros((xs.size, ys.size), dtype=np.int64)
        for a_end, b_end in ((u, v), (v, u)):
            m = (xi[a_end] >= 0) & (yi[b_end] >= 0)
            A[xi[a_end[m]], yi[b_end[m]]] = 1
        out.append((A, np.searchsorted(p[ys], p[xs])))
    return out


def _masked_core_gram(g, K):
    """The core part as a product of 0/1 matrices: row i of A masked to the
    middles below x_i, a[i, i'] = (masked A[i]) · A[i'] for the ends i' < i.
    Returns (Σ a, Σ C(a, 2))."""
    s1 = s2 = 0
    for A, t in _core_blocks(g, K):
        Am = A * (np.arange(A.shape[1])[None, :] < t[:, None])
        a = np.tril(Am @ A.T, k=-1)                 # ends below the start
        s1 += int(a.sum())
        s2 += int((a * (a - 1) // 2).sum())
    return s1, s2


def _tiled_core_pairs(A, t, tm, tj):
    """The same product as a tensor-core kernel would tile it: output tiles
    (I, I') with I' <= I only, accumulated over contraction blocks J below
    t[last row of I]; the per-row mask is applied only in the blocks that
    straddle t[first row of I] .. t[last row of I].  Returns (a, MACs)."""
    X, Y = A.shape
    acc = np.zeros((X, X), dtype=np.int64)
    macs = 0
    for i0 in range(0, X, tm):
        i1 = min(i0 + tm, X)
        tmin, tmax = int(t[i0]), int(t[i1 - 1])
        for j0 in range(0, tmax, tj):
            j1 = min(j0 + tj, Y)
            rows = A[i0:i1, j0:j1]
            if j1 > tmin:   # some row of the tile stops inside this block
                rows = rows * (np.arange(j0, j1)[None, :] < t[i0:i1, None])
            for k0 in range(0, i1, tm):
                k1 = min(k0 + tm, X)
                acc[i0:i1, k0:k1] += rows @ A[k0:k1, j0:j1].T
                macs += (i1 - i0) * (k1 - k0) * (j1 - j0)
    return np.tril(acc, k=-1), macs


def test_tiled_core_product_matches_the_core_split():
    g = G.chung_lu_bipartite(300, 200, 4000, 2.1, 2.1, 8)
    n = g.num_u + g.num_l
    for K in (n // 8, n // 3, n):
        tot, skipped, c2a, _ = oracle.vp_core_split(g, K)
        for tm, tj in ((4, 3), (8, 8), (16, 5)):
            s1 = s2 = 0
            macs = dense = 0
            for A, t in _core_blocks(g, K):
                assert np.all(np.diff(t) >= 0)
                a, m = _tiled_core_pairs(A, t, tm, tj)
                s1 += int(a.sum())
                s2 += int((a * (a - 1) // 2).sum())
                macs += m
                dense += A.shape[0] ** 2 * A.shape[1]
            assert (s1, s2) == (skipped, c2a), (K, tm, tj)
            assert macs <= dense


@pytest.mark.parametrize("gi", range(5))
def test_core_split_is_exact(gi):
    g = [G.complete_bipartite(4, 6), G.complete_bipartite(7, 5), G.chung_lu_bipartite(120, 80, 1200, 2.1, 2.1, 4),
         G.uniform_bipartite(60, 40, 500, 3), G.random_tiny(9, 8, 3, 6, 17)][gi]
    ref = oracle.vp(g)
    n = g.num_u + g.num_l
    for K in sorted({0, 1, 2, 7, n // 4, n // 2, n - 1, n}):
        tot, skipped, c2a, _ = oracle.vp_core_split(g, K)
        assert tot == ref["total"], K
        # the skipped wedges and the core's own pairs, from the matrix product
        assert (skipped, c2a) == _masked_core_gram(g, K), K
    assert oracle.vp_core_split(g, 0)[1:] == (0, 0, 0)
    tot, skipped, c2a, cross = oracle.vp_core_split(g, n)
    # the whole graph is the core: no middle outside it, the product gives all
    assert skipped == ref["wedges"] and c2a == ref["total"] and cross == 0


def test_core_split_cross_term_matters():
    # with a core strictly inside the graph some core pair has middles on both
    # sides, so a·b is needed: C(a, 2) + C(b, 2) alone falls short
    g = G.chung_lu_bipartite(120, 80, 1200, 2.1, 2.1, 4)
    n = g.num_u + g.num_l
    ref = oracle.vp(g)["total"]
    for K in (n // 8, n // 4, n // 2):
        tot, skipped, c2a, cross = oracle.vp_core_split(g, K)
        assert tot == ref and skipped > 0 and cross > 0
        assert tot - cross < ref


# ---------------------------------------------------------------------------
# Section 6.3's pair formulation: a second exact path by sorting wedge pairs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("gi", range(6))
def test_pair_formulation_agrees(gi):
    g = [G.complete_bipartite(4, 6), G.paper_fig3(), G.cycle(6), G.uniform_bipartite(300, 200, 3000, 11),
         G.chung_lu_bipartite(800, 500, 6000, 2.1, 2.1, 13), G.random_tiny(9, 7, 3, 5, 21)][gi]
    tot, pairs = oracle.pairs_total(g)
    r = oracle.vp(g)
    assert tot == r["total"] and pairs == r["wedges"]          # Lemma 1, Lemma 4
    if gi == 0:
        assert tot == c2(4) * c2(6)


# ---------------------------------------------------------------------------
# caterpillars (three-paths) of the clustering coefficient (Section 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("a,b", [(1, 1), (2, 2), (3, 4), (5, 2)])
def test_caterpillars_complete_bipartite(a, b):
    # every edge of K_{a,b} is the middle of (a-1)(b-1) three-paths; the
    # clustering coefficient 4·C(a,2)C(b,2) / (a b (a-1)(b-1)) is 1
    g = G.complete_bipartite(a, b)
    cat = oracle.caterpillars(g)
    assert cat == a * b * (a - 1) * (b - 1) == oracle.enumerate_three_paths(g)
    if cat:
        assert 4 * oracle.vp(g)["total"] == cat


def test_caterpillars_closed_forms():
    assert oracle.caterpillars(G.cycle(7)) == 14            # C_14: one per edge
    assert oracle.caterpillars(G.star(9)) == 0               # leaves end every path
    assert oracle.caterpillars(G.path(6)) == 4               # a path of 6 edges holds 4
    assert oracle.caterpillars(G.from_edges(3, 3, [], [])) == 0


@pytest.mark.parametrize("seed", range(12))
def test_caterpillars_against_enumeration(seed):
    g = G.random_tiny(4 + seed % 5, 3 + seed % 6, 2, 5, 100 + seed)
    assert oracle.caterpillars(g) == oracle.enumerate_three_paths(g)


@pytest.mark.parametrize("k", [3, 4, 5, 10])
def test_long_cycles_have_none(k):
    g = G.cycle(k)
    assert oracle.vp(g)["total"] == 0
    assert oracle.brute_total(g) == 0


def test_c4():
    g = G.cycle(2)
    r = oracle.vp(g, vertices=True, edges=True)
    assert r["total"] == 1
    assert np.all(r["pe"] == 1) and np.all(r["pv_u"] == 1) and np.all(r["pv_l"] == 1)


@pytest.mark.parametrize("seed", range(6))
def test_forests_stars_paths_have_none(seed):
    for g in [G.random_forest(30 + seed, 25, seed), G.star(17 + seed), G.star(9, False),
              G.path(11 + seed)]:
        r = oracle.vp(g, vertices=True, edges=True)
        assert r["total"] == 0
        assert r["pe"].sum() == 0 and r["pv_u"].sum() == 0 and r["pv_l"].sum() == 0
        assert oracle.ibs(g)[0] == 0 and oracle.vppp(g)[0] == 0


def test_empty_and_isolated():
    g = G.from_edges(5, 4, [], [])
    assert oracle.vp(g)["total"] == 0 and oracle.vp(g)["wedges"] == 0
    h = G.from_edges(6, 6, [0, 0, 1, 1], [0, 1, 0, 1])   # C4 plus isolated vertices
    assert oracle.vp(h)["total"] == 1
    assert oracle.brute_total(h) == 1


def test_disjoint_union_is_additive():
    a = G.complete_bipartite(4, 3)
    b = G.uniform_bipartite(60, 50, 500, 3)
    u = G.disjoint_union(a, b)
    assert oracle.vp(u)["total"] == oracle.vp(a)["total"] + oracle.vp(b)["total"]


# ---------------------------------------------------------------------------
# the paper's worked examples
# ---------------------------------------------------------------------------

def test_paper_examples():
    gold = json.load(open(os.path.join(GOLDEN, "paper_examples.json")))
    for name, g in [("paper_fig2a", G.paper_fig2a()), ("paper_fig3", G.paper_fig3())]:
        exp = gold[name]
        r = oracle.vp(g)
        assert r["wedges"] == exp["vp_wedges"]["value"], name
        assert r["total"] == exp["total"]["value"], name
        t, w, _ = oracle.ibs(g)
        assert w == exp["ibs_wedges"]["value"], name
        assert t == exp["total"]["value"]
        assert oracle.vppp(g) == (exp["total"]["value"], exp["vp_wedges"]["value"])
        assert oracle.brute_total(g, 0) == exp["total"]["value"]


def test_paper_fig3_priority_order():
    gold = json.load(open(os.path.join(GOLDEN, "paper_examples.json")))["paper_fig3"]
    g = G.paper_fig3()
    ru, rl, p = oracle.priority(g)
    l = g.num_l

    def gid(name):
        return (l + int(name[1:])) if name[0] == "u" else int(name[1:])

    n = g.num_u + g.num_l
    top = [gid(x) for x in gold["priority_top"]["value"]]
    assert [p[x] for x in top] == list(range(n, n - len(top), -1))
    bottom = [gid(x) for x in gold["priority_bottom"]["value"]]
    assert [p[x] for x in bottom] == [2, 1]
    # per-layer ranks agree with p
    assert ru[1] == g.num_u - 1 and ru[0] == g.num_u - 2
    assert rl[1001] == l - 1 and rl[1000] == l - 2 and rl[0] == 0


# ---------------------------------------------------------------------------
# exhaustive enumeration on tiny graphs (Definition 2 taken literally)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(120))
def test_tiny_graphs_against_enumeration(seed):
    r_ = 2 + seed % 6
    l_ = 2 + (seed // 6) % 6
    pnum = 1 + seed % 4
    g = G.random_tiny(r_, l_, pnum, 5, seed)
    ref = oracle.enumerate_butterflies(g)
    vp = oracle.vp(g, threads=1, vertices=True, edges=True)
    assert vp["total"] == ref["total"]
    assert np.array_equal(vp["pv_u"], ref["pv_u"]) and np.array_equal(vp["pv_l"], ref["pv_l"])
    assert np.array_equal(vp["pe"], ref["pe"])
    assert oracle.brute_total(g, 0) == ref["total"] == oracle.brute_total(g, 1)
    bu, bl = oracle.brute_vertices(g)
    assert np.array_equal(bu, ref["pv_u"]) and np.array_equal(bl, ref["pv_l"])
    assert np.array_equal(oracle.brute_edges(g), ref["pe"])
    assert oracle.ibs(g)[0] == ref["total"]
    assert oracle.vppp(g)[0] == ref["total"]
    # the sampled forms of Eq. 1 and Eq. 7 for every vertex and edge
    assert np.array_equal(oracle.vertices_sampled(g, 0, np.arange(g.num_u)), ref["pv_u"])
    assert np.array_equal(oracle.vertices_sampled(g, 1, np.arange(g.num_l)), ref["pv_l"])
    assert np.array_equal(oracle.edges_sampled(g, np.arange(g.num_edges)), ref["pe"])


@pytest.mark.parametrize("a,b", [(2, 2), (3, 5), (6, 4)])
def test_sampled_closed_forms(a, b):
    g = G.complete_bipartite(a, b)
    assert np.all(oracle.vertices_sampled(g, 0, np.arange(a)) == (a - 1) * c2(b))
    assert np.all(oracle.vertices_sampled(g, 1, np.arange(b)) == (b - 1) * c2(a))
    assert np.all(oracle.edges_sampled(g, np.arange(a * b)) == (a - 1) * (b - 1))
    # any order, repeats allowed
    assert list(oracle.vertices_sampled(g, 1, [b - 1, 0, b - 1])) == [(b - 1) * c2(a)] * 3
    with pytest.raises(ValueError):
        oracle.vertices_sampled(g, 0, [a])
    with pytest.raises(ValueError):
        oracle.edges_sampled(g, [a * b])


def test_sampled_on_larger_graph_agrees_with_full_oracle():
    g = G.chung_lu_bipartite(3000, 1500, 40000, 2.1, 2.1, 16)
    ref = oracle.vp(g, vertices=True, edges=True)
    xs = np.arange(0, g.num_u, 7)
    ys = np.arange(0, g.num_l, 5)
    es = np.arange(0, g.num_edges, 13)
    assert np.array_equal(oracle.vertices_sampled(g, 0, xs), ref["pv_u"][xs])
    assert np.array_equal(oracle.vertices_sampled(g, 1, ys), ref["pv_l"][ys])
    assert np.array_equal(oracle.edges_sampled(g, es), ref["pe"][es])


# ---------------------------------------------------------------------------
# identities on larger random graphs
# ---------------------------------------------------------------------------

def _graphs():
    return [G.uniform_bipartite(300, 200, 3000, 11), G.uniform_bipartite(50, 400, 2500, 12),
            G.chung_lu_bipartite(800, 500, 6000, 2.1, 2.1, 13),
            G.chung_lu_bipartite(1500, 100, 8000, 2.5, 1.8, 14, max_l=600),
            G.chung_lu_bipartite(400, 900, 5000, 1.9, 2.4, 15)]


@pytest.mark.parametrize("gi", range(5))
def test_identities(gi):
    g = _graphs()[gi]
    r = oracle.vp(g, threads=2, vertices=True, edges=True)
    B = r["total"]
    # Lemma 1, Eq. 2: Σ_U ⋈_u = Σ_L ⋈_v = 2 ⋈_G
    assert int(r["pv_u"].sum()) == 2 * B == int(r["pv_l"].sum())
    # every butterfly has four edges
    assert int(r["pe"].sum()) == 4 * B
    # every butterfly through x uses two of x's edges: Σ_{e ∋ x} ⋈_e = 2 ⋈_x
    u, v = g.edges()
    su = np.bincount(u, weights=r["pe"].astype(np.float64), minlength=g.num_u)
    sl = np.bincount(v, weights=r["pe"].astype(np.float64), minlength=g.num_l)
    assert np.array_equal(su.astype(np.uint64), 2 * r["pv_u"])
    assert np.array_equal(sl.astype(np.uint64), 2 * r["pv_l"])
    # Theorems 1 and 4 / Lemma 4: all orders agree, VP and VP++ process the same wedges
    assert oracle.ibs(g)[0] == B == oracle.brute_total(g, 0) == oracle.brute_total(g, 1)
    t3, w3 = oracle.vppp(g)
    assert t3 == B and w3 == r["wedges"]
    # Lemma 3: W <= Σ_E min(deg) <= min(Σ_U deg², Σ_L deg²)
    tc, du2, dl2 = oracle.degree_stats(g)
    assert r["wedges"] <= tc <= min(du2, dl2)
    # the definitions per vertex / per edge
    bu, bl = oracle.brute_vertices(g)
    assert np.array_equal(bu, r["pv_u"]) and np.array_equal(bl, r["pv_l"])
    assert np.array_equal(oracle.brute_edges(g), r["pe"])


@pytest.mark.parametrize("a,b", [(1, 1), (1, 6), (3, 7), (6, 4), (5, 5)])
def test_degree_stats_closed_forms_complete_bipartite(a, b):
    # K_{a,b}: every U vertex has degree b, every L vertex degree a, so each of
    # the a·b edges has min(deg) = min(a, b); Σ_U deg² = a·b², Σ_L deg² = b·a²
    tc, du2, dl2 = oracle.degree_stats(G.complete_bipartite(a, b))
    assert tc == a * b * min(a, b)
    assert du2 == a * b * b and dl2 == b * a * a


def test_degree_stats_closed_forms_sparse_shapes():
    # star with k leaves, centre in U: every edge has min(deg) = 1
    k = 9
    assert oracle.degree_stats(G.star(k)) == (k, k * k, k)
    assert oracle.degree_stats(G.star(k, center_in_u=False)) == (k, k, k * k)
    # C_{2k}: every vertex has degree 2
    for k in (2, 3, 8):
        assert oracle.degree_stats(G.cycle(k)) == (4 * k, 4 * k, 4 * k)
    # path with e >= 2 edges: the two end edges have min(deg) = 1, the rest 2;
    # U holds the even path positions (degrees 1, 2, ..., ending in 1 or 2)
    for e in (2, 5, 8):
        tc, du2, dl2 = oracle.degree_stats(G.path(e))
        assert tc == 2 + 2 * (e - 2)
        degs = [1] + [2] * (e - 1) + [1]     # degree of path position 0..e
        assert du2 == sum(d * d for d in degs[0::2]) and dl2 == sum(d * d for d in degs[1::2])
    # disjoint unions add
    a, b = G.complete_bipartite(3, 7), G.cycle(4)
    sa, sb = oracle.degree_stats(a), oracle.degree_stats(b)
    assert oracle.degree_stats(G.disjoint_union(a, b)) == tuple(x + y for x, y in zip(sa, sb))


@pytest.mark.parametrize("gi", range(5))
def test_relabel_and_list_order_invariance(gi):
    g = _graphs()[gi]
    B = oracle.vp(g)["total"]
    assert oracle.vp(G.relabel(g, 5 + gi))["total"] == B
    s = G.shuffle_lists(g, 9 + gi)
    rs = oracle.vp(s, edges=True)
    assert rs["total"] == B
    # per-edge counts follow their edges through the shuffle
    r0 = oracle.vp(g, edges=True)
    u0, v0 = g.edges()
    us, vs = s.edges()
    k0 = dict(zip(zip(u0.tolist(), v0.tolist()), r0["pe"].tolist()))
    assert all(k0[(a, b)] == c for a, b, c in zip(us.tolist(), vs.tolist(), rs["pe"].tolist()))


def test_thread_count_invariance():
    g = G.chung_lu_bipartite(3000, 2000, 30000, 2.1, 2.1, 21)
    a = oracle.vp(g, threads=1, vertices=True, edges=True)
    b = oracle.vp(g, threads=4, vertices=True, edges=True)
    assert a["total"] == b["total"] and a["wedges"] == b["wedges"]
    assert np.array_equal(a["pe"], b["pe"]) and np.array_equal(a["pv_u"], b["pv_u"])


def test_uniform_small_golden_values():
    gold = json.load(open(os.path.join(GOLDEN, "uniform_small.json")))
    g = G.uniform_small()
    r = oracle.vp(g, threads=2, vertices=True, edges=True)
    assert r["total"] == gold["total"] == gold["brute_total"] == gold["ibs_total"]
    assert r["wedges"] == gold["vp_wedges"]
    assert hashlib.sha256(r["pe"].tobytes()).hexdigest() == gold["pe_sha256"]
    assert hashlib.sha256(r["pv_u"].tobytes()).hexdigest() == gold["pv_u_sha256"]


# ---------------------------------------------------------------------------
# Definition 3 / Definition 4 and the per-start work (used by the GPU's
# prepare parity tests)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("gi", range(5))
def test_priority_and_projection(gi):
    g = _graphs()[gi]
    ru, rl, p = oracle.priority(g)
    l, r = g.num_l, g.num_u
    n = l + r
    u, v = g.edges()
    deg = np.concatenate([np.bincount(v, minlength=l), np.diff(g.off_u.astype(np.int64))])
    # p sorts gids by (deg, gid): check against numpy's lexsort
    order = np.lexsort((np.arange(n), deg))
    assert np.array_equal(p[order], np.arange(1, n + 1))
    assert sorted(ru.tolist()) == list(range(r)) and sorted(rl.tolist()) == list(range(l))
    P = oracle.projection(g)
    # structure preserved: mapping G* back gives the edge set of G
    star_u, star_l = l + ru, rl
    pairs_star = set()
    for x in range(n):
        for y in P["adj"][P["off"][x]:P["off"][x + 1]]:
            pairs_star.add((x, int(y)))
    pairs = {(int(star_u[a]), int(star_l[b])) for a, b in zip(u, v)}
    assert pairs | {(b, a) for a, b in pairs} == pairs_star
    # every list ascending; eid points back at the edge
    for x in range(n):
        seg = P["adj"][P["off"][x]:P["off"][x + 1]]
        assert np.all(np.diff(seg) > 0)
    for k in range(0, 2 * g.num_edges, 7):
        x = int(np.searchsorted(P["off"], k, side="right") - 1)
        y = int(P["adj"][k])
        e = int(P["eid"][k])
        uu, vv = (x, y) if x >= l else (y, x)
        assert star_u[u[e]] == uu and star_l[v[e]] == vv
    # Σ work = processed wedges of Algorithm 2
    assert int(P["work"].sum()) == oracle.vp(g)["wedges"]
    assert int(P["cut"].sum()) == g.num_edges   # every edge oriented exactly once


def test_malformed_inputs_rejected():
    g = G.complete_bipartite(3, 3)
    bad = G.BipartiteCSR(3, 3, g.off_u.copy(), g.adj_u.copy())
    bad.adj_u[4] = bad.adj_u[3]       # duplicate edge
    with pytest.raises(ValueError):
        oracle.vp(bad)
    bad2 = G.BipartiteCSR(3, 3, g.off_u.copy(), g.adj_u.copy())
    bad2.adj_u[0] = 7                 # id out of range
    with pytest.raises(ValueError):
        oracle.vp(bad2)
    bad3 = G.BipartiteCSR(3, 3, g.off_u[::-1].copy(), g.adj_u.copy())
    with pytest.raises(ValueError):
        oracle.vp(bad3)
