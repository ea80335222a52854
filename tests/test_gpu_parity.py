"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work, so the bar is bit-exact everywhere: totals, per-vertex and
per-edge counts, and the intermediate arrays of steps a2-a4 (ranks, the
projection graph, cut, per-start work).
"""
import numpy as np
import pytest

import oracle
from bfc_inputs import generators as G

from gpu_path import run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def c2(x):
    return x * (x - 1) // 2


def _opts(**kw):
    from paper_1812_00283_gb300 import bfc
    return bfc.bfc_options_init(**kw)


# bins: default, everything dense, everything CTA-hash, everything warp-hash where allowed
BIN_SETTINGS = {
    "default": {},
    "all_dense": dict(warp_max_work=0, hash_max_work=0),
    "hash_only": dict(warp_max_work=0, team_max_work=0, hash_max_work=24576),
    "warp_heavy": dict(warp_max_work=256, hash_max_work=256),
    "team_small": dict(warp_max_work=32, team_max_work=512, hash_max_work=4096),
    # team tables may fill up: escalation to a CTA table in the retry pass
    "team_only": dict(warp_max_work=0, team_max_work=16384, hash_max_work=16384),
    "wide_positions": dict(wide_positions=1),
    "all_dense_wide_positions": dict(warp_max_work=0, hash_max_work=0, wide_positions=1),
    "team_only_wide_positions": dict(warp_max_work=0, team_max_work=16384, hash_max_work=16384,
                                     wide_positions=1),
    # Algorithm 3's orientation: team / CTA hash tables with the retry pass
    "vpp": dict(orientation=1),
    "vpp_retry_all": dict(orientation=1, warp_max_work=0, hash_max_work=0),
    "vpp_retry_beyond_warp": dict(orientation=1, warp_max_work=256, hash_max_work=0),
    "vpp_no_warp": dict(orientation=1, warp_max_work=0),
    "vpp_no_team": dict(orientation=1, team_max_work=0),
    "vpp_team_small": dict(orientation=1, team_max_work=2048),
    "vpp_wide_positions": dict(orientation=1, wide_positions=1),
}


def _check_against_oracle(g, opts=None, vertices=True, edges=True):
    ref = oracle.vp(g, vertices=vertices, edges=edges)
    got = run_gpu(g, vertices=vertices, edges=edges, options=opts)
    assert got["total"] == ref["total"]
    assert got["info"]["wedges"] == ref["wedges"]
    if vertices:
        assert got["total_v"] == ref["total"]
        assert np.array_equal(got["pv_u"], ref["pv_u"])
        assert np.array_equal(got["pv_l"], ref["pv_l"])
    if edges:
        assert got["total_e"] == ref["total"]
        assert np.array_equal(got["pe"], ref["pe"])
    if vertices and edges:
        assert got["total_all"] == ref["total"]
        assert np.array_equal(got["all_pv_u"], ref["pv_u"]) and np.array_equal(got["all_pv_l"], ref["pv_l"])
        assert np.array_equal(got["all_pe"], ref["pe"])
    return got, ref


# ---------------------------------------------------------------------------
# closed forms and the paper's examples
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("a,b", [(2, 2), (3, 5), (5, 3), (7, 7), (1, 9), (40, 60), (300, 200)])
def test_complete_bipartite(a, b):
    g = G.complete_bipartite(a, b)
    got = run_gpu(g, vertices=True, edges=True)
    assert got["total"] == c2(a) * c2(b)
    assert np.all(got["pv_u"] == (a - 1) * c2(b)) and np.all(got["pv_l"] == (b - 1) * c2(a))
    assert np.all(got["pe"] == (a - 1) * (b - 1))
    x, y = (a, b) if b >= a else (b, a)
    assert got["info"]["wedges"] == y * c2(x)


@pytest.mark.parametrize("orientation", [0, 1])
@pytest.mark.parametrize("a", [2, 3])
def test_wide_counters(a, orientation):
    # one start with more than 65,535 middles: count_wedge reaches 70,000 and
    # must not wrap in 16 bits
    b = 70_000
    g = G.complete_bipartite(a, b)
    got = run_gpu(g, vertices=True, edges=True, options=_opts(orientation=orientation))
    assert got["total"] == c2(a) * c2(b)
    assert np.all(got["pv_u"] == (a - 1) * c2(b))
    assert np.all(got["pv_l"] == (b - 1) * c2(a))
    assert np.all(got["pe"] == (a - 1) * (b - 1))


def test_zero_cases():
    for g in [G.cycle(5), G.cycle(2), G.random_forest(200, 150, 3), G.star(1000), G.path(50),
              G.from_edges(10, 7, [], []), G.from_edges(3, 0, [], []), G.from_edges(0, 0, [], [])]:
        got = run_gpu(g, vertices=True, edges=True)
        expect = 1 if g.name == "C_4" else 0
        assert got["total"] == expect, g.name
        assert int(got["pe"].sum()) == 4 * expect
        assert int(got["pv_u"].sum()) == 2 * expect


def test_paper_examples():
    for g, tot in [(G.paper_fig2a(), 0), (G.paper_fig3(), 999_000)]:
        got = run_gpu(g, export=True)
        assert got["total"] == tot
        assert got["info"]["wedges"] == 2000       # printed in Sections 1 and 4
    # Definition 3 order printed for Figure 3: p(u1) > p(u0) > p(v1001) > p(v1000)
    got = run_gpu(G.paper_fig3(), export=True)
    assert got["rank_u"][1] == 1001 and got["rank_u"][0] == 1000
    assert got["rank_l"][1001] == 1001 and got["rank_l"][1000] == 1000
    assert got["rank_l"][0] == 0 and got["rank_l"][1] == 1


# ---------------------------------------------------------------------------
# steps a2-a4: bit-exact intermediate arrays
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("gi", range(4))
def test_prepare_arrays(gi):
    g = [G.uniform_small(), G.chung_lu_bipartite(5000, 3000, 40000, 2.1, 2.1, 31),
         G.shuffle_lists(G.chung_lu_bipartite(3000, 800, 30000, 2.5, 1.8, 32, max_l=2000), 4),
         G.paper_fig3()][gi]
    got = run_gpu(g, export=True)
    ru, rl, _ = oracle.priority(g)
    assert np.array_equal(got["rank_u"], ru) and np.array_equal(got["rank_l"], rl)
    P = oracle.projection(g)
    assert np.array_equal(got["off"], P["off"])
    assert np.array_equal(got["adj"], P["adj"])
    assert np.array_equal(got["eid"], P["eid"])
    assert np.array_equal(got["cut"], P["cut"])
    assert np.array_equal(got["work"], P["work"])


@pytest.mark.parametrize("gi", range(3))
def test_long_list_graphs(gi):
    # one side's lists average 256 entries or more (Algorithm 2's run lengths
    # are searched in long lists): G*, cut, work and every output
    g = [G.chung_lu_bipartite(60_000, 500, 200_000, 2.5, 1.8, 5),
         G.chung_lu_bipartite(400, 50_000, 150_000, 1.8, 2.5, 6),
         G.shuffle_lists(G.complete_bipartite(300, 40), 3)][gi]
    assert g.num_edges >= 256 * min(g.num_u, g.num_l)
    got = run_gpu(g, export=True, vertices=True, edges=True)
    P = oracle.projection(g)
    for k in ("off", "adj", "eid", "cut", "work"):
        assert np.array_equal(got[k], P[k]), k
    ref = oracle.vp(g, vertices=True, edges=True)
    assert got["total"] == ref["total"] and got["total_all"] == ref["total"]
    assert np.array_equal(got["all_pv_u"], ref["pv_u"]) and np.array_equal(got["all_pv_l"], ref["pv_l"])
    assert np.array_equal(got["pe"], ref["pe"]) and np.array_equal(got["all_pe"], ref["pe"])


# U lists on both sides of each construction threshold (warp ranking up to 32
# neighbours, warp sort up to 256, CTA sort up to 4,096, radix above), with
# repeated degrees so that Definition 3's tie-break decides ranks
ROW_DEGREES = [1, 2, 31, 32, 32, 33, 64, 255, 256, 256, 257, 1000, 4095, 4096, 4096, 4097, 9000]


def _rows_graph():
    degs = ROW_DEGREES + [(7 * i) % 40 + 1 for i in range(300)]
    return G.rows_of_degrees(degs, 12000, 61)


def test_prepare_arrays_across_row_tiers():
    g = _rows_graph()
    got = run_gpu(g, export=True, vertices=True, edges=True)
    ru, rl, _ = oracle.priority(g)
    assert np.array_equal(got["rank_u"], ru) and np.array_equal(got["rank_l"], rl)
    P = oracle.projection(g)
    for k in ("off", "adj", "eid", "cut", "work"):
        assert np.array_equal(got[k], P[k]), k
    ref = oracle.vp(g, vertices=True, edges=True)
    assert got["total"] == ref["total"]
    assert np.array_equal(got["pe"], ref["pe"])


@pytest.mark.parametrize("deg", [2, 32, 200, 3000, 5000])
def test_duplicate_rejected_in_every_row_tier(deg):
    from paper_1812_00283_gb300 import BfcError, ButterflyGraph
    g = G.rows_of_degrees([deg, 3, 40], 6000, 62)
    adj = g.adj_u.copy()
    adj[deg - 1] = adj[0]          # the last neighbour of row 0 repeats its first
    with pytest.raises(BfcError) as ei:
        ButterflyGraph(torch.from_numpy(g.off_u).cuda(), torch.from_numpy(adj).cuda(), 3, 6000)
    assert ei.value.status == 2


# ---------------------------------------------------------------------------
# totals / per-vertex / per-edge against the oracle, every bin
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bins", sorted(BIN_SETTINGS))
def test_uniform_small_all_outputs(bins):
    g = G.uniform_small()
    _check_against_oracle(g, _opts(**BIN_SETTINGS[bins]))


@pytest.mark.parametrize("bins", sorted(BIN_SETTINGS))
@pytest.mark.parametrize("seed", [41, 42])
def test_powerlaw_all_outputs(bins, seed):
    g = G.chung_lu_bipartite(20000, 8000, 150000, 2.1, 2.0, seed)
    _check_against_oracle(g, _opts(**BIN_SETTINGS[bins]))


@pytest.mark.parametrize("wide", [0, 1])
def test_multi_chunk_end_ranges(wide):
    # U layer larger than one dense chunk (98,304 counters) so heavy U starts
    # are split into several end-range chunks with a ragged last chunk
    g = G.chung_lu_bipartite(230_000, 20_000, 900_000, 2.1, 2.1, 43)
    got, ref = _check_against_oracle(g, _opts(warp_max_work=0, hash_max_work=0, wide_positions=wide))
    assert got["info"]["dense_items"] > got["info"]["dense_starts"]


@pytest.mark.parametrize("opts", [{}, dict(warp_max_work=0, hash_max_work=0)])
def test_byte_counter_chunks(opts):
    # dense starts with at most 255 middles count in 8-bit counters: a
    # 400k-vertex U layer spans several 196,608-counter chunks (46 such
    # starts with the default bins)
    g = G.chung_lu_bipartite(400_000, 2_000, 3_000_000, 2.5, 1.8, 91, max_u=2000)
    got, ref = _check_against_oracle(g, _opts(**opts))
    assert got["info"]["dense_items"] > got["info"]["dense_starts"]


@pytest.mark.parametrize("wide", [0, 1])
def test_multi_chunk_retry_pass(wide):
    # Algorithm 3 with every start sent to the chunked dense pass: low starts
    # of the 230k-vertex U layer span several chunks above them
    g = G.chung_lu_bipartite(230_000, 20_000, 900_000, 2.1, 2.1, 43)
    _check_against_oracle(g, _opts(orientation=1, warp_max_work=0, hash_max_work=0,
                                   wide_positions=wide))


# Regular circulants on Sidon shift sets: starts at either end of the U order
# have ~3p^2 distinct ends, more than a team table (3,072 at load 3/4) holds
# for p = 37 and more than a CTA table (24,576) for p = 97.
SIDON = {37: (37, 3000, 12000), 97: (97, 20000, 78000)}


@pytest.mark.parametrize("p,mode,retries", [(37, "vpp", True), (37, "team_only", True),
                                            (37, "vpp_team_small", False), (97, "vpp", True),
                                            (97, "vpp_no_team", True), (97, "team_only", True)])
def test_retry_escalation(p, mode, retries):
    # team table full -> CTA table in the retry pass; CTA table full -> dense
    # chunks of the end range (Algorithm 3), all bit-exact.  Team starts of at
    # most 2,048 wedges always fit (vpp_team_small).
    g = G.shifted_sidon_circulant(*SIDON[p])
    got, ref = _check_against_oracle(g, _opts(**BIN_SETTINGS[mode]), edges=(p == 37))
    assert (got["retries"] > 0) == retries


def test_orientations_agree_on_wedges_and_work():
    # Lemma 4: both orientations process the same number of wedges
    g = G.chung_lu_bipartite(20000, 8000, 150000, 2.1, 2.0, 47)
    a = run_gpu(g, options=_opts(orientation=0))
    b = run_gpu(g, options=_opts(orientation=1))
    assert a["total"] == b["total"] and a["info"]["wedges"] == b["info"]["wedges"]


@pytest.mark.parametrize("orientation", [0, 1])
def test_shopping_shape_small(orientation):
    g = G.shopping_300m(scale=0.01)   # 100k users, 1k items, 3M edges
    _check_against_oracle(g, _opts(orientation=orientation))


def test_list_order_and_relabel_invariance():
    g = G.chung_lu_bipartite(6000, 4000, 50000, 2.1, 2.1, 44)
    base = run_gpu(g, edges=True)
    s = G.shuffle_lists(g, 3)
    got = run_gpu(s, edges=True)
    assert got["total"] == base["total"]
    u0, v0 = g.edges()
    us, vs = s.edges()
    k0 = dict(zip(zip(u0.tolist(), v0.tolist()), base["pe"].tolist()))
    assert all(k0[(a, b)] == c for a, b, c in zip(us.tolist(), vs.tolist(), got["pe"].tolist()))
    assert run_gpu(G.relabel(g, 7))["total"] == base["total"]


def test_repeated_counts_identical():
    import torch
    from paper_1812_00283_gb300 import ButterflyGraph
    g = G.chung_lu_bipartite(20000, 10000, 200000, 2.1, 2.1, 45)
    off = torch.from_numpy(g.off_u).cuda()
    adj = torch.from_numpy(g.adj_u).cuda()
    bg = ButterflyGraph(off, adj, g.num_u, g.num_l)
    vals = [bg.count() for _ in range(5)]
    pe1, _ = bg.count_edges()
    pe2, _ = bg.count_edges()
    bg.release()
    assert len(set(vals)) == 1 and torch.equal(pe1, pe2)
    assert vals[0] == oracle.vp(g)["total"]


def test_count_host_end_to_end():
    from paper_1812_00283_gb300 import bfc
    g = G.chung_lu_bipartite(10000, 5000, 80000, 2.1, 2.1, 46)
    off = np.ascontiguousarray(g.off_u)
    adj = np.ascontiguousarray(g.adj_u)
    total, wedges = bfc.bfc_count_host(g.num_u, g.num_l, g.num_edges, off.ctypes.data,
                                       adj.ctypes.data)
    ref = oracle.vp(g)
    assert (total, wedges) == (ref["total"], ref["wedges"])


# ---------------------------------------------------------------------------
# malformed input is rejected on the host side, never faults
# ---------------------------------------------------------------------------

def test_invalid_graphs_rejected():
    from paper_1812_00283_gb300 import BfcError, ButterflyGraph
    g = G.complete_bipartite(4, 4)
    cases = []
    adj = g.adj_u.copy(); adj[1] = adj[0]; cases.append((g.off_u, adj, "duplicate"))
    adj = g.adj_u.copy(); adj[3] = 99; cases.append((g.off_u, adj, "id"))
    adj = g.adj_u.copy(); adj[3] = -1; cases.append((g.off_u, adj, "negative id"))
    off = g.off_u.copy(); off[2] = 1; cases.append((off, g.adj_u, "offsets"))
    off = g.off_u.copy(); off[-1] = 15; cases.append((off, g.adj_u[:16], "end offset"))
    for off, adj, what in cases:
        with pytest.raises(BfcError) as ei:
            ButterflyGraph(torch.from_numpy(off).cuda(), torch.from_numpy(adj).cuda(), 4, 4)
        assert ei.value.status == 2, what


# ---------------------------------------------------------------------------
# derived statistics: caterpillars and the clustering coefficient (Section 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("gi", range(4))
def test_caterpillars_and_clustering(gi):
    from paper_1812_00283_gb300 import ButterflyGraph
    g = [G.complete_bipartite(6, 9), G.uniform_small(), G.chung_lu_bipartite(20000, 8000, 150000, 2.1, 2.0, 48),
         G.from_edges(5, 4, [], [])][gi]
    adj = g.adj_u if g.num_edges else np.zeros(1, np.int32)
    bg = ButterflyGraph(torch.from_numpy(g.off_u).cuda(), torch.from_numpy(adj).cuda()[:g.num_edges],
                        g.num_u, g.num_l)
    try:
        cat = bg.caterpillars()
        cc = bg.clustering_coefficient()
    finally:
        bg.release()
    ref = oracle.caterpillars(g)
    assert cat == ref
    tot = oracle.vp(g)["total"]
    assert cc == (4.0 * tot / ref if ref else 0.0)
    if gi == 0:
        assert cc == 1.0
