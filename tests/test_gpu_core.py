"""The dense-core hybrid: the top-K priority core counted by a masked 0/1
matrix product on the tensor cores (tcgen05), the rest by Algorithm 2's
walk, which skips every wedge with start, middle and end in the core and
adds a·b + C(a, 2) per core pair (Lemma 1).

* ⋈_G against the oracle for core sizes from 1 to every vertex.
* The products against the oracle's own core split (Σ a = the wedges its
  walk skips, Σ C(a, 2)), and element by element against a numpy masked
  product built from the oracle's priorities.
* The core sizes per layer against the oracle's top-K by Definition 3.
* Per-vertex and per-edge counts of a graph prepared with a core (the core
  only serves total counts) and repeated counts stay exact.
"""
import numpy as np
import pytest

import oracle
from bfc_inputs import generators as G

from gpu_path import as_u64

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _graphs():
    return [G.complete_bipartite(9, 14), G.paper_fig3(), G.uniform_small(),
            G.chung_lu_bipartite(4000, 2500, 30000, 2.1, 2.1, 7),
            G.chung_lu_bipartite(20000, 8000, 150000, 2.1, 2.0, 48),
            G.chung_lu_bipartite(30000, 3000, 200000, 2.5, 1.8, 11)]


def _core_count(g, K, repeat=1, products=True):
    from paper_1812_00283_gb300 import ButterflyGraph, bfc
    opts = bfc.bfc_options_init(core_vertices=K)
    bg = ButterflyGraph(torch.from_numpy(g.off_u).cuda(), torch.from_numpy(g.adj_u).cuda(),
                        g.num_u, g.num_l, opts)
    try:
        tots = [bg.count() for _ in range(repeat)]
        info = bg.info()
        if not products:
            return dict(totals=tots, info=info)
        pu = bg.export(bfc.BFC_CORE_PRODUCT_U).cpu().numpy().view(np.uint16)
        pl = bg.export(bfc.BFC_CORE_PRODUCT_L).cpu().numpy().view(np.uint16)
        ku, kl = info["core_u"], info["core_l"]
        return dict(totals=tots, info=info, pu=pu[:ku * ku].reshape(ku, ku).astype(np.int64),
                    pl=pl[:kl * kl].reshape(kl, kl).astype(np.int64))
    finally:
        bg.release()


def _ks(g):
    n = g.num_u + g.num_l
    return sorted({1, 7, 128, 129, min(600, n), min(2000, n), n})


CASES = [(gi, K) for gi, g in enumerate(_graphs()) for K in _ks(g)]


@pytest.mark.parametrize("gi,K", CASES)
def test_core_total_and_split_match_oracle(gi, K):
    g = _graphs()[gi]
    got = _core_count(g, K)
    ref_total = oracle.vp(g)["total"]
    assert got["totals"][0] == ref_total
    # the core is the oracle's top K by Definition 3 (p of U vertex u is p[l + u])
    _, _, p = oracle.priority(g)
    n, l = g.num_u + g.num_l, g.num_l
    top = p > n - min(K, n)
    assert got["info"]["core_u"] == int(top[l:].sum()) and got["info"]["core_l"] == int(top[:l].sum())
    # the products are the oracle split's a: Σ a = the wedges its walk skips
    tot, skipped, c2a, _ = oracle.vp_core_split(g, min(K, n))
    assert tot == ref_total
    a = np.concatenate([got["pu"][np.tril_indices(len(got["pu"]), -1)],
                        got["pl"][np.tril_indices(len(got["pl"]), -1)]])
    assert int(a.sum()) == skipped
    assert int((a * (a - 1) // 2).sum()) == c2a


def _numpy_products(g, K):
    """a(u, w) of both cores from the oracle's priorities, by a plain masked
    0/1 matrix product (rows and columns in ascending priority)."""
    _, _, p = oracle.priority(g)
    n, l = g.num_u + g.num_l, g.num_l
    u_e, v_e = g.edges()
    gu = l + u_e.astype(np.int64)          # gid of the U end of each edge
    gv = v_e.astype(np.int64)
    core = p > n - K
    cu = np.flatnonzero(core[l:]) + l      # core U gids
    cl = np.flatnonzero(core[:l])          # core L gids
    cu = cu[np.argsort(p[cu])]
    cl = cl[np.argsort(p[cl])]
    iu = {int(x): i for i, x in enumerate(cu)}
    il = {int(x): i for i, x in enumerate(cl)}
    B = np.zeros((len(cu), len(cl)), dtype=np.int64)
    for a, b in zip(gu, gv):
        if int(a) in iu and int(b) in il:
            B[iu[int(a)], il[int(b)]] = 1
    below_u = (p[cl][None, :] < p[cu][:, None]).astype(np.int64)   # p(v) < p(u)
    below_l = (p[cu][None, :] < p[cl][:, None]).astype(np.int64)   # p(u) < p(v)
    AU = (B * below_u) @ B.T
    AL = (B.T * below_l) @ B
    return AU, AL


@pytest.mark.parametrize("gi,K", [(0, 23), (2, 700), (3, 300), (4, 900), (5, 1500)])
def test_core_products_elementwise(gi, K):
    g = _graphs()[gi]
    got = _core_count(g, K)
    AU, AL = _numpy_products(g, K)
    assert AU.shape == got["pu"].shape and AL.shape == got["pl"].shape
    lu, ll = np.tril_indices(len(AU), -1), np.tril_indices(len(AL), -1)
    assert np.array_equal(got["pu"][lu], AU[lu])
    assert np.array_equal(got["pl"][ll], AL[ll])


def test_core_graph_keeps_other_outputs_and_repeats():
    from paper_1812_00283_gb300 import ButterflyGraph, bfc
    g = G.chung_lu_bipartite(20000, 8000, 150000, 2.1, 2.0, 48)
    ref = oracle.vp(g, vertices=True, edges=True)
    bg = ButterflyGraph(torch.from_numpy(g.off_u).cuda(), torch.from_numpy(g.adj_u).cuda(),
                        g.num_u, g.num_l, bfc.bfc_options_init(core_vertices=800))
    try:
        assert [bg.count() for _ in range(3)] == [ref["total"]] * 3
        pu, pl, pe, t = bg.count_all()
        assert t == ref["total"]
        assert np.array_equal(as_u64(pu), ref["pv_u"]) and np.array_equal(as_u64(pl), ref["pv_l"])
        assert np.array_equal(as_u64(pe), ref["pe"])
        assert bg.count() == ref["total"]   # the core again after a full walk
        assert bg.info()["wedges"] == ref["wedges"]
    finally:
        bg.release()


@pytest.mark.parametrize("gi", range(6))
@pytest.mark.parametrize("hash_max", [None, 0])
def test_core_automatic_size(gi, hash_max):
    # -1 (the default): as many core vertices as starts heavier than the
    # CTA-hash bin (at most 8,192), if each layer then holds 1,024 of them
    from paper_1812_00283_gb300 import ButterflyGraph, bfc
    g = _graphs()[gi]
    opts = bfc.bfc_options_init() if hash_max is None else \
        bfc.bfc_options_init(warp_max_work=0, hash_max_work=hash_max)
    assert opts.core_vertices == -1
    bg = ButterflyGraph(torch.from_numpy(g.off_u).cuda(), torch.from_numpy(g.adj_u).cuda(),
                        g.num_u, g.num_l, opts)
    try:
        total, info, work = bg.count(), bg.info(), as_u64(bg.export(bfc.BFC_WORK))
    finally:
        bg.release()
    assert total == oracle.vp(g)["total"]
    K = min(int((work > opts.hash_max_work).sum()), 8192)
    _, _, p = oracle.priority(g)
    n, l = g.num_u + g.num_l, g.num_l
    top = p > n - K
    ku, kl = int(top[l:].sum()), int(top[:l].sum())
    if ku >= 1024 and kl >= 1024:
        assert (info["core_u"], info["core_l"]) == (ku, kl)
    else:
        assert (info["core_u"], info["core_l"]) == (0, 0)


def test_core_powerlaw_20m_against_oracle():
    g = G.powerlaw_20m(device="cuda")
    ref = oracle.vp(g)["total"]
    for K in (-1, 4096, 16384):
        got = _core_count(g, K, repeat=2, products=False)
        assert got["totals"] == [ref, ref]
