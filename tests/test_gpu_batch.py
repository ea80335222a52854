"""Batched counting: one prepare over the disjoint union, one persistent
count launch, per-graph totals bit-exact against the oracle per graph."""
import numpy as np
import pytest

import oracle
from bfc_inputs import generators as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _batch_graphs(k=40, seed=0):
    out = [G.complete_bipartite(5, 7), G.from_edges(6, 4, [], []), G.cycle(2), G.paper_fig3(),
           G.complete_bipartite(2, 70_000)]
    for i in range(k):
        nu, nl, m, gu, gl = G.batch_graph_params(i, 9000 + seed)
        # small versions of the batched workload's size distribution
        nu, nl = max(2, nu // 20), max(2, nl // 20)
        m = max(1, min(m // 100, nu * nl // 2))
        out.append(G.chung_lu_bipartite(nu, nl, m, gu, gl, 9000 + seed + i))
    return out


def _prepare(b, options=None):
    from paper_1812_00283_gb300 import bfc
    dev = torch.device("cuda")
    t = dict(off=torch.from_numpy(b.union.off_u).to(dev), adj=torch.from_numpy(b.union.adj_u).to(dev),
             us=torch.from_numpy(b.u_start).to(dev), ls=torch.from_numpy(b.l_start).to(dev))
    h = bfc.bfc_prepare_batch(b.union.num_u, b.union.num_l, b.union.num_edges, t["off"].data_ptr(),
                              t["adj"].data_ptr(), b.num_graphs, t["us"].data_ptr(),
                              t["ls"].data_ptr(), options, torch.cuda.current_stream().cuda_stream)
    return h, t


def _count(h, nG):
    from paper_1812_00283_gb300 import bfc
    s = torch.cuda.current_stream().cuda_stream
    tot = torch.zeros(nG, dtype=torch.int64, device="cuda")
    one = torch.zeros(1, dtype=torch.int64, device="cuda")
    bfc.bfc_count_batch(h, s, tot.data_ptr(), one.data_ptr())
    bfc.bfc_sync(h, s)
    return tot.cpu().numpy().view(np.uint64), int(one.item())


@pytest.mark.parametrize("opts", [{}, dict(warp_max_work=0, hash_max_work=0), dict(warp_max_work=128, hash_max_work=256),
                                  dict(warp_max_work=0, team_max_work=16384),
                                  dict(orientation=1), dict(orientation=1, warp_max_work=0, hash_max_work=0),
                                  dict(orientation=1, team_max_work=0)])
def test_batch_totals_match_oracle(opts):
    from paper_1812_00283_gb300 import bfc
    graphs = _batch_graphs()
    b = G.union_batch(graphs)
    h, keep = _prepare(b, bfc.bfc_options_init(**opts) if opts else None)
    try:
        tot, whole = _count(h, b.num_graphs)
        wed = torch.zeros(b.num_graphs, dtype=torch.int64, device="cuda")
        bfc.bfc_batch_wedges(h, torch.cuda.current_stream().cuda_stream, wed.data_ptr())
        wed = wed.cpu().numpy().view(np.uint64)
    finally:
        bfc.bfc_release(h)
    refs = [oracle.vp(g) for g in graphs]
    assert [int(x) for x in tot] == [r["total"] for r in refs]
    assert [int(x) for x in wed] == [r["wedges"] for r in refs]
    assert whole == sum(r["total"] for r in refs)


@pytest.mark.parametrize("opts", [{}, dict(warp_max_work=0, hash_max_work=0)])
def test_batch_chunked_dense_items_match_oracle(opts):
    # layers above 98,304 vertices in two graphs of different shapes: heavy
    # starts count their ends in several dense chunks, whose run bounds come
    # from the chunk-boundary table relative to each graph's range
    from paper_1812_00283_gb300 import bfc
    graphs = [G.complete_bipartite(3, 4),
              G.chung_lu_bipartite(150_000, 5_000, 400_000, 1.8, 2.5, 71),
              G.chung_lu_bipartite(200, 300, 2_000, 2.1, 2.1, 72),
              G.chung_lu_bipartite(6_000, 120_000, 300_000, 2.5, 1.8, 73),
              G.from_edges(4, 5, [], [])]
    b = G.union_batch(graphs)
    h, keep = _prepare(b, bfc.bfc_options_init(**opts) if opts else None)
    try:
        info = bfc.bfc_graph_info(h)
        tot, whole = _count(h, b.num_graphs)
    finally:
        bfc.bfc_release(h)
    refs = [oracle.vp(g)["total"] for g in graphs]
    assert info["dense_items"] > info["dense_starts"] > 0
    assert [int(x) for x in tot] == refs and whole == sum(refs)


def test_batch_autotune_and_graph_capture():
    from paper_1812_00283_gb300 import bfc
    graphs = _batch_graphs(k=60, seed=1)
    b = G.union_batch(graphs)
    h, keep = _prepare(b)
    try:
        s = torch.cuda.current_stream()
        chosen = bfc.bfc_autotune(h, s.cuda_stream, 1)
        assert chosen.warp_max_work in (32, 128, 384) and chosen.hash_max_work in (4096, 24576)
        expect, _ = _count(h, b.num_graphs)          # first call outside capture
        tot = torch.zeros(b.num_graphs, dtype=torch.int64, device="cuda")
        cg = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(s)
        with torch.cuda.graph(cg, stream=cap):
            bfc.bfc_count_batch(h, cap.cuda_stream, tot.data_ptr(), None)
        for _ in range(2):
            tot.fill_(-1)
            cg.replay()
            torch.cuda.synchronize()
            assert np.array_equal(tot.cpu().numpy().view(np.uint64), expect)
    finally:
        bfc.bfc_release(h)
    assert [int(x) for x in expect] == [oracle.vp(g)["total"] for g in graphs]


def test_batch_rejects_cross_graph_edge():
    from paper_1812_00283_gb300 import BfcError
    graphs = [G.complete_bipartite(3, 3), G.complete_bipartite(2, 2)]
    b = G.union_batch(graphs)
    b.union.adj_u[0] = 4      # an L vertex of the second graph
    with pytest.raises(BfcError) as ei:
        _prepare(b)
    assert ei.value.status == 2


def test_tuned_bounds_kept_per_size_class():
    # bfc_autotune keeps its choice for the size class; a later batch of the
    # same class prepared with use_tuned gets the same bins as one prepared
    # with the chosen bounds given explicitly, and counts exactly
    from paper_1812_00283_gb300 import bfc
    graphs = _batch_graphs(k=50, seed=3)
    b = G.union_batch(graphs)
    h, keep = _prepare(b)
    try:
        chosen = bfc.bfc_autotune(h, torch.cuda.current_stream().cuda_stream, 1)
    finally:
        bfc.bfc_release(h)
    other = [G.relabel(g, 40 + i) for i, g in enumerate(graphs)]   # same sizes
    b2 = G.union_batch(other)
    h1, k1 = _prepare(b2, bfc.bfc_options_init(use_tuned=1))
    h2, k2 = _prepare(b2, bfc.bfc_options_init(warp_max_work=chosen.warp_max_work,
                                               team_max_work=chosen.team_max_work,
                                               hash_max_work=chosen.hash_max_work))
    try:
        i1, i2 = bfc.bfc_graph_info(h1), bfc.bfc_graph_info(h2)
        for key in ("warp_starts", "team_starts", "hash_starts", "dense_starts", "dense_items"):
            assert i1[key] == i2[key], key
        tot, _ = _count(h1, b2.num_graphs)
    finally:
        bfc.bfc_release(h1)
        bfc.bfc_release(h2)
    assert [int(x) for x in tot] == [oracle.vp(g)["total"] for g in other]
