"""Batch plans: a batch of a fixed shape prepared and counted on the stream
with no host synchronisation and no allocation, so the whole step (ranks,
projection, cut and work, bins, the persistent count and the per-graph
totals) is recorded once in a CUDA graph and replayed on new contents.

* Per-graph totals against the oracle, under several bin settings, with rows
  in every construction tier (the largest rows are placed by the bitmap
  tier).
* A captured step replayed on two batches of the same shape written into the
  same buffers, each against the oracle.
* Malformed input gives a status, not a fault, and zero totals; the next
  valid run is exact.
"""
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


def _graphs(seed=0, k=30):
    # K_{3,6000}: U rows of 6,000 neighbours (the bitmap tier); a power-law
    # graph with hubs above 4,096 and rows in the warp and CTA sort tiers
    out = [G.complete_bipartite(5, 7), G.from_edges(6, 4, [], []), G.cycle(2), G.paper_fig3(),
           G.complete_bipartite(3, 6000),
           G.chung_lu_bipartite(3000, 20000, 120000, 2.1, 2.1, 31 + seed, max_u=9000)]
    for i in range(k):
        nu, nl, m, gu, gl = G.batch_graph_params(i, 9500 + seed)
        nu, nl = max(2, nu // 20), max(2, nl // 20)
        m = max(1, min(m // 100, nu * nl // 2))
        out.append(G.chung_lu_bipartite(nu, nl, m, gu, gl, 9500 + seed + i))
    return out


def _same_shape(graphs, seed):
    """Other graphs with the same layer sizes and edge counts, one by one."""
    out = []
    for i, g in enumerate(graphs):
        if g.num_edges == 0 or g.num_edges >= g.num_u * g.num_l:
            out.append(G.relabel(g, seed + i))   # nothing else has this shape
        else:
            out.append(G.uniform_bipartite(g.num_u, g.num_l, g.num_edges, seed + i))
    return out


def _device(b):
    dev = torch.device("cuda")
    return dict(off=torch.from_numpy(b.union.off_u).to(dev), adj=torch.from_numpy(b.union.adj_u).to(dev),
                us=torch.from_numpy(b.u_start).to(dev), ls=torch.from_numpy(b.l_start).to(dev))


def _max_layer(graphs):
    return max(max(g.num_u, g.num_l) for g in graphs)


def _plan(b, max_layer, options=None):
    from paper_1812_00283_gb300 import bfc
    s = torch.cuda.current_stream().cuda_stream
    return bfc.bfc_batch_plan_create(b.union.num_u, b.union.num_l, b.union.num_edges, b.num_graphs,
                                     max_layer, options, s)


def _run(plan, t, num_graphs, stream=None):
    from paper_1812_00283_gb300 import bfc
    s = torch.cuda.current_stream() if stream is None else stream
    tot = torch.full((num_graphs,), -1, dtype=torch.int64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    bfc.bfc_batch_plan_run(plan, t["off"].data_ptr(), t["adj"].data_ptr(), t["us"].data_ptr(),
                           t["ls"].data_ptr(), s.cuda_stream, tot.data_ptr(), st.data_ptr())
    s.synchronize()
    return tot.cpu().numpy().view(np.uint64), int(st.item())


@pytest.mark.parametrize("opts", [{}, dict(warp_max_work=0, hash_max_work=0),
                                  dict(warp_max_work=128, hash_max_work=256),
                                  dict(warp_max_work=32, team_max_work=512, hash_max_work=4096),
                                  dict(warp_max_work=0, team_max_work=0)])
def test_plan_totals_match_oracle(opts):
    from paper_1812_00283_gb300 import bfc
    graphs = _graphs()
    b = G.union_batch(graphs)
    t = _device(b)
    plan = _plan(b, _max_layer(graphs), bfc.bfc_options_init(**opts))
    try:
        tot, st = _run(plan, t, b.num_graphs)
        tot2, st2 = _run(plan, t, b.num_graphs)   # the plan's arrays are reused
    finally:
        bfc.bfc_batch_plan_destroy(plan)
    ref = [oracle.vp(g)["total"] for g in graphs]
    assert st == 0 and st2 == 0
    assert [int(x) for x in tot] == ref and [int(x) for x in tot2] == ref


def test_plan_step_captured_and_replayed_on_new_contents():
    from paper_1812_00283_gb300 import bfc
    ga = _graphs(seed=1, k=20)
    gb = _same_shape(ga, 77)
    ba, bb = G.union_batch(ga), G.union_batch(gb)
    assert (ba.union.num_u, ba.union.num_l, ba.union.num_edges) == \
        (bb.union.num_u, bb.union.num_l, bb.union.num_edges)
    assert np.array_equal(ba.u_start, bb.u_start) and np.array_equal(ba.l_start, bb.l_start)
    t = _device(ba)
    ref_a = [oracle.vp(g)["total"] for g in ga]
    ref_b = [oracle.vp(g)["total"] for g in gb]
    assert ref_a != ref_b
    plan = _plan(ba, max(_max_layer(ga), _max_layer(gb)))
    try:
        s = torch.cuda.current_stream()
        tot_a, st = _run(plan, t, ba.num_graphs)        # a first run outside capture
        assert st == 0 and [int(x) for x in tot_a] == ref_a
        tot = torch.zeros(ba.num_graphs, dtype=torch.int64, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        cg = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        cap.wait_stream(s)
        with torch.cuda.graph(cg, stream=cap):
            bfc.bfc_batch_plan_run(plan, t["off"].data_ptr(), t["adj"].data_ptr(), t["us"].data_ptr(),
                                   t["ls"].data_ptr(), cap.cuda_stream, tot.data_ptr(), status.data_ptr())
        for batch, ref in [(bb, ref_b), (ba, ref_a), (bb, ref_b)]:
            t["off"].copy_(torch.from_numpy(batch.union.off_u))
            t["adj"].copy_(torch.from_numpy(batch.union.adj_u))
            tot.fill_(-1)
            status.fill_(-1)
            cg.replay()
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            assert [int(x) for x in tot.cpu().numpy().view(np.uint64)] == ref
    finally:
        bfc.bfc_batch_plan_destroy(plan)


def test_plan_flags_malformed_input():
    from paper_1812_00283_gb300 import bfc
    graphs = _graphs(seed=2, k=8)
    b = G.union_batch(graphs)
    ref = [oracle.vp(g)["total"] for g in graphs]
    plan = _plan(b, _max_layer(graphs))
    try:
        good = b.union.adj_u.copy()
        # the first row of graph 5 (the power-law graph) with two neighbours or more
        off_u = b.union.off_u.astype(np.int64)
        u = next(x for x in range(int(b.u_start[5]), int(b.u_start[6])) if off_u[x + 1] - off_u[x] >= 2)
        e0 = int(off_u[u])
        cases = []
        bad = good.copy(); bad[e0] = b.union.num_l + 5; cases.append(("id out of range", bad, None))
        bad = good.copy(); bad[e0] = 0; cases.append(("edge across graphs", bad, None))
        bad = good.copy(); bad[e0 + 1] = bad[e0]; cases.append(("duplicate edge", bad, None))
        off = b.union.off_u.copy(); off[3] = off[4] + 1; cases.append(("offsets", good, off))
        t = _device(b)
        for what, adj, off in cases:
            t["adj"].copy_(torch.from_numpy(adj))
            t["off"].copy_(torch.from_numpy(b.union.off_u if off is None else off))
            tot, st = _run(plan, t, b.num_graphs)
            assert st == 2, what
            if what != "duplicate edge":
                assert not tot.any(), what   # nothing counted after failed checks
        t["adj"].copy_(torch.from_numpy(good))
        t["off"].copy_(torch.from_numpy(b.union.off_u))
        tot, st = _run(plan, t, b.num_graphs)
        assert st == 0 and [int(x) for x in tot] == ref
    finally:
        bfc.bfc_batch_plan_destroy(plan)


def test_plan_flags_graph_above_max_layer():
    from paper_1812_00283_gb300 import bfc
    graphs = [G.complete_bipartite(4, 5), G.complete_bipartite(3, 40)]
    b = G.union_batch(graphs)
    plan = _plan(b, 20)   # the second graph's L layer has 40 vertices
    try:
        tot, st = _run(plan, _device(b), b.num_graphs)
    finally:
        bfc.bfc_batch_plan_destroy(plan)
    assert st == 2 and not tot.any()
