"""The continuous-batching server: every request's result equals its graph's
count alone, whatever mix, timing, batch limit or memory budget it meets."""
import random
import threading
import time

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


def _pool(k=48, seed=5):
    out = [G.complete_bipartite(6, 9), G.from_edges(7, 3, [], []), G.paper_fig3(), G.cycle(2)]
    for i in range(k):
        nu, nl, m, gu, gl = G.batch_graph_params(i, 7000 + seed)
        nu, nl = max(2, nu // 10), max(2, nl // 10)
        m = max(1, min(m // 50, nu * nl // 2))
        out.append(G.chung_lu_bipartite(nu, nl, m, gu, gl, 7000 + seed + i))
    return out


def _alone(g):
    from paper_1812_00283_gb300 import ButterflyGraph
    if g.num_edges == 0:
        return 0
    bg = ButterflyGraph(torch.from_numpy(g.off_u).cuda(), torch.from_numpy(g.adj_u).cuda(),
                        g.num_u, g.num_l)
    try:
        return bg.count()
    finally:
        bg.release()


def _serve(graphs, order, cfg, delays=None):
    from paper_1812_00283_gb300 import bfc
    sv = bfc.bfc_server_create(cfg)
    ids = [None] * len(order)
    arrays = [(np.ascontiguousarray(g.off_u), np.ascontiguousarray(g.adj_u if g.num_edges else
                                                                  np.zeros(1, np.int32)))
              for g in graphs]
    try:
        def submit():
            for j, gi in enumerate(order):
                if delays:
                    time.sleep(delays[j])
                g = graphs[gi]
                off, adj = arrays[gi]
                ids[j] = bfc.bfc_server_submit(sv, g.num_u, g.num_l, g.num_edges, off.ctypes.data,
                                               adj.ctypes.data)
        t = threading.Thread(target=submit)
        t.start()
        t.join()
        res = [bfc.bfc_server_poll(sv, rid, True) for rid in ids]
        stats = bfc.bfc_server_get_stats(sv)
    finally:
        bfc.bfc_server_destroy(sv)
    return res, stats


def test_server_results_equal_alone_results():
    from paper_1812_00283_gb300 import bfc
    graphs = _pool()
    alone = [_alone(g) for g in graphs]
    assert alone[:4] == [15 * 36, 0, 999_000, 1]
    # every graph counted alone on the GPU equals the oracle's count
    assert alone == [oracle.vp(g)["total"] for g in graphs]
    rng = random.Random(3)
    order = [rng.randrange(len(graphs)) for _ in range(300)]
    delays = [rng.expovariate(20000.0) for _ in order]     # ~50 us apart: requests overlap
    for cfg in [bfc.bfc_server_config_init(),                                  # batching, 2 workers
                bfc.bfc_server_config_init(max_batch_graphs=1, workers=1),     # one graph per launch
                bfc.bfc_server_config_init(workers=3, max_batch_graphs=7),
                bfc.bfc_server_config_init(memory_budget_bytes=200 << 20)]:   # tight budget
        res, stats = _serve(graphs, order, cfg, delays)
        assert all(st == 0 for st, _, _ in res)
        assert [tot for _, tot, _ in res] == [alone[gi] for gi in order]
        assert stats["submitted"] == stats["completed"] == len(order) and stats["failed"] == 0
        assert stats["peak_bytes_in_use"] <= cfg.memory_budget_bytes
        # the admission estimate bounds the memory the batches really took
        # from the library's pool (its measured high-water mark)
        assert stats["pool_bytes_high"] <= stats["pool_bytes_at_create"] + stats["peak_bytes_in_use"]
        if cfg.max_batch_graphs == 1:
            assert stats["batches"] == len(order)


def test_server_rejects_request_over_budget():
    from paper_1812_00283_gb300 import BfcError, bfc
    g = G.chung_lu_bipartite(20000, 10000, 300000, 2.1, 2.1, 3)
    sv = bfc.bfc_server_create(bfc.bfc_server_config_init(memory_budget_bytes=8 << 20))
    try:
        with pytest.raises(BfcError) as ei:
            bfc.bfc_server_submit(sv, g.num_u, g.num_l, g.num_edges, g.off_u.ctypes.data,
                                  g.adj_u.ctypes.data)
        assert ei.value.status == 3
    finally:
        bfc.bfc_server_destroy(sv)


def test_server_bad_request_fails_alone():
    """A malformed request fails on its own; the requests batched with it
    get the oracle's counts."""
    from paper_1812_00283_gb300 import BfcError, bfc
    graphs = [G.chung_lu_bipartite(40000, 20000, 400000, 2.1, 2.1, 17)] + _pool(k=16, seed=9)
    expect = [oracle.vp(g)["total"] for g in graphs]
    arrays = [(np.ascontiguousarray(g.off_u), np.ascontiguousarray(g.adj_u if g.num_edges else
                                                                  np.zeros(1, np.int32)))
              for g in graphs]
    sv = bfc.bfc_server_create(bfc.bfc_server_config_init(workers=1))
    try:
        # not a CSR, and an id out of range: refused at submission
        for off, adj in [(np.array([0, 3, 2], np.int32), np.array([0, 1, 0], np.int32)),
                         (np.array([0, 1, 3], np.int32), np.array([0, 1, 5], np.int32))]:
            with pytest.raises(BfcError) as ei:
                bfc.bfc_server_submit(sv, 2, 2, 3, off.ctypes.data, adj.ctypes.data)
            assert ei.value.status == 2
        # a duplicate edge is found on the device while the large first graph
        # keeps the worker busy, so it meets the others in one batch
        dup_off, dup_adj = np.array([0, 2, 3], np.int32), np.array([1, 1, 0], np.int32)
        ids = []
        for i, (g, (off, adj)) in enumerate(zip(graphs, arrays)):
            ids.append(bfc.bfc_server_submit(sv, g.num_u, g.num_l, g.num_edges, off.ctypes.data,
                                             adj.ctypes.data))
            if i == 5:
                dup_id = bfc.bfc_server_submit(sv, 2, 2, 3, dup_off.ctypes.data, dup_adj.ctypes.data)
        res = [bfc.bfc_server_poll(sv, rid, True) for rid in ids]
        dup = bfc.bfc_server_poll(sv, dup_id, True)
        stats = bfc.bfc_server_get_stats(sv)
    finally:
        bfc.bfc_server_destroy(sv)
    assert dup[0] == 2
    assert [st for st, _, _ in res] == [0] * len(graphs)
    assert [tot for _, tot, _ in res] == expect
    assert stats["failed"] == 1 and stats["completed"] == len(graphs)


def test_server_rejects_batch_limit_beyond_int32_offsets():
    from paper_1812_00283_gb300 import BfcError, bfc
    with pytest.raises(BfcError) as ei:
        bfc.bfc_server_create(bfc.bfc_server_config_init(max_batch_edges=1 << 31))
    assert ei.value.status == 1
