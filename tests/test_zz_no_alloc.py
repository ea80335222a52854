"""bfc_count_small_noalloc: the allocation-free entry point for callers that
may not allocate device memory where they count (their device memory is
reserved up front by their own allocator, or they run in a loop that must
not enter the driver's allocator).  Its result must equal the regular entry
point's (bfc_prepare + bfc_count) and the oracle's bit for bit, on
consecutive calls that share the library's fixed scratch array.

This file is collected last on purpose: a failure here leaves every other
test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
from bfc_inputs import generators as G

torch = pytest.importorskip("torch")


def _graphs():
    return [G.uniform_small(), G.chung_lu_bipartite(20000, 8000, 150000, 2.1, 2.0, 41),
            G.complete_bipartite(30, 40), G.cycle(2), G.from_edges(10, 7, [], []),
            G.paper_fig3(), G.chung_lu_bipartite(40000, 25000, 1_000_000, 2.3, 1.9, 5)]


def test_no_alloc_rejects_oversized_graphs():
    # size checks come before any GPU work
    from paper_1812_00283_gb300 import bfc
    lib = bfc.library()
    tot = ctypes.c_uint64(0)
    for r, l, m in [(49153, 10, 10), (10, 49153, 10), (40000, 30000, 10), (10, 10, (1 << 20) + 1)]:
        rc = lib.bfc_count_small_noalloc(r, l, m, 16, 16, None, ctypes.addressof(tot), None)
        assert rc == 1 and "too large" in bfc.bfc_last_error()


@pytest.mark.gpu
def test_no_alloc_matches_regular_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00283_gb300 import ButterflyGraph, bfc
    stream = torch.cuda.current_stream()
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for g in _graphs():
        off = torch.from_numpy(np.ascontiguousarray(g.off_u)).cuda()
        adj = torch.from_numpy(np.ascontiguousarray(g.adj_u if g.num_edges else
                                                    np.zeros(1, np.int32))).cuda()
        bg = ButterflyGraph(off, adj[:g.num_edges], g.num_u, g.num_l)
        expect = bg.count()
        bg.release()
        assert expect == oracle.vp(g)["total"], g.name
        for _ in range(2):   # two calls in a row on the shared scratch
            total.fill_(-1)
            status.fill_(-1)
            bfc.bfc_count_small_noalloc(g.num_u, g.num_l, g.num_edges, off.data_ptr(),
                                        adj.data_ptr(), stream.cuda_stream, total.data_ptr(),
                                        status.data_ptr())
            stream.synchronize()
            assert int(status.item()) == 0, g.name
            assert (int(total.item()) & ((1 << 64) - 1)) == expect, g.name


@pytest.mark.gpu
def test_no_alloc_flags_invalid_csr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00283_gb300 import bfc
    g = G.complete_bipartite(4, 4)
    stream = torch.cuda.current_stream()
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    adj = g.adj_u.copy()
    adj[5] = 17   # id out of range
    off_t = torch.from_numpy(g.off_u).cuda()
    adj_t = torch.from_numpy(adj).cuda()
    bfc.bfc_count_small_noalloc(4, 4, 16, off_t.data_ptr(), adj_t.data_ptr(), stream.cuda_stream,
                                total.data_ptr(), status.data_ptr())
    stream.synchronize()
    assert int(status.item()) == 2 and int(total.item()) == 0
    # the next valid call is unaffected
    adj_t = torch.from_numpy(g.adj_u).cuda()
    bfc.bfc_count_small_noalloc(4, 4, 16, off_t.data_ptr(), adj_t.data_ptr(), stream.cuda_stream,
                                total.data_ptr(), status.data_ptr())
    stream.synchronize()
    assert int(status.item()) == 0 and int(total.item()) == 36
