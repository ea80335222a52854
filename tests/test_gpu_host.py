"""End to end from host memory: bfc_count_all_host and bfc_count_host copy
the CSR in and the outputs out (by the SMs for page-locked buffers, by the
copy engines for pageable ones); every output against the oracle."""
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


def _buffers(g, pinned, shift):
    """Host input and output buffers; `shift` int32 words of slack in front of
    the outputs make them 4-byte aligned only (the narrow copy path)."""
    mk = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
    off = mk(torch.from_numpy(np.ascontiguousarray(g.off_u)))
    adj = mk(torch.from_numpy(np.ascontiguousarray(g.adj_u if g.num_edges else np.zeros(1, np.int32))))
    outs = []
    for n in (g.num_u, g.num_l, g.num_edges):
        raw = mk(torch.zeros(2 * max(n, 1) + shift, dtype=torch.int32))
        outs.append((raw, raw.data_ptr() + 4 * shift))
    return off, adj, outs


def _view(raw, ptr_shift_words, n):
    return raw.numpy()[ptr_shift_words:ptr_shift_words + 2 * n].view(np.uint64)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("gi", range(4))
def test_count_all_host_matches_oracle(pinned, shift, gi):
    from paper_1812_00283_gb300 import bfc
    g = [G.complete_bipartite(6, 9), G.uniform_small(), G.from_edges(5, 3, [], []),
         G.chung_lu_bipartite(20000, 8000, 150000, 2.1, 2.0, 48)][gi]
    ref = oracle.vp(g, vertices=True, edges=True)
    off, adj, outs = _buffers(g, pinned, shift)
    s = torch.cuda.current_stream().cuda_stream
    tot, wed = bfc.bfc_count_all_host(g.num_u, g.num_l, g.num_edges, off.data_ptr(), adj.data_ptr(), None, s,
                                      outs[0][1], outs[1][1], outs[2][1])
    assert tot == ref["total"] and wed == ref["wedges"]
    assert np.array_equal(_view(outs[0][0], shift, g.num_u), ref["pv_u"])
    assert np.array_equal(_view(outs[1][0], shift, g.num_l), ref["pv_l"])
    assert np.array_equal(_view(outs[2][0], shift, g.num_edges), ref["pe"])
    t2, w2 = bfc.bfc_count_host(g.num_u, g.num_l, g.num_edges, off.data_ptr(), adj.data_ptr(), None, s)
    assert (t2, w2) == (ref["total"], ref["wedges"])


def test_count_all_host_rejects_missing_edge_output():
    from paper_1812_00283_gb300 import BfcError, bfc
    g = G.complete_bipartite(3, 3)
    off, adj = g.off_u.copy(), g.adj_u.copy()
    with pytest.raises(BfcError) as ei:
        bfc.bfc_count_all_host(3, 3, 9, off.ctypes.data, adj.ctypes.data, None, 0, None, None, None)
    assert ei.value.status == 1
