"""Parity at the benchmark sizes, in the launch configuration the benchmark
times (default options, Algorithm 2, one CTA per SM).

* The 20M-edge power-law graph: every output against the full oracle.
* The 300M-edge shopping graph (10M users, 100k items): every output
  (⋈_G, W, per-vertex of both layers, per-edge) against the full oracle run
  on the host cores, which works while the GPU counts.  Two checks that do
  not go through the oracle's Algorithm 2 stand beside it: identities that
  hold at any size (Σ per-vertex over each layer = 2⋈, Σ per-edge = 4⋈,
  Algorithm 3 gives the same ⋈ and W by Lemma 4) and sampled vertices and
  edges, including the heaviest of each kind, computed one by one from
  Eq. 1 and Eq. 7.
"""
import threading

import numpy as np
import pytest

import oracle
from bfc_inputs import generators as G

from gpu_path import as_u64, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_powerlaw_20m_all_outputs_against_oracle():
    g = G.powerlaw_20m(device="cuda")
    got = run_gpu(g, vertices=True, edges=True)
    ref = oracle.vp(g, vertices=True, edges=True)
    assert got["total"] == ref["total"] and got["info"]["wedges"] == ref["wedges"]
    for key in ("total_v", "total_e", "total_all"):
        assert got[key] == ref["total"]
    assert np.array_equal(got["pv_u"], ref["pv_u"]) and np.array_equal(got["pv_l"], ref["pv_l"])
    assert np.array_equal(got["pe"], ref["pe"])
    assert np.array_equal(got["all_pv_u"], ref["pv_u"]) and np.array_equal(got["all_pv_l"], ref["pv_l"])
    assert np.array_equal(got["all_pe"], ref["pe"])


def _sample(rng, n, k, must):
    pick = set(int(x) for x in must)
    while len(pick) < min(n, k + len(must)):
        pick.add(int(rng.integers(n)))
    return np.array(sorted(pick), dtype=np.int64)


def test_shopping_300m_all_outputs_against_oracle():
    from paper_1812_00283_gb300 import ButterflyGraph, bfc
    g = G.shopping_300m(device="cuda")
    # the oracle (Algorithm 2 with the two-walk attribution, all host cores)
    # runs in a thread while the GPU counts; ctypes releases the GIL
    ref, failure = {}, []

    def run_oracle():
        try:
            ref.update(oracle.vp(g, vertices=True, edges=True))
        except Exception as e:   # re-raised in the test thread
            failure.append(e)
    th = threading.Thread(target=run_oracle)
    th.start()
    try:
        off = torch.from_numpy(g.off_u).cuda()
        adj = torch.from_numpy(g.adj_u).cuda()
        bg = ButterflyGraph(off, adj, g.num_u, g.num_l)
        try:
            tot = bg.count()
            W = bg.info()["wedges"]
            pu, pl, pe, t_all = bg.count_all()
            pu, pl, pe = as_u64(pu), as_u64(pl), as_u64(pe)
            pe2, t_e = bg.count_edges()
            pe2 = as_u64(pe2)
        finally:
            bg.release()
        del off, adj
        torch.cuda.empty_cache()
        # Lemma 4: Algorithm 3 processes the same wedges and finds the same total
        alt = run_gpu(g, options=bfc.bfc_options_init(orientation=1))
        torch.cuda.empty_cache()
    finally:
        th.join()
    if failure:
        raise failure[0]
    assert tot > 0 and t_all == tot and t_e == tot
    assert alt["total"] == tot and alt["info"]["wedges"] == W
    # element by element against the oracle
    assert tot == ref["total"] and W == ref["wedges"]
    assert np.array_equal(pu, ref["pv_u"]) and np.array_equal(pl, ref["pv_l"])
    assert np.array_equal(pe, ref["pe"]) and np.array_equal(pe2, ref["pe"])
    # identities (uint64 sums wrap like the counts; the totals stay far below 2^64)
    assert int(pu.sum(dtype=np.uint64)) == 2 * tot
    assert int(pl.sum(dtype=np.uint64)) == 2 * tot
    assert int(pe.sum(dtype=np.uint64)) == 4 * tot
    # sampled outputs, one by one from the definitions (Eq. 1, Eq. 7)
    deg_u = np.diff(g.off_u.astype(np.int64))
    deg_l = np.bincount(g.adj_u, minlength=g.num_l)
    rng = np.random.default_rng(7)
    xs = _sample(rng, g.num_u, 8, [int(np.argmax(deg_u))])
    ys = _sample(rng, g.num_l, 4, [int(np.argmax(deg_l))])
    top_item_edge = int(np.flatnonzero(g.adj_u == int(np.argmax(deg_l)))[0])
    es = _sample(rng, g.num_edges, 8, [top_item_edge, int(g.off_u[int(np.argmax(deg_u))])])
    assert np.array_equal(pu[xs], oracle.vertices_sampled(g, 0, xs))
    assert np.array_equal(pl[ys], oracle.vertices_sampled(g, 1, ys))
    assert np.array_equal(pe[es], oracle.edges_sampled(g, es))
