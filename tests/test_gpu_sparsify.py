"""Approximate counting by edge sparsification on the GPU (Section 7's
estimator with the exact counter as its inner block), against the oracle.

* Every sample's exact count and kept edges, bit for bit, against the oracle
  sampling with the same keep rule (SplitMix64 per sample and edge), over
  keep probabilities from 0.02 to 1, several seeds and sample counts, rows
  shorter and longer than a warp, and the empty graph.
* The estimate and its standard error against the oracle's (double).
* The prepared samples: wedges per sample and in total against the oracle.
* The 20M-edge power-law graph at the bench's setting (p = 0.1, 16 samples),
  every sample against the oracle.
* Invalid arguments and malformed graphs give errors, not faults.
"""
import math

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


def _dev(g):
    return (torch.from_numpy(np.ascontiguousarray(g.off_u)).cuda(),
            torch.from_numpy(np.ascontiguousarray(g.adj_u) if g.num_edges else np.zeros(1, np.int32)).cuda())


def _gpu(g, p, seed, samples):
    from paper_1812_00283_gb300 import bfc
    off, adj = _dev(g)
    s = torch.cuda.current_stream()
    edges = torch.zeros(samples, dtype=torch.int64, device="cuda")
    h = bfc.bfc_prepare_sparsified(g.num_u, g.num_l, g.num_edges, off.data_ptr(), adj.data_ptr(), p, seed,
                                   samples, None, s.cuda_stream, edges.data_ptr())
    try:
        counts = torch.zeros(samples, dtype=torch.int64, device="cuda")
        wed = torch.zeros(samples, dtype=torch.int64, device="cuda")
        est = torch.zeros(2, dtype=torch.float64, device="cuda")
        bfc.bfc_count_batch(h, s.cuda_stream, counts.data_ptr())
        bfc.bfc_batch_wedges(h, s.cuda_stream, wed.data_ptr())
        bfc.bfc_sparsified_estimate(counts.data_ptr(), samples, p, s.cuda_stream, est.data_ptr())
        bfc.bfc_sync(h, s.cuda_stream)
        info = bfc.bfc_graph_info(h)
    finally:
        bfc.bfc_release(h)
    u64 = lambda t: [int(x) for x in t.cpu().numpy().view(np.uint64)]
    e = est.cpu().tolist()
    return dict(counts=u64(counts), edges=u64(edges), wedges=u64(wed), estimate=e[0], std_error=e[1],
                info=info)


def _oracle(g, p, seed, samples):
    r = oracle.sparsified_estimate(g, p, seed, samples)
    r["wedges"] = [oracle.vp(oracle.sparsify(g, p, seed, j))["wedges"] for j in range(samples)]
    return r


def _graphs():
    return [G.complete_bipartite(9, 14), G.paper_fig3(), G.uniform_small(),
            G.chung_lu_bipartite(4000, 2500, 30000, 2.1, 2.1, 7),
            G.chung_lu_bipartite(3000, 20000, 120000, 2.1, 2.1, 31, max_u=9000),
            G.from_edges(6, 4, [], [])]


CASES = [(0, 0.5, 3, 16), (0, 1.0, 0, 2), (1, 0.3, 2**63 + 9, 5), (2, 0.1, 42, 16), (2, 0.77, 1, 1),
         (3, 0.02, 5, 7), (3, 0.25, 6, 32), (4, 0.05, 2**64 - 1, 9), (4, 0.6, 17, 3), (5, 0.5, 1, 4)]


@pytest.mark.parametrize("gi,p,seed,samples", CASES)
def test_samples_match_oracle(gi, p, seed, samples):
    g = _graphs()[gi]
    got = _gpu(g, p, seed, samples)
    ref = _oracle(g, p, seed, samples)
    assert got["edges"] == ref["edges"]
    assert got["counts"] == ref["counts"]
    assert got["wedges"] == ref["wedges"]
    assert got["info"]["wedges"] == sum(ref["wedges"])
    assert got["info"]["num_edges"] == sum(ref["edges"])
    assert got["info"]["num_u"] == samples * g.num_u and got["info"]["num_l"] == samples * g.num_l
    assert got["estimate"] == pytest.approx(ref["estimate"], rel=1e-12, abs=0)
    if samples == 1:
        assert math.isnan(got["std_error"])
    else:
        assert got["std_error"] == pytest.approx(ref["std_error"], rel=1e-9, abs=1e-12)


def test_one_call_entry_point_and_package_api():
    from paper_1812_00283_gb300 import estimate_butterflies
    g = G.chung_lu_bipartite(4000, 2500, 30000, 2.1, 2.1, 7)
    ref = oracle.sparsified_estimate(g, 0.4, 99, 12)
    off, adj = _dev(g)
    r = estimate_butterflies(off, adj, g.num_u, g.num_l, 0.4, 12, seed=99)
    assert [int(x) for x in r["counts"].cpu().numpy().view(np.uint64)] == ref["counts"]
    assert r["estimate"] == pytest.approx(ref["estimate"], rel=1e-12)
    assert r["std_error"] == pytest.approx(ref["std_error"], rel=1e-9)
    # p = 1: every sample is the graph itself
    exact = oracle.vp(g)["total"]
    r1 = estimate_butterflies(off, adj, g.num_u, g.num_l, 1.0, 3, seed=5)
    assert [int(x) for x in r1["counts"].cpu()] == [exact] * 3
    assert r1["estimate"] == float(exact) and r1["std_error"] == 0.0


def test_powerlaw_20m_bench_setting_against_oracle():
    # the 20M-edge power-law graph, p = 0.1, 16 samples (the bench's setting)
    g = G.powerlaw_20m(device="cuda")
    got = _gpu(g, 0.1, 7, 16)
    ref = _oracle(g, 0.1, 7, 16)
    assert got["edges"] == ref["edges"] and got["counts"] == ref["counts"]
    assert got["wedges"] == ref["wedges"]
    assert got["estimate"] == pytest.approx(ref["estimate"], rel=1e-12)
    assert got["std_error"] == pytest.approx(ref["std_error"], rel=1e-9)


def test_errors_are_reported():
    from paper_1812_00283_gb300 import bfc
    g = G.complete_bipartite(5, 6)
    off, adj = _dev(g)
    s = torch.cuda.current_stream().cuda_stream
    counts = torch.zeros(4, dtype=torch.int64, device="cuda")

    def run(p=0.5, samples=4, off_t=off, adj_t=adj, num_u=g.num_u, num_l=g.num_l):
        bfc.bfc_estimate_sparsified(num_u, num_l, g.num_edges, off_t.data_ptr(), adj_t.data_ptr(), p, 1,
                                    samples, None, s, counts.data_ptr(), None)

    for p in (0.0, -0.1, 1.5, float("nan")):
        with pytest.raises(bfc.BfcError) as e:
            run(p=p)
        assert e.value.status == 1
    for samples in (0, -3, 2**30):
        with pytest.raises(bfc.BfcError) as e:
            run(samples=samples)
        assert e.value.status == 1
    bad_off = off.clone()
    bad_off[2] = bad_off[3] + 1
    with pytest.raises(bfc.BfcError) as e:
        run(off_t=bad_off)
    assert e.value.status == 2
    bad_adj = adj.clone()
    bad_adj[4] = g.num_l + 3
    with pytest.raises(bfc.BfcError) as e:
        run(adj_t=bad_adj)
    assert e.value.status == 2
    # still usable afterwards
    run(p=1.0)
    assert [int(x) for x in counts.cpu()] == [oracle.vp(g)["total"]] * 4
