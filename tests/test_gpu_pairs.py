"""Section 6.3's pair formulation on the GPU (bfc_count_pairs): every wedge
of the prepared orientation becomes the key (start, end), a radix sort groups
equal keys and a run of c keys adds C(c, 2).  ⋈_G against the oracle for
both orientations, with and without the dense core, and against the walk."""
import pytest

import oracle
from bfc_inputs import generators as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


GRAPHS = [lambda: G.complete_bipartite(7, 11), lambda: G.paper_fig3(), lambda: G.cycle(5),
          lambda: G.from_edges(4, 3, [], []), lambda: G.uniform_small(),
          lambda: G.chung_lu_bipartite(20000, 8000, 150000, 2.1, 2.0, 48),
          lambda: G.chung_lu_bipartite(30000, 3000, 200000, 2.5, 1.8, 11)]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("orientation", [0, 1])
def test_pairs_total_matches_oracle(gi, orientation):
    from paper_1812_00283_gb300 import ButterflyGraph, bfc
    g = GRAPHS[gi]()
    ref = oracle.vp(g)["total"]
    adj = torch.from_numpy(g.adj_u).cuda() if g.num_edges else torch.zeros(0, dtype=torch.int32).cuda()
    bg = ButterflyGraph(torch.from_numpy(g.off_u).cuda(), adj, g.num_u, g.num_l,
                        bfc.bfc_options_init(orientation=orientation))
    try:
        assert bg.count_pairs() == ref
        assert bg.count() == ref
        assert bg.count_pairs() == ref   # again, after a walk on the same graph
    finally:
        bg.release()


def test_pairs_powerlaw_20m():
    from paper_1812_00283_gb300 import ButterflyGraph
    g = G.powerlaw_20m(device="cuda")
    bg = ButterflyGraph(torch.from_numpy(g.off_u).cuda(), torch.from_numpy(g.adj_u).cuda(), g.num_u, g.num_l)
    try:
        total = bg.count_pairs()
    finally:
        bg.release()
    assert total == oracle.vp(g)["total"]
