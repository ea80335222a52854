"""The disjoint-union batch layout (CPU only)."""
import numpy as np

import oracle
from bfc_inputs import generators as G


def test_union_batch_layout_and_additivity():
    graphs = [G.complete_bipartite(3, 4), G.from_edges(5, 2, [], []), G.cycle(2),
              G.uniform_bipartite(40, 30, 200, 3), G.chung_lu_bipartite(60, 50, 400, 2.1, 2.1, 4)]
    b = G.union_batch(graphs)
    assert b.num_graphs == len(graphs)
    u, v = b.union.edges()
    for i, g in enumerate(graphs):
        sl = slice(int(b.e_start[i]), int(b.e_start[i + 1]))
        assert np.all((u[sl] >= b.u_start[i]) & (u[sl] < b.u_start[i + 1]))
        assert np.all((v[sl] >= b.l_start[i]) & (v[sl] < b.l_start[i + 1]))
        gu, gv = g.edges()
        assert np.array_equal(u[sl] - b.u_start[i], gu) and np.array_equal(v[sl] - b.l_start[i], gv)
    # butterflies never span graphs of a disjoint union
    assert oracle.vp(b.union)["total"] == sum(oracle.vp(g)["total"] for g in graphs)
