"""Writes tests/golden/uniform_small.json from the CPU oracle only.

Run:  python tests/golden/make_golden.py
The graph is the integer-only uniform generator (|U| = 2,000, |L| = 3,000,
20,000 edges, seed 1001), so the stored values do not depend on libm.
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from bfc_inputs import generators as G  # noqa: E402


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.uint64).tobytes()).hexdigest()


def main():
    g = G.uniform_small()
    vp = oracle.vp(g, threads=1, vertices=True, edges=True)
    ibs_total, ibs_wedges, ibs_layer = oracle.ibs(g)
    tc_new, du2, dl2 = oracle.degree_stats(g)
    out = dict(
        graph=dict(name=g.name, num_u=g.num_u, num_l=g.num_l, num_edges=g.num_edges,
                   seed=1001, adj_sha256=hashlib.sha256(g.adj_u.tobytes()).hexdigest(),
                   off_sha256=hashlib.sha256(g.off_u.tobytes()).hexdigest()),
        total=vp["total"], vp_wedges=vp["wedges"], brute_total=oracle.brute_total(g, 0),
        ibs_total=ibs_total, ibs_wedges=ibs_wedges, ibs_start_layer=ibs_layer,
        tc_new=tc_new, sum_du2=du2, sum_dl2=dl2,
        pv_u_sha256=digest(vp["pv_u"]), pv_l_sha256=digest(vp["pv_l"]), pe_sha256=digest(vp["pe"]),
        pv_u_sum=int(vp["pv_u"].sum()), pe_sum=int(vp["pe"].sum()),
    )
    with open(os.path.join(HERE, "uniform_small.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
