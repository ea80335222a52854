"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the pins catch each one.  The real oracle source is never modified."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from bfc_inputs import generators as G
import oracle

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "bfc_oracle.c")

MUTANTS = {
    "end_filter_le": ("if (!(p[w] < p[u])) break;\n                    if (count_wedge[w] == 0)",
                      "if (!(p[w] <= p[u])) break;\n                    if (count_wedge[w] == 0)"),
    "middle_filter_flipped": ("if (!(p[v] < p[u])) break;           /* sorted",
                              "if (!(p[v] > p[u])) continue;           /* sorted"),
    "choose2_off_by_one": ("return c < 2 ? 0 : c * (c - 1) / 2;", "return c < 2 ? 0 : c * (c + 1) / 2;"),
    "priority_reversed": ("p[key[i] & 0xffffffffLL] = i + 1;", "p[key[i] & 0xffffffffLL] = n - i;"),
    "edge_delta_off": ("uint64_t delta = (uint64_t)count_wedge[w] - 1;",
                       "uint64_t delta = (uint64_t)count_wedge[w];"),
    "edge_uv_dropped": ("pe[g.eid[i]] += sum;", "pe[g.eid[i]] += 0;"),
    "vertex_end_dropped": ("pv[w] += c2;", "pv[w] += 0;"),
    "middle_vertex_dropped": ("pv[v] += sum;", "pv[v] += 0;"),
    "priority_ignores_degree": ("key[x] = ((int64_t)g->deg[x] << 32) | (int64_t)x;",
                                "key[x] = (int64_t)x;"),
}


def _build_mutant(name, tmp_path):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    src = src.replace(old, new)
    d = tmp_path / name
    d.mkdir()
    c = d / "m.c"
    c.write_text(src)
    so = d / "m.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-I",
                    os.path.dirname(SRC), "-o", str(so), str(c)], check=True)
    lib = ctypes.CDLL(str(so))
    return lib


def _vp(lib, g):
    i32 = ctypes.POINTER(ctypes.c_int32)
    u64 = ctypes.POINTER(ctypes.c_uint64)
    off = np.ascontiguousarray(g.off_u, dtype=np.int32)
    adj = np.ascontiguousarray(g.adj_u if g.num_edges else np.zeros(1, np.int32), dtype=np.int32)
    t = np.zeros(1, np.uint64); w = np.zeros(1, np.uint64)
    pu = np.zeros(max(g.num_u, 1), np.uint64); pl = np.zeros(max(g.num_l, 1), np.uint64)
    pe = np.zeros(max(g.num_edges, 1), np.uint64)
    lib.orc_vp.restype = ctypes.c_int
    rc = lib.orc_vp(ctypes.c_int32(g.num_u), ctypes.c_int32(g.num_l), off.ctypes.data_as(i32),
                    adj.ctypes.data_as(i32), ctypes.c_int(1), t.ctypes.data_as(u64),
                    w.ctypes.data_as(u64), pu.ctypes.data_as(u64), pl.ctypes.data_as(u64),
                    pe.ctypes.data_as(u64))
    assert rc == 0
    return dict(total=int(t[0]), wedges=int(w[0]), pv_u=pu[:g.num_u], pv_l=pl[:g.num_l],
                pe=pe[:g.num_edges])


def _pins_pass(lib) -> bool:
    """The subset of the oracle pins that exercise orc_vp."""
    for a, b in [(3, 5), (4, 4), (6, 2)]:
        r = _vp(lib, G.complete_bipartite(a, b))
        x, y = (a, b) if b >= a else (b, a)
        if r["total"] != (a * (a - 1) // 2) * (b * (b - 1) // 2):
            return False
        if r["wedges"] != y * x * (x - 1) // 2:
            return False
        if not (np.all(r["pv_u"] == (a - 1) * (b * (b - 1) // 2)) and np.all(r["pe"] == (a - 1) * (b - 1))):
            return False
    for g, (tot, wed) in [(G.paper_fig2a(), (0, 2000)), (G.paper_fig3(), (999000, 2000))]:
        r = _vp(lib, g)
        if (r["total"], r["wedges"]) != (tot, wed):
            return False
    for seed in range(40):
        g = G.random_tiny(2 + seed % 5, 2 + (seed // 5) % 5, 2, 3, seed)
        ref = oracle.enumerate_butterflies(g)
        r = _vp(lib, g)
        if r["total"] != ref["total"] or not np.array_equal(r["pe"], ref["pe"]) \
                or not np.array_equal(r["pv_u"], ref["pv_u"]) or not np.array_equal(r["pv_l"], ref["pv_l"]):
            return False
    # Definition 3 order printed in Section 4, Example 1 (Figure 3)
    g = G.paper_fig3()
    return _fig3_order_ok(lib, g)


def _fig3_order_ok(lib, g):
    i32 = ctypes.POINTER(ctypes.c_int32)
    off = np.ascontiguousarray(g.off_u, dtype=np.int32)
    adj = np.ascontiguousarray(g.adj_u, dtype=np.int32)
    ru = np.zeros(g.num_u, np.int32); rl = np.zeros(g.num_l, np.int32)
    p = np.zeros(g.num_u + g.num_l, np.int32)
    rc = lib.orc_priority(ctypes.c_int32(g.num_u), ctypes.c_int32(g.num_l), off.ctypes.data_as(i32),
                          adj.ctypes.data_as(i32), ru.ctypes.data_as(i32), rl.ctypes.data_as(i32),
                          p.ctypes.data_as(i32))
    assert rc == 0
    n, l = g.num_u + g.num_l, g.num_l
    return p[l + 1] == n and p[l + 0] == n - 1 and p[1001] == n - 2 and p[1000] == n - 3 \
        and p[0] == 1 and p[1] == 2


def test_unmutated_copy_passes(tmp_path):
    src = open(SRC).read()
    d = tmp_path / "orig"
    d.mkdir()
    (d / "m.c").write_text(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-I",
                    os.path.dirname(SRC), "-o", str(d / "m.so"), str(d / "m.c")], check=True)
    assert _pins_pass(ctypes.CDLL(str(d / "m.so")))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    lib = _build_mutant(name, tmp_path)
    assert not _pins_pass(lib), f"planted mistake {name} went unnoticed"


# ---------------------------------------------------------------------------
# The second exact paths: split end ranges, the core split, the pair formulation
# ---------------------------------------------------------------------------

EXTRA_MUTANTS = {
    "core_cross_dropped": [("t += aw * (uint64_t)b[w] + aw * (aw - 1) / 2;", "t += aw * (aw - 1) / 2;")],
    # skips core-start, core-middle wedges whatever their end: the total
    # survives (any split of the middles adds up), the skipped count does not
    "core_skip_ignores_end": [("if (cu && cv && p[w] > n - K) {", "if (cu && cv) {")],
    "core_running_form_after_increment": [("t += b[w];       /* running form", "t += b[w] + 1;   /* running form")],
    "chunk_boundary_inclusive": [("p[w] >= lo && p[w] < hi)", "p[w] >= lo && p[w] <= hi)")],
    "pairs_include_self": [("if (p[g.adj[j]] < p[w]) ++np;", "if (p[g.adj[j]] <= p[w]) ++np;"),
                           ("if (p[u] < p[w]) key[k++]", "if (p[u] <= p[w]) key[k++]")],
    "pairs_run_off_by_one": [("t += run - 1;", "t += run;")],
}


def _build_extra(name, tmp_path):
    src = open(SRC).read()
    for old, new in EXTRA_MUTANTS[name]:
        assert src.count(old) == 1, f"mutation site for {name} not found once"
        src = src.replace(old, new)
    d = tmp_path / name
    d.mkdir()
    (d / "m.c").write_text(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-I",
                    os.path.dirname(SRC), "-o", str(d / "m.so"), str(d / "m.c")], check=True)
    return ctypes.CDLL(str(d / "m.so"))


def _csr_args(g):
    i32 = ctypes.POINTER(ctypes.c_int32)
    off = np.ascontiguousarray(g.off_u, dtype=np.int32)
    adj = np.ascontiguousarray(g.adj_u if g.num_edges else np.zeros(1, np.int32), dtype=np.int32)
    return (off, adj), (ctypes.c_int32(g.num_u), ctypes.c_int32(g.num_l), off.ctypes.data_as(i32),
                        adj.ctypes.data_as(i32))


def _core_wedges(g, K):
    """Wedges of Algorithm 2 with start, middle and end among the top-K by
    priority, counted from the edge list (priorities from the real oracle)."""
    _, _, p = oracle.priority(g)
    l, n = g.num_l, g.num_u + g.num_l
    core = p > n - K
    u = np.repeat(np.arange(g.num_u), np.diff(g.off_u.astype(np.int64))) + l
    v = g.adj_u.astype(np.int64)
    keep = core[u] & core[v]
    mid = np.concatenate([u[keep], v[keep]]); nb = np.concatenate([v[keep], u[keep]])
    o = np.lexsort((p[nb], mid)); mid, nb = mid[o], nb[o]
    idx = np.arange(mid.size) - np.searchsorted(mid, mid, side="left")
    return int(idx[p[nb] > p[mid]].sum())


def _extra_pins_pass(lib) -> bool:
    u64 = ctypes.POINTER(ctypes.c_uint64)
    graphs = [G.complete_bipartite(4, 6), G.complete_bipartite(5, 7),
              G.chung_lu_bipartite(120, 80, 1200, 2.1, 2.1, 4), G.uniform_bipartite(60, 40, 500, 3),
              G.random_tiny(9, 8, 3, 6, 17)]
    for g in graphs:
        ref = oracle.vp(g)
        n = g.num_u + g.num_l
        keep, args = _csr_args(g)
        for K in (n // 4, n // 2, n):
            out = np.zeros(4, np.uint64)
            rc = lib.orc_vp_core_split(*args, ctypes.c_int32(K), *(out[i:].ctypes.data_as(u64) for i in range(4)))
            if rc != 0 or int(out[0]) != ref["total"] or int(out[1]) != _core_wedges(g, K):
                return False
        for chunk in (2, 3):
            out = np.zeros(1, np.uint64)
            rc = lib.orc_vp_chunked(*args, ctypes.c_int32(chunk), out.ctypes.data_as(u64))
            if rc != 0 or int(out[0]) != ref["total"]:
                return False
        out = np.zeros(2, np.uint64)
        rc = lib.orc_pairs_total(*args, out[0:].ctypes.data_as(u64), out[1:].ctypes.data_as(u64))
        if rc != 0 or (int(out[0]), int(out[1])) != (ref["total"], ref["wedges"]):
            return False
    return True


def test_unmutated_copy_passes_extra_pins(tmp_path):
    d = tmp_path / "orig"
    d.mkdir()
    (d / "m.c").write_text(open(SRC).read())
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-I",
                    os.path.dirname(SRC), "-o", str(d / "m.so"), str(d / "m.c")], check=True)
    assert _extra_pins_pass(ctypes.CDLL(str(d / "m.so")))


@pytest.mark.parametrize("name", sorted(EXTRA_MUTANTS))
def test_extra_mutant_is_caught(name, tmp_path):
    assert not _extra_pins_pass(_build_extra(name, tmp_path)), f"planted mistake {name} went unnoticed"
