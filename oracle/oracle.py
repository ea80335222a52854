"""Python front end of the CPU oracle (``bfc_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline arm of ``bench.py``; the product package never imports
it, and it never imports the product package.

Besides binding the C routines, this module holds the smallest oracle of all:
:func:`enumerate_butterflies`, which lists every (2,2)-biclique of a tiny graph
straight from Definition 2.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading
import types
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfc_oracle.c")
_LIB = os.path.join(_HERE, "libbfc_oracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libbfc_oracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "bfc_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            c = ctypes
            sig = {
                "orc_brute_total": [c.c_int32, c.c_int32, _i32p, _i32p, c.c_int, _u64p],
                "orc_brute_vertices": [c.c_int32, c.c_int32, _i32p, _i32p, _u64p, _u64p],
                "orc_brute_edges": [c.c_int32, c.c_int32, _i32p, _i32p, _u64p],
                "orc_vertices_sampled": [c.c_int32, c.c_int32, _i32p, _i32p, c.c_int, _i32p,
                                         c.c_int64, _u64p],
                "orc_edges_sampled": [c.c_int32, c.c_int32, _i32p, _i32p, _i64p, c.c_int64, _u64p],
                "orc_ibs": [c.c_int32, c.c_int32, _i32p, _i32p, _u64p, _u64p, c.POINTER(c.c_int)],
                "orc_priority": [c.c_int32, c.c_int32, _i32p, _i32p, _i32p, _i32p, _i32p],
                "orc_projection": [c.c_int32, c.c_int32, _i32p, _i32p, _i64p, _i32p, _i32p,
                                   _i32p, _u64p],
                "orc_vp": [c.c_int32, c.c_int32, _i32p, _i32p, c.c_int, _u64p, _u64p, _u64p,
                           _u64p, _u64p],
                "orc_vppp": [c.c_int32, c.c_int32, _i32p, _i32p, _u64p, _u64p],
                "orc_degree_stats": [c.c_int32, c.c_int32, _i32p, _i32p, _u64p, _u64p, _u64p],
                "orc_caterpillars": [c.c_int32, c.c_int32, _i32p, _i32p, _u64p],
                "orc_pairs_total": [c.c_int32, c.c_int32, _i32p, _i32p, _u64p, _u64p],
                "orc_vp_chunked": [c.c_int32, c.c_int32, _i32p, _i32p, c.c_int32, _u64p],
                "orc_vp_core_split": [c.c_int32, c.c_int32, _i32p, _i32p, c.c_int32, _u64p, _u64p, _u64p,
                                      _u64p],
                "orc_sparsify": [c.c_int32, c.c_int32, _i32p, _i32p, c.c_uint64, c.c_uint64,
                                 c.c_uint64, c.c_int, _i32p, _i32p, _i64p],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = c.c_int
            lib.orc_splitmix64.argtypes = [c.c_uint64, c.c_uint64]
            lib.orc_splitmix64.restype = c.c_uint64
            _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t) if a is not None else None


def _csr(g):
    off = np.ascontiguousarray(g.off_u, dtype=np.int32)
    adj = np.ascontiguousarray(g.adj_u, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)
    return off, adj


def _check(rc: int, what: str):
    if rc == -1:
        raise ValueError(f"{what}: malformed graph")
    if rc != 0:
        raise MemoryError(f"{what}: failed ({rc})")


def brute_total(g, pair_layer: int = 0) -> int:
    """Definition 2 / Lemma 1: Σ over vertex pairs of one layer of C(common, 2)."""
    off, adj = _csr(g)
    out = np.zeros(1, dtype=np.uint64)
    _check(_load().orc_brute_total(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p),
                                   pair_layer, _p(out, _u64p)), "brute_total")
    return int(out[0])


def brute_vertices(g) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 1 for every vertex: (per-U, per-L) uint64 arrays."""
    off, adj = _csr(g)
    pu = np.zeros(max(g.num_u, 1), dtype=np.uint64)
    pl = np.zeros(max(g.num_l, 1), dtype=np.uint64)
    _check(_load().orc_brute_vertices(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p),
                                      _p(pu, _u64p), _p(pl, _u64p)), "brute_vertices")
    return pu[:g.num_u], pl[:g.num_l]


def brute_edges(g) -> np.ndarray:
    """Eq. 7 for every edge, U-side slot order."""
    off, adj = _csr(g)
    pe = np.zeros(max(g.num_edges, 1), dtype=np.uint64)
    _check(_load().orc_brute_edges(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p),
                                   _p(pe, _u64p)), "brute_edges")
    return pe[:g.num_edges]


def vertices_sampled(g, layer: int, xs) -> np.ndarray:
    """Eq. 1 for the listed vertices of one layer (0 = U, 1 = L), by counting
    two-hop paths; for graphs too large for the full oracle."""
    off, adj = _csr(g)
    xs = np.ascontiguousarray(np.asarray(xs, dtype=np.int32))
    out = np.zeros(max(xs.size, 1), dtype=np.uint64)
    _check(_load().orc_vertices_sampled(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p), int(layer),
                                        _p(xs, _i32p), xs.size, _p(out, _u64p)), "vertices_sampled")
    return out[:xs.size]


def edges_sampled(g, es) -> np.ndarray:
    """Eq. 7 for the listed edges (U-side slots)."""
    off, adj = _csr(g)
    es = np.ascontiguousarray(np.asarray(es, dtype=np.int64))
    out = np.zeros(max(es.size, 1), dtype=np.uint64)
    _check(_load().orc_edges_sampled(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p),
                                     _p(es, _i64p), es.size, _p(out, _u64p)), "edges_sampled")
    return out[:es.size]


def ibs(g) -> tuple[int, int, int]:
    """Algorithm 1: (total, wedges passing the id filter, start layer 0=U/1=L)."""
    off, adj = _csr(g)
    t = np.zeros(1, dtype=np.uint64)
    w = np.zeros(1, dtype=np.uint64)
    layer = ctypes.c_int(0)
    _check(_load().orc_ibs(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p), _p(t, _u64p),
                           _p(w, _u64p), ctypes.byref(layer)), "ibs")
    return int(t[0]), int(w[0]), int(layer.value)


def priority(g) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Definition 3 / 4: (rank_u[r], rank_l[l], p[n] indexed by gid)."""
    off, adj = _csr(g)
    ru = np.zeros(max(g.num_u, 1), dtype=np.int32)
    rl = np.zeros(max(g.num_l, 1), dtype=np.int32)
    pr = np.zeros(max(g.num_u + g.num_l, 1), dtype=np.int32)
    _check(_load().orc_priority(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p),
                                _p(ru, _i32p), _p(rl, _i32p), _p(pr, _i32p)), "priority")
    return ru[:g.num_u], rl[:g.num_l], pr[:g.num_u + g.num_l]


def projection(g) -> dict:
    """The projection graph G* with ascending-priority lists, cut and work."""
    off, adj = _csr(g)
    n, m = g.num_u + g.num_l, g.num_edges
    poff = np.zeros(n + 1, dtype=np.int64)
    padj = np.zeros(max(2 * m, 1), dtype=np.int32)
    peid = np.zeros(max(2 * m, 1), dtype=np.int32)
    cut = np.zeros(max(n, 1), dtype=np.int32)
    work = np.zeros(max(n, 1), dtype=np.uint64)
    _check(_load().orc_projection(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p),
                                  _p(poff, _i64p), _p(padj, _i32p), _p(peid, _i32p),
                                  _p(cut, _i32p), _p(work, _u64p)), "projection")
    return dict(off=poff, adj=padj[:2 * m], eid=peid[:2 * m], cut=cut[:n], work=work[:n])


def vp(g, threads: int = 0, vertices: bool = False, edges: bool = False) -> dict:
    """Algorithm 2 scheduled as Algorithm 5.  Returns total, wedges and, on
    request, per-vertex (pv_u, pv_l) and per-edge (pe) counts."""
    off, adj = _csr(g)
    t = np.zeros(1, dtype=np.uint64)
    w = np.zeros(1, dtype=np.uint64)
    pu = np.zeros(max(g.num_u, 1), dtype=np.uint64) if vertices else None
    pl = np.zeros(max(g.num_l, 1), dtype=np.uint64) if vertices else None
    pe = np.zeros(max(g.num_edges, 1), dtype=np.uint64) if edges else None
    _check(_load().orc_vp(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p), int(threads),
                          _p(t, _u64p), _p(w, _u64p), _p(pu, _u64p), _p(pl, _u64p),
                          _p(pe, _u64p)), "vp")
    out = dict(total=int(t[0]), wedges=int(w[0]))
    if vertices:
        out["pv_u"], out["pv_l"] = pu[:g.num_u], pl[:g.num_l]
    if edges:
        out["pe"] = pe[:g.num_edges]
    return out


def vppp(g) -> tuple[int, int]:
    """Algorithm 3: (total, processed wedges)."""
    off, adj = _csr(g)
    t = np.zeros(1, dtype=np.uint64)
    w = np.zeros(1, dtype=np.uint64)
    _check(_load().orc_vppp(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p), _p(t, _u64p),
                            _p(w, _u64p)), "vppp")
    return int(t[0]), int(w[0])


def degree_stats(g) -> tuple[int, int, int]:
    """(Σ_E min(deg u, deg v), Σ_U deg², Σ_L deg²) — the quantities of Lemma 3."""
    off, adj = _csr(g)
    a = np.zeros(3, dtype=np.uint64)
    _check(_load().orc_degree_stats(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p),
                                    _p(a[0:], _u64p), _p(a[1:], _u64p), _p(a[2:], _u64p)),
           "degree_stats")
    return int(a[0]), int(a[1]), int(a[2])


def vp_chunked(g, chunk: int) -> int:
    """Algorithm 2 with each start's end set split into priority ranges of
    `chunk`, each counted separately (tiny graphs)."""
    off, adj = _csr(g)
    a = np.zeros(1, dtype=np.uint64)
    _check(_load().orc_vp_chunked(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p), int(chunk),
                                  _p(a, _u64p)), "vp_chunked")
    return int(a[0])


def vp_core_split(g, K: int) -> tuple[int, int, int, int]:
    """Algorithm 2 with the top-K priority core counted apart (tiny graphs):
    (total, wedges skipped by the walk, Σ C(a_uw, 2) and Σ a_uw·b_uw over
    core pairs)."""
    off, adj = _csr(g)
    a = np.zeros(4, dtype=np.uint64)
    _check(_load().orc_vp_core_split(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p), int(K),
                                     _p(a[0:], _u64p), _p(a[1:], _u64p), _p(a[2:], _u64p),
                                     _p(a[3:], _u64p)), "vp_core_split")
    return int(a[0]), int(a[1]), int(a[2]), int(a[3])


def pairs_total(g) -> tuple[int, int]:
    """Section 6.3's pair formulation in memory: (total, pairs written)."""
    off, adj = _csr(g)
    a = np.zeros(2, dtype=np.uint64)
    _check(_load().orc_pairs_total(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p), _p(a[0:], _u64p),
                                   _p(a[1:], _u64p)), "pairs_total")
    return int(a[0]), int(a[1])


def caterpillars(g) -> int:
    """Three-paths of the graph: Σ over edges of (deg u − 1)(deg v − 1)."""
    off, adj = _csr(g)
    a = np.zeros(1, dtype=np.uint64)
    _check(_load().orc_caterpillars(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p), _p(a, _u64p)),
           "caterpillars")
    return int(a[0])


def enumerate_three_paths(g) -> int:
    """Three-paths a-b-c-d (three distinct edges, a path read either way counted
    once) by walking every path from every vertex, for tiny graphs."""
    if g.num_u > 60 or g.num_l > 60:
        raise ValueError("exhaustive enumeration is for tiny graphs only")
    u, v = g.edges()
    nbr = {}
    for a, b in zip(u.tolist(), v.tolist()):
        nbr.setdefault(("U", a), set()).add(("L", b))
        nbr.setdefault(("L", b), set()).add(("U", a))
    paths = set()
    for a in nbr:
        for b in nbr[a]:
            for c in nbr[b]:
                if c == a:
                    continue
                for d in nbr[c]:
                    if d == b:
                        continue
                    p = (a, b, c, d)
                    paths.add(min(p, p[::-1]))
    return len(paths)


def enumerate_butterflies(g) -> dict:
    """Definition 2 taken literally, for tiny graphs: every choice of two U
    vertices and two L vertices that are joined by all four edges is one
    butterfly.  Returns the total and the per-vertex and per-edge counts."""
    if g.num_u > 40 or g.num_l > 40:
        raise ValueError("exhaustive enumeration is for tiny graphs only")
    u_of, v_of = g.edges()
    slot = {(int(a), int(b)): k for k, (a, b) in enumerate(zip(u_of, v_of))}
    total = 0
    pv_u = np.zeros(g.num_u, dtype=np.uint64)
    pv_l = np.zeros(g.num_l, dtype=np.uint64)
    pe = np.zeros(g.num_edges, dtype=np.uint64)
    for u1, u2 in itertools.combinations(range(g.num_u), 2):
        for v1, v2 in itertools.combinations(range(g.num_l), 2):
            es = [(u1, v1), (u1, v2), (u2, v1), (u2, v2)]
            if all(e in slot for e in es):
                total += 1
                pv_u[u1] += 1; pv_u[u2] += 1; pv_l[v1] += 1; pv_l[v2] += 1
                for e in es:
                    pe[slot[e]] += 1
    return dict(total=total, pv_u=pv_u, pv_l=pv_l, pe=pe)


# ---------------------------------------------------------------------------
# Approximate counting by edge sparsification (Section 7)
# ---------------------------------------------------------------------------

def splitmix64(seed: int, k: int) -> int:
    """The k-th output (k >= 1) of SplitMix64 seeded with `seed` (C routine)."""
    return int(_load().orc_splitmix64(seed & (2**64 - 1), k & (2**64 - 1)))


def keep_threshold(p: float) -> tuple[int, bool]:
    """(floor(p * 2^64), keep_all) for a keep probability 0 < p <= 1, in exact
    rational arithmetic."""
    if not (0.0 < p <= 1.0):
        raise ValueError("keep probability must lie in (0, 1]")
    if p == 1.0:
        return 0, True
    return int(Fraction(p) * 2**64), False


def sparsify(g, p: float, seed: int, j: int):
    """Sample j of graph g: every edge kept independently with probability p
    (the keep rule of ``orc_sparsify``).  Returns a graph with the same vertex
    sets and the kept edges (in their original order)."""
    off, adj = _csr(g)
    t, keep_all = keep_threshold(p)
    m = max(g.num_edges, 1)
    oo = np.zeros(g.num_u + 1, dtype=np.int32)
    oa = np.zeros(m, dtype=np.int32)
    kept = np.zeros(1, dtype=np.int64)
    _check(_load().orc_sparsify(g.num_u, g.num_l, _p(off, _i32p), _p(adj, _i32p), seed & (2**64 - 1),
                                int(j), t, int(keep_all), _p(oo, _i32p), _p(oa, _i32p),
                                _p(kept, _i64p)), "sparsify")
    k = int(kept[0])
    return types.SimpleNamespace(num_u=g.num_u, num_l=g.num_l, num_edges=k, off_u=oo,
                                 adj_u=oa[:k].copy())


def sparsified_estimate(g, p: float, seed: int, samples: int, threads: int = 0) -> dict:
    """The sampling estimator with the exact counter as its inner block: each
    of `samples` sparsified graphs (sample j = ``sparsify(g, p, seed, j)``) is
    counted by Algorithm 2; a butterfly survives a sample iff its four edges
    do (probability p^4), so estimate = Σ_j ⋈(G_j) / (samples · p^4).
    std_error = the sample standard deviation of ⋈(G_j) / p^4 over
    sqrt(samples) (NaN for one sample)."""
    if samples < 1:
        raise ValueError("at least one sample")
    counts, edges = [], []
    for j in range(samples):
        h = sparsify(g, p, seed, j)
        counts.append(vp(h, threads=threads)["total"])
        edges.append(h.num_edges)
    p4 = p ** 4
    est = float(sum(counts)) / (samples * p4)
    if samples > 1:
        mean = sum(counts) / samples
        var = sum((c - mean) ** 2 for c in counts) / (samples - 1)
        se = (var / samples) ** 0.5 / p4
    else:
        se = float("nan")
    return dict(counts=counts, edges=edges, estimate=est, std_error=se)
