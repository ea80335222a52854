"""Seeded synthetic bipartite graphs.

This module only draws inputs.  It holds none of the butterfly-counting
arithmetic, so both the CPU oracle and the CUDA path can be fed from it
without sharing any of the method's code.

Graph format (shared by every consumer)
---------------------------------------
A bipartite graph G(U, L, E) (paper Section 2) is given by its U-side CSR:

* ``num_u`` = r = |U|, ``num_l`` = l = |L|, ``num_edges`` = m.
* ``off_u``: int32[r + 1], non-decreasing, ``off_u[0] == 0``, ``off_u[r] == m``.
* ``adj_u``: int32[m]; ``adj_u[off_u[u]:off_u[u+1]]`` are the L-ids adjacent
  to u.  Ids are 0-based inside each layer.  Edges are distinct (E is a set).
* The edge stored at U-side slot k (``0 <= k < m``) has edge id k; per-edge
  outputs are indexed by that slot.

Random numbers
--------------
All draws come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: output i of stream s is ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)``.
It is implemented twice, once on numpy uint64 and once on torch int64 (with
logical shifts emulated), and the two must agree bit for bit; the torch
version runs on the GPU for the large configurations.

Chung-Lu weights use float64 ``pow`` on the host (numpy) and are quantised
to integers once; every draw after that is integer-only.  A different libm
on another machine can therefore change a few weights in their last bit, so
stored expected values are only ever kept for integer-only graphs (the
uniform generator and the closed-form families); parity tests on power-law
graphs run the oracle on the graph generated in the same process.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

_GOLD = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK64 = (1 << 64) - 1


def _to_i64(x: int) -> int:
    x &= _MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


# ---------------------------------------------------------------------------
# SplitMix64, numpy (uint64) and torch (int64) versions
# ---------------------------------------------------------------------------

def splitmix64_np(idx: np.ndarray, seed: int) -> np.ndarray:
    """Output ``idx`` of the SplitMix64 stream ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(_GOLD)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def _srl_t(x, k: int):
    return (x >> k) & ((1 << (64 - k)) - 1)


def splitmix64_torch(idx, seed: int):
    """Same stream as :func:`splitmix64_np`, on torch int64 (any device).

    The bit pattern of each int64 output equals the uint64 numpy output.
    """
    z = (idx + 1) * _to_i64(_GOLD) + _to_i64(seed)
    z = (z ^ _srl_t(z, 30)) * _to_i64(_M1)
    z = (z ^ _srl_t(z, 27)) * _to_i64(_M2)
    z = z ^ _srl_t(z, 31)
    return z


# ---------------------------------------------------------------------------
# Graph container
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class BipartiteCSR:
    """U-side CSR of a simple bipartite graph (see the module docstring)."""
    num_u: int
    num_l: int
    off_u: np.ndarray  # int32[r+1]
    adj_u: np.ndarray  # int32[m]
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def num_edges(self) -> int:
        return int(self.adj_u.shape[0])

    def edges(self) -> tuple[np.ndarray, np.ndarray]:
        """(u, v) arrays in U-side slot order."""
        deg = np.diff(self.off_u.astype(np.int64))
        u = np.repeat(np.arange(self.num_u, dtype=np.int64), deg)
        return u, self.adj_u.astype(np.int64)


def from_edges(num_u: int, num_l: int, u, v, name: str = "", sort_lists: bool = True,
               meta: Optional[dict] = None) -> BipartiteCSR:
    """Build a U-side CSR from edge arrays.  Rejects duplicates and bad ids."""
    u = np.asarray(u, dtype=np.int64).ravel()
    v = np.asarray(v, dtype=np.int64).ravel()
    if u.shape != v.shape:
        raise ValueError("u and v differ in length")
    if u.size and (u.min() < 0 or u.max() >= num_u or v.min() < 0 or v.max() >= num_l):
        raise ValueError("vertex id out of range")
    key = u * max(num_l, 1) + v
    order = np.argsort(key, kind="stable") if sort_lists else np.argsort(u, kind="stable")
    if np.unique(key).size != key.size:
        raise ValueError("duplicate edge")
    u, v = u[order], v[order]
    off = np.zeros(num_u + 1, dtype=np.int64)
    np.add.at(off, u + 1, 1)
    off = np.cumsum(off)
    if off[-1] > np.iinfo(np.int32).max:
        raise ValueError("too many edges for int32 offsets")
    return BipartiteCSR(num_u, num_l, off.astype(np.int32), v.astype(np.int32), name,
                        dict(meta or {}))


def shuffle_lists(g: BipartiteCSR, seed: int) -> BipartiteCSR:
    """Same graph with every adjacency list in a seeded random order.

    Edge ids follow their slots, so per-edge outputs must be compared through
    :func:`edge_slot_map`.
    """
    u, v = g.edges()
    h = splitmix64_np(np.arange(v.size, dtype=np.uint64), seed).view(np.int64)
    order = np.lexsort((h, u))
    return BipartiteCSR(g.num_u, g.num_l, g.off_u.copy(), v[order].astype(np.int32),
                        g.name + "+shuffled", dict(g.meta))


def relabel(g: BipartiteCSR, seed: int) -> BipartiteCSR:
    """Same graph under seeded random permutations of both layers' ids."""
    pu = _perm_np(g.num_u, seed * 2 + 1)
    pl = _perm_np(g.num_l, seed * 2 + 2)
    u, v = g.edges()
    return from_edges(g.num_u, g.num_l, pu[u], pl[v], g.name + "+relabelled", meta=g.meta)


def sample_u(g: BipartiteCSR, frac: float, seed: int) -> BipartiteCSR:
    """The subgraph of the edges of a seeded random fraction of U (same id
    spaces; the other U vertices become isolated)."""
    h = splitmix64_np(np.arange(g.num_u, dtype=np.uint64), seed)
    keep = (h >> np.uint64(11)).astype(np.float64) / float(1 << 53) < frac
    deg = np.diff(g.off_u.astype(np.int64))
    mask = np.repeat(keep, deg)
    off = np.zeros(g.num_u + 1, dtype=np.int64)
    off[1:] = np.cumsum(np.where(keep, deg, 0))
    return BipartiteCSR(g.num_u, g.num_l, off.astype(np.int32), g.adj_u[mask].copy(),
                        f"{g.name}+u{frac}", dict(g.meta))


def _perm_np(n: int, seed: int) -> np.ndarray:
    h = splitmix64_np(np.arange(n, dtype=np.uint64), seed).view(np.int64)
    order = np.argsort(h, kind="stable")
    perm = np.empty(n, dtype=np.int64)
    perm[order] = np.arange(n, dtype=np.int64)
    return perm


# ---------------------------------------------------------------------------
# Closed-form families and the paper's worked examples
# ---------------------------------------------------------------------------

def complete_bipartite(a: int, b: int) -> BipartiteCSR:
    """K_{a,b}: |U| = a, |L| = b, every pair joined."""
    u = np.repeat(np.arange(a), b)
    v = np.tile(np.arange(b), a)
    return from_edges(a, b, u, v, f"K_{a},{b}")


def cycle(k: int) -> BipartiteCSR:
    """C_{2k}: u_i - v_i - u_{i+1} - ... (k >= 2; C_4 when k = 2)."""
    u = np.concatenate([np.arange(k), np.arange(k)])
    v = np.concatenate([np.arange(k), (np.arange(k) - 1) % k])
    return from_edges(k, k, u, v, f"C_{2 * k}")


def star(leaves: int, center_in_u: bool = True) -> BipartiteCSR:
    if center_in_u:
        return from_edges(1, leaves, np.zeros(leaves), np.arange(leaves), f"star_{leaves}")
    return from_edges(leaves, 1, np.arange(leaves), np.zeros(leaves), f"star_{leaves}_L")


def path(num_edges: int) -> BipartiteCSR:
    """Path with ``num_edges`` edges alternating U, L, U, ..."""
    us, vs = [], []
    for i in range(num_edges):
        # edge i joins vertex i and vertex i+1 of the path; even positions are U
        a, b = i, i + 1
        if a % 2 == 0:
            us.append(a // 2); vs.append(b // 2)
        else:
            us.append(b // 2); vs.append(a // 2)
    r = num_edges // 2 + 1
    l = (num_edges + 1) // 2
    return from_edges(r, l, us, vs, f"path_{num_edges}")


def random_forest(num_u: int, num_l: int, seed: int) -> BipartiteCSR:
    """A seeded random forest: each vertex after the first joins one earlier
    vertex of the other layer, so no cycle (and no butterfly) can form."""
    order = _perm_np(num_u + num_l, seed)  # interleave the two layers randomly
    us, vs = [], []
    seen_u, seen_l = [], []
    rnd = splitmix64_np(np.arange(num_u + num_l, dtype=np.uint64), seed + 7)
    for t, x in enumerate(np.argsort(order)):
        if x < num_u:
            if seen_l and (int(rnd[t]) % 4) != 0:
                us.append(x); vs.append(seen_l[int(rnd[t] >> np.uint64(8)) % len(seen_l)])
            seen_u.append(x)
        else:
            y = x - num_u
            if seen_u and (int(rnd[t]) % 4) != 0:
                us.append(seen_u[int(rnd[t] >> np.uint64(8)) % len(seen_u)]); vs.append(y)
            seen_l.append(y)
    return from_edges(num_u, num_l, us, vs, f"forest_{num_u}_{num_l}_{seed}")


def disjoint_union(a: BipartiteCSR, b: BipartiteCSR) -> BipartiteCSR:
    ua, va = a.edges()
    ub, vb = b.edges()
    return from_edges(a.num_u + b.num_u, a.num_l + b.num_l,
                      np.concatenate([ua, ub + a.num_u]), np.concatenate([va, vb + a.num_l]),
                      f"{a.name}+{b.name}")


def paper_fig2a() -> BipartiteCSR:
    """Section 1, Figure 2(a): u0 joined to v0..v999, v1000 joined to
    u1..u1000, and v_i joined to u_{i+1} for 0 <= i <= 999 (2,002 vertices,
    3,000 edges)."""
    us = [0] * 1000 + list(range(1, 1001)) + [i + 1 for i in range(1000)]
    vs = list(range(1000)) + [1000] * 1000 + list(range(1000))
    return from_edges(1001, 1001, us, vs, "paper_fig2a")


def paper_fig3() -> BipartiteCSR:
    """Section 4, Figure 3: u0 and u1 joined to v0..v999; v1000 and v1001
    joined to u2..u1001 (2,004 vertices, 4,000 edges)."""
    us, vs = [], []
    for u in (0, 1):
        us += [u] * 1000; vs += list(range(1000))
    for v in (1000, 1001):
        us += list(range(2, 1002)); vs += [v] * 1000
    return from_edges(1002, 1002, us, vs, "paper_fig3")


def shifted_sidon_circulant(p: int, c: int, n: int) -> BipartiteCSR:
    """A regular circulant: U vertex u is joined to L vertex (u + s) mod n for
    every distinct shift s mod n in T and in T + c, where T = {2pk + (k^2 mod
    p)} (p prime) is the Erdős-Turán Sidon set (its differences are pairwise
    distinct).
    Every vertex has degree 2p, so priorities tie on degree and every U vertex
    lies above every L vertex.  The two-hop neighbourhood of a U vertex has
    about 3p^2 distinct vertices, most reached once and the differences of T
    twice: a start near either end of the U order has that many distinct
    ends (hash-table stress), with butterflies from the doubled differences."""
    t = np.array([2 * p * k + (k * k) % p for k in range(p)], dtype=np.int64)
    shifts = np.unique(np.concatenate([t, t + c]) % n)
    u = np.repeat(np.arange(n, dtype=np.int64), shifts.size)
    v = (u + np.tile(shifts, n)) % n
    return from_edges(n, n, u, v, f"sidon_{p}_{c}_{n}")


def rows_of_degrees(degs, num_l: int, seed: int) -> BipartiteCSR:
    """U vertex i gets degs[i] distinct L neighbours (a + j·s mod num_l,
    j < degs[i], with a seeded start a and a stride s coprime to num_l):
    lists of chosen lengths, for exercising degree thresholds."""
    degs = [int(d) for d in degs]
    if max(degs, default=0) > num_l:
        raise ValueError("a degree exceeds num_l")
    h = splitmix64_np(np.arange(2 * len(degs), dtype=np.uint64), seed)
    us, vs = [], []
    for i, d in enumerate(degs):
        a = int(h[2 * i] % np.uint64(num_l))
        st = int(h[2 * i + 1] % np.uint64(num_l)) | 1
        while math.gcd(st, num_l) != 1:
            st += 2
        us.append(np.full(d, i, dtype=np.int64))
        vs.append((a + np.arange(d, dtype=np.int64) * st) % num_l)
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    return from_edges(len(degs), num_l, u, v, f"rows_{len(degs)}_{num_l}_{seed}")


def random_tiny(num_u: int, num_l: int, p_num: int, p_den: int, seed: int) -> BipartiteCSR:
    """Each of the r*l pairs is an edge with probability p_num/p_den."""
    k = np.arange(num_u * num_l, dtype=np.uint64)
    keep = (splitmix64_np(k, seed) % np.uint64(p_den)) < np.uint64(p_num)
    idx = np.nonzero(keep)[0]
    return from_edges(num_u, num_l, idx // max(num_l, 1), idx % max(num_l, 1),
                      f"tiny_{num_u}_{num_l}_{seed}")


# ---------------------------------------------------------------------------
# Uniform and Chung-Lu generators (numpy or torch back end)
# ---------------------------------------------------------------------------

class _NumpyOps:
    name = "numpy"

    def arange(self, a, b):
        return np.arange(a, b, dtype=np.uint64)

    def rand(self, ctr, seed):
        # 63-bit non-negative value as int64
        return (splitmix64_np(ctr, seed) >> np.uint64(1)).astype(np.int64)

    def hash(self, keys, seed):
        return splitmix64_np(keys.astype(np.uint64), seed).view(np.int64)

    def searchsorted_right(self, table, x):
        return np.searchsorted(table, x, side="right").astype(np.int64)

    def unique(self, x):
        return np.unique(x)

    def cat(self, a, b):
        return np.concatenate([a, b])

    def take_smallest(self, keys, h, m):
        order = np.argsort(h, kind="stable")[:m]
        return np.sort(keys[order])

    def size(self, x):
        return int(x.shape[0])

    def empty(self):
        return np.zeros(0, dtype=np.int64)

    def table(self, t):
        return t

    def to_numpy(self, x):
        return x


class _TorchOps:
    name = "torch"

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = torch.device(device)

    def arange(self, a, b):
        return self.torch.arange(a, b, dtype=self.torch.int64, device=self.device)

    def rand(self, ctr, seed):
        return _srl_t(splitmix64_torch(ctr, seed), 1)

    def hash(self, keys, seed):
        return splitmix64_torch(keys, seed)

    def searchsorted_right(self, table, x):
        return self.torch.searchsorted(table, x, right=True)

    def unique(self, x):
        return self.torch.unique(x, sorted=True)

    def cat(self, a, b):
        return self.torch.cat([a, b])

    def take_smallest(self, keys, h, m):
        order = self.torch.argsort(h, stable=True)[:m]
        return self.torch.sort(keys[order]).values

    def size(self, x):
        return int(x.shape[0])

    def empty(self):
        return self.torch.zeros(0, dtype=self.torch.int64, device=self.device)

    def table(self, t):
        return self.torch.from_numpy(np.ascontiguousarray(t)).to(self.device)

    def to_numpy(self, x):
        return x.cpu().numpy()


def _ops(device):
    return _NumpyOps() if device is None else _TorchOps(device)


def _draw_distinct(num_u: int, num_l: int, m: int, seed: int, ops,
                   sample_u: Callable, sample_v: Callable) -> np.ndarray:
    """Draw (u, v) pairs in rounds until at least m distinct pairs exist, then
    keep the m pairs of smallest hash.  Returns sorted keys u*l + v (numpy).
    After 48 rounds (only near-saturated skewed graphs get there) the
    remaining draws are uniform."""
    if m > num_u * num_l:
        raise ValueError("more edges requested than vertex pairs")
    s_u, s_v, s_h = seed * 4 + 1, seed * 4 + 2, seed * 4 + 3
    keys = ops.empty()
    drawn, need, factor = 0, m, 1.1
    for rnd in range(200):
        k = max(1024, int(math.ceil(need * factor)))
        ctr = ops.arange(drawn, drawn + k)
        if rnd < 48:
            u = sample_u(ops.rand(ctr, s_u))
            v = sample_v(ops.rand(ctr, s_v))
        else:
            # near-saturated skewed graphs: top up with uniform draws
            u = ops.rand(ctr, s_u) % num_u
            v = ops.rand(ctr, s_v) % num_l
        before = ops.size(keys)
        keys = ops.unique(ops.cat(keys, u * num_l + v))
        drawn += k
        have = ops.size(keys)
        if have >= m:
            break
        added = have - before
        need = m - have
        if added < need // 2:
            factor = min(factor * 2.0, 4096.0)
    else:
        raise RuntimeError("generator did not reach the requested edge count")
    if ops.size(keys) > m:
        keys = ops.take_smallest(keys, ops.hash(keys, s_h), m)
    return ops.to_numpy(keys).astype(np.int64)


def _keys_to_csr(num_u: int, num_l: int, keys: np.ndarray, name: str, meta: dict) -> BipartiteCSR:
    u = keys // num_l
    v = keys % num_l
    off = np.searchsorted(u, np.arange(num_u + 1, dtype=np.int64), side="left")
    return BipartiteCSR(num_u, num_l, off.astype(np.int32), v.astype(np.int32), name, meta)


def uniform_bipartite(num_u: int, num_l: int, m: int, seed: int, device=None) -> BipartiteCSR:
    """m distinct edges, each endpoint drawn uniformly in its layer."""
    ops = _ops(device)
    keys = _draw_distinct(num_u, num_l, m, seed, ops,
                          lambda x: x % num_u, lambda x: x % num_l)
    return _keys_to_csr(num_u, num_l, keys, f"uniform_{num_u}_{num_l}_{m}_s{seed}",
                        dict(kind="uniform", seed=seed))


def chung_lu_weights(n: int, total: float, gamma: float, w_max: float,
                     fast: bool = False) -> tuple[np.ndarray, float]:
    """Expected degrees w_i = C (i + i0)^(-1/(gamma-1)), i = 0..n-1, with C set
    so that sum(w) = total and i0 solved (bisection) so that w_0 = w_max.

    fast=True evaluates the sum inside the bisection as 256 exact terms plus
    the midpoint integral of the tail (used for the many small batch graphs)."""
    alpha = 1.0 / (gamma - 1.0)
    i = np.arange(n, dtype=np.float64)
    head = np.arange(min(n, 256), dtype=np.float64)

    def tail(i0: float) -> float:
        k = head.size
        if k >= n:
            return 0.0
        a, b = k - 0.5 + i0, n - 0.5 + i0
        if abs(alpha - 1.0) < 1e-12:
            return math.log(b / a)
        return (b ** (1.0 - alpha) - a ** (1.0 - alpha)) / (1.0 - alpha)

    def top(i0: float) -> float:
        if fast:
            s = np.sum((head + i0) ** (-alpha)) + tail(i0)
        else:
            s = np.sum((i + i0) ** (-alpha))
        return total * i0 ** (-alpha) / s

    lo, hi = 1e-9, 1e12
    if top(hi) > w_max:  # even a flat profile exceeds w_max: use a flat one
        return np.full(n, total / n), hi
    if top(lo) < w_max:
        lo = lo
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if top(mid) > w_max:
            lo = mid
        else:
            hi = mid
    i0 = math.sqrt(lo * hi)
    w = (i + i0) ** (-alpha)
    w *= total / w.sum()
    return w, i0


def _quantised_cdf(w: np.ndarray) -> np.ndarray:
    q = np.maximum(1, np.floor(w / w.sum() * float(1 << 40))).astype(np.int64)
    return np.cumsum(q)


def chung_lu_bipartite(num_u: int, num_l: int, m: int, gamma_u: float, gamma_l: float,
                       seed: int, max_u: Optional[float] = None, max_l: Optional[float] = None,
                       device=None, fast_weights: bool = False) -> BipartiteCSR:
    """Chung-Lu style power-law bipartite graph with exactly m distinct edges.

    Endpoints are drawn independently with probability proportional to the
    expected-degree weights of :func:`chung_lu_weights`; duplicates are
    removed and the draw is topped up until m distinct edges exist.  Vertex
    ids are then scattered by a seeded permutation of each layer, so that id
    and degree are uncorrelated.  ``max_u``/``max_l`` default to 0.1 x the
    size of the other layer.
    """
    ops = _ops(device)
    max_u = 0.1 * num_l if max_u is None else max_u
    max_l = 0.1 * num_u if max_l is None else max_l
    wu, i0u = chung_lu_weights(num_u, m, gamma_u, max_u, fast_weights)
    wl, i0l = chung_lu_weights(num_l, m, gamma_l, max_l, fast_weights)
    cu, cl = _quantised_cdf(wu), _quantised_cdf(wl)
    pu, pl = _perm_np(num_u, seed * 4 + 5), _perm_np(num_l, seed * 4 + 6)
    tcu, tcl, tpu, tpl = ops.table(cu), ops.table(cl), ops.table(pu), ops.table(pl)
    tu, tl = int(cu[-1]), int(cl[-1])
    keys = _draw_distinct(
        num_u, num_l, m, seed, ops,
        lambda x: tpu[ops.searchsorted_right(tcu, x % tu)],
        lambda x: tpl[ops.searchsorted_right(tcl, x % tl)])
    meta = dict(kind="chung_lu", seed=seed, gamma_u=gamma_u, gamma_l=gamma_l,
                i0_u=i0u, i0_l=i0l, w_max_u=float(wu[0]), w_max_l=float(wl[0]))
    return _keys_to_csr(num_u, num_l, keys,
                        f"chunglu_{num_u}_{num_l}_{m}_g{gamma_u}_{gamma_l}_s{seed}", meta)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def uniform_small(seed: int = 1001, device=None) -> BipartiteCSR:
    """Uniform bipartite graph, |U| = 2,000, |L| = 3,000, 20,000 edges."""
    g = uniform_bipartite(2000, 3000, 20000, seed, device)
    g.name = "uniform_u2k_l3k_m20k"
    return g


def powerlaw_20m(seed: int = 2001, device=None) -> BipartiteCSR:
    """Chung-Lu, |U| = 1M, |L| = 500k, 20M edges, exponent 2.1 on both layers."""
    g = chung_lu_bipartite(1_000_000, 500_000, 20_000_000, 2.1, 2.1, seed, device=device)
    g.name = "chunglu_u1m_l500k_m20m_g2.1"
    return g


def shopping_300m(seed: int = 3001, device=None, scale: float = 1.0) -> BipartiteCSR:
    """Shopping-like: 10M users (exponent 2.5), 100k items (exponent 1.8,
    expected top item degree 1M), 300M edges.  ``scale`` shrinks every size
    proportionally (for tests)."""
    r = int(10_000_000 * scale)
    l = int(100_000 * scale)
    m = int(300_000_000 * scale)
    g = chung_lu_bipartite(r, l, m, 2.5, 1.8, seed, max_u=0.1 * l, max_l=1_000_000 * scale,
                           device=device)
    g.name = f"shopping_u{r}_l{l}_m{m}"
    return g


def batch_graph_params(g: int, seed_base: int = 4000) -> tuple[int, int, int, float, float]:
    """Sizes of graph g of the batched workload: |U|, |L| log-uniform in
    [100, 50,000], m log-uniform in [1,000, 2,000,000] clamped to
    floor(0.5 |U| |L|), exponents uniform in [1.8, 2.6]."""
    r = splitmix64_np(np.arange(5, dtype=np.uint64), seed_base + g)
    f = (r >> np.uint64(11)).astype(np.float64) / float(1 << 53)

    def logu(x, lo, hi):
        return int(round(math.exp(math.log(lo) + x * (math.log(hi) - math.log(lo)))))

    nu = logu(f[0], 100, 50_000)
    nl = logu(f[1], 100, 50_000)
    m = min(logu(f[2], 1_000, 2_000_000), (nu * nl) // 2)
    gu = 1.8 + 0.8 * float(f[3])
    gl = 1.8 + 0.8 * float(f[4])
    return nu, nl, m, gu, gl


def batch_graph(g: int, seed_base: int = 4000, device=None) -> BipartiteCSR:
    nu, nl, m, gu, gl = batch_graph_params(g, seed_base)
    gr = chung_lu_bipartite(nu, nl, m, gu, gl, seed_base + g, device=device, fast_weights=True)
    gr.name = f"batch{g}"
    return gr


# ---------------------------------------------------------------------------
# Batches as disjoint unions
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Batch:
    """Several graphs laid side by side as one disjoint union.

    ``union`` is the U-side CSR of the union (graph g's U vertices are
    ``u_start[g]:u_start[g+1]``, its L vertices ``l_start[g]:l_start[g+1]``,
    L ids global); ``e_start[g]`` is the first edge slot of graph g, so graph
    g's per-edge outputs are the union's slots ``e_start[g]:e_start[g+1]``.
    """
    union: BipartiteCSR
    u_start: np.ndarray  # int32[G+1]
    l_start: np.ndarray  # int32[G+1]
    e_start: np.ndarray  # int64[G+1]

    @property
    def num_graphs(self) -> int:
        return int(self.u_start.shape[0] - 1)


def union_batch(graphs) -> Batch:
    us = np.zeros(len(graphs) + 1, dtype=np.int64)
    ls = np.zeros(len(graphs) + 1, dtype=np.int64)
    es = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        us[i + 1] = us[i] + g.num_u
        ls[i + 1] = ls[i] + g.num_l
        es[i + 1] = es[i] + g.num_edges
    if us[-1] + ls[-1] > np.iinfo(np.int32).max - 1 or es[-1] > np.iinfo(np.int32).max:
        raise ValueError("batch too large for int32 ids and offsets")
    off = np.zeros(us[-1] + 1, dtype=np.int64)
    adj = np.zeros(es[-1], dtype=np.int32)
    for i, g in enumerate(graphs):
        off[us[i] + 1:us[i + 1] + 1] = es[i] + g.off_u[1:].astype(np.int64)
        adj[es[i]:es[i + 1]] = g.adj_u + ls[i]
    u = BipartiteCSR(int(us[-1]), int(ls[-1]), off.astype(np.int32), adj, f"union_{len(graphs)}")
    return Batch(u, us.astype(np.int32), ls.astype(np.int32), es)
