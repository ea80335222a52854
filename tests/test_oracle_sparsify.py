"""Pins of the oracle's approximate counting by edge sparsification (Section
7: the exact counter as the inner block of a sampling estimator).

* The generator: SplitMix64's published first output, and agreement with the
  input module's separate numpy SplitMix64 over many draws.
* The keep rule: the threshold floor(p * 2^64) in exact arithmetic; p = 1 is
  the whole graph; the kept edges of a sample are exactly those whose draw is
  below the threshold, in their original order.
* The sampling law: the kept fraction is p and two samples are independent
  (p^2 kept in both), within binomial bounds.
* The estimator: Σ over all edge subsets of P(S)·⋈(S) = p^4·⋈(G) exactly on
  tiny graphs (brute-force counts, rational arithmetic), so dividing by p^4 is
  unbiased; the oracle's estimate lies within 5 standard errors of the exact
  count; p = 1 gives the exact count with zero spread.
* Planted mistakes in a copy of the C source are caught.
"""
import ctypes
import itertools
import math
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from bfc_inputs import generators as G
import oracle

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "bfc_oracle.c")


def test_splitmix64_published_first_output():
    # SplitMix64 from state 0: first output 0xE220A8397B1DCDAF (Steele et al.)
    assert oracle.splitmix64(0, 1) == 0xE220A8397B1DCDAF


def test_splitmix64_matches_input_module():
    rng = np.random.default_rng(3)
    for seed in [0, 1, 2**63 + 5, int(rng.integers(0, 2**62))]:
        ks = [1, 2, 3, 1000, 2**40 + 7, 2**64 - 1]
        ref = G.splitmix64_np(np.array([k - 1 for k in ks], dtype=np.uint64), seed)
        assert [oracle.splitmix64(seed, k) for k in ks] == [int(x) for x in ref]


def test_keep_threshold_exact():
    assert oracle.keep_threshold(0.5) == (2**63, False)
    assert oracle.keep_threshold(0.375) == (3 * 2**61, False)
    assert oracle.keep_threshold(2.0**-64) == (1, False)
    assert oracle.keep_threshold(1.0) == (0, True)
    t, _ = oracle.keep_threshold(0.1)
    assert t <= 0.1 * 2**64 < t + 1          # floor of the double's exact value
    for bad in [0.0, -0.5, 1.5, float("nan")]:
        with pytest.raises(ValueError):
            oracle.keep_threshold(bad)


def test_sparsify_keep_all_is_the_graph():
    g = G.chung_lu_bipartite(500, 300, 4000, 2.1, 2.0, 9)
    h = oracle.sparsify(g, 1.0, 123, 4)
    assert h.num_edges == g.num_edges
    assert np.array_equal(h.off_u, g.off_u) and np.array_equal(h.adj_u, g.adj_u)


@pytest.mark.parametrize("p,seed,j", [(0.3, 11, 0), (0.3, 11, 5), (0.05, 2**63 + 1, 2), (0.9, 0, 1)])
def test_sparsify_keeps_exactly_the_draws_below_threshold(p, seed, j):
    g = G.chung_lu_bipartite(2000, 1500, 20000, 2.1, 2.0, 21)
    m = g.num_edges
    t, _ = oracle.keep_threshold(p)
    draws = G.splitmix64_np(np.arange(m, dtype=np.uint64) + np.uint64(j * m), seed)
    keep = draws < np.uint64(t)
    h = oracle.sparsify(g, p, seed, j)
    assert np.array_equal(h.adj_u, g.adj_u[keep])
    rows = np.repeat(np.arange(g.num_u), np.diff(g.off_u.astype(np.int64)))
    assert np.array_equal(np.diff(h.off_u.astype(np.int64)), np.bincount(rows[keep], minlength=g.num_u))


@pytest.mark.parametrize("p", [0.05, 0.5])
def test_sparsify_rate_and_independence(p):
    g = G.uniform_bipartite(3000, 3000, 200000, 5)
    m = g.num_edges
    a = oracle.sparsify(g, p, 77, 0)
    b = oracle.sparsify(g, p, 77, 1)
    sd = math.sqrt(m * p * (1 - p))
    assert abs(a.num_edges - p * m) <= 6 * sd and abs(b.num_edges - p * m) <= 6 * sd
    # kept in both samples: probability p^2 when the samples are independent
    ka = set(zip(np.repeat(np.arange(g.num_u), np.diff(a.off_u.astype(np.int64))).tolist(), a.adj_u.tolist()))
    kb = set(zip(np.repeat(np.arange(g.num_u), np.diff(b.off_u.astype(np.int64))).tolist(), b.adj_u.tolist()))
    both = len(ka & kb)
    q = p * p
    assert abs(both - q * m) <= 6 * math.sqrt(m * q * (1 - q))


def _subgraph(g, keep):
    u_of, v_of = g.edges()
    return G.from_edges(g.num_u, g.num_l, u_of[keep], v_of[keep])


@pytest.mark.parametrize("gi,p", [(0, Fraction(1, 2)), (1, Fraction(1, 3)), (2, Fraction(2, 5))])
def test_expected_sampled_count_is_p4_times_count(gi, p):
    # enumerate the sampling distribution: every edge subset S with its
    # probability p^|S| (1-p)^(m-|S|), counted by brute force (Definition 2)
    g = [G.complete_bipartite(3, 3), G.random_tiny(4, 4, 2, 3, 5), G.complete_bipartite(2, 5)][gi]
    m = g.num_edges
    assert m <= 12
    expect = Fraction(0)
    for bits in itertools.product([False, True], repeat=m):
        keep = np.array(bits, dtype=bool)
        k = int(keep.sum())
        c = oracle.brute_total(_subgraph(g, keep)) if k >= 4 else 0
        expect += p**k * (1 - p)**(m - k) * c
    assert expect == p**4 * oracle.brute_total(g)


@pytest.mark.parametrize("gi,p,samples", [(0, 0.5, 600), (1, 0.3, 300), (2, 0.6, 200)])
def test_estimate_within_five_standard_errors(gi, p, samples):
    g = [G.complete_bipartite(6, 6), G.chung_lu_bipartite(300, 200, 3000, 2.1, 1.9, 8),
         G.uniform_bipartite(120, 90, 2000, 4)][gi]
    exact = oracle.vp(g)["total"]
    r = oracle.sparsified_estimate(g, p, 1000 + gi, samples)
    assert len(r["counts"]) == samples and r["std_error"] > 0
    assert abs(r["estimate"] - exact) <= 5 * r["std_error"]
    # the spread is that of a mean: the standard error shrinks as 1/sqrt(samples)
    sd = float(np.std(np.array(r["counts"], dtype=np.float64), ddof=1)) / p**4
    assert r["std_error"] == pytest.approx(sd / math.sqrt(samples), rel=1e-9)


def test_estimate_keep_all_is_exact():
    g = G.chung_lu_bipartite(400, 300, 5000, 2.1, 2.0, 3)
    exact = oracle.vp(g)["total"]
    r = oracle.sparsified_estimate(g, 1.0, 5, 3)
    assert r["counts"] == [exact] * 3 and r["edges"] == [g.num_edges] * 3
    assert r["estimate"] == float(exact) and r["std_error"] == 0.0
    one = oracle.sparsified_estimate(g, 0.5, 5, 1)
    assert math.isnan(one["std_error"])


def test_sparsify_rejects_malformed():
    g = G.complete_bipartite(3, 4)
    bad = G.complete_bipartite(3, 4)
    bad.adj_u = bad.adj_u.copy()
    bad.adj_u[2] = 9
    with pytest.raises(ValueError):
        oracle.sparsify(bad, 0.5, 1, 0)
    assert oracle.sparsify(g, 0.5, 1, 0).num_edges <= g.num_edges


# ---------------------------------------------------------------------------
# planted mistakes (in a copy of the C source, on the CPU)
# ---------------------------------------------------------------------------

MUTANTS = {
    "keep_flipped": ("< threshold)", ">= threshold)"),
    "draw_index_without_offset": ("j * m + (uint64_t)e + 1)", "j * m + (uint64_t)e)"),
    "draw_ignores_sample": ("j * m + (uint64_t)e + 1)", "(uint64_t)e + 1)"),
    "mix_shift": ("z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;"),
    "golden_gamma": ("seed + k * 0x9E3779B97F4A7C15ull", "seed + k * 0x9E3779B97F4A7C17ull"),
}


def _build(tmp_path, name, pair=None):
    src = open(SRC).read()
    if pair:
        assert src.count(pair[0]) == 1, f"mutation site for {name} not found once"
        src = src.replace(*pair)
    d = tmp_path / name
    d.mkdir()
    (d / "m.c").write_text(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-I",
                    os.path.dirname(SRC), "-o", str(d / "m.so"), str(d / "m.c")], check=True)
    lib = ctypes.CDLL(str(d / "m.so"))
    lib.orc_splitmix64.restype = ctypes.c_uint64
    lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    return lib


def _sparsify(lib, g, t, seed, j):
    i32 = ctypes.POINTER(ctypes.c_int32)
    off = np.ascontiguousarray(g.off_u, dtype=np.int32)
    adj = np.ascontiguousarray(g.adj_u, dtype=np.int32)
    oo = np.zeros(g.num_u + 1, np.int32)
    oa = np.zeros(max(g.num_edges, 1), np.int32)
    kept = np.zeros(1, np.int64)
    rc = lib.orc_sparsify(ctypes.c_int32(g.num_u), ctypes.c_int32(g.num_l), off.ctypes.data_as(i32),
                          adj.ctypes.data_as(i32), ctypes.c_uint64(seed), ctypes.c_uint64(j),
                          ctypes.c_uint64(t), ctypes.c_int(0), oo.ctypes.data_as(i32),
                          oa.ctypes.data_as(i32), kept.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    assert rc == 0
    return oa[:int(kept[0])]


def _pins_pass(lib) -> bool:
    if lib.orc_splitmix64(0, 1) != 0xE220A8397B1DCDAF:
        return False
    g = G.uniform_bipartite(2000, 2000, 60000, 6)
    m = g.num_edges
    for p, j in [(0.05, 0), (0.3, 3)]:
        t, _ = oracle.keep_threshold(p)
        got = _sparsify(lib, g, t, 99, j)
        draws = G.splitmix64_np(np.arange(m, dtype=np.uint64) + np.uint64(j * m), 99)
        if not np.array_equal(got, g.adj_u[draws < np.uint64(t)]):
            return False
    return True


def test_unmutated_copy_passes(tmp_path):
    assert _pins_pass(_build(tmp_path, "orig"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    assert not _pins_pass(_build(tmp_path, name, MUTANTS[name])), f"planted mistake {name} went unnoticed"
