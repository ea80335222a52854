"""The Chung-Lu input recipe: expected-degree weights w_i = C (i + i0)^(-1/(γ-1))
with Σ w = m and w_0 = the requested maximum, and realised graphs whose
degrees follow those weights.  Deterministic checks of the weights, loose
statistical checks of one realised graph."""
import numpy as np
import pytest

from bfc_inputs import generators as G


@pytest.mark.parametrize("gamma", [1.8, 2.1, 2.5])
def test_weights_closed_form(gamma):
    n, total, w_max = 10_000, 50_000.0, 500.0
    w, i0 = G.chung_lu_weights(n, total, gamma, w_max)
    assert w.shape == (n,)
    assert abs(w.sum() - total) < 1e-9 * total
    assert abs(w[0] - w_max) < 1e-6 * w_max
    assert np.all(np.diff(w) < 0)
    # ratios follow the power law exactly: w_i / w_j = ((i + i0) / (j + i0))^(-1/(γ-1))
    i = np.array([0, 1, 10, 100, 1000, n - 1], dtype=np.float64)
    alpha = 1.0 / (gamma - 1.0)
    np.testing.assert_allclose(w[i.astype(int)] / w[0], ((i + i0) / i0) ** (-alpha), rtol=1e-9)


def test_weights_fast_sum_matches_exact():
    for gamma in (1.8, 2.1, 2.6):
        _, i0 = G.chung_lu_weights(200_000, 1e6, gamma, 2_000.0)
        wf, i0f = G.chung_lu_weights(200_000, 1e6, gamma, 2_000.0, fast=True)
        assert abs(i0f - i0) < 1e-3 * i0
        assert abs(wf.sum() - 1e6) < 1e-6 * 1e6


def test_weights_flat_when_the_maximum_is_below_the_mean():
    # a top weight below the mean degree cannot be met: the profile is flat
    w, _ = G.chung_lu_weights(1000, 5000.0, 2.1, 4.0)
    assert np.allclose(w, 5.0)


def test_realised_degrees_follow_the_weights():
    nu, nl, m, gamma = 20_000, 10_000, 100_000, 2.1
    g = G.chung_lu_bipartite(nu, nl, m, gamma, gamma, 11)
    deg_u = np.diff(g.off_u.astype(np.int64))
    deg_l = np.bincount(g.adj_u, minlength=nl)
    assert deg_u.sum() == m and deg_l.sum() == m
    # heavy tails on both layers: the top vertex is far above the mean, and
    # a few percent of the vertices carry a large share of the edges
    for deg, n, other in ((deg_u, nu, nl), (deg_l, nl, nu)):
        mean = m / n
        assert deg.max() > 20 * mean
        assert deg.max() <= 0.1 * other * 1.05   # the requested top weight, 0.1 x the other layer
        top = np.sort(deg)[::-1][: n // 100]
        assert top.sum() > 0.15 * m
    # ids are scattered: degree is not monotone in the id
    assert not np.all(np.diff(deg_u) <= 0)
    # the ranking by weight survives the draw: weight rank vs degree rank
    w, _ = G.chung_lu_weights(nu, float(m), gamma, 0.1 * nl)
    perm = G._perm_np(nu, 11 * 4 + 5)   # weight index i sits at id perm[i]
    d_by_weight = deg_u[perm]
    head = d_by_weight[:200].astype(np.float64)
    assert np.corrcoef(np.log1p(head), np.log(w[:200]))[0, 1] > 0.9
