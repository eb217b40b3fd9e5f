"""Pins of the MCMC oracle (oracle/mcmc.py) against things other than itself:
the stationary marginals of exp(-Abar / kT) integrated on a fine grid of the
CV torus (1-D and 2-D), and the limiting cases of the Metropolis rule (a flat
free energy accepts every move; at kT -> 0 only downhill moves are taken).
"""
import math

import numpy as np
import pytest

from oracle import mcmc as MC
from oracle import train as T


def _net(D, L, H, seed, scale):
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 1.0, size=(1, T.param_count(D, L, H)))
    return w * scale


def _exact_bin_probs(weights, C, L, H, bins, kT, sub=24):
    # p(s) ~ exp(-Abar(s)/kT) on a (bins * sub)^C midpoint grid, summed per bin
    n = bins * sub
    g = -math.pi + (np.arange(n) + 0.5) * (2 * math.pi / n)
    grids = np.meshgrid(*([g] * C), indexing="ij")
    s = np.stack([x.ravel() for x in grids], axis=1)
    A = MC.ensemble_mean_value(weights, 2 * C, L, H, False, s)
    p = np.exp(-(A - A.min()) / kT).reshape([n] * C)
    p /= p.sum()
    for ax in range(C):
        p = np.add.reduceat(p, np.arange(0, n, sub), axis=ax)
    return p, A.max() - A.min()


def test_one_cv_histogram_matches_the_stationary_marginal():
    C, L, H, bins, kT = 1, 2, 8, 16, 1.0
    w = _net(2 * C, L, H, 3, 0.9)
    p, span = _exact_bin_probs(w, C, L, H, bins, kT)
    assert span > 2.0 * kT                      # a landscape the rule must follow
    rng = np.random.default_rng(3)
    s0 = rng.uniform(-math.pi, math.pi, size=(200, C))
    r = MC.run(w, C, L, H, False, s0, 600, 100, kT, 0.8, 11, bins, (0, 0))
    h = r["hist1"][0]
    assert h.sum() == 200 * 500
    tv = 0.5 * np.abs(h / h.sum() - p).sum()
    assert tv < 0.04, tv
    # the inverted landscape is far off: the pin separates the sign of the rule
    q, _ = _exact_bin_probs(-w, C, L, H, bins, kT)
    assert 0.5 * np.abs(h / h.sum() - q).sum() > 0.2


def test_two_cv_joint_histogram_matches_the_stationary_joint():
    C, L, H, bins, kT = 2, 2, 8, 12, 1.0
    w = _net(2 * C, L, H, 2, 0.7)
    p, span = _exact_bin_probs(w, C, L, H, bins, kT, sub=12)
    assert span > 2.0 * kT
    rng = np.random.default_rng(4)
    s0 = rng.uniform(-math.pi, math.pi, size=(400, C))
    r = MC.run(w, C, L, H, False, s0, 500, 100, kT, 0.9, 12, bins, (0, 1))
    h2 = r["hist2"]
    assert h2.sum() == 400 * 400
    tv = 0.5 * np.abs(h2 / h2.sum() - p).sum()
    assert tv < 0.06, tv
    # the 1-D histograms are the joint's marginals
    np.testing.assert_array_equal(r["hist1"][0], h2.sum(axis=1))
    np.testing.assert_array_equal(r["hist1"][1], h2.sum(axis=0))


def test_flat_free_energy_accepts_every_move():
    C, L, H = 3, 2, 4
    w = np.zeros((2, T.param_count(2 * C, L, H)))
    w[:, -1] = 1.5                                  # b_out only
    s0 = np.zeros((16, C))
    r = MC.run(w, C, L, H, False, s0, 20, 0, 1.0, 0.5, 5, 8, (0, 1))
    assert r["n_accepted"] == 16 * 20


def test_zero_temperature_takes_only_downhill_moves():
    C, L, H = 2, 2, 6
    w = _net(2 * C, L, H, 6, 0.8)
    rng = np.random.default_rng(6)
    s0 = rng.uniform(-math.pi, math.pi, size=(64, C))
    A0 = MC.ensemble_mean_value(w, 2 * C, L, H, False, s0)
    sp = MC.wrap(s0 + 0.7 * MC.proposal_normals(64, C, 0, 9))
    Ap = MC.ensemble_mean_value(w, 2 * C, L, H, False, sp)
    r = MC.run(w, C, L, H, False, s0, 1, 0, 1e-12, 0.7, 9, 8, (0, 1))
    down = Ap < A0
    assert r["n_accepted"] == int(down.sum())
    np.testing.assert_allclose(r["s"][down], sp[down])
    np.testing.assert_allclose(r["s"][~down], s0[~down])


def test_binning_edges_and_projection():
    b = MC.bin_index(np.array([-math.pi, -math.pi + 1e-12, 0.0, math.pi - 1e-12, math.pi]), 10)
    np.testing.assert_array_equal(b, [0, 0, 5, 9, 9])
    f = MC.projected_pmf(np.array([10, 0, 40, 50]), 2.0)
    assert f[3] == 0.0 and math.isinf(f[1])
    assert f[0] == pytest.approx(-2.0 * math.log(10 / 50))


def test_path_cv_limits():
    # nodes far apart on the torus: at node k, s -> k and z -> 0; between two
    # neighbouring nodes s is the weighted index; large and small lambda agree
    # with the plain formula
    nodes = np.array([[-2.0, 0.0], [-1.0, 0.5], [0.0, 1.0], [1.0, 0.5], [2.0, 0.0]])
    pts = np.zeros((5, 3))
    pts[:, [0, 2]] = nodes
    sp, z = MC.path_cv(pts, nodes, [0, 2], 40.0)
    np.testing.assert_allclose(sp, np.arange(1, 6), atol=1e-6)
    np.testing.assert_allclose(z, 0.0, atol=1e-6)
    rng = np.random.default_rng(8)
    q = np.zeros((50, 3))
    q[:, [0, 2]] = rng.uniform(-0.8, 0.8, size=(50, 2))   # no difference wraps
    for lam in (0.25, 3.0):
        sp, z = MC.path_cv(q, nodes, [0, 2], lam)
        d2 = ((q[:, None, [0, 2]] - nodes[None]) ** 2).sum(-1)
        e = np.exp(-lam * d2)
        np.testing.assert_allclose(sp, (e * np.arange(1, 6)).sum(1) / e.sum(1), rtol=1e-12)
        np.testing.assert_allclose(z, -np.log(e.sum(1)) / lam, rtol=1e-12)
    # periodic: a point just across pi from the last node
    far = np.zeros((1, 3))
    far[0, 0] = 2.0 - 2 * math.pi
    sp, z = MC.path_cv(far, nodes, [0, 2], 40.0)
    assert sp[0] == pytest.approx(5.0, abs=1e-6) and z[0] == pytest.approx(0.0, abs=1e-6)
    bs, bz = MC.path_bins(np.array([1.0, 3.0, 5.0]), np.array([-1.0, 0.5, 9.0]), 5, 0.0, 1.0, 10)
    np.testing.assert_array_equal(bs, [0, 5, 9])
    np.testing.assert_array_equal(bz, [0, 5, 9])


# --------------------------------------------------------------------------- distance CVs
def _exact_mixed_bin_probs(weights, L, H, bins, kT, dist, lo, hi, sub=12):
    """p(s) ~ exp(-Abar(s)/kT) on a midpoint grid of the box: [-pi, pi) for a
    torsion, [lo, hi] for a distance CV, summed per bin."""
    C = len(dist)
    n = bins * sub
    axes = []
    for c in range(C):
        a, b = (lo[c], hi[c]) if dist[c] else (-math.pi, math.pi)
        axes.append(a + (np.arange(n) + 0.5) * ((b - a) / n))
    grids = np.meshgrid(*axes, indexing="ij")
    s = np.stack([x.ravel() for x in grids], axis=1)
    A = MC.ensemble_mean_value(weights, 2 * C, L, H, False, s, np.asarray(dist))
    p = np.exp(-(A - A.min()) / kT).reshape([n] * C)
    p /= p.sum()
    for ax in range(C):
        p = np.add.reduceat(p, np.arange(0, n, sub), axis=ax)
    return p, A.max() - A.min()


def test_distance_cv_marginal_and_mixed_joint_match_the_stationary_density():
    """A distance CV in [1, 4] next to a torsion: the walk must sample
    exp(-Abar/kT) restricted to the box (moves leaving the range refused)."""
    L, H, bins, kT = 2, 8, 12, 1.0
    dist, lo, hi = np.array([False, True]), np.array([0.0, 1.0]), np.array([0.0, 4.0])
    w = _net(4, L, H, 7, 1.3)
    p, span = _exact_mixed_bin_probs(w, L, H, bins, kT, dist, lo, hi)
    assert span > 2.0 * kT
    rng = np.random.default_rng(5)
    W = 400
    s0 = np.stack([rng.uniform(-math.pi, math.pi, W), rng.uniform(1.0, 4.0, W)], axis=1)
    r = MC.run(w, 2, L, H, False, s0, 500, 100, kT, 0.6, 13, bins, (0, 1), dist=dist, lo=lo, hi=hi)
    assert np.all((r["s"][:, 1] >= 1.0) & (r["s"][:, 1] <= 4.0))
    h2 = r["hist2"]
    tv = 0.5 * np.abs(h2 / h2.sum() - p).sum()
    assert tv < 0.06, tv
    h1 = r["hist1"][1]
    tv1 = 0.5 * np.abs(h1 / h1.sum() - p.sum(axis=0)).sum()
    assert tv1 < 0.04, tv1
    # read as a torsion (wrapped, (cos, sin) input) the same walk is a different density
    q, _ = _exact_mixed_bin_probs(w, L, H, bins, kT, np.array([False, False]), lo, hi)
    assert 0.5 * np.abs(h2 / h2.sum() - q).sum() > 0.1


def test_distance_cv_range_refuses_moves_and_bins_span_it():
    # a flat landscape: every proposal inside the range is taken, none outside
    C, L, H = 1, 1, 4
    w = np.zeros((1, T.param_count(2 * C, L, H)))
    s0 = np.full((64, 1), 1.05)
    r = MC.run(w, C, L, H, False, s0, 40, 0, 1.0, 0.5, 21, 10, (0, 0), dist=[True], lo=[1.0], hi=[2.0])
    assert np.all((r["s"] >= 1.0) & (r["s"] <= 2.0))
    moves = 0
    s = s0[:, 0].astype(np.float64).copy()
    for t in range(40):
        sp = s + 0.5 * MC.proposal_normals(64, 1, t, 21)[:, 0]
        ok = (sp >= 1.0) & (sp <= 2.0)
        s[ok] = sp[ok]
        moves += int(ok.sum())
    assert r["n_accepted"] == moves
    np.testing.assert_allclose(r["s"][:, 0], s, rtol=0, atol=0)
    # bins over [lo, hi]
    b = MC.bin_index(np.array([[1.0], [1.0999], [1.1], [1.95], [2.0]]), 10, [True], [1.0], [2.0])
    assert list(b[:, 0]) == [0, 0, 1, 9, 9]


def test_path_over_a_distance_cv_uses_plain_differences():
    nodes = np.array([[0.5], [3.5]])
    s = np.array([[6.3]])
    sp, z = MC.path_cv(s, nodes, [0], 2.0, dist=np.array([True]))
    d2 = np.array([5.8 ** 2, 2.8 ** 2])
    e = np.exp(-2.0 * (d2 - d2.min()))
    assert sp[0] == pytest.approx((e * [1, 2]).sum() / e.sum(), rel=1e-12)
    assert z[0] == pytest.approx(d2.min() - math.log(e.sum()) / 2.0, rel=1e-12)
    # a torsion reading would wrap 6.3 - 0.5 onto -0.48: node 1 nearest instead
    sp_t, _ = MC.path_cv(s, nodes, [0], 2.0)
    assert sp_t[0] < 1.5 < sp[0]
