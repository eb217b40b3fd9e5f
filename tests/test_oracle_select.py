"""Pins of the selection oracle (oracle/select.py): hand-worked clusterings,
the invariants of leader clustering checked by brute force, the periodic and
weighted distance against float64, the trust window, and a threshold search
on separated blobs whose right cluster count is known.
"""
import math

import numpy as np

from oracle import select as S


def test_hand_worked_line():
    cv = np.array([[0.0], [0.1], [5.0], [5.05], [0.2], [10.0], [9.5]])
    r = S.select(cv, np.full(7, 2.5), 2.0, 3.0, 1.0, 1, 100, False, 100, periodic=[False])
    np.testing.assert_array_equal(r["selected"], [0, 2, 5])
    assert r["n_clusters"] == 3


def test_periodic_wrap_joins_both_ends_and_weights_mask_a_cv():
    cv = np.array([[-3.1, 0.0], [3.1, 2.0]])
    e = np.full(2, 2.5)
    assert S.select(cv, e, 2, 3, 0.5, 1, 9, False, 9, w=[1, 0])["n_clusters"] == 1
    assert S.select(cv, e, 2, 3, 0.5, 1, 9, False, 9, w=[1, 0], periodic=[False, True])["n_clusters"] == 2
    assert S.select(cv, e, 2, 3, 0.5, 1, 9, False, 9, w=[1, 1])["n_clusters"] == 2


def test_fp32_distance_against_float64():
    rng = np.random.default_rng(1)
    a = rng.uniform(-math.pi, math.pi, size=(500, 6)).astype(np.float32)
    b = rng.uniform(-math.pi, math.pi, size=6).astype(np.float32)
    w = np.array([1.0, 0.5, 2.0, 1.0, 0.25, 1.0])
    per = np.array([1, 1, 0, 1, 0, 1], bool)
    d = a.astype(np.float64) - b.astype(np.float64)
    d[:, per] = (d[:, per] + math.pi) % (2 * math.pi) - math.pi
    exact = (w * d * d).sum(axis=1)
    np.testing.assert_allclose(S.dist2(a, b, w, per), exact, rtol=2e-6, atol=1e-6)


def test_leader_invariants_by_brute_force():
    rng = np.random.default_rng(2)
    x = rng.uniform(-math.pi, math.pi, size=(400, 3)).astype(np.float32)
    w, per, t = np.ones(3), np.ones(3, bool), 1.3
    lead, assign = S.leaders(x, w, per, t)
    t2 = np.float32(t * t)
    for k in range(x.shape[0]):
        d2 = S.dist2(x[lead], x[k], w, per)
        first = np.nonzero(d2 <= t2)[0]
        # a row joins the first leader within the threshold that existed before it
        earlier = lead <= k
        assert assign[k] == (first[earlier[first]][0])
    for i, li in enumerate(lead):                 # leaders are apart from every earlier leader
        if i:
            assert np.all(S.dist2(x[lead[:i]], x[li], w, per) > t2)


def test_trust_window_selects_candidates():
    eps = np.array([0.5, 2.0, 2.9, 3.0, 3.5, 2.5])
    np.testing.assert_array_equal(S.candidates(eps, 2.0, 3.0), [1, 2, 5])


def test_threshold_search_finds_the_blob_count():
    rng = np.random.default_rng(3)
    centres = rng.uniform(-2.5, 2.5, size=(12, 2))
    # keep centres apart by more than 1
    while True:
        d = np.linalg.norm(centres[:, None] - centres[None], axis=-1) + np.eye(12) * 9
        if d.min() > 1.0:
            break
        centres = rng.uniform(-2.5, 2.5, size=(12, 2))
    x = (centres[rng.integers(0, 12, 600)] + rng.normal(0, 0.05, size=(600, 2))).astype(np.float32)
    r = S.select(x, np.full(600, 2.5), 2, 3, 0.02, 12, 12, True, 50, periodic=[False, False])
    assert r["n_clusters"] == 12
    assert 0.2 < r["threshold"] < 1.0
    assert S.select(x, np.full(600, 2.5), 2, 3, 0.02, 12, 12, True, 5, periodic=[False, False])["selected"].size == 5
