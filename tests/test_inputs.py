"""The seeded input generators (paper_2408_14070_gb300.inputs) against the
recipe they state: chain geometry (bond lengths, bond angles, self-avoidance,
centring), CV placement, force-field parameter ranges, Glorot-uniform weight
bounds and the packed layout's size, label targets on the torus,
determinism per seed, and the job mixes' ranges and arrival process.  CPU
only."""
import math

import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I


@pytest.mark.parametrize("n,W,seed", [(22, 16, 1), (200, 8, 2), (60, 5, 7)])
def test_chains_follow_the_recipe(n, W, seed):
    sp = I.make_system(n, 4, seed)
    x = I.make_chains(W, sp, seed).astype(np.float64)
    assert x.shape == (W, n, 3)
    b = np.linalg.norm(x[:, 1:] - x[:, :-1], axis=-1)
    assert np.max(np.abs(b - sp.bond_r0)) < 1e-5                    # bonds at r0 (float32 storage)
    u, v = x[:, :-2] - x[:, 1:-1], x[:, 2:] - x[:, 1:-1]
    ang = np.arccos(np.sum(u * v, -1) / (np.linalg.norm(u, axis=-1) * np.linalg.norm(v, axis=-1)))
    assert np.max(np.abs(ang - sp.angle_theta0)) < 1e-4              # angles at theta0
    d = np.linalg.norm(x[:, :, None] - x[:, None, :], axis=-1)
    i, j = np.triu_indices(n, 3)                                     # non-excluded pairs |i - j| >= 3
    assert d[:, i, j].min() >= 0.9 - 1e-5                            # self-avoiding at 0.9
    assert np.max(np.abs(x.mean(axis=1))) < 1e-4                     # centred
    assert not np.allclose(x[0], x[1])                               # walkers differ


def test_generators_are_deterministic_per_seed():
    sp = I.make_system(40, 6, 3)
    sp2 = I.make_system(40, 6, 3)
    assert np.array_equal(sp.dihedral_k, sp2.dihedral_k) and np.array_equal(sp.dihedral_delta, sp2.dihedral_delta)
    assert np.array_equal(I.make_chains(4, sp, 5), I.make_chains(4, sp, 5))
    assert not np.array_equal(I.make_chains(4, sp, 5), I.make_chains(4, sp, 6))
    e1, e2 = I.make_ensemble(2, 12, 3, 32, 9), I.make_ensemble(2, 12, 3, 32, 9)
    assert np.array_equal(e1.weights, e2.weights)
    assert not np.array_equal(e1.weights, I.make_ensemble(2, 12, 3, 32, 10).weights)
    assert np.array_equal(I.make_label_targets(3, 4, 1), I.make_label_targets(3, 4, 1))


def test_force_field_parameters_and_cv_placement():
    n, C = 120, 9
    sp = I.make_system(n, C, 4)
    assert sp.dihedral_k.shape == (n - 3, 3) and sp.dihedral_delta.shape == (n - 3, 3)
    assert sp.dihedral_k.min() >= 0 and sp.dihedral_k.max() < 2
    assert sp.dihedral_delta.min() >= 0 and sp.dihedral_delta.max() < 2 * math.pi
    first = np.floor((np.arange(C) + 0.5) * (n - 3) / C).astype(int)
    assert np.array_equal(sp.cv_atoms, first[:, None] + np.arange(4)[None, :])
    assert sp.cv_atoms.max() < n and len(set(first)) == C            # distinct, in range
    assert (sp.bond_k, sp.bond_r0, sp.angle_k, sp.lj_eps, sp.lj_sigma, sp.lj_rc) == (100.0, 1.0, 20.0, 1.0, 1.0, 2.5)
    assert sp.angle_theta0 == pytest.approx(math.radians(110.0))
    with pytest.raises(ValueError):
        I.evenly_spaced_cvs(3, 1)


def test_ensemble_layout_and_weight_bounds():
    M, D, L, H = 3, 10, 3, 32
    e = I.make_ensemble(M, D, L, H, 2)
    P = H * D + H + (L - 1) * (H * H + H) + H + 1
    assert e.weights.shape == (M, P) and I.ensemble_param_count(D, L, H) == P
    w = e.weights[0].astype(np.float64)
    o, fin = 0, D
    for _ in range(L):
        W = w[o:o + H * fin]
        o += H * fin
        a = math.sqrt(6.0 / (fin + H))
        assert np.abs(W).max() <= a and np.abs(W).max() > 0.8 * a   # Glorot-uniform bound, filled
        assert np.abs(w[o:o + H]).max() <= 0.2                       # biases U(-0.2, 0.2)
        o += H
        fin = H
    assert np.abs(w[o:o + H]).max() <= math.sqrt(6.0 / (H + 1))
    assert o + H + 1 == P


def test_label_targets_on_the_torus():
    s0 = I.make_label_targets(2000, 3, 8)
    assert s0.shape == (2000, 3) and s0.min() >= -math.pi and s0.max() < math.pi
    assert abs(s0.mean()) < 0.1


def test_job_mixes_follow_their_ranges():
    jobs = I.label_batch_jobs(300, 3)
    b = I.chain_length_buckets(50, 500)
    assert all(j["n_beads"] in b for j in jobs)
    assert all(4 <= j["n_cv"] <= min(40, j["n_beads"] - 3) for j in jobs)
    assert all(50 <= j["kappa"].min() and j["kappa"].max() <= 500 and j["kappa"].size == j["n_cv"] for j in jobs)
    assert all(j["width"] % 32 == 0 and 128 <= j["width"] <= 512 for j in jobs)
    # log-uniform lengths: about as many jobs below the geometric mean as above it
    n = np.array([j["n_beads"] for j in jobs])
    assert 0.35 < np.mean(n < math.sqrt(50 * 500)) < 0.65
    reqs = I.serving_requests(2000, 200.0, 5)
    t = np.array([r["t"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.min() > 0 and abs(gaps.mean() - 1 / 200.0) < 5 * (1 / 200.0) / math.sqrt(len(gaps))
    frac = np.mean([r["kind"] == "label" for r in reqs])
    assert abs(frac - 0.7) < 5 * math.sqrt(0.7 * 0.3 / len(reqs))
    assert all(r["walkers"] == (1 if r["kind"] == "label" else 12) for r in reqs)
    assert all(500 <= r["n_steps"] <= 5000 and 2 <= r["n_cv"] <= 64 for r in reqs)
