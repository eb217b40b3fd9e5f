"""MCMC dimension reduction (rid_mcmc) against the FP64 MCMC oracle: walker
trajectories step by step, exact integer counting and binning, the
stationary 2-D marginal of a small landscape, the projected PMF, residual
nets, host / device arguments and errors.

Tolerances: both sides draw the same Philox numbers, so a walker's path is the
same as long as every accept decision is: the FP32 free energy differs from
the FP64 one by about 1e-6 relative, and a decision whose margin
|kT ln u + dAbar| came within 1e-3 of zero on the oracle side may go either
way (such walkers are excluded from the path comparison; there are few).
Along a path, the CVs agree to 1e-4 rad (FP32 sums of up to 40 proposals).
Bins are integer decisions taken from FP32 states; the counting test bins the
GPU's own states with the same FP32 operations.
"""
import math

import numpy as np
import pytest

from oracle import mcmc as MC
from oracle import train as T
from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def _wrapdiff(a, b):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return np.abs(d - 2 * math.pi * np.round(d / (2 * math.pi)))


def _bins_f32(s, bins):
    # floor((s + pi) * (1 / 2 pi) * bins), each operation rounded to FP32
    t = (np.float32(s) + np.float32(math.pi)).astype(np.float32)
    t = (t * np.float32(0.159154943091895)).astype(np.float32)
    t = (t * np.float32(bins)).astype(np.float32)
    return np.clip(np.floor(t).astype(np.int64), 0, bins - 1)


@pytest.mark.parametrize("M,C,L,H,resnet,W,K", [(4, 20, 4, 256, False, 256, 30), (2, 3, 3, 40, True, 100, 40)])
def test_trajectories_follow_the_oracle(R, M, C, L, H, resnet, W, K):
    ens = I.make_ensemble(M, 2 * C, L, H, 31, resnet=resnet)
    rng = np.random.default_rng(1)
    s0 = rng.uniform(-math.pi, math.pi, size=(W, C)).astype(np.float32)
    kT, step, seed, bins = 1.0, 0.25, 77, 101
    s = np.zeros_like(s0)
    nacc = R.mcmc(ens.weights, M, C, L, H, s0, K, 0, kT, step, seed, bins=bins, pair=(0, C - 1), resnet=resnet,
                  s_out=s)
    ref = MC.run(ens.weights, C, L, H, resnet, s0, K, 0, kT, step, seed, bins, (0, C - 1))
    safe = ref["min_margin"] > 1e-3
    print(f"\n[{M}x{H}x{L}] walkers with a near-threshold decision: {int((~safe).sum())} of {W}; "
          f"accepted {nacc} (oracle {ref['n_accepted']})")
    assert safe.mean() > 0.9
    assert np.max(_wrapdiff(s[safe], ref["s"][safe])) < 1e-4
    assert abs(nacc - ref["n_accepted"]) <= K * int((~safe).sum())
    assert 0 < nacc < W * K                      # moves are taken and refused


def test_counting_and_binning_are_exact(R):
    M, C, L, H, W, K = 2, 5, 2, 32, 300, 7
    ens = I.make_ensemble(M, 2 * C, L, H, 32)
    s0 = np.random.default_rng(2).uniform(-math.pi, math.pi, size=(W, C)).astype(np.float32)
    bins = 37
    s = np.zeros_like(s0)
    h1 = np.zeros((C, bins), np.uint64)
    h2 = np.zeros((bins, bins), np.uint64)
    f1 = np.zeros((C, bins))
    f2 = np.zeros((bins, bins))
    R.mcmc(ens.weights, M, C, L, H, s0, K, K - 1, 1.0, 0.6, 5, bins=bins, pair=(3, 1), s_out=s, hist1=h1, hist2=h2,
           pmf1=f1, pmf2=f2)
    b = _bins_f32(s, bins)                       # only the last step is counted: the final states
    for c in range(C):
        np.testing.assert_array_equal(h1[c], np.bincount(b[:, c], minlength=bins))
    want2 = np.zeros((bins, bins), np.int64)
    np.add.at(want2, (b[:, 3], b[:, 1]), 1)
    np.testing.assert_array_equal(h2, want2)
    for c in range(C):
        np.testing.assert_allclose(f1[c], MC.projected_pmf(h1[c], 1.0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(f2, MC.projected_pmf(h2, 1.0), rtol=1e-12, atol=1e-12)


def test_joint_histogram_matches_the_stationary_marginal(R):
    C, L, H, bins, kT = 2, 2, 8, 12, 1.0
    rng = np.random.default_rng(2)
    w = (rng.normal(0.0, 1.0, size=(1, T.param_count(2 * C, L, H))) * 0.7).astype(np.float32)
    n = bins * 12
    g = -math.pi + (np.arange(n) + 0.5) * (2 * math.pi / n)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    A = MC.ensemble_mean_value(w, 2 * C, L, H, False, np.stack([gx.ravel(), gy.ravel()], 1))
    p = np.exp(-(A - A.min()) / kT).reshape(n, n)
    p = np.add.reduceat(np.add.reduceat(p, np.arange(0, n, 12), axis=0), np.arange(0, n, 12), axis=1)
    p /= p.sum()
    W, K, burn = 4096, 1500, 300
    s0 = rng.uniform(-math.pi, math.pi, size=(W, C)).astype(np.float32)
    h2 = np.zeros((bins, bins), np.uint64)
    R.mcmc(w, 1, C, L, H, s0, K, burn, kT, 0.9, 3, bins=bins, pair=(0, 1), hist2=h2)
    assert int(h2.sum()) == W * (K - burn)
    tv = 0.5 * np.abs(h2 / h2.sum() - p).sum()
    print(f"\ntotal variation against the exact joint: {tv:.4f}")
    assert tv < 0.02, tv


def test_device_arguments_match_host_arguments(R):
    import torch
    M, C, L, H, W, K = 2, 4, 2, 48, 200, 12
    ens = I.make_ensemble(M, 2 * C, L, H, 33)
    s0 = np.random.default_rng(3).uniform(-math.pi, math.pi, size=(W, C)).astype(np.float32)
    sh = np.zeros_like(s0)
    h1 = np.zeros((C, 21), np.uint64)
    na = R.mcmc(ens.weights, M, C, L, H, s0, K, 2, 1.0, 0.4, 8, bins=21, s_out=sh, hist1=h1)
    sd = torch.zeros((W, C), dtype=torch.float32, device="cuda")
    hd = torch.zeros((C, 21), dtype=torch.uint64, device="cuda")
    nd = R.mcmc(torch.from_numpy(ens.weights).cuda(), M, C, L, H, torch.from_numpy(s0).cuda(), K, 2, 1.0, 0.4, 8,
                bins=21, s_out=sd, hist1=hd)
    assert na == nd
    assert np.array_equal(sh, sd.cpu().numpy())
    assert np.array_equal(h1, hd.cpu().numpy())


def test_errors(R):
    ens = I.make_ensemble(1, 4, 2, 16, 34)
    s0 = np.zeros((4, 2), np.float32)
    with pytest.raises(R.RidError) as e:
        R.mcmc(ens.weights, 1, 2, 2, 16, s0, 5, 0, 1.0, 0.3, 1, bins=10, pair=(0, 2))
    assert e.value.code == R.RID_ERR_ARG
    with pytest.raises(R.RidError) as e:
        R.mcmc(ens.weights, 1, 2, 2, 16, s0, 5, 0, 0.0, 0.3, 1, bins=10)
    assert e.value.code == R.RID_ERR_ARG


def test_path_projection_follows_the_oracle(R):
    # path nodes along a line in the (CV 0, CV 2) plane; the walkers' path
    # histogram against the oracle's on the same trajectories: the walkers
    # whose accept decisions came near the threshold may differ, and FP32
    # against FP64 can move a count across a bin edge
    M, C, L, H, W, K = 2, 4, 2, 32, 256, 30
    ens = I.make_ensemble(M, 2 * C, L, H, 35)
    s0 = np.random.default_rng(4).uniform(-math.pi, math.pi, size=(W, C)).astype(np.float32)
    nodes = np.stack([np.linspace(-2.5, 2.5, 9), np.linspace(1.0, -1.0, 9)], axis=1).astype(np.float32)
    path = (nodes, [0, 2], 2.0, -1.0, 3.0)
    bins = 25
    hp = np.zeros((bins, bins), np.uint64)
    fp = np.zeros((bins, bins))
    R.mcmc(ens.weights, M, C, L, H, s0, K, 10, 1.0, 0.4, 12, bins=bins, path=path, hist_path=hp, pmf_path=fp)
    ref = MC.run(ens.weights, C, L, H, False, s0, K, 10, 1.0, 0.4, 12, bins, (0, 1), path=path)
    unsafe = int((ref["min_margin"] <= 1e-3).sum())
    diff = int(np.abs(hp.astype(np.int64) - ref["hist_path"]).sum())
    print(f"\npath histogram: |GPU - oracle|_1 = {diff} of {W * (K - 10)} counts, near-threshold walkers {unsafe}")
    assert int(hp.sum()) == W * (K - 10)
    assert diff <= 2 * unsafe * (K - 10) + 0.01 * W * (K - 10)
    np.testing.assert_allclose(fp, MC.projected_pmf(hp, 1.0), rtol=1e-12, atol=1e-12)


def test_system_path_fp32_follows_the_oracle(R):
    # the system's own FP32 ensemble kernels evaluate the proposals
    M, C, L, H, W, K = 4, 6, 3, 64, 192, 25
    sp = I.make_system(40, C, 36)
    ens = I.make_ensemble(M, 2 * C, L, H, 36)
    s0 = np.random.default_rng(6).uniform(-math.pi, math.pi, size=(W, C)).astype(np.float32)
    s = np.zeros_like(s0)
    with R.System(sp) as sysobj:
        sysobj.set_ensemble(ens, precision=R.RID_PREC_FP32)
        nacc = sysobj.mcmc(s0, K, 0, 1.0, 0.3, 21, bins=51, s_out=s)
    ref = MC.run(ens.weights, C, L, H, False, s0, K, 0, 1.0, 0.3, 21, 51, (0, 1))
    safe = ref["min_margin"] > 1e-3
    assert safe.mean() > 0.9
    assert np.max(_wrapdiff(s[safe], ref["s"][safe])) < 1e-4
    assert abs(nacc - ref["n_accepted"]) <= K * int((~safe).sum())


def test_system_path_projection_follows_the_oracle(R):
    # the path projection through rid_mcmc_system (FP32 ensemble kernels of a
    # system) against the oracle's path histogram on the same trajectories,
    # with the bound of the standalone path test
    M, C, L, H, W, K, burn, bins = 2, 4, 2, 32, 256, 30, 10, 25
    ens = I.make_ensemble(M, 2 * C, L, H, 38)
    s0 = np.random.default_rng(8).uniform(-math.pi, math.pi, size=(W, C)).astype(np.float32)
    nodes = np.stack([np.linspace(-2.5, 2.5, 9), np.linspace(1.0, -1.0, 9)], axis=1).astype(np.float32)
    path = (nodes, [1, 3], 2.0, -1.0, 3.0)
    hp = np.zeros((bins, bins), np.uint64)
    fp = np.zeros((bins, bins))
    h2 = np.zeros((bins, bins), np.uint64)
    with R.System(I.make_system(30, C, 38)) as sysobj:
        sysobj.set_ensemble(ens, precision=R.RID_PREC_FP32)
        sysobj.mcmc(s0, K, burn, 1.0, 0.4, 14, bins=bins, hist2=h2, path=path, hist_path=hp, pmf_path=fp)
        h2b = np.zeros_like(h2)
        sysobj.mcmc(s0, K, burn, 1.0, 0.4, 14, bins=bins, hist2=h2b)
    ref = MC.run(ens.weights, C, L, H, False, s0, K, burn, 1.0, 0.4, 14, bins, (0, 1), path=path)
    unsafe = int((ref["min_margin"] <= 1e-3).sum())
    diff = int(np.abs(hp.astype(np.int64) - ref["hist_path"]).sum())
    print(f"\nsystem path histogram: |GPU - oracle|_1 = {diff} of {W * (K - burn)} counts, near-threshold {unsafe}")
    assert int(hp.sum()) == W * (K - burn)
    assert diff <= 2 * unsafe * (K - burn) + 0.01 * W * (K - burn)
    np.testing.assert_allclose(fp, MC.projected_pmf(hp, 1.0), rtol=1e-12, atol=1e-12)
    # the projection only counts: the chain and its other histograms are those of a run without it
    assert np.array_equal(h2, h2b)


def test_system_path_errors(R):
    C = 3
    ens = I.make_ensemble(1, 2 * C, 2, 32, 39)
    s0 = np.zeros((4, C), np.float32)
    nodes = np.zeros((3, 2), np.float32)
    with R.System(I.make_system(22, C, 39)) as sysobj:
        sysobj.set_ensemble(ens, precision=R.RID_PREC_FP32)
        for bad in ((nodes[:1], [0, 1], 1.0, 0.0, 1.0), (nodes, [0, 3], 1.0, 0.0, 1.0),
                    (nodes, [0, 1], 0.0, 0.0, 1.0), (nodes, [0, 1], 1.0, 1.0, 1.0)):
            with pytest.raises(R.RidError) as e:
                sysobj.mcmc(s0, 5, 0, 1.0, 0.3, 1, bins=10, path=bad)
            assert e.value.code == R.RID_ERR_ARG


@pytest.mark.parametrize("prec,bound", [("bf16", 0.02), ("fp8", 0.06)])
def test_system_path_tensor_cores_sample_the_stationary_marginal(R, prec, bound):
    # BF16 / FP8 ensembles on the tensor cores: the sampled joint of two CVs
    # against exp(-Abar/kT) of the FP64 network.  The low-precision forward
    # pass moves Abar by its relative error (BF16 about 5e-3, FP8 e4m3 about
    # 2e-2, the precision sweep's figures) times a landscape spanning a few kT,
    # so bin weights move by up to ~1% (BF16) and ~5% (FP8); the sampling
    # noise adds about 3e-3.  Measured: 3e-3 (BF16), 2.8e-2 (FP8).
    C, L, H, bins, kT = 2, 2, 32, 12, 1.0
    rng = np.random.default_rng(2)
    w = (rng.normal(0.0, 1.0, size=(1, T.param_count(2 * C, L, H))) * 0.5).astype(np.float32)
    n = bins * 12
    g = -math.pi + (np.arange(n) + 0.5) * (2 * math.pi / n)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    A = MC.ensemble_mean_value(w, 2 * C, L, H, False, np.stack([gx.ravel(), gy.ravel()], 1))
    p = np.exp(-(A - A.min()) / kT).reshape(n, n)
    p = np.add.reduceat(np.add.reduceat(p, np.arange(0, n, 12), axis=0), np.arange(0, n, 12), axis=1)
    p /= p.sum()
    W, K, burn = 4096, 1200, 200
    s0 = rng.uniform(-math.pi, math.pi, size=(W, C)).astype(np.float32)
    h2 = np.zeros((bins, bins), np.uint64)
    ens = I.EnsembleParams(1, 2 * C, L, H, False, w, 1e9, 2e9)
    with R.System(I.make_system(22, C, 37)) as sysobj:
        sysobj.set_ensemble(ens, precision={"bf16": R.RID_PREC_BF16, "fp8": R.RID_PREC_FP8}[prec])
        sysobj.mcmc(s0, K, burn, kT, 0.9, 3, bins=bins, pair=(0, 1), hist2=h2)
    assert int(h2.sum()) == W * (K - burn)
    tv = 0.5 * np.abs(h2 / h2.sum() - p).sum()
    print(f"\n[{prec}] total variation against the exact joint: {tv:.4f}")
    assert tv < bound, tv


# ------------------------------------------------------------------ distance CVs
def _mixed_diff(a, b, dist):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    d[:, ~dist] = d[:, ~dist] - 2 * math.pi * np.round(d[:, ~dist] / (2 * math.pi))
    return np.abs(d)


def _bins_f32_range(s, lo, hi, bins):
    # floor((s - lo) / (hi - lo) * bins), each operation rounded to FP32
    t = (np.float32(s) - np.float32(lo)).astype(np.float32)
    t = (t / (np.float32(hi) - np.float32(lo))).astype(np.float32)
    t = (t * np.float32(bins)).astype(np.float32)
    return np.clip(np.floor(t).astype(np.int64), 0, bins - 1)


def _mixed_start(W, C, dist, lo, hi, seed):
    rng = np.random.default_rng(seed)
    s0 = rng.uniform(-math.pi, math.pi, size=(W, C))
    for c in np.flatnonzero(dist):
        s0[:, c] = rng.uniform(lo[c], hi[c], size=W)
    return s0.astype(np.float32)


def test_distance_cvs_follow_the_oracle_and_bin_exactly(R):
    """rid_mcmc with two distance CVs (ranges [1, 3] and [2, 5]) beside three
    torsions: walker paths against the oracle (near-threshold and near-edge
    walkers left out), every state inside its range, exact counting in the
    range bins."""
    M, C, L, H, W, K = 3, 5, 3, 48, 256, 30
    dist = np.array([False, True, False, True, False])
    lo = np.array([0.0, 1.0, 0.0, 2.0, 0.0])
    hi = np.array([0.0, 3.0, 0.0, 5.0, 0.0])
    ens = I.make_ensemble(M, 2 * C, L, H, 41, resnet=True)
    s0 = _mixed_start(W, C, dist, lo, hi, 41)
    bins = 23
    s = np.zeros_like(s0)
    h1 = np.zeros((C, bins), np.uint64)
    h2 = np.zeros((bins, bins), np.uint64)
    nacc = R.mcmc(ens.weights, M, C, L, H, s0, K, K - 1, 1.0, 0.4, 19, bins=bins, pair=(1, 2), resnet=True,
                  s_out=s, hist1=h1, hist2=h2, cv_dist=dist, cv_range=(lo, hi))
    ref = MC.run(ens.weights, C, L, H, True, s0, K, K - 1, 1.0, 0.4, 19, bins, (1, 2), dist=dist, lo=lo, hi=hi)
    safe = ref["min_margin"] > 1e-3
    print(f"\n[mixed] near-threshold / near-edge walkers: {int((~safe).sum())} of {W}; accepted {nacc} "
          f"(oracle {ref['n_accepted']})")
    assert safe.mean() > 0.9
    assert np.max(_mixed_diff(s[safe], ref["s"][safe], dist)) < 1e-4
    assert abs(nacc - ref["n_accepted"]) <= K * int((~safe).sum())
    assert 0 < nacc < W * K
    for c in np.flatnonzero(dist):
        assert np.all((s[:, c] >= lo[c]) & (s[:, c] <= hi[c]))
    # only the last step is counted: the final states, binned with the FP32 operations
    for c in range(C):
        b = _bins_f32_range(s[:, c], lo[c], hi[c], bins) if dist[c] else _bins_f32(s[:, c], bins)
        np.testing.assert_array_equal(h1[c], np.bincount(b, minlength=bins))
    want2 = np.zeros((bins, bins), np.int64)
    np.add.at(want2, (_bins_f32_range(s[:, 1], lo[1], hi[1], bins), _bins_f32(s[:, 2], bins)), 1)
    np.testing.assert_array_equal(h2, want2)


def test_system_with_distance_cvs_follows_the_oracle(R):
    """rid_mcmc_system on a system mixing torsions and distances (FP32
    ensemble kernels; the kinds come from the system's cv_atoms)."""
    M, C, L, H, W, K = 4, 6, 3, 64, 192, 25
    sp = I.make_system(40, C, 42, n_dist=2)
    dist = I.cv_is_distance(sp)
    lo = np.where(dist, 1.5, 0.0)
    hi = np.where(dist, 4.5, 0.0)
    ens = I.make_ensemble(M, 2 * C, L, H, 42)
    s0 = _mixed_start(W, C, dist, lo, hi, 42)
    s = np.zeros_like(s0)
    with R.System(sp) as sysobj:
        sysobj.set_ensemble(ens, precision=R.RID_PREC_FP32)
        nacc = sysobj.mcmc(s0, K, 0, 1.0, 0.3, 23, bins=51, s_out=s, cv_range=(lo, hi))
        with pytest.raises(R.RidError) as e:
            sysobj.mcmc(s0, 5, 0, 1.0, 0.3, 23, bins=51)            # distance CVs need their ranges
        assert e.value.code == R.RID_ERR_ARG
        with pytest.raises(R.RidError) as e:
            sysobj.mcmc(s0, 5, 0, 1.0, 0.3, 23, bins=51, cv_range=(hi, lo))
        assert e.value.code == R.RID_ERR_ARG
    ref = MC.run(ens.weights, C, L, H, False, s0, K, 0, 1.0, 0.3, 23, 51, (0, 1), dist=dist, lo=lo, hi=hi)
    safe = ref["min_margin"] > 1e-3
    assert safe.mean() > 0.9
    assert np.max(_mixed_diff(s[safe], ref["s"][safe], dist)) < 1e-4
    assert abs(nacc - ref["n_accepted"]) <= K * int((~safe).sum())


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_system_with_distance_cvs_on_the_tensor_cores(R, prec):
    """The same mixed system with a BF16 / FP8 ensemble: runs, keeps every
    distance CV inside its range, and accepts moves."""
    M, C, L, H, W, K = 4, 6, 3, 64, 512, 40
    sp = I.make_system(40, C, 43, n_dist=2)
    dist = I.cv_is_distance(sp)
    lo, hi = np.where(dist, 1.5, 0.0), np.where(dist, 4.5, 0.0)
    ens = I.make_ensemble(M, 2 * C, L, H, 43)
    s0 = _mixed_start(W, C, dist, lo, hi, 43)
    s = np.zeros_like(s0)
    with R.System(sp) as sysobj:
        sysobj.set_ensemble(ens, precision=R.RID_PREC_BF16 if prec == "bf16" else R.RID_PREC_FP8)
        nacc = sysobj.mcmc(s0, K, 0, 1.0, 0.3, 29, bins=51, s_out=s, cv_range=(lo, hi))
    assert 0 < nacc < W * K
    for c in np.flatnonzero(dist):
        assert np.all((s[:, c] >= lo[c]) & (s[:, c] <= hi[c]))
