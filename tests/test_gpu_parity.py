"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (fixed here, from the FP32 arithmetic of the kernels):
  forces, CVs, member gradients:  |d| <= 1e-5 (|ref| + rms(ref))   (rel 1e-5)
  20-step trajectories:           |d| <= 1e-4 (|ref| + 1)
  Philox words, pair sets:        bit-exact
  normals:                        |d| <= 1e-6 (1 + r), r = Box-Muller radius
  mean-force labels:              within 2 combined standard errors (>= 90%
                                  of entries, none beyond 4)
"""
import math

import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORCE_RTOL = 1e-5
TRAJ_RTOL = 1e-4


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def close_rel(got, ref, rtol, axis=None):
    """Largest elementwise error relative to |ref| + rms(ref), in units of
    rtol: below 1 when every element is within rtol."""
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    scale = np.sqrt(np.mean(ref ** 2, axis=axis, keepdims=True)) if axis is not None else np.sqrt(np.mean(ref ** 2))
    err = np.abs(got - ref) / (np.abs(ref) + scale)
    return err.max() / rtol


def wrapd(d):
    return d - 2 * np.pi * np.floor(d / (2 * np.pi) + 0.5)


def setup(R, n_beads, n_cv, seed, W, M=4, L=3, H=64, ens_seed=None, **kw):
    sp = I.make_system(n_beads, n_cv, seed, **kw)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * n_cv, L, H, seed if ens_seed is None else ens_seed)
    return sp, x, ens


def set_trust_at_percentiles(R, sys, sp, x, ens, orc):
    """Put trust_lo / trust_hi at the 25th / 75th percentile of eps over x, so
    every switching region is exercised."""
    eps = np.array([orc.ensemble(ens, orc.cvs(sp, xi.astype(np.float64))[0])["eps"] for xi in x])
    ens.trust_lo, ens.trust_hi = float(np.percentile(eps, 25)), float(np.percentile(eps, 75))
    sys.set_ensemble(ens)
    return eps


# ------------------------------------------------------------------ Philox
def test_philox_words_bit_exact_and_normals(R, orc):
    rng = np.random.default_rng(0)
    n = 20000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 0], [5, 0, 7, 1]]
    seed = 0xDEADBEEF12345678
    words = np.zeros((n, 4), np.uint32)
    z = np.zeros((n, 3), np.float32)
    R.philox(ctr, seed, words, z)
    assert np.array_equal(words, orc.philox(ctr, seed))
    zr = orc.normals(ctr, seed)
    rad = np.hypot(zr[:, 0], zr[:, 1])
    assert np.all(np.abs(z[:, :2] - zr[:, :2]) <= 1e-6 * (1 + rad)[:, None])
    assert np.all(np.abs(z[:, 2] - zr[:, 2]) <= 1e-6 * (1 + np.abs(zr[:, 2]) * 2 + 2))


def test_philox_extreme_words(R, orc):
    # counters whose first / third output words sit near 0 and 2^32 are found by
    # search on the oracle; the normal transform must stay accurate there
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(400000, 4), dtype=np.uint64).astype(np.uint32)
    w = orc.philox(ctr, 3)
    pick = np.argsort(w[:, 0])[[0, 1, 2, -3, -2, -1]]
    c = np.ascontiguousarray(ctr[pick])
    z = np.zeros((len(pick), 3), np.float32)
    R.philox(c, 3, None, z)
    zr = orc.normals(c, 3)
    assert np.all(np.abs(z - zr) <= 2e-6 * (1 + np.abs(zr)))


# ------------------------------------------------------------------ pairs
@pytest.mark.parametrize("n,W,seed", [(22, 16, 1), (200, 8, 2), (37, 5, 3)])
def test_pair_inclusion_bit_exact(R, orc, n, W, seed):
    sp = I.make_system(n, 2, seed)
    x = I.make_chains(W, sp, seed)
    # squeeze some walkers so many pairs sit near the cutoff
    x[1::2] *= np.float32(0.83)
    with R.System(sp) as sys:
        nw = (n + 31) // 32
        mask = np.zeros((W, n, nw), np.uint32)
        sys.pair_mask(x, mask)
    for w in range(W):
        got = set()
        for i in range(n):
            for j in range(n):
                if (mask[w, i, j >> 5] >> (j & 31)) & 1:
                    got.add((min(i, j), max(i, j)))
                    assert (mask[w, j, i >> 5] >> (i & 31)) & 1   # symmetric
        want = {tuple(p) for p in orc.lj_pairs(x[w], sp.lj_rc)}
        assert got == want


# ------------------------------------------------------------------ forces
@pytest.mark.parametrize("n,C,W,seed,squeeze", [
    (22, 2, 16, 1, False), (200, 20, 40, 2, False), (61, 9, 33, 4, False), (4, 1, 3, 5, False),
    (200, 20, 12, 6, True),        # compressed walkers: many pairs and cluster boxes near the cutoff
    (257, 9, 5, 7, False),         # two passes of the bead loop, last warp holds one bead
    (1500, 16, 3, 8, False),       # beyond the shared-memory bonded slots, warps past the last bead
    (4096, 64, 2, 9, False),       # largest chain
])
def test_force_field_and_cvs(R, orc, n, C, W, seed, squeeze):
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    if squeeze:
        x[1::2] *= np.float32(0.83)
    f = np.zeros((W, n, 3), np.float32)
    s = np.zeros((W, C), np.float32)
    with R.System(sp) as sys:
        sys.eval_forces(x, R.RID_BIAS_NONE, f_out=f, s_out=s)
    for w in range(W):
        r = orc.total(sp, x[w].astype(np.float64), mode=0)
        assert close_rel(f[w], r["f"], FORCE_RTOL) < 1.0, w
        assert np.all(np.abs(wrapd(s[w] - r["s"])) <= FORCE_RTOL * np.maximum(1.0, np.abs(r["s"])))


@pytest.mark.parametrize("n,C,W,M,L,H,resnet,seed", [
    (22, 2, 16, 4, 3, 64, False, 1),
    (200, 20, 37, 4, 4, 256, False, 2),
    (60, 12, 70, 3, 2, 96, True, 6),
    (30, 1, 5, 2, 2, 32, True, 8),          # five walkers, one CV, width 32 (member in shared memory)
    (140, 64, 33, 2, 2, 96, False, 9),      # 128 inputs at width 96: the largest member held in shared memory
])
def test_biased_forces_eps_and_member_gradients(R, orc, n, C, W, M, L, H, resnet, seed):
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, resnet=resnet)
    f = np.zeros((W, n, 3), np.float32)
    s = np.zeros((W, C), np.float32)
    eps = np.zeros(W, np.float32)
    abar = np.zeros(W, np.float32)
    g = np.zeros((M, W, C), np.float32)
    with R.System(sp) as sys:
        epsr = set_trust_at_percentiles(R, sys, sp, x, ens, orc)
        sys.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=f, s_out=s, eps_out=eps, abar_out=abar, grad_out=g)
    sigmas = []
    for w in range(W):
        xd = x[w].astype(np.float64)
        r = orc.total(sp, xd, ens=ens, mode=1)
        e = orc.ensemble(ens, r["s"])
        sigmas.append(e["sigma"])
        assert close_rel(g[:, w], e["gradA"], FORCE_RTOL) < 1.0
        assert abs(eps[w] - e["eps"]) <= FORCE_RTOL * (abs(e["eps"]) + 1e-3)
        assert abs(abar[w] - e["Abar"]) <= FORCE_RTOL * (abs(e["Abar"]) + 1.0)
        # near the switching band edges a 1e-5 change in eps moves sigma; the
        # FF part is still compared tightly and the CV force through sigma
        # with the slope of the switch
        slope = math.pi / 2 / (ens.trust_hi - ens.trust_lo)
        tol = FORCE_RTOL + slope * abs(eps[w] - e["eps"])
        assert close_rel(f[w], r["f"], tol) < 1.0, w
    sig = np.array(sigmas)
    assert (sig == 1).any() and (sig == 0).any() and ((sig > 0) & (sig < 1)).any()
    assert np.allclose(eps, epsr, rtol=1e-4)


@pytest.mark.parametrize("n,C,W,M,L,H,resnet,seed", [
    (40, 6, 1003, 2, 3, 64, False, 31),     # 8-walker tiles, a ragged last tile of 3
    (30, 4, 4096, 4, 2, 32, True, 32),      # 32-walker tiles, residual
    (50, 8, 300, 3, 3, 96, True, 33),       # 2-walker tiles at width 96
])
def test_small_ensembles_on_walker_tiles(R, orc, n, C, W, M, L, H, resnet, seed):
    """Ensembles whose members fit in shared memory run one CTA per (tile,
    member) with the tile's walker count set by the walker count; sampled
    walkers (first, tile edges, last) against the oracle at 1e-5."""
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, resnet=resnet, trust_lo=1e9, trust_hi=2e9)
    g = np.zeros((M, W, C), np.float32)
    abar = np.zeros(W, np.float32)
    with R.System(sp) as sys:
        sys.set_ensemble(ens)
        sys.eval_forces(x, R.RID_BIAS_ENSEMBLE, abar_out=abar, grad_out=g)
    for w in sorted({0, 1, 7, 8, 31, 32, W // 2, W - 2, W - 1}):
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])
        assert close_rel(g[:, w], e["gradA"], FORCE_RTOL) < 1.0, w
        assert abs(abar[w] - e["Abar"]) <= FORCE_RTOL * (abs(e["Abar"]) + 1.0), w


def test_fp32_ensemble_at_the_size_limits(R, orc):
    # 128 torsion CVs (256 MLP inputs) and width 512: the FP32 ensemble
    # kernel's largest shared-memory footprint (activations, inputs and the
    # weight ring: 212 KB); two walker tiles, the second ragged
    n, C, W, M, L, H, seed = 140, 128, 40, 2, 3, 512, 12
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, trust_lo=1e9, trust_hi=2e9)
    eps = np.zeros(W, np.float32)
    abar = np.zeros(W, np.float32)
    g = np.zeros((M, W, C), np.float32)
    with R.System(sp) as sys:
        sys.set_ensemble(ens, precision=R.RID_PREC_FP32)
        sys.eval_forces(x, R.RID_BIAS_ENSEMBLE, eps_out=eps, abar_out=abar, grad_out=g)
    for w in (0, 1, 31, 32, 39):
        r = orc.total(sp, x[w].astype(np.float64), ens=ens, mode=1)
        e = orc.ensemble(ens, r["s"])
        assert close_rel(g[:, w], e["gradA"], FORCE_RTOL) < 1.0, w
        assert abs(eps[w] - e["eps"]) <= FORCE_RTOL * (abs(e["eps"]) + 1e-3)
        assert abs(abar[w] - e["Abar"]) <= FORCE_RTOL * (abs(e["Abar"]) + 1.0)


def test_restraint_forces(R, orc):
    sp = I.make_system(50, 7, 3)
    W = 9
    x = I.make_chains(W, sp, 3)
    s0 = I.make_label_targets(W, 7, 3)
    kap = np.random.default_rng(0).uniform(50, 500, size=(W, 7))
    f = np.zeros((W, 50, 3), np.float32)
    with R.System(sp) as sys:
        sys.eval_forces(x, R.RID_BIAS_RESTRAINT, s0=s0, kappa=kap, f_out=f)
    for w in range(W):
        r = orc.total(sp, x[w].astype(np.float64), mode=2, s0=s0[w], kappa=kap[w])
        assert close_rel(f[w], r["f"], FORCE_RTOL) < 1.0


def test_device_pointer_path_matches_host_path(R, orc):
    torch = pytest.importorskip("torch")
    sp = I.make_system(30, 4, 7)
    x = I.make_chains(12, sp, 7)
    ens = I.make_ensemble(4, 8, 2, 32, 7)
    fh = np.zeros((12, 30, 3), np.float32)
    with R.System(sp) as sys:
        sys.set_ensemble(ens)
        sys.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=fh)
        xd = torch.from_numpy(x).cuda()
        fd = torch.zeros((12, 30, 3), dtype=torch.float32, device="cuda")
        sys.eval_forces(xd, R.RID_BIAS_ENSEMBLE, f_out=fd, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
    assert np.array_equal(fd.cpu().numpy(), fh)


# ------------------------------------------------------------------ dynamics
@pytest.mark.parametrize("n,C,W,H,seed", [(22, 2, 16, 64, 1), (200, 20, 8, 256, 2), (45, 6, 35, 64, 9),
                                          (300, 12, 3, 64, 10)])   # two batches of the integrator loop
def test_twenty_step_biased_trajectories(R, orc, n, C, W, H, seed):
    sp = I.make_system(n, C, seed, output_freq=1)
    x0 = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(4, 2 * C, 3, H, seed)
    steps = 20
    cv = np.zeros((W, steps, C), np.float32)
    eps = np.zeros((W, steps), np.float32)
    xo = np.zeros((W, n, 3), np.float32)
    vo = np.zeros((W, n, 3), np.float32)
    with R.System(sp) as sys:
        set_trust_at_percentiles(R, sys, sp, x0, ens, orc)
        sys.explore(x0, steps, cv_out=cv, eps_out=eps, x_out=xo, v_out=vo)
    ref = orc.explore(sp, x0, steps, ens=ens)
    assert np.all(np.abs(xo - ref["x"]) <= TRAJ_RTOL * (np.abs(ref["x"]) + 1))
    assert np.all(np.abs(vo - ref["v"]) <= TRAJ_RTOL * (np.abs(ref["v"]) + 1))
    assert np.all(np.abs(wrapd(cv - ref["cv"])) <= TRAJ_RTOL * (np.abs(ref["cv"]) + 1))
    assert np.all(np.abs(eps - ref["eps"]) <= TRAJ_RTOL * (np.abs(ref["eps"]) + 1))


def test_unbiased_trajectory_and_mb_start(R, orc):
    sp = I.make_system(30, 3, 5, output_freq=5)
    x0 = I.make_chains(7, sp, 5)
    xo = np.zeros_like(x0)
    with R.System(sp) as sys:
        sys.explore(x0, 20, x_out=xo)
    ref = orc.explore(sp, x0, 20)
    assert np.all(np.abs(xo - ref["x"]) <= TRAJ_RTOL * (np.abs(ref["x"]) + 1))


def test_resume_is_bit_identical_and_runs_are_deterministic(R):
    sp = I.make_system(40, 4, 6, output_freq=4)
    x0 = I.make_chains(10, sp, 6)
    ens = I.make_ensemble(4, 8, 2, 64, 6)
    with R.System(sp) as sys:
        sys.set_ensemble(ens)
        xa, va = np.zeros_like(x0), np.zeros_like(x0)
        sys.explore(x0, 40, x_out=xa, v_out=va)
        xb, vb = np.zeros_like(x0), np.zeros_like(x0)
        sys.explore(x0, 40, x_out=xb, v_out=vb)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        x1, v1 = np.zeros_like(x0), np.zeros_like(x0)
        sys.explore(x0, 20, x_out=x1, v_out=v1)
        x2, v2 = np.zeros_like(x0), np.zeros_like(x0)
        sys.explore(x1, 20, v0=v1, step0=20, x_out=x2, v_out=v2)
        assert np.array_equal(x2, xa) and np.array_equal(v2, va)


def test_nve_energy_drift_within_twice_the_oracle(R, orc):
    sp = I.make_system(22, 2, 1, gamma=0.0, output_freq=50)
    x0 = I.make_chains(8, sp, 1)
    ens = I.make_ensemble(4, 4, 3, 64, 1, trust_lo=1e9, trust_hi=2e9)
    steps = 10000
    T = steps // 50
    en = np.zeros((8, T, 3))
    with R.System(sp) as sys:
        sys.set_ensemble(ens)
        sys.explore(x0, steps, energy_out=en)
    ref = orc.explore(sp, x0, steps, ens=ens, energy=True)
    def drift(e):
        E = e.sum(-1)
        return np.abs(E - E[:, :1]).max(axis=1) / (3 * sp.n_beads * sp.kT)
    dg, do = drift(en), drift(ref["energy"])
    # FP32 and FP64 trajectories decorrelate over 10k steps, so the bound is
    # on the walker average of the per-walker maximum deviation
    assert dg.mean() <= 2 * do.mean(), (dg, do)
    assert dg.max() < 2e-3
    # the first recorded frame agrees with the oracle's energy terms
    assert np.allclose(en[:, 0], ref["energy"][:, 0], rtol=1e-3, atol=1e-3)


def test_labels_within_two_standard_errors(R, orc):
    sp = I.make_system(22, 2, 1)
    Rn = 16
    x0 = I.make_chains(Rn, sp, 11)
    s0 = I.make_label_targets(Rn, 2, 11)
    kap = np.full((Rn, 2), 50.0)
    n_steps, n_equil, B = 4000, 400, 20
    mf, se, sd = (np.zeros((Rn, 2)) for _ in range(3))
    with R.System(sp) as sys:
        sys.label(x0, s0, kap, n_steps, n_equil, B, mf, se, sd)
    ref = orc.label(sp, x0, s0, kap, n_steps, n_equil, B)
    z = (mf - ref["mf"]) / np.sqrt(se ** 2 + ref["se"] ** 2)
    assert np.mean(np.abs(z) <= 2) >= 0.9 and np.all(np.abs(z) < 4), z
    assert np.all(se > 0) and np.all(sd > 0)
    assert np.allclose(sd, ref["std"], rtol=0.3)


def test_label_statistics_exact_on_first_steps(R, orc):
    """With n_equil = 0 and a short run the GPU and oracle trajectories are
    still close, so the label statistics agree tightly (checks the FP64 sums,
    block rule and finishing formulas, not just the statistics)."""
    sp = I.make_system(30, 4, 2)
    x0 = I.make_chains(6, sp, 2)
    s0 = I.make_label_targets(6, 4, 2)
    kap = np.full((6, 4), 200.0)
    mf, se, sd = (np.zeros((6, 4)) for _ in range(3))
    with R.System(sp) as sys:
        sys.label(x0, s0, kap, 23, 0, 7, mf, se, sd)
    ref = orc.label(sp, x0, s0, kap, 23, 0, 7)
    assert np.allclose(mf, ref["mf"], rtol=1e-4, atol=1e-3)
    assert np.allclose(se, ref["se"], rtol=1e-2, atol=1e-3)
    assert np.allclose(sd, ref["std"], rtol=1e-2, atol=1e-3)


# ------------------------------------------------------------------ edges & errors
def test_nonfinite_detection(R):
    sp = I.make_system(12, 2, 1)
    x = I.make_chains(3, sp, 1)
    x[1, 7] = x[1, 3]          # two non-excluded beads on top of each other: infinite LJ force
    with R.System(sp) as sys:
        with pytest.raises(R.RidError) as e:
            sys.explore(x, 2)
        assert e.value.code == R.RID_ERR_NONFINITE
        xo = np.zeros_like(x)
        sys.explore(x[[0, 2]].copy(), 2, x_out=xo[:2])   # the system stays usable
        assert np.isfinite(xo[:2]).all()


def test_argument_errors(R):
    sp = I.make_system(12, 2, 1)
    x = I.make_chains(2, sp, 1)
    with R.System(sp) as sys:
        with pytest.raises(R.RidError) as e:
            sys.set_ensemble(I.make_ensemble(2, 6, 2, 32, 1))      # n_in != 2 C
        assert e.value.code == R.RID_ERR_ARG
        with pytest.raises(R.RidError) as e:
            sys.label(x, np.zeros((2, 2)), np.ones((2, 2)), 10, 5, 20, *(np.zeros((2, 2)) for _ in range(3)))
        assert e.value.code == R.RID_ERR_ARG
        with pytest.raises(R.RidError) as e:
            sys.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=np.zeros((2, 12, 3), np.float32))
        assert e.value.code == R.RID_ERR_STATE


def test_full_size_chain200_w1024_sampled(R, orc):
    """The benchmark's workload size (1024 walkers, 200 beads, 20 CVs, 4 x
    40->256x4->1): every walker evaluated on the GPU, a sample checked
    against the oracle one by one, plus a short trajectory on a sample."""
    wl = I.workload("chain_n200_w1024")
    sp = I.make_system(wl["n_beads"], wl["n_cv"], 1)
    x = I.make_chains(wl["n_walkers"], sp, 1)
    ens = I.make_ensemble(wl["n_models"], 2 * wl["n_cv"], wl["n_layers"], wl["width"], 1)
    W = wl["n_walkers"]
    f = np.zeros((W, sp.n_beads, 3), np.float32)
    eps = np.zeros(W, np.float32)
    g = np.zeros((ens.n_models, W, sp.n_cv), np.float32)
    with R.System(sp) as sys:
        sys.set_ensemble(ens)
        sys.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=f, eps_out=eps, grad_out=g)
        for w in [0, 1, 31, 32, 511, 777, 1000, 1023]:
            r = orc.total(sp, x[w].astype(np.float64), ens=ens)
            e = orc.ensemble(ens, r["s"])
            assert close_rel(g[:, w], e["gradA"], FORCE_RTOL) < 1.0
            assert close_rel(f[w], r["f"], FORCE_RTOL) < 1.0
        xo = np.zeros_like(x)
        sys.explore(x, 20, x_out=xo)
    sample = [0, 513, 1023]
    ref = orc.explore(sp, x[sample], 20, ens=ens)
    # the oracle numbers walkers 0..2 in its Philox counters; rerun those three
    # on the GPU with the same numbering for the trajectory comparison
    with R.System(sp) as sys:
        sys.set_ensemble(ens)
        xs = np.zeros((3, sp.n_beads, 3), np.float32)
        sys.explore(np.ascontiguousarray(x[sample]), 20, x_out=xs)
    assert np.all(np.abs(xs - ref["x"]) <= TRAJ_RTOL * (np.abs(ref["x"]) + 1))
    assert np.isfinite(xo).all()
