"""GPU parity of the BF16 tensor-core ensemble path (tcgen05 + TMA) against
the FP64 oracle.

Tolerance (derived from the arithmetic, BF16 operands with FP32
accumulation): weights and activations are rounded to BF16 (unit roundoff
u = 2^-9) before each of the 2L GEMMs, and tanh uses the hardware
approximation (relative error ~2^-11).  Each GEMM adds a relative error of a
few u in the normwise sense, so after 2L = 8 GEMMs the member gradients carry
~1e-2; the test bound is 3e-2 normwise per walker (member gradients, mean
force) and 5e-2 on the model deviation eps (a difference of gradients).
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GRAD_TOL = 3e-2
EPS_TOL = 5e-2


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def normwise(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


def run_eval(R, sp, ens, x, prec):
    W = x.shape[0]
    f = np.zeros((W, sp.n_beads, 3), np.float32)
    eps = np.zeros(W, np.float32)
    abar = np.zeros(W, np.float32)
    g = np.zeros((ens.n_models, W, sp.n_cv), np.float32)
    with R.System(sp) as sys:
        sys.set_ensemble(ens, precision=prec)
        sys.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=f, eps_out=eps, abar_out=abar, grad_out=g)
    return f, eps, abar, g


@pytest.mark.parametrize("n,C,W,M,L,H,seed", [
    (200, 20, 300, 4, 4, 256, 1),      # the benchmark shape, ragged walker count
    (22, 2, 16, 4, 3, 64, 2),          # tiny chain: D = 4 padded to 64
    (60, 9, 130, 3, 2, 96, 3),         # width not a multiple of 64 (partial K-chunks)
    (80, 16, 200, 4, 3, 160, 7),       # width 160: three chunks, the last half full
    (150, 64, 129, 2, 2, 64, 8),       # 128 inputs (two input chunks) wider than the hidden layers
])
def test_bf16_member_gradients_eps_and_values(R, orc, n, C, W, M, L, H, seed):
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, trust_lo=1e9, trust_hi=2e9)
    f, eps, abar, g = run_eval(R, sp, ens, x, R.RID_PREC_BF16)
    sample = sorted(set([0, 1, W // 2, W - 1] + list(range(0, W, max(1, W // 12)))))
    for w in sample:
        xd = x[w].astype(np.float64)
        r = orc.total(sp, xd, ens=ens)
        e = orc.ensemble(ens, r["s"])
        for m in range(M):
            assert normwise(g[m, w], e["gradA"][m]) < GRAD_TOL, (w, m)
        assert abs(eps[w] - e["eps"]) <= EPS_TOL * abs(e["eps"]) + 1e-4
        assert abs(abar[w] - e["Abar"]) <= GRAD_TOL * (abs(e["Abar"]) + 0.1)
        fb = f[w] - orc.total(sp, xd)["f"]          # the CV (bias) part of the force
        rb = r["f"] - orc.total(sp, xd)["f"]
        assert normwise(fb, rb) < GRAD_TOL, w


def test_bf16_width512_eight_members(R, orc):
    """The precision-sweep shape (64 -> 512 x 4 -> 1, 8 members) on a sample:
    one accumulator (512 TMEM columns) and two 256-row weight halves per chunk."""
    sp = I.make_system(100, 32, 4)
    W = 150
    x = I.make_chains(W, sp, 4)
    ens = I.make_ensemble(8, 64, 4, 512, 4, trust_lo=1e9, trust_hi=2e9)
    f, eps, abar, g = run_eval(R, sp, ens, x, R.RID_PREC_BF16)
    for w in [0, 77, 128, 149]:
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])
        for m in range(8):
            assert normwise(g[m, w], e["gradA"][m]) < GRAD_TOL
        assert abs(eps[w] - e["eps"]) <= EPS_TOL * abs(e["eps"]) + 1e-4


def test_bf16_runs_are_deterministic_and_close_to_fp32(R):
    sp = I.make_system(200, 20, 5)
    x = I.make_chains(256, sp, 5)
    ens = I.make_ensemble(4, 40, 4, 256, 5)
    a = run_eval(R, sp, ens, x, R.RID_PREC_BF16)
    b = run_eval(R, sp, ens, x, R.RID_PREC_BF16)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))
    c = run_eval(R, sp, ens, x, R.RID_PREC_FP32)
    for w in range(0, 256, 17):
        assert normwise(a[3][:, w], c[3][:, w]) < GRAD_TOL


def test_bf16_switching_and_trajectory(R, orc):
    sp = I.make_system(200, 20, 6, output_freq=1)
    W = 8
    x0 = I.make_chains(W, sp, 6)
    ens = I.make_ensemble(4, 40, 4, 256, 6)
    eps_r = np.array([orc.ensemble(ens, orc.cvs(sp, xi.astype(np.float64))[0])["eps"] for xi in x0])
    ens.trust_lo, ens.trust_hi = float(np.percentile(eps_r, 25)), float(np.percentile(eps_r, 75))
    steps = 20
    xo = np.zeros_like(x0)
    eps = np.zeros((W, steps), np.float32)
    with R.System(sp) as sys:
        sys.set_ensemble(ens, precision=R.RID_PREC_BF16)
        sys.explore(x0, steps, eps_out=eps, x_out=xo)
    ref = orc.explore(sp, x0, steps, ens=ens)
    # BF16 bias forces perturb the trajectory by ~1e-2 of the bias force, dt^2 scaled
    assert np.all(np.abs(xo - ref["x"]) <= 1e-3 * (np.abs(ref["x"]) + 1))
    assert np.all(np.abs(eps - ref["eps"]) <= EPS_TOL * np.abs(ref["eps"]) + 1e-3)


# Residual networks and widths that are not a multiple of 32 (padded inside the
# library with zero units, an exact transformation).  The first case is the
# paper's own ensemble (Sec. "Training phase": four models, neurons
# [300, 300, 300, 300], resnet) on 18 torsion CVs, the count of its chignolin
# example (Sec. "CV selection").
RESNET_CASES = [
    (120, 18, 200, 4, 4, 300, True, 21),   # 4 x 36->300x4->1, resnet: width 320 inside, five K-chunks
    (60, 9, 130, 3, 3, 96, True, 22),      # resnet, width not a multiple of 64
    (100, 32, 150, 8, 4, 512, True, 23),   # resnet at width 512 (a single TMEM accumulator)
    (40, 6, 70, 2, 3, 300, False, 24),     # width 300 without residuals
    (30, 3, 20, 2, 2, 45, True, 25),       # odd width 45 (64 inside)
    (22, 2, 9, 4, 1, 64, True, 26),        # one hidden layer: no residual term to add
]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("n,C,W,M,L,H,resnet,seed", RESNET_CASES)
def test_resnet_and_any_width(R, orc, prec, n, C, W, M, L, H, resnet, seed):
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, resnet=resnet, trust_lo=1e9, trust_hi=2e9)
    p = dict(fp32=R.RID_PREC_FP32, bf16=R.RID_PREC_BF16, fp8=R.RID_PREC_FP8)[prec]
    f, eps, abar, g = run_eval(R, sp, ens, x, p)
    worst = 0.0
    for w in sorted(set([0, 1, W // 2, W - 1] + list(range(0, W, max(1, W // 10))))):
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])
        if prec == "fp32":
            # the FP32 SIMT path: element-wise 1e-5 as in the unit parity tests
            ref = e["gradA"]
            sc = np.sqrt(np.mean(ref ** 2))
            assert (np.abs(g[:, w] - ref) / (np.abs(ref) + sc)).max() < 1e-5, w
            assert abs(eps[w] - e["eps"]) <= 1e-5 * (abs(e["eps"]) + 1e-3)
            assert abs(abar[w] - e["Abar"]) <= 1e-5 * (abs(e["Abar"]) + 1.0)
            continue
        if prec == "bf16":
            for m in range(M):
                assert normwise(g[m, w], e["gradA"][m]) < GRAD_TOL, (w, m)
            assert abs(abar[w] - e["Abar"]) <= GRAD_TOL * (abs(e["Abar"]) + 0.1)
        fbar = g[:, w].astype(np.float64).mean(axis=0)
        worst = max(worst, normwise(fbar, e["gradA"].mean(axis=0)))
        assert abs(eps[w] - e["eps"]) <= EPS_TOL * abs(e["eps"]) + 1e-4, w
    assert worst < (GRAD_TOL if prec == "bf16" else 6e-2)
    assert np.all(np.isfinite(f))


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_paper_network_trajectory(R, orc, prec):
    """20 biased steps with the paper's 4 x [300]^4 residual ensemble on the
    tensor cores, the switching band placed inside the walkers' eps range."""
    sp = I.make_system(120, 18, 27, output_freq=1)
    W = 12                                     # the paper's walker count
    x0 = I.make_chains(W, sp, 27)
    ens = I.make_ensemble(4, 36, 4, 300, 27, resnet=True)
    eps_r = np.array([orc.ensemble(ens, orc.cvs(sp, xi.astype(np.float64))[0])["eps"] for xi in x0])
    ens.trust_lo, ens.trust_hi = float(np.percentile(eps_r, 25)), float(np.percentile(eps_r, 75))
    steps = 20
    xo = np.zeros_like(x0)
    eps = np.zeros((W, steps), np.float32)
    with R.System(sp) as sysobj:
        sysobj.set_ensemble(ens, precision=R.RID_PREC_BF16 if prec == "bf16" else R.RID_PREC_FP8)
        sysobj.explore(x0, steps, eps_out=eps, x_out=xo)
    ref = orc.explore(sp, x0, steps, ens=ens)
    tol = 1e-3 if prec == "bf16" else 2e-3
    assert np.all(np.abs(xo - ref["x"]) <= tol * (np.abs(ref["x"]) + 1))
    assert np.all(np.abs(eps - ref["eps"]) <= (EPS_TOL if prec == "bf16" else 1e-1) * np.abs(ref["eps"]) + 1e-3)


@pytest.mark.parametrize("n,C,W,M,L,H,seed", [
    (200, 20, 300, 4, 4, 256, 1),      # the benchmark shape
    (60, 9, 130, 3, 2, 96, 3),         # width 96: the FP8 K-chunk (128 columns) is partly padding
    (80, 16, 200, 4, 3, 160, 7),       # width 160: two FP8 K-chunks, the second partly padding
    (150, 64, 129, 2, 2, 64, 8),       # 128 inputs (one FP8 chunk), width 64 (half a chunk)
])
def test_fp8_mean_force_and_eps(R, orc, n, C, W, M, L, H, seed):
    """FP8 e4m3 forward GEMMs (BF16 input gradient): mean force within 6e-2
    and eps within 5e-2 of the oracle (host emulation: about 2e-2)."""
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, trust_lo=1e9, trust_hi=2e9)
    f, eps, abar, g = run_eval(R, sp, ens, x, R.RID_PREC_FP8)
    worst_f = worst_e = 0.0
    for w in sorted(set([0, 1, W // 2, W - 1] + list(range(0, W, max(1, W // 12))))):
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])
        fbar = g[:, w].astype(np.float64).mean(axis=0)
        worst_f = max(worst_f, normwise(fbar, e["gradA"].mean(axis=0)))
        worst_e = max(worst_e, abs(eps[w] - e["eps"]) / e["eps"])
    print(f"\n[fp8 {n},{C},{H}] mean force {worst_f:.2e} eps {worst_e:.2e}")
    assert worst_f < 6e-2 and worst_e < 5e-2


def test_fp8_trajectory_is_deterministic(R):
    sp = I.make_system(100, 16, 9, output_freq=5)
    x0 = I.make_chains(40, sp, 9)
    ens = I.make_ensemble(4, 32, 3, 128, 9)
    outs = []
    for _ in range(2):
        xo = np.zeros_like(x0)
        eps = np.zeros((40, 4), np.float32)
        with R.System(sp) as sysobj:
            sysobj.set_ensemble(ens, precision=R.RID_PREC_FP8)
            sysobj.explore(x0, 20, eps_out=eps, x_out=xo)
        outs.append((xo, eps))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.all(np.isfinite(outs[0][0]))


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("n,C,W,M,L,H,seed", [
    (300, 128, 40, 16, 8, 512, 11),    # largest ensemble: 16 members, 8 layers, width 512, 256 inputs
    (60, 9, 1, 4, 3, 64, 12),          # a single walker (one mostly empty tile)
    (40, 8, 129, 4, 3, 96, 13),        # one walker past a full tile
    (4, 1, 7, 2, 1, 32, 14),           # minimal chain and network: one CV, one hidden layer of 32
])
def test_tensor_core_limits(R, orc, prec, n, C, W, M, L, H, seed):
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, trust_lo=1e9, trust_hi=2e9)
    f, eps, abar, g = run_eval(R, sp, ens, x, R.RID_PREC_BF16 if prec == "bf16" else R.RID_PREC_FP8)
    # the per-GEMM rounding errors add up roughly as the square root of the
    # number of GEMMs (2L): the 4-layer bounds scaled by sqrt(L / 4) for deeper nets
    scale = max(1.0, (L / 4) ** 0.5)
    tol = (GRAD_TOL if prec == "bf16" else 6e-2) * scale
    for w in sorted(set([0, W // 2, W - 1])):
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])
        fbar = g[:, w].astype(np.float64).mean(axis=0)
        ref = e["gradA"].mean(axis=0)
        assert np.linalg.norm(fbar - ref) <= tol * np.linalg.norm(ref) + 1e-4, w
        assert abs(eps[w] - e["eps"]) <= EPS_TOL * scale * abs(e["eps"]) + 1e-3, w
    assert np.all(np.isfinite(f))


# The ensemble kernel's cluster variants (each GEMM's output columns split over
# 2 or 4 CTAs, the next operand exchanged through distributed shared memory)
# must give the same bits as the one-CTA kernel; the autotuner may pick any.
CLUSTER_CASES = [
    (200, 20, 300, 4, 4, 256, False, 1),   # the benchmark's ensemble, ragged walker count
    (120, 18, 200, 4, 4, 300, True, 21),   # the paper's residual network: 80- and 160-column slices
    (60, 9, 130, 3, 3, 96, True, 22),      # 48-column slices at S = 2; 32, 32, 32 and none at S = 4
    (22, 2, 16, 4, 3, 64, False, 2),       # last GEMM N = 64 (D = 4 padded): 16-column slices at S = 4
    (150, 64, 100, 2, 2, 32, False, 32),   # 128 inputs, width 32: an operand buffer reused at a narrower K
    (40, 8, 700, 2, 2, 32, False, 33),     # width 32 at S = 4: two CTAs with 16 columns, two with none
]


def small_batch_tiles(H, D):
    """128-output tiles of the widest GEMM (hidden width H, or the input
    gradient's D inputs padded to 64)."""
    return -(-max(H, -(-D // 64) * 64) // 128)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("n,C,W,M,L,H,resnet,seed", CLUSTER_CASES)
def test_cluster_sizes_give_identical_bits(R, orc, prec, n, C, W, M, L, H, resnet, seed):
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, resnet=resnet)
    eps_r = np.array([orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])["eps"] for w in range(0, W, 7)])
    ens.trust_lo, ens.trust_hi = float(np.percentile(eps_r, 25)), float(np.percentile(eps_r, 75))
    p = R.RID_PREC_BF16 if prec == "bf16" else R.RID_PREC_FP8
    outs = {}
    for cs in (1, 2, 4):
        f = np.zeros((W, n, 3), np.float32)
        eps = np.zeros(W, np.float32)
        abar = np.zeros(W, np.float32)
        g = np.zeros((M, W, C), np.float32)
        with R.System(sp) as sysobj:
            sysobj.set_ensemble(ens, precision=p)
            sysobj.set_mlp_cluster(cs)
            sysobj.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=f, eps_out=eps, abar_out=abar, grad_out=g)
            # up to 16 walkers a BF16 ensemble runs the small-batch kernel, its 128-output
            # tiles split over at most cs CTAs
            t = small_batch_tiles(H, 2 * C)
            assert sysobj.mlp_cluster() == (min(cs, t) if W <= 16 and prec == "bf16" and t <= 4 else cs)
            xo = np.zeros_like(x[:9])
            sysobj.explore(np.ascontiguousarray(x[:9]), 6, x_out=xo)
        outs[cs] = (f, eps, abar, g, xo)
    for cs in (2, 4):
        for a, b in zip(outs[cs], outs[1]):
            assert np.array_equal(a, b), cs
    # and the shared result is the oracle's within the precision's bound
    f, eps, abar, g, _ = outs[4]
    tol = GRAD_TOL if prec == "bf16" else 6e-2
    for w in sorted(set([0, W // 2, W - 1])):
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])
        fbar = g[:, w].astype(np.float64).mean(axis=0)
        assert normwise(fbar, e["gradA"].mean(axis=0)) < tol, w
        if prec == "bf16":
            # (FP8 member values carry the e4m3 forward error; they are checked
            # through the MCMC sampling tests)
            assert abs(abar[w] - e["Abar"]) <= tol * (abs(e["Abar"]) + 0.1), w


def test_cluster_size_argument_errors(R):
    sp = I.make_system(22, 2, 1)
    with R.System(sp) as sysobj:
        with pytest.raises(R.RidError) as e:
            sysobj.set_mlp_cluster(3)
        assert e.value.code == R.RID_ERR_ARG
        # width 512 with 256 inputs: two operand buffers do not fit shared memory
        # (65 walkers: above the small-batch kernel's range (16), which runs
        # whatever the cluster setting)
        sp2 = I.make_system(140, 128, 2)
        with R.System(sp2) as s2:
            s2.set_ensemble(I.make_ensemble(2, 256, 2, 512, 2), precision=R.RID_PREC_BF16)
            s2.set_mlp_cluster(4)
            x = I.make_chains(65, sp2, 2)
            with pytest.raises(R.RidError) as e:
                s2.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=np.zeros((65, 140, 3), np.float32))
            assert e.value.code == R.RID_ERR_ARG
            s2.set_mlp_cluster(0)
            s2.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=np.zeros((65, 140, 3), np.float32))
            # up to 16 walkers the small-batch kernel runs, its four 128-output tiles
            # split over at most the fixed number of CTAs
            x3 = np.ascontiguousarray(x[:3])
            for cs, used in ((4, 4), (2, 2), (1, 1), (0, 4)):
                s2.set_mlp_cluster(cs)
                s2.eval_forces(x3, R.RID_BIAS_ENSEMBLE, f_out=np.zeros((3, 140, 3), np.float32))
                assert s2.mlp_cluster() == used, cs


def test_full_size_as_benched(R, orc):
    """The benchmark's workload and launch configuration: 1024 walkers of the
    200-bead chain, 20 torsions, the BF16 ensemble 4 x 40->256x4->1 with the
    default trust levels, inputs drawn as the benchmark draws them.  One force
    evaluation, member gradients and eps checked against the oracle on a
    sample of walkers one by one (tiles 0, 1, 3 and 7, first and last rows);
    then 20 resident steps, the path the benchmark times, with the CV and eps
    traces' last slot checked against the oracle at the final positions the
    GPU reached."""
    sp = I.make_system(200, 20, 1, output_freq=10)
    W = 1024
    x = I.make_chains(W, sp, 1)
    ens = I.make_ensemble(4, 40, 4, 256, 1)
    sample = [0, 1, 127, 128, 511, 777, 1000, 1023]
    s = np.zeros((W, 20), np.float32)
    f, eps, abar, g = (np.zeros((W, 200, 3), np.float32), np.zeros(W, np.float32), np.zeros(W, np.float32),
                       np.zeros((4, W, 20), np.float32))
    with R.System(sp) as sysm:
        sysm.set_ensemble(ens, precision=R.RID_PREC_BF16)
        sysm.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=f, s_out=s, eps_out=eps, abar_out=abar, grad_out=g)
        for w in sample:
            sr, _ = orc.cvs(sp, x[w].astype(np.float64))
            assert np.abs(np.angle(np.exp(1j * (s[w] - sr)))).max() < 1e-5
            e = orc.ensemble(ens, sr)
            for m in range(4):
                assert normwise(g[m, w], e["gradA"][m]) < GRAD_TOL, (w, m)
            assert normwise(g[:, w].mean(axis=0), e["gradA"].mean(axis=0)) < GRAD_TOL, w
            assert abs(eps[w] - e["eps"]) <= EPS_TOL * abs(e["eps"]) + 1e-4, w
        assert np.isfinite(f).all()
        sysm.walkers_load(x)
        cv = np.zeros((W, 2, 20), np.float32)
        et = np.zeros((W, 2), np.float32)
        sysm.walkers_advance(20, cv_out=cv, eps_out=et)
        xo = np.zeros_like(x)
        sysm.walkers_read(x_out=xo)
    assert np.isfinite(xo).all() and np.isfinite(cv).all()
    for w in sample:
        sr, _ = orc.cvs(sp, xo[w].astype(np.float64))
        assert np.abs(np.angle(np.exp(1j * (cv[w, -1] - sr)))).max() < 1e-4, w
        e = orc.ensemble(ens, sr)
        assert abs(et[w, -1] - e["eps"]) <= EPS_TOL * abs(e["eps"]) + 1e-4, w
