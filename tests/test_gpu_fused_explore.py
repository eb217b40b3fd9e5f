"""Fused steps.  Exploration (k_explore_small): for small systems with FP32
ensembles every step of a call runs in one persistent launch, one CTA per
walker.  Each step is the per-step kernels' arithmetic in the same order, so
traces (CVs, model deviation), final positions and velocities are the same
bits as through the per-step kernels: checked on the paper's small
configuration's shape, with distance CVs, eight members, a 96-wide ensemble,
step counts with and without a final trace slot, calls continued from a
previous call, and a Maxwell-Boltzmann start.  Ineligible shapes (residual
networks, energy traces) take the per-step path with the switch on.  Labels:
rid_label of chains below 768 beads runs in one launch of the persistent label
kernel, with the same bits as through the per-step kernels."""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def run(R, sp, ens, x0, n_steps, fused, calls=1, v0=None, res=False):
    W, C = x0.shape[0], sp.n_cv
    T = n_steps // sp.output_freq
    out = []
    with R.System(sp) as sysm:
        sysm.set_ensemble(ens, precision=R.RID_PREC_FP32)
        sysm.set_fused_steps(fused)
        l0 = sysm.launch_count()
        sysm.walkers_load(x0, v0)
        for _ in range(calls):
            cv = np.zeros((W, T, C), np.float32)
            eps = np.zeros((W, T), np.float32)
            sysm.walkers_advance(n_steps, cv_out=cv, eps_out=eps)
            out += [cv, eps]
        xo, vo = np.zeros_like(x0), np.zeros_like(x0)
        sysm.walkers_read(x_out=xo, v_out=vo)
        launches = sysm.launch_count() - l0
    return out + [xo, vo], launches


CASES = [
    # n, C, nd, W, M, L, H, steps, of, calls, seed
    (22, 2, 0, 16, 4, 3, 64, 200, 10, 1, 1),     # the paper's small configuration's shape
    (22, 2, 0, 16, 4, 3, 64, 207, 10, 2, 2),     # no trace at the last step; a continued call
    (61, 9, 3, 8, 8, 2, 32, 150, 7, 1, 3),       # distance CVs, eight members
    (120, 12, 0, 5, 2, 2, 96, 60, 1, 1, 4),      # 96 wide, a trace every step
    (40, 4, 0, 33, 2, 4, 48, 90, 9, 1, 5),       # four hidden layers, ragged widths
]


@pytest.mark.parametrize("n,C,nd,W,M,L,H,steps,of,calls,seed", CASES)
def test_fused_steps_equal_per_step_kernels(R, n, C, nd, W, M, L, H, steps, of, calls, seed):
    sp = I.make_system(n, C, seed, n_dist=nd, dist_span=5, output_freq=of)
    x0 = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed)
    a, la = run(R, sp, ens, x0, steps, True, calls)
    b, lb = run(R, sp, ens, x0, steps, False, calls)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    assert np.all(np.isfinite(a[-2]))
    assert la < lb   # one launch per call instead of three per step


def test_fused_with_maxwell_boltzmann_start_and_trust_band(R, orc):
    sp = I.make_system(22, 2, 9, output_freq=5)
    x0 = I.make_chains(16, sp, 9)
    ens = I.make_ensemble(4, 4, 3, 64, 9)
    eps0 = np.array([orc.ensemble(ens, orc.cvs(sp, x0[w].astype(np.float64))[0])["eps"] for w in range(16)])
    ens.trust_lo, ens.trust_hi = float(np.percentile(eps0, 25)), float(np.percentile(eps0, 75))
    a, _ = run(R, sp, ens, x0, 100, True)
    b, _ = run(R, sp, ens, x0, 100, False)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("n,resnet", [(30, True), (200, False)])
def test_ineligible_shapes_take_the_per_step_path(R, n, resnet):
    """A residual ensemble, a chain above 128 beads."""
    sp = I.make_system(n, 3, 11, output_freq=5)
    x0 = I.make_chains(8, sp, 11)
    ens = I.make_ensemble(4, 6, 3, 64, 11, resnet=resnet)
    a, la = run(R, sp, ens, x0, 50, True)
    b, lb = run(R, sp, ens, x0, 50, False)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    assert la == lb
    with R.System(sp) as sysm:
        with pytest.raises(R.RidError) as e:
            R._check(R.lib().rid_set_fused_steps(sysm.h, 2))
        assert e.value.code == R.RID_ERR_ARG


@pytest.mark.parametrize("n,C,R_,steps,seed", [(22, 2, 16, 300, 21), (200, 20, 3, 240, 22), (700, 9, 40, 120, 23)])
def test_fused_labels_equal_per_step_kernels(R, n, C, R_, steps, seed):
    """rid_label of chains below 768 beads runs in one launch of the persistent
    label kernel; with the switch off, through the per-step kernels: the same
    bits (mean force, standard error, std, final positions and velocities),
    with a Maxwell-Boltzmann start and with given velocities."""
    sp = I.make_system(n, C, seed)
    x0 = I.make_chains(R_, sp, seed)
    rng = np.random.default_rng(seed)
    kap = rng.uniform(50.0, 500.0, size=(R_, C))
    outs = []
    for fused in (True, False):
        with R.System(sp) as sysm:
            sysm.set_fused_steps(fused)
            s = np.zeros((R_, C), np.float32)
            sysm.eval_forces(x0, R.RID_BIAS_NONE, s_out=s)
            s0 = s.astype(np.float64) + np.random.default_rng(seed + 1).uniform(-0.3, 0.3, size=s.shape)
            res = []
            for v0 in (None, (0.5 * rng.standard_normal(x0.shape)).astype(np.float32)):
                mf, se, sd = (np.zeros((R_, C)) for _ in range(3))
                xo, vo = np.zeros_like(x0), np.zeros_like(x0)
                sysm.label(x0, s0, kap, steps, steps // 5, 8, mf, se, sd, v0=v0, x_out=xo, v_out=vo)
                res += [mf, se, sd, xo, vo]
            outs.append(res)
        rng = np.random.default_rng(seed)
        kap = rng.uniform(50.0, 500.0, size=(R_, C))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert np.all(np.isfinite(outs[0][0]))


def test_small_configuration_as_benched(R, orc):
    """The paper's small configuration in the calls the benchmark times: 16
    walkers x 2000 biased steps in one exploration call (the fused kernel) and
    16 restrained runs (kappa 50, centres uniform on the torus) x 1000 steps in
    one label call (the persistent label kernel).  The first trace slot
    against the oracle's first 10 steps (1e-4), the last slot against the
    oracle's CVs and model deviation at the final positions the GPU reached
    (1e-5), labels within two combined standard errors of the oracle's."""
    sp = I.make_system(22, 2, 1, output_freq=10)
    W = 16
    x0 = I.make_chains(W, sp, 1)
    ens = I.make_ensemble(4, 4, 3, 64, 1)
    cv = np.zeros((W, 200, 2), np.float32)
    eps = np.zeros((W, 200), np.float32)
    xo = np.zeros_like(x0)
    s0 = I.make_label_targets(W, 2, 1)
    kap = np.full((W, 2), 50.0)
    mf, se, sd = (np.zeros((W, 2)) for _ in range(3))
    with R.System(sp) as sysm:
        sysm.set_ensemble(ens, precision=R.RID_PREC_FP32)
        sysm.explore(x0, 2000, cv_out=cv, eps_out=eps, x_out=xo)
        sysm.label(x0, s0, kap, 1000, 100, 20, mf, se, sd)
    assert np.isfinite(xo).all() and np.isfinite(cv).all() and np.isfinite(eps).all()
    first = orc.explore(sp, x0, 10, ens=ens)
    assert np.abs(np.angle(np.exp(1j * (cv[:, 0] - first["cv"][:, 0])))).max() < 1e-4
    assert np.allclose(eps[:, 0], first["eps"][:, 0], rtol=1e-4, atol=1e-5)
    for w in range(W):
        sr, _ = orc.cvs(sp, xo[w].astype(np.float64))
        assert np.abs(np.angle(np.exp(1j * (cv[w, -1] - sr)))).max() < 1e-5, w
        e = orc.ensemble(ens, sr)
        assert abs(eps[w, -1] - e["eps"]) <= 1e-4 * e["eps"] + 1e-6, w
    ref = orc.label(sp, x0, s0, kap, 1000, 100, 20)
    z = (mf - ref["mf"]) / np.sqrt(se ** 2 + ref["se"] ** 2)
    assert np.mean(np.abs(z) <= 2) >= 0.9 and np.all(np.abs(z) < 4), z
    assert np.all(se > 0) and np.allclose(sd, ref["std"], rtol=0.3)
