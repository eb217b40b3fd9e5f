"""The force-field kernel's CTA-size tuner and its split of a walker's chain
over several CTAs at few walkers: every size it may pick and every split give
the same forces bit for bit (each thread sums its own beads in a fixed order), the
energy trace does not depend on the size (energy launches keep the default),
and a whole biased trajectory is the same with a fixed small size, the tuned
size and the default.  Forces are also checked against the oracle at 1e-5,
whichever size the tuner kept."""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def default_threads(N):
    return min(224, max(32, (N + 31) // 32 * 32))


@pytest.mark.parametrize("n,W,seed", [(200, 96, 1), (150, 40, 2), (61, 33, 3), (22, 16, 4), (480, 8, 5)])
def test_every_cta_size_gives_the_same_forces(R, orc, n, W, seed):
    sp = I.make_system(n, 4, seed)
    x = I.make_chains(W, sp, seed)
    dth = default_threads(n)
    outs = {}
    with R.System(sp) as sysm:
        for th in [0] + list(range(32, dth + 1, 32)):
            sysm.set_ff_threads(th)
            f = np.zeros((W, n, 3), np.float32)
            sysm.eval_forces(x, R.RID_BIAS_NONE, f_out=f)
            got = sysm.ff_threads()
            if th:
                assert got == th
            else:
                assert got % 32 == 0 and 64 <= got <= dth or got == dth
            outs[th] = f
    for th, f in outs.items():
        assert np.array_equal(f, outs[0]), th
    for w in (0, W // 2, W - 1):
        ref = orc.total(sp, x[w].astype(np.float64))["f"]
        scale = np.abs(ref) + np.sqrt(np.mean(ref ** 2))
        assert (np.abs(outs[0][w] - ref) / scale).max() < 1e-5


def test_trajectory_and_energy_trace_do_not_depend_on_the_size(R):
    sp = I.make_system(120, 6, 7, output_freq=2)
    x0 = I.make_chains(24, sp, 7)
    ens = I.make_ensemble(4, 12, 3, 64, 7)
    res = []
    for th in (64, 0, default_threads(120)):
        xo, vo = np.zeros_like(x0), np.zeros_like(x0)
        cv = np.zeros((24, 10, 6), np.float32)
        en = np.zeros((24, 10, 3))
        with R.System(sp) as sysm:
            sysm.set_ensemble(ens, precision=R.RID_PREC_BF16)
            sysm.set_ff_threads(th)
            sysm.explore(x0, 20, cv_out=cv, energy_out=en, x_out=xo, v_out=vo)
        res.append((xo, vo, cv, en))
    for r in res[1:]:
        for a, b in zip(r, res[0]):
            assert np.array_equal(a, b)


def test_cta_size_argument_errors(R):
    sp = I.make_system(70, 3, 8)
    with R.System(sp) as sysm:
        for bad in (16, 33, 128, -32):
            with pytest.raises(R.RidError) as e:
                sysm.set_ff_threads(bad)
            assert e.value.code == R.RID_ERR_ARG
        sysm.set_ff_threads(96)
        assert sysm.ff_threads() == 96
        sysm.set_ff_threads(0)
        assert sysm.ff_threads() == 96   # the default for 70 beads, before any evaluation


@pytest.mark.parametrize("n,seed", [(200, 11), (700, 12), (2000, 13)])
def test_walker_split_over_ctas_gives_the_same_forces(R, orc, n, seed):
    """With fewer walkers than two per SM each walker's passes over its chain are
    split over up to 8 CTAs; a bead's force is the same code and order whatever
    the split, so 6 walkers alone (split) and the same 6 inside a batch of 312
    (one CTA per walker) give the same bits, at every CTA size."""
    sp = I.make_system(n, 6, seed)
    x = I.make_chains(6, sp, seed)
    xb = np.ascontiguousarray(np.tile(x, (52, 1, 1)))
    with R.System(sp) as sysm:
        for th in (0, 64):
            sysm.set_ff_threads(th)
            f = np.zeros((6, n, 3), np.float32)
            sysm.eval_forces(x, R.RID_BIAS_NONE, f_out=f)
            fb = np.zeros((312, n, 3), np.float32)
            sysm.eval_forces(xb, R.RID_BIAS_NONE, f_out=fb)
            assert np.array_equal(f, fb[:6]), th
            assert np.array_equal(fb[6:12], fb[:6])
    ref = orc.total(sp, x[0].astype(np.float64))["f"]
    scale = np.abs(ref) + np.sqrt(np.mean(ref ** 2))
    assert (np.abs(f[0] - ref) / scale).max() < 1e-5
