"""The per-walker split of the step kernels at few walkers: with fewer walkers
than two per SM, k_head runs each walker as a thread-block cluster over its
bead batches (new positions exchanged through distributed shared memory for
the CVs) and k_ff splits each walker's passes over several CTAs.  A bead's
update and a CV are the same arithmetic whatever the split, so a few walkers
alone give the same bits as the same walkers inside a batch of 312 (one CTA
per walker): CVs and Jacobian-weighted forces at given positions, restrained
labels (mean force, standard error, std) and final states after many steps.
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu

COPIES = 52   # 6 walkers x 52 = 312 >= two per SM on 152 SMs: no split


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def tiled(a):
    return np.ascontiguousarray(np.tile(a, (COPIES,) + (1,) * (a.ndim - 1)))


@pytest.mark.parametrize("n,C,seed,nd,span", [(200, 20, 1, 0, 5), (700, 33, 2, 0, 5), (2000, 64, 3, 0, 5),
                                              (517, 7, 4, 0, 5), (1500, 12, 7, 4, 600)])
def test_cvs_and_forces_alone_equal_inside_a_batch(R, orc, n, C, seed, nd, span):
    """(the last case has distance CVs between beads 600 apart: their atoms lie
    in different CTAs' slices)"""
    sp = I.make_system(n, C, seed, n_dist=nd, dist_span=span)
    x = I.make_chains(6, sp, seed)
    with R.System(sp) as sysm:
        s1, f1 = np.zeros((6, C), np.float32), np.zeros((6, n, 3), np.float32)
        sysm.eval_forces(x, R.RID_BIAS_NONE, s_out=s1, f_out=f1)
        sb, fb = np.zeros((6 * COPIES, C), np.float32), np.zeros((6 * COPIES, n, 3), np.float32)
        sysm.eval_forces(tiled(x), R.RID_BIAS_NONE, s_out=sb, f_out=fb)
    assert np.array_equal(s1, sb[:6]) and np.array_equal(f1, fb[:6])
    ref = orc.cvs(sp, x[5].astype(np.float64))[0]
    dist = I.cv_is_distance(sp)
    d = np.where(dist, (s1[5] - ref) / np.maximum(np.abs(ref), 1.0), np.angle(np.exp(1j * (s1[5] - ref))))
    assert np.abs(d).max() < 1e-5


@pytest.mark.parametrize("n,C,seed,nd,span", [(300, 12, 5, 0, 5), (2000, 40, 6, 0, 5), (1200, 10, 8, 3, 500)])
def test_labels_alone_equal_inside_a_batch(R, n, C, seed, nd, span):
    sp = I.make_system(n, C, seed, n_dist=nd, dist_span=span)
    x = I.make_chains(6, sp, seed)
    rng = np.random.default_rng(seed)
    with R.System(sp) as sysm:
        s = np.zeros((6, C), np.float32)
        sysm.eval_forces(x, R.RID_BIAS_NONE, s_out=s)
        s0 = s.astype(np.float64) + rng.uniform(-0.2, 0.2, size=s.shape)
        kap = rng.uniform(50.0, 500.0, size=(6, C))
        outs = []
        for xs, s0s, ks in ((x, s0, kap), (tiled(x), tiled(s0), tiled(kap))):
            W = xs.shape[0]
            mf, se, sd = (np.zeros((W, C)) for _ in range(3))
            xo, vo = np.zeros_like(xs), np.zeros_like(xs)
            sysm.label(xs, s0s, ks, 400, 40, 10, mf, se, sd, x_out=xo, v_out=vo)
            outs.append([a[:6] for a in (mf, se, sd, xo, vo)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert np.all(np.isfinite(outs[0][3]))
