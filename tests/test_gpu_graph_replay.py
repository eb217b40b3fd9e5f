"""Long exploration runs (rid_explore / rid_walkers_advance of at least two
chunks of about 256 steps) are replayed as CUDA graphs of one chunk.  The
replay must give the same bits as the direct launches: checked against the
same run cut into short calls (each below the replay threshold), with FP32 and
BF16 ensembles, trace slots across chunk boundaries, a remainder that is not
a whole chunk, and a step count that is not a multiple of the output stride.
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


@pytest.mark.parametrize("prec,n_steps,of", [("fp32", 2000, 10), ("bf16", 1337, 7), ("fp32", 530, 1)])
def test_replayed_run_equals_short_calls(R, prec, n_steps, of):
    sp = I.make_system(22, 2, 81, output_freq=of)
    W = 16
    x0 = I.make_chains(W, sp, 81)
    ens = I.make_ensemble(4, 4, 3, 64, 81)
    p = R.RID_PREC_FP32 if prec == "fp32" else R.RID_PREC_BF16
    T = n_steps // of
    with R.System(sp) as sysm:
        sysm.set_ensemble(ens, precision=p)
        sysm.set_fused_steps(False)   # the per-step kernels (this FP32 shape would run fused)
        cv = np.zeros((W, T, 2), np.float32)
        eps = np.zeros((W, T), np.float32)
        xo, vo = np.zeros_like(x0), np.zeros_like(x0)
        l0 = sysm.launch_count()
        sysm.explore(x0, n_steps, cv_out=cv, eps_out=eps, x_out=xo, v_out=vo)
        launches = sysm.launch_count() - l0
        # the same run in calls of `of` steps (the direct path)
        sysm.walkers_load(x0)
        cvs, epss = [], []
        for _ in range(T):
            c = np.zeros((W, 1, 2), np.float32)
            e = np.zeros((W, 1), np.float32)
            sysm.walkers_advance(of, cv_out=c, eps_out=e)
            cvs.append(c)
            epss.append(e)
        if n_steps % of:
            sysm.walkers_advance(n_steps % of)
        x2, v2 = np.zeros_like(x0), np.zeros_like(x0)
        sysm.walkers_read(x_out=x2, v_out=v2)
    assert np.array_equal(xo, x2) and np.array_equal(vo, v2)
    assert np.array_equal(cv, np.concatenate(cvs, axis=1))
    assert np.array_equal(eps, np.concatenate(epss, axis=1))
    assert np.all(np.isfinite(xo))
    # every replayed kernel is counted: three per step at least
    assert launches >= 3 * n_steps
