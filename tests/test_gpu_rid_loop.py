"""One iteration of the RiD cycle through the library (Sec. "Overall Automatic
Workflow"): biased exploration with an ensemble, selection of frames by model
deviation, restrained labelling of the selected configurations, training of
the ensemble on the new labels, and exploration with the trained ensemble.

Each stage is checked against its own definition: selected frames lie in the
trust window and come from the explored trajectories; the labels are finite
and their restraint centres are the selected CVs; training lowers the loss on
the labels; the trained members, handed back through rid_set_ensemble, give
the same CV gradients as the training path's own forward pass, and drive a
finite exploration.
"""
import numpy as np
import pytest

from oracle import train as T
from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def test_one_rid_iteration(R):
    sp = I.make_system(22, 2, 41, output_freq=50)
    M, L, H = 4, 3, 64
    ens = I.make_ensemble(M, 4, L, H, 41)
    W, chunks, per = 64, 6, 100
    x = I.make_chains(W, sp, 41)
    v = None
    frames_x, frames_cv, frames_eps = [], [], []
    with R.System(sp) as s:
        s.set_ensemble(ens, precision=R.RID_PREC_FP32)
        # exploration in chunks, the configuration kept at the end of each chunk
        for k in range(chunks):
            T_ = per // sp.output_freq
            cv = np.zeros((W, T_, 2), np.float32)
            eps = np.zeros((W, T_), np.float32)
            xo, vo = np.zeros_like(x), np.zeros_like(x)
            s.explore(x, per, v0=v, step0=k * per, cv_out=cv, eps_out=eps, x_out=xo, v_out=vo)
            frames_x.append(xo)
            frames_cv.append(cv[:, -1])
            frames_eps.append(eps[:, -1])
            x, v = xo, vo
        fx = np.concatenate(frames_x)                  # [chunks * W][N][3], chunk-major
        fcv = np.ascontiguousarray(np.concatenate(frames_cv))
        feps = np.ascontiguousarray(np.concatenate(frames_eps))
        # selection: trust window between the 20th and 90th percentiles of eps
        lo, hi = np.quantile(feps, [0.2, 0.9])
        sel, nc, thr = R.select(fcv, feps, lo, hi, 0.3, 6, 12, True, 10)
        assert 1 <= sel.size <= 10
        assert np.all((feps[sel] >= np.float32(lo)) & (feps[sel] < np.float32(hi)))
        # restrained labels at the selected configurations, centred on their CVs
        x0 = np.ascontiguousarray(fx[sel])
        s0 = fcv[sel].astype(np.float64)
        kappa = np.full_like(s0, 100.0)
        mf, se, sd = (np.zeros_like(s0) for _ in range(3))
        s.label(x0, s0, kappa, 2000, 200, 10, mf, se, sd)
        assert np.all(np.isfinite(mf)) and np.all(se > 0)
        # training on the new labels
        n = sel.size
        lab_s = s0.astype(np.float32)
        lab_mf = mf.astype(np.float32)
        steps = 300
        idx = np.stack([np.stack([np.arange(n) for _ in range(M)]) for _ in range(steps)]).astype(np.int32)
        losses = np.zeros((steps, M), np.float32)
        with R.Trainer(M, 2, L, H, ens.weights, batch_size=n, init_lr=3e-3) as tr:
            tr.set_data(lab_s, lab_mf)
            tr.run(idx, losses)
            w, _ = tr.weights()
        assert np.all(losses[-1] < 0.5 * losses[0]), losses[[0, -1]]
        # the trained members through the exploration path: the ensemble's CV
        # gradients at the labels equal the trained networks' own (FP32)
        trained = I.EnsembleParams(M, 4, L, H, False, w, ens.trust_lo, ens.trust_hi)
        s.set_ensemble(trained, precision=R.RID_PREC_FP32)
        g = np.zeros((M, n, 2), np.float32)
        xs = np.ascontiguousarray(x0)
        s.eval_forces(xs, R.RID_BIAS_ENSEMBLE, grad_out=g)
        cvs = np.zeros((n, 2), np.float32)
        s.eval_forces(xs, R.RID_BIAS_ENSEMBLE, s_out=cvs)
        want_at = np.array([[T.member_value_and_grad(w[m].astype(np.float64), 4, L, H, False, q)[1]
                             for q in cvs.astype(np.float64)] for m in range(M)])
        np.testing.assert_allclose(g, want_at, rtol=1e-4, atol=1e-4)
        # and a further exploration with the trained ensemble stays finite
        cv = np.zeros((W, 2, 2), np.float32)
        eps = np.zeros((W, 2), np.float32)
        s.explore(x, 100, v0=v, step0=chunks * per, cv_out=cv, eps_out=eps)
        assert np.all(np.isfinite(cv)) and np.all(np.isfinite(eps))
