"""Degenerate calls: empty inputs and zero-length runs return what their
definitions give, with no device error.  Selection of no frames finds no
cluster and keeps its threshold; a batch of no jobs does nothing; an
exploration of zero steps returns the loaded state unchanged, bit for bit;
an MCMC run of zero steps leaves the walkers where they started, with empty
histograms and an all-infinite PMF; a training run of zero steps takes no
step."""
import math

import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def test_selection_of_no_frames(R):
    cv, eps = np.zeros((0, 3), np.float32), np.zeros(0, np.float32)
    for adapt in (False, True):
        sel, nc, thr = R.select(cv, eps, 0.0, 5.0, 1.25, 1, 5, adapt, 10)
        assert sel.size == 0 and nc == 0 and thr == 1.25


def test_batch_of_no_jobs(R):
    with R.Server(64 << 20) as srv:
        assert srv.label_batch([]) == []


def test_zero_step_exploration_returns_the_loaded_state(R):
    sp = I.make_system(30, 3, 5)
    W = 4
    x0 = I.make_chains(W, sp, 5)
    v0 = np.random.default_rng(2).standard_normal(x0.shape).astype(np.float32)
    xo, vo = np.zeros_like(x0), np.zeros_like(x0)
    cv, eps = np.zeros((W, 0, 3), np.float32), np.zeros((W, 0), np.float32)
    with R.System(sp) as s:
        s.set_ensemble(I.make_ensemble(2, 6, 2, 32, 5), precision=R.RID_PREC_FP32)
        s.explore(x0, 0, v0=v0, cv_out=cv, eps_out=eps, x_out=xo, v_out=vo)
    assert np.array_equal(xo, x0) and np.array_equal(vo, v0)


def test_zero_step_mcmc(R):
    M, C, L, H, W, bins = 2, 3, 2, 16, 50, 10
    ens = I.make_ensemble(M, 2 * C, L, H, 6)
    s0 = np.random.default_rng(3).uniform(-math.pi, math.pi, size=(W, C)).astype(np.float32)
    s = np.zeros_like(s0)
    h1 = np.ones((C, bins), np.uint64)
    f1 = np.zeros((C, bins))
    nacc = R.mcmc(ens.weights, M, C, L, H, s0, 0, 0, 1.0, 0.3, 1, bins=bins, s_out=s, hist1=h1, pmf1=f1)
    assert nacc == 0 and np.array_equal(s, s0)
    assert not h1.any() and np.all(np.isposinf(f1))


def test_zero_step_training_run(R):
    M, C, L, H, B = 2, 3, 2, 16, 8
    ens = I.make_ensemble(M, 2 * C, L, H, 7)
    rng = np.random.default_rng(4)
    s = rng.uniform(-math.pi, math.pi, size=(20, C)).astype(np.float32)
    mf = rng.normal(size=(20, C)).astype(np.float32)
    with R.Trainer(M, C, L, H, ens.weights, batch_size=B) as tr:
        tr.set_data(s, mf)
        tr.run(np.zeros((0, M, B), np.int32))
        w, steps = tr.weights()
    assert steps == 0 and np.array_equal(w, ens.weights)
