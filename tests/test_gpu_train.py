"""Ensemble training on mean-force labels (rid_trainer_*) against the FP64
training oracle: batch loss and its gradient through the input-gradient pass,
with and without dropout,
Adam steps with the exponential learning-rate decay, bit-for-bit
reproducibility, host / device arguments, errors, a fit of a teacher's
gradient field, and the hand-off of the trained weights to the ensemble path.

Tolerances: the GEMMs accumulate in FP32 over K <= 2 * 128 terms and tanh is
FP32, so the gradient carries relative errors of order 1e-6 (normwise bound
1e-4 below, 1e-5 on the loss).  The Adam step is pinned on its own: given the
trainer's gradient, the new weights equal the oracle's FP64 update to FP32
rounding.  End to end over a few steps, a weight whose gradient sits at the
rounding level can take an Adam step of another size or sign (Adam
normalises by the gradient's own magnitude); up to 1e-3 of the weights may
then differ from the oracle's by more than 1e-6 (measured: about 1e-4).
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


def _problem(M, C, L, H, B, n, seed, resnet=False):
    ens = I.make_ensemble(M, 2 * C, L, H, seed, resnet=resnet)
    rng = np.random.default_rng(seed + 50)
    s = rng.uniform(-np.pi, np.pi, size=(n, C)).astype(np.float32)
    mf = rng.normal(0.0, 2.0, size=(n, C)).astype(np.float32)
    idx = np.stack([rng.choice(n, size=B, replace=B > n) for _ in range(M)]).astype(np.int32)
    return ens, s, mf, idx


SHAPES = [  # M, C, L, H, B, n, resnet
    (4, 20, 4, 256, 128, 1000, False),   # the exploration model of the 200-bead workload
    (2, 3, 3, 40, 50, 77, True),         # ragged tiles, residual layers
    (1, 1, 1, 8, 1, 3, False),           # one member, one CV, one sample
]


@pytest.mark.parametrize("M,C,L,H,B,n,resnet", SHAPES)
def test_loss_and_gradient_match_the_oracle(R, M, C, L, H, B, n, resnet):
    ens, s, mf, idx = _problem(M, C, L, H, B, n, 3, resnet)
    loss = np.zeros(M, np.float32)
    grad = np.zeros((M, ens.weights.shape[1]), np.float32)
    with R.Trainer(M, C, L, H, ens.weights, batch_size=B, resnet=resnet) as tr:
        tr.set_data(s, mf)
        tr.grad(idx, loss, grad)
        w_after, steps = tr.weights()
    assert steps == 0 and np.array_equal(w_after, ens.weights)      # grad() takes no step
    for m in range(M):
        lo, go = T.loss_and_grad(ens.weights[m].astype(np.float64), 2 * C, L, H, resnet, s[idx[m]], mf[idx[m]])
        assert abs(loss[m] - lo) <= 1e-5 * lo
        err = np.linalg.norm(grad[m] - go) / np.linalg.norm(go)
        assert err < 1e-4, err
        assert grad[m, -1] == 0.0                                   # b_out does not enter the loss


@pytest.mark.parametrize("M,C,L,H,B,n,resnet", SHAPES[:2])
def test_each_step_is_adam_on_the_batch_gradient(R, M, C, L, H, B, n, resnet):
    # the step itself: w_{k+1} must be the oracle's Adam update (FP64) applied
    # to the trainer's own gradient at w_k, with the decayed learning rate
    ens, s, mf, _ = _problem(M, C, L, H, B, n, 4, resnet)
    rng = np.random.default_rng(9)
    K = 4
    kw = dict(init_lr=2e-3, decay_rate=0.5, decay_steps=2)      # a visible decay within K steps
    P = ens.weights.shape[1]
    m = np.zeros((M, P))
    v = np.zeros((M, P))
    with R.Trainer(M, C, L, H, ens.weights, batch_size=B, resnet=resnet, **kw) as tr:
        tr.set_data(s, mf)
        w = ens.weights.astype(np.float64)
        for k in range(K):
            idx = np.stack([rng.choice(n, size=B, replace=B > n) for _ in range(M)]).astype(np.int32)
            g = np.zeros((M, P), np.float32)
            tr.grad(idx, grad_out=g)
            lr = T.learning_rate(k, kw["init_lr"], kw["decay_rate"], kw["decay_steps"])
            want = np.empty_like(w)
            for i in range(M):
                want[i], m[i], v[i] = T.adam_update(w[i], g[i].astype(np.float64), m[i], v[i], k, lr,
                                                    0.9, 0.999, 1e-8)
            tr.run(idx[None])
            got, steps = tr.weights()
            assert steps == k + 1
            tol = 1e-6 * kw["init_lr"] + 4 * np.finfo(np.float32).eps * np.abs(want).max()
            assert np.max(np.abs(got - want)) <= tol
            w = got.astype(np.float64)


@pytest.mark.parametrize("M,C,L,H,B,n,resnet", SHAPES[:2])
def test_trajectory_follows_the_oracle(R, M, C, L, H, B, n, resnet):
    # K steps end to end against the FP64 oracle.  The losses agree to FP32
    # accuracy.  A weight whose gradient sits at the rounding level can take
    # an Adam step of different size or sign (|step| <= lr per step), so a
    # small fraction of weights is allowed beyond 1e-6.
    ens, s, mf, _ = _problem(M, C, L, H, B, n, 4, resnet)
    rng = np.random.default_rng(9)
    K = 4
    idx = np.stack([np.stack([rng.choice(n, size=B, replace=B > n) for _ in range(M)]) for _ in range(K)])
    idx = idx.astype(np.int32)
    kw = dict(init_lr=2e-3, decay_rate=0.5, decay_steps=2)
    losses = np.zeros((K, M), np.float32)
    with R.Trainer(M, C, L, H, ens.weights, batch_size=B, resnet=resnet, **kw) as tr:
        tr.set_data(s, mf)
        tr.run(idx, losses)
        w, steps = tr.weights()
    assert steps == K
    wo, lo, _, _ = T.train(ens.weights, 2 * C, L, H, resnet, s, mf, idx, **kw)
    np.testing.assert_allclose(losses, lo, rtol=1e-5)
    d = np.abs(w.astype(np.float64) - wo)
    print(f"\n[{M}x{H}x{L}] weights beyond 1e-6 of the oracle: {np.mean(d > 1e-6):.2e}, max {d.max():.2e}")
    assert np.mean(d > 1e-6) <= 1e-3
    assert d.max() <= K * kw["init_lr"]
    assert not np.array_equal(w, ens.weights)


@pytest.mark.parametrize("rate", [0.1, 0.5])
@pytest.mark.parametrize("M,C,L,H,B,n,resnet", SHAPES[:2])
def test_dropout_loss_and_gradient_match_the_oracle(R, M, C, L, H, B, n, resnet, rate):
    # the thinned network of the trainer's next step (t = 0): the masks are
    # the oracle's own Philox draws, so the comparison is the no-dropout one
    ens, s, mf, idx = _problem(M, C, L, H, B, n, 13, resnet)
    seed = 0x5EED0000DEADBEEF
    loss = np.zeros(M, np.float32)
    grad = np.zeros((M, ens.weights.shape[1]), np.float32)
    with R.Trainer(M, C, L, H, ens.weights, batch_size=B, resnet=resnet, dropout_rate=rate,
                   dropout_seed=seed) as tr:
        tr.set_data(s, mf)
        tr.grad(idx, loss, grad)
    q = T.dropout_scales(M, B, L, H, 0, seed, rate)
    for m in range(M):
        lo, go = T.loss_and_grad(ens.weights[m].astype(np.float64), 2 * C, L, H, resnet, s[idx[m]], mf[idx[m]],
                                 q[m])
        _, gp = T.loss_and_grad(ens.weights[m].astype(np.float64), 2 * C, L, H, resnet, s[idx[m]], mf[idx[m]])
        assert np.linalg.norm(go - gp) > 0.3 * np.linalg.norm(gp)   # the masks change the gradient
        assert abs(loss[m] - lo) <= 1e-5 * lo
        err = np.linalg.norm(grad[m] - go) / np.linalg.norm(go)
        assert err < 1e-4, err


@pytest.mark.parametrize("M,C,L,H,B,n,resnet", SHAPES[:2])
def test_dropout_trajectory_follows_the_oracle(R, M, C, L, H, B, n, resnet):
    # K steps with the paper's rate: every step draws its own masks
    ens, s, mf, _ = _problem(M, C, L, H, B, n, 14, resnet)
    rng = np.random.default_rng(10)
    K, rate, seed = 4, 0.1, 99
    idx = np.stack([np.stack([rng.choice(n, size=B, replace=B > n) for _ in range(M)]) for _ in range(K)])
    idx = idx.astype(np.int32)
    kw = dict(init_lr=2e-3, decay_rate=0.5, decay_steps=2)
    losses = np.zeros((K, M), np.float32)
    with R.Trainer(M, C, L, H, ens.weights, batch_size=B, resnet=resnet, dropout_rate=rate, dropout_seed=seed,
                   **kw) as tr:
        tr.set_data(s, mf)
        tr.run(idx, losses)
        w, _ = tr.weights()
    wo, lo, _, _ = T.train(ens.weights, 2 * C, L, H, resnet, s, mf, idx, dropout_rate=rate, dropout_seed=seed, **kw)
    np.testing.assert_allclose(losses, lo, rtol=1e-5)
    d = np.abs(w.astype(np.float64) - wo)
    print(f"\n[{M}x{H}x{L} dropout] weights beyond 1e-6 of the oracle: {np.mean(d > 1e-6):.2e}, max {d.max():.2e}")
    assert np.mean(d > 1e-6) <= 1e-3
    assert d.max() <= K * kw["init_lr"]


def test_runs_are_reproducible_and_split_runs_equal_one_run(R):
    M, C, L, H, B, n = 2, 6, 3, 64, 64, 500
    ens, s, mf, _ = _problem(M, C, L, H, B, n, 5)
    rng = np.random.default_rng(2)
    idx = rng.integers(0, n, size=(10, M, B)).astype(np.int32)
    out = []
    for split in (False, True):
        with R.Trainer(M, C, L, H, ens.weights, batch_size=B) as tr:
            tr.set_data(s, mf)
            if split:
                tr.run(idx[:3])
                tr.run(idx[3:])
            else:
                tr.run(idx)
            out.append(tr.weights()[0])
    assert np.array_equal(out[0], out[1])
    # with dropout the masks follow the trainer's step count across calls
    out = []
    for split in (False, True):
        with R.Trainer(M, C, L, H, ens.weights, batch_size=B, dropout_rate=0.2, dropout_seed=4) as tr:
            tr.set_data(s, mf)
            if split:
                tr.run(idx[:3])
                tr.run(idx[3:])
            else:
                tr.run(idx)
            out.append(tr.weights()[0])
    assert np.array_equal(out[0], out[1])


def test_device_arguments_match_host_arguments(R):
    import torch
    M, C, L, H, B, n = 2, 5, 2, 48, 40, 300
    ens, s, mf, _ = _problem(M, C, L, H, B, n, 6)
    idx = np.random.default_rng(3).integers(0, n, size=(3, M, B)).astype(np.int32)
    res = []
    for dev in (False, True):
        with R.Trainer(M, C, L, H, ens.weights, batch_size=B) as tr:
            if dev:
                tr.set_data(torch.from_numpy(s).cuda(), torch.from_numpy(mf).cuda())
                loss = torch.zeros((3, M), dtype=torch.float32, device="cuda")
                tr.run(torch.from_numpy(idx).cuda(), loss)
                w = torch.zeros((M, ens.weights.shape[1]), dtype=torch.float32, device="cuda")
                tr.weights(w)
                res.append((loss.cpu().numpy(), w.cpu().numpy()))
            else:
                tr.set_data(s, mf)
                loss = np.zeros((3, M), np.float32)
                tr.run(idx, loss)
                res.append((loss, tr.weights()[0]))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_errors(R):
    M, C, L, H, B, n = 1, 2, 2, 16, 8, 20
    ens, s, mf, idx = _problem(M, C, L, H, B, n, 7)
    with R.Trainer(M, C, L, H, ens.weights, batch_size=B) as tr:
        with pytest.raises(R.RidError) as e:
            tr.run(idx[None])
        assert e.value.code == R.RID_ERR_STATE                     # no data yet
        tr.set_data(s, mf)
        bad = idx.copy()
        bad[0, 3] = n
        with pytest.raises(R.RidError) as e:
            tr.run(bad[None])
        assert e.value.code == R.RID_ERR_ARG
        tr.run(idx[None])                                          # usable afterwards
    with pytest.raises(R.RidError) as e:
        R.Trainer(M, C, L, H, ens.weights, batch_size=0)
    assert e.value.code == R.RID_ERR_ARG
    for rate in (1.0, -0.1):
        with pytest.raises(R.RidError) as e:
            R.Trainer(M, C, L, H, ens.weights, batch_size=B, dropout_rate=rate)
        assert e.value.code == R.RID_ERR_ARG


def test_fit_of_a_teacher_gradient_field_and_hand_off_to_the_ensemble(R):
    # labels: the exact CV gradient of a teacher net; the trained members are
    # then evaluated through the exploration path's FP32 ensemble gradient
    import torch
    M, C, L, H, B, n = 4, 4, 3, 64, 128, 4096
    teacher = I.make_ensemble(1, 2 * C, L, H, 21)
    rng = np.random.default_rng(8)
    s = rng.uniform(-np.pi, np.pi, size=(n, C)).astype(np.float32)
    mf = np.array([T.member_value_and_grad(teacher.weights[0], 2 * C, L, H, False, x)[1] for x in s],
                  dtype=np.float32)
    student = I.make_ensemble(M, 2 * C, L, H, 22)
    steps = 1500
    idx = rng.integers(0, n, size=(steps, M, B)).astype(np.int32)
    losses = np.zeros((steps, M), np.float32)
    with R.Trainer(M, C, L, H, student.weights, batch_size=B, init_lr=3e-3, decay_steps=300) as tr:
        tr.set_data(s, mf)
        tr.run(idx, losses)
        w, _ = tr.weights()
    assert np.all(losses[-50:].mean(axis=0) < 0.02 * losses[:10].mean(axis=0)), losses[[0, -1]]
    # the trained weights through rid_ensemble_grad_noalloc (packed layout, FP32)
    P = 512
    sd = torch.from_numpy(s[:P]).cuda()
    g = torch.zeros((M, P, C), dtype=torch.float32, device="cuda")
    R.ensemble_grad_noalloc(sd, torch.from_numpy(w).cuda(), M, L, H, g)
    mse = ((g.cpu().numpy() - mf[None, :P]) ** 2).mean(axis=(1, 2))
    start = ((np.array([[T.member_value_and_grad(student.weights[m], 2 * C, L, H, False, x)[1] for x in s[:64]]
                        for m in range(M)]) - mf[None, :64]) ** 2).mean(axis=(1, 2))
    assert np.all(mse < 0.05 * start), (mse, start)


# ------------------------------------------------------------------ distance CVs
@pytest.mark.parametrize("resnet", [False, True])
def test_distance_cvs_loss_gradient_and_trajectory_match_the_oracle(R, resnet):
    """Labels over torsions and distance CVs (a distance enters the network as
    (s, 0)): the batch loss and gradient, then four Adam steps, against the
    oracle with the same kinds, at the tolerances above."""
    M, C, L, H, B, n = 3, 6, 3, 64, 40, 200
    dist = np.array([False, True, False, True, True, False])
    ens, s, mf, idx = _problem(M, C, L, H, B, n, 7, resnet)
    rng = np.random.default_rng(8)
    s[:, dist] = rng.uniform(1.0, 4.0, size=(n, dist.sum())).astype(np.float32)
    loss = np.zeros(M, np.float32)
    grad = np.zeros((M, ens.weights.shape[1]), np.float32)
    kw = dict(init_lr=2e-3, decay_rate=0.5, decay_steps=2)
    K = 4
    idxs = np.stack([np.stack([rng.choice(n, size=B) for _ in range(M)]) for _ in range(K)]).astype(np.int32)
    losses = np.zeros((K, M), np.float32)
    with R.Trainer(M, C, L, H, ens.weights, batch_size=B, resnet=resnet, cv_dist=dist, **kw) as tr:
        tr.set_data(s, mf)
        tr.grad(idx, loss, grad)
        tr.run(idxs, losses)
        w, _ = tr.weights()
    for m in range(M):
        lo, go = T.loss_and_grad(ens.weights[m].astype(np.float64), 2 * C, L, H, resnet, s[idx[m]], mf[idx[m]],
                                 None, dist)
        assert abs(loss[m] - lo) <= 1e-5 * lo
        assert np.linalg.norm(grad[m] - go) / np.linalg.norm(go) < 1e-4
        # the torsion reading of the same labels has another gradient
        _, gt = T.loss_and_grad(ens.weights[m].astype(np.float64), 2 * C, L, H, resnet, s[idx[m]], mf[idx[m]])
        assert np.linalg.norm(gt - go) > 1e-2 * np.linalg.norm(go)
    wo, lo, _, _ = T.train(ens.weights, 2 * C, L, H, resnet, s, mf, idxs, dist=dist, **kw)
    np.testing.assert_allclose(losses, lo, rtol=1e-5)
    d = np.abs(w.astype(np.float64) - wo)
    assert np.mean(d > 1e-6) <= 1e-3 and d.max() <= K * kw["init_lr"]
