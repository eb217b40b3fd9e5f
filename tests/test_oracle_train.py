"""Pins of the training oracle (oracle/train.py) against things other than
itself: central finite differences of its own loss (which uses only the
forward and input-gradient passes), a second-order derivative taken by
torch.autograd in float64 (an independent library route), the closed form of
Adam's first step, the exponential learning-rate decay of the training
section, and a fit that must reproduce a teacher network's gradient field.
Dropout: the same derivative pins with masks, the special cases that reduce
to no dropout and to a network whose last layer is dropped entirely, the
counter mapping written out element by element, and the mask statistics
(keep fraction within binomial bounds, unit mean scale).
"""
import numpy as np
import pytest

from oracle import train as T


def _net(D, L, H, seed):
    rng = np.random.default_rng(seed)
    P = T.param_count(D, L, H)
    return rng.normal(0.0, 0.6, size=P)


def _masks(B, L, H, seed, rate=0.3):
    # dropout scales with zeros in every layer (independent of the oracle's generator)
    keep = np.random.default_rng(seed).uniform(size=(B, L, H)) >= rate
    return np.where(keep, 1.0 / (1.0 - rate), 0.0)


@pytest.mark.parametrize("resnet,dropout", [(False, False), (True, False), (False, True), (True, True)])
def test_gradient_matches_central_differences(resnet, dropout):
    C, L, H, B = 2, 3, 5, 3
    D = 2 * C
    rng = np.random.default_rng(7)
    w = _net(D, L, H, 1)
    s = rng.uniform(-np.pi, np.pi, size=(B, C))
    mf = rng.normal(0.0, 1.0, size=(B, C))
    q = _masks(B, L, H, 3) if dropout else None
    loss, g = T.loss_and_grad(w, D, L, H, resnet, s, mf, q)
    assert loss == pytest.approx(T.loss(w, D, L, H, resnet, s, mf, q), rel=1e-13)
    h = 1e-6
    fd = np.empty_like(w)
    for p in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[p] += h
        wm[p] -= h
        fd[p] = (T.loss(wp, D, L, H, resnet, s, mf, q) - T.loss(wm, D, L, H, resnet, s, mf, q)) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))
    assert g[-1] == 0.0                       # b_out does not enter the loss


@pytest.mark.parametrize("resnet,dropout", [(False, False), (True, False), (False, True), (True, True)])
def test_gradient_matches_torch_double_backward(resnet, dropout):
    torch = pytest.importorskip("torch")
    C, L, H, B = 3, 4, 8, 5
    D = 2 * C
    rng = np.random.default_rng(11)
    w = _net(D, L, H, 2)
    s = rng.uniform(-np.pi, np.pi, size=(B, C))
    mf = rng.normal(0.0, 1.0, size=(B, C))
    q = _masks(B, L, H, 4) if dropout else np.ones((B, L, H))
    loss, g = T.loss_and_grad(w, D, L, H, resnet, s, mf, q if dropout else None)
    qt = torch.tensor(q, dtype=torch.float64)

    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    st = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    o, fin, h = 0, D, None
    u = torch.stack([torch.cos(st), torch.sin(st)], dim=-1).reshape(B, D)
    h = u
    for l in range(L):
        W = wt[o:o + H * fin].reshape(H, fin)
        o += H * fin
        b = wt[o:o + H]
        o += H
        t = torch.tanh(h @ W.T + b) * qt[:, l]       # torch.nn dropout's inverted form, masks given
        h = t + h if (resnet and l >= 1) else t
        fin = H
    A = h @ wt[o:o + H] + wt[o + H]
    (dAds,) = torch.autograd.grad(A.sum(), st, create_graph=True)
    lt = ((dAds - torch.tensor(mf)) ** 2).mean()
    (gt,) = torch.autograd.grad(lt, wt)
    assert lt.item() == pytest.approx(loss, rel=1e-12)
    np.testing.assert_allclose(g, gt.numpy(), rtol=1e-10, atol=1e-13)


def test_adam_first_step_is_signed_learning_rate():
    # from zero moments, mhat = g and vhat = g^2: the step is lr g / (|g| + eps)
    g = np.array([3.0, -2e-3, 0.0, 1e-9])
    w0 = np.array([0.5, 0.5, 0.5, 0.5])
    w1, m, v = T.adam_update(w0, g, np.zeros(4), np.zeros(4), 0, 1e-3, 0.9, 0.999, 1e-8)
    np.testing.assert_allclose(w1, w0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_learning_rate_decays_by_rate_every_decay_steps():
    assert T.learning_rate(0, 8e-4, 0.96, 120) == 8e-4
    assert T.learning_rate(120, 8e-4, 0.96, 120) == pytest.approx(8e-4 * 0.96, rel=1e-15)
    assert T.learning_rate(60, 8e-4, 0.96, 120) == pytest.approx(8e-4 * 0.96 ** 0.5, rel=1e-15)
    assert T.learning_rate(2400, 8e-4, 0.96, 120) == pytest.approx(8e-4 * 0.96 ** 20, rel=1e-13)


def test_training_recovers_a_teacher_gradient_field():
    # labels are the exact CV gradient of a teacher network of the same shape
    C, L, H = 2, 2, 12
    D = 2 * C
    rng = np.random.default_rng(5)
    teacher = _net(D, L, H, 3) * 0.8
    s = rng.uniform(-np.pi, np.pi, size=(256, C))
    mf = np.array([T.member_value_and_grad(teacher, D, L, H, False, x)[1] for x in s])
    student = _net(D, L, H, 4)[None, :] * 0.5
    idx = np.array([[rng.choice(256, size=32, replace=False)] for _ in range(400)])
    w, losses, _, _ = T.train(student, D, L, H, False, s, mf, idx, init_lr=1e-2)
    first = losses[:20, 0].mean()
    last = losses[-20:, 0].mean()
    assert last < 0.1 * first, (first, last)


def test_dropout_with_every_unit_kept_is_no_dropout():
    C, L, H, B = 2, 3, 6, 4
    rng = np.random.default_rng(5)
    w = _net(2 * C, L, H, 3)
    s = rng.uniform(-np.pi, np.pi, size=(B, C))
    mf = rng.normal(0.0, 1.0, size=(B, C))
    for resnet in (False, True):
        a = T.loss_and_grad(w, 2 * C, L, H, resnet, s, mf)
        b = T.loss_and_grad(w, 2 * C, L, H, resnet, s, mf, np.ones((B, L, H)))
        assert a[0] == b[0] and np.array_equal(a[1], b[1])
    q = T.dropout_scales(2, 3, L, H, 0, 9, 0.0)
    assert np.array_equal(q, np.ones_like(q))


def test_dropping_the_last_layer_leaves_a_constant_network():
    # every unit of the last hidden layer dropped (plain net): A = b_out for
    # every s, so dA/ds = 0, the loss is the mean of MF^2 and no weight moves it
    C, L, H, B = 2, 3, 5, 4
    rng = np.random.default_rng(6)
    w = _net(2 * C, L, H, 4)
    s = rng.uniform(-np.pi, np.pi, size=(B, C))
    mf = rng.normal(0.0, 1.0, size=(B, C))
    q = _masks(B, L, H, 5)
    q[:, L - 1] = 0.0
    loss, g = T.loss_and_grad(w, 2 * C, L, H, False, s, mf, q)
    assert loss == pytest.approx(np.mean(mf ** 2), rel=1e-15)
    assert np.array_equal(g, np.zeros_like(g))
    A, dads = T.member_value_and_grad(w, 2 * C, L, H, False, s[0], q[0])
    assert A == w[-1] and np.array_equal(dads, np.zeros(C))


def test_dropout_counters_follow_their_definition():
    # the vectorised mask against the counter mapping written out per unit
    import oracle
    M, B, L, H, step, seed, rate = 2, 3, 2, 7, 11, 1234567, 0.37
    q = T.dropout_scales(M, B, L, H, step, seed, rate)
    nw = (H + 3) // 4
    thr = int(np.floor(rate * 2 ** 32))
    for m in range(M):
        for b in range(B):
            for l in range(L):
                for j in range(H):
                    word = oracle.philox(np.array([[j // 4 + nw * (l + L * m), b, step, 4]]), seed)[0, j % 4]
                    want = 1.0 / (1.0 - rate) if int(word) >= thr else 0.0
                    assert q[m, b, l, j] == want


@pytest.mark.parametrize("rate", [0.1, 0.5])
def test_dropout_mask_statistics(rate):
    # kept fraction within 5 sigma of 1 - rate; the mean scale is 1 (inverted
    # dropout keeps the expected activation); masks differ between steps
    M, B, L, H = 4, 128, 4, 64
    q = T.dropout_scales(M, B, L, H, 0, 77, rate)
    n = q.size
    keep = np.count_nonzero(q)
    assert set(np.unique(q)) <= {0.0, 1.0 / (1.0 - rate)}
    assert abs(keep - n * (1 - rate)) < 5 * np.sqrt(n * rate * (1 - rate))
    assert abs(q.mean() - 1.0) < 5 * np.sqrt(rate / (1 - rate) / n)
    assert T.dropout_threshold(0.5) == 2 ** 31 and T.dropout_threshold(0.25) == 2 ** 30
    q1 = T.dropout_scales(M, B, L, H, 1, 77, rate)
    assert 0.5 < np.mean((q > 0) == (q1 > 0)) < 1.0


# --------------------------------------------------------------------------- distance CVs
def test_mixed_cv_gradient_matches_finite_differences_and_torch():
    """Training on labels over torsions and distance CVs (a distance enters as
    (s, 0), dA/ds = dA/du_2j): the weight gradient against central differences
    of the oracle's loss and against torch double backward."""
    torch = pytest.importorskip("torch")
    C, L, H, B = 3, 3, 6, 4
    D = 2 * C
    dist = np.array([False, True, True])
    rng = np.random.default_rng(13)
    w = _net(D, L, H, 5)
    s = np.stack([rng.uniform(-np.pi, np.pi, B), rng.uniform(1.0, 4.0, B), rng.uniform(1.0, 4.0, B)], axis=1)
    mf = rng.normal(0.0, 1.0, size=(B, C))
    loss, g = T.loss_and_grad(w, D, L, H, True, s, mf, None, dist)
    assert loss == pytest.approx(T.loss(w, D, L, H, True, s, mf, None, dist), rel=1e-13)
    h = 1e-6
    fd = np.empty_like(w)
    for p in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[p] += h
        wm[p] -= h
        fd[p] = (T.loss(wp, D, L, H, True, s, mf, None, dist) - T.loss(wm, D, L, H, True, s, mf, None, dist)) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    st = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    dt = torch.tensor(dist)
    u = torch.stack([torch.where(dt, st, torch.cos(st)), torch.where(dt, torch.zeros_like(st), torch.sin(st))],
                    dim=-1).reshape(B, D)
    o, fin, hh = 0, D, u
    for l in range(L):
        W = wt[o:o + H * fin].reshape(H, fin)
        o += H * fin
        b = wt[o:o + H]
        o += H
        t = torch.tanh(hh @ W.T + b)
        hh = t + hh if l >= 1 else t
        fin = H
    A = hh @ wt[o:o + H] + wt[o + H]
    (dAds,) = torch.autograd.grad(A.sum(), st, create_graph=True)
    lt = ((dAds - torch.tensor(mf)) ** 2).mean()
    (gt,) = torch.autograd.grad(lt, wt)
    assert lt.item() == pytest.approx(loss, rel=1e-12)
    np.testing.assert_allclose(g, gt.numpy(), rtol=1e-10, atol=1e-13)
    # the torsion reading of the same CVs is a different loss
    assert abs(T.loss(w, D, L, H, True, s, mf) - loss) > 1e-3 * loss
