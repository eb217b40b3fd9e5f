"""Pins of the training oracle (oracle/train.py) against things other than
itself: central finite differences of its own loss (which uses only the
forward and input-gradient passes), a second-order derivative taken by
torch.autograd in float64 (an independent library route), the closed form of
Adam's first step, the exponential learning-rate decay of the training
section, and a fit that must reproduce a teacher network's gradient field.
"""
import numpy as np
import pytest

from oracle import train as T


def _net(D, L, H, seed):
    rng = np.random.default_rng(seed)
    P = T.param_count(D, L, H)
    return rng.normal(0.0, 0.6, size=P)


@pytest.mark.parametrize("resnet", [False, True])
def test_gradient_matches_central_differences(resnet):
    C, L, H, B = 2, 3, 5, 3
    D = 2 * C
    rng = np.random.default_rng(7)
    w = _net(D, L, H, 1)
    s = rng.uniform(-np.pi, np.pi, size=(B, C))
    mf = rng.normal(0.0, 1.0, size=(B, C))
    loss, g = T.loss_and_grad(w, D, L, H, resnet, s, mf)
    assert loss == pytest.approx(T.loss(w, D, L, H, resnet, s, mf), rel=1e-13)
    h = 1e-6
    fd = np.empty_like(w)
    for p in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[p] += h
        wm[p] -= h
        fd[p] = (T.loss(wp, D, L, H, resnet, s, mf) - T.loss(wm, D, L, H, resnet, s, mf)) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))
    assert g[-1] == 0.0                       # b_out does not enter the loss


@pytest.mark.parametrize("resnet", [False, True])
def test_gradient_matches_torch_double_backward(resnet):
    torch = pytest.importorskip("torch")
    C, L, H, B = 3, 4, 8, 5
    D = 2 * C
    rng = np.random.default_rng(11)
    w = _net(D, L, H, 2)
    s = rng.uniform(-np.pi, np.pi, size=(B, C))
    mf = rng.normal(0.0, 1.0, size=(B, C))
    loss, g = T.loss_and_grad(w, D, L, H, resnet, s, mf)

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
        t = torch.tanh(h @ W.T + b)
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
