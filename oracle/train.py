"""FP64 CPU oracle for training the ensemble on mean-force labels.

TEST INFRASTRUCTURE ONLY: imported by the tests (and by the benchmark's
CPU-baseline leg) -- never by the product path.  It shares no code with the
CUDA library; both read the arrays made by ``paper_2408_14070_gb300.inputs``.

What it computes (Sec. "Training phase" and Sec. "Training"; Introduction:
the free energy is learnt by fitting its derivatives, the mean forces).  Every
member i of the ensemble is a tanh MLP A_i(s) of u = (cos s_0, sin s_0, ...)
(a distance CV enters as (s_j, 0)),
with the packed weight layout of the exploration kernels.  On a batch of
labels (s_k, MF_k) the member's loss is the mean squared difference between
its CV gradient and the label,

    L_i = 1 / (B C) * sum_k sum_j (dA_i/ds_j(s_k) - MF_kj)^2,

and its weights take one Adam step (beta1, beta2, eps) with the learning
rate lr_t = init_lr * decay_rate ** (t / decay_steps) of the training
section's exponential decay (t = 0, 1, ... counts the steps taken).

The gradient dL/dtheta differentiates through the input-gradient pass (a
second-order quantity).  It is written out here pass by pass in the order a
reader would derive it:
  1. forward:   t_l = tanh(z_l), z_l = W_l h_{l-1} + b_l,
                h_l = t_l + r_l h_{l-1}  (r_l = 1 for l >= 1 with resnet),
                h_{-1} = u, A = w_out . h_{L-1} + b_out;
  2. input gradient: g_{L-1} = w_out,
                g_{l-1} = W_l^T (g_l * (1 - t_l^2)) + r_l g_l,  dA/du = g_{-1};
  3. loss: dA/ds_j = -sin s_j g[2j] + cos s_j g[2j+1], residual and the
     adjoint gbar_{-1} of dA/du;
  4. adjoint of pass 2, layers in increasing order:
                dbar_l = W_l gbar_{l-1},  dL/dW_l += d_l (x) gbar_{l-1},
                gbar_l = dbar_l * (1 - t_l^2) + r_l gbar_{l-1},
                tbar_l = -2 t_l * g_l * dbar_l,       dL/dw_out = gbar_{L-1};
  5. back through pass 1, layers in decreasing order (hbar_{L-1} = 0):
                zbar_l = (tbar_l + hbar_l) * (1 - t_l^2),
                dL/dW_l += zbar_l (x) h_{l-1},  dL/db_l = zbar_l,
                hbar_{l-1} = W_l^T zbar_l + r_l hbar_l.
b_out does not enter the loss (its gradient is exactly zero).

Dropout (the training section's drop_out_rate; the paper gives the rate, not
the form).  Reading: inverted dropout on the output of every hidden layer,
during training only.  Unit j of hidden layer l for batch row b of member m at
training step t is kept iff word j % 4 of the Philox4x32-10 block at counter
(j // 4 + ceil(H / 4) (l + L m), b, t, 4), key = dropout seed, is at least
floor(rate 2^32); a kept unit is scaled by q = 1 / (1 - rate), a dropped one
by q = 0.  With q_l the scales of layer l the passes above become
  h_l = q_l t_l + r_l h_{l-1},  d_l = g_l q_l (1 - t_l^2),
  gbar_l = dbar_l q_l (1 - t_l^2) + r_l gbar_{l-1},  tbar_l = -2 q_l t_l g_l dbar_l,
  zbar_l = (tbar_l + q_l hbar_l) (1 - t_l^2):
every derivative of the activation q tanh(z) carries q, and the input
gradient dA/ds of the loss is that of the thinned network of the step.

Everything is float64 numpy; batches are plain loops over samples where that
keeps the formulas readable.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

DROPOUT_STREAM = 4


def param_count(D: int, L: int, H: int) -> int:
    return H * D + H + (L - 1) * (H * H + H) + H + 1


def unpack(w, D: int, L: int, H: int):
    """Views of one member's packed weights: [(W_l, b_l)] * L, w_out, b_out."""
    w = np.asarray(w)
    layers, o, fin = [], 0, D
    for _ in range(L):
        W = w[o:o + H * fin].reshape(H, fin)
        o += H * fin
        b = w[o:o + H]
        o += H
        layers.append((W, b))
        fin = H
    w_out = w[o:o + H]
    b_out = w[o + H:o + H + 1]
    assert o + H + 1 == w.shape[0]
    return layers, w_out, b_out


def features(s, dist=None):
    """u = (cos s_0, sin s_0, cos s_1, sin s_1, ...) for s [..., C]; a distance
    CV (dist [C] true) enters as (s_j, 0)."""
    s = np.asarray(s, dtype=np.float64)
    u = np.empty(s.shape[:-1] + (2 * s.shape[-1],))
    u[..., 0::2] = np.cos(s)
    u[..., 1::2] = np.sin(s)
    if dist is not None and np.any(dist):
        d = np.asarray(dist, dtype=bool)
        u[..., 0::2][..., d] = s[..., d]
        u[..., 1::2][..., d] = 0.0
    return u


def cv_gradient(s, g, dist=None):
    """dA/ds from dA/du through the input map: -sin s g[2j] + cos s g[2j+1] for
    a torsion, g[2j] for a distance CV."""
    s = np.asarray(s, dtype=np.float64)
    out = -np.sin(s) * g[0::2] + np.cos(s) * g[1::2]
    if dist is not None and np.any(dist):
        d = np.asarray(dist, dtype=bool)
        out[d] = g[0::2][d]
    return out


def cv_gradient_adjoint(s, v, dist=None):
    """The adjoint of cv_gradient: d(v . dA/ds) / d(dA/du)."""
    s = np.asarray(s, dtype=np.float64)
    gbar = np.empty(2 * s.shape[-1])
    gbar[0::2] = -np.sin(s) * v
    gbar[1::2] = np.cos(s) * v
    if dist is not None and np.any(dist):
        d = np.asarray(dist, dtype=bool)
        gbar[0::2][d] = v[d]
        gbar[1::2][d] = 0.0
    return gbar


def dropout_threshold(rate: float) -> int:
    """A unit is kept iff its 32-bit Philox word is >= this integer."""
    return int(math.floor(rate * 2.0 ** 32))


def dropout_scales(M, B, L, H, step, seed, rate):
    """q [M][B][L][H] of training step `step`: 1 / (1 - rate) for a kept unit,
    0 for a dropped one (counters as in the module docstring)."""
    nw = (H + 3) // 4
    m, b, l, k = np.meshgrid(np.arange(M), np.arange(B), np.arange(L), np.arange(nw), indexing="ij")
    ctr = np.stack([k + nw * (l + L * m), b, np.full_like(b, step), np.full_like(b, DROPOUT_STREAM)], axis=-1)
    words = oracle.philox(ctr.reshape(-1, 4), seed).reshape(M, B, L, 4 * nw)[..., :H]
    keep = words.astype(np.int64) >= dropout_threshold(rate)
    return np.where(keep, 1.0 / (1.0 - rate), 0.0)


def member_value_and_grad(w, D, L, H, resnet, s, q=None, dist=None):
    """A(s) and dA/ds for one member at one point (passes 1 and 2); q [L][H]
    are the dropout scales of the point (None: no dropout); dist [C] marks
    distance CVs (None: all torsions)."""
    layers, w_out, b_out = unpack(np.asarray(w, dtype=np.float64), D, L, H)
    q = np.ones((L, H)) if q is None else np.asarray(q, dtype=np.float64)
    u = features(s, dist)
    h, ts = u, []
    for l, (W, b) in enumerate(layers):
        t = np.tanh(W @ h + b)
        ts.append(t)
        h = q[l] * t + (h if (resnet and l >= 1) else 0.0)
    A = float(w_out @ h + b_out[0])
    g = w_out.copy()
    for l in range(L - 1, -1, -1):
        W = layers[l][0]
        g = W.T @ (g * q[l] * (1.0 - ts[l] ** 2)) + (g if (resnet and l >= 1) else 0.0)
    return A, cv_gradient(s, g, dist)


def loss(w, D, L, H, resnet, s_batch, mf_batch, q=None, dist=None):
    """L = mean over the batch and the C components of (dA/ds - MF)^2; q
    [B][L][H] dropout scales (None: no dropout)."""
    s_batch = np.asarray(s_batch, dtype=np.float64)
    tot = 0.0
    for k, (s, mf) in enumerate(zip(s_batch, np.asarray(mf_batch, dtype=np.float64))):
        _, g = member_value_and_grad(w, D, L, H, resnet, s, None if q is None else q[k], dist)
        tot += float(np.sum((g - mf) ** 2))
    return tot / s_batch.size


def loss_and_grad(w, D, L, H, resnet, s_batch, mf_batch, q=None, dist=None):
    """Loss of one member on a batch and dL/dtheta in the packed layout; q
    [B][L][H] dropout scales of the batch rows (None: no dropout); dist [C]
    marks distance CVs."""
    w = np.asarray(w, dtype=np.float64)
    s_batch = np.asarray(s_batch, dtype=np.float64)
    mf_batch = np.asarray(mf_batch, dtype=np.float64)
    B, C = s_batch.shape
    q = np.ones((B, L, H)) if q is None else np.asarray(q, dtype=np.float64)
    layers, w_out, _ = unpack(w, D, L, H)
    grad = np.zeros_like(w)
    glayers, gw_out, _ = unpack(grad, D, L, H)   # views into grad
    tot = 0.0
    for s, mf, qs in zip(s_batch, mf_batch, q):
        r_ = [bool(resnet and l >= 1) for l in range(L)]
        # 1. forward
        hs = [features(s, dist)]                 # hs[l + 1] = h_l, hs[0] = u
        ts = []
        for l, (W, b) in enumerate(layers):
            t = np.tanh(W @ hs[l] + b)
            ts.append(t)
            hs.append(qs[l] * t + (hs[l] if r_[l] else 0.0))
        # 2. input gradient
        gs = [None] * (L + 1)                    # gs[l + 1] = g_l, gs[0] = dA/du
        ds = [None] * L                          # d_l = g_l * q_l * (1 - t_l^2)
        gs[L] = w_out.copy()
        for l in range(L - 1, -1, -1):
            ds[l] = gs[l + 1] * qs[l] * (1.0 - ts[l] ** 2)
            gs[l] = layers[l][0].T @ ds[l] + (gs[l + 1] if r_[l] else 0.0)
        # 3. loss and its adjoint with respect to dA/du
        dAds = cv_gradient(s, gs[0], dist)
        res = dAds - mf
        tot += float(np.sum(res ** 2))
        v = 2.0 * res / (B * C)
        gbar = cv_gradient_adjoint(s, v, dist)
        # 4. adjoint of the input-gradient pass, increasing l
        tbar = [None] * L
        for l in range(L):
            W = layers[l][0]
            dbar = W @ gbar
            glayers[l][0][...] += np.outer(ds[l], gbar)
            tbar[l] = -2.0 * qs[l] * ts[l] * gs[l + 1] * dbar
            gbar = dbar * qs[l] * (1.0 - ts[l] ** 2) + (gbar if r_[l] else 0.0)
        gw_out[...] += gbar
        # 5. back through the forward pass, decreasing l
        hbar = np.zeros(H)
        for l in range(L - 1, -1, -1):
            W = layers[l][0]
            zbar = (tbar[l] + qs[l] * hbar) * (1.0 - ts[l] ** 2)
            glayers[l][0][...] += np.outer(zbar, hs[l])
            glayers[l][1][...] += zbar
            hbar = W.T @ zbar + (hbar if r_[l] else 0.0)
    return tot / (B * C), grad


def learning_rate(step: int, init_lr: float, decay_rate: float, decay_steps: int) -> float:
    """Exponential decay: init_lr * decay_rate ** (step / decay_steps)."""
    return init_lr * decay_rate ** (step / decay_steps)


def adam_update(w, g, m, v, step: int, lr: float, beta1: float, beta2: float, eps: float):
    """One Adam step (Kingma & Ba, Algorithm 1) at 0-based step index `step`;
    returns the new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** (step + 1))
    vhat = v / (1.0 - beta2 ** (step + 1))
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(weights, D, L, H, resnet, s_data, mf_data, idx, init_lr=8e-4, decay_rate=0.96, decay_steps=120,
          beta1=0.9, beta2=0.999, eps=1e-8, step0=0, m=None, v=None, dropout_rate=0.0, dropout_seed=0, dist=None):
    """Run len(idx) steps; idx [n_steps][M][B] holds each member's batch of
    sample indices.  Returns (weights [M][P], losses [n_steps][M], m, v)."""
    w = np.array(weights, dtype=np.float64)
    Mn = w.shape[0]
    m = np.zeros_like(w) if m is None else np.array(m, dtype=np.float64)
    v = np.zeros_like(w) if v is None else np.array(v, dtype=np.float64)
    s_data = np.asarray(s_data, dtype=np.float64)
    mf_data = np.asarray(mf_data, dtype=np.float64)
    idx = np.asarray(idx)
    losses = np.zeros((idx.shape[0], Mn))
    for k in range(idx.shape[0]):
        t = step0 + k
        lr = learning_rate(t, init_lr, decay_rate, decay_steps)
        q = None
        if dropout_rate > 0:
            q = dropout_scales(Mn, idx.shape[2], L, H, t, dropout_seed, dropout_rate)
        for i in range(Mn):
            b = idx[k, i]
            losses[k, i], g = loss_and_grad(w[i], D, L, H, resnet, s_data[b], mf_data[b],
                                            None if q is None else q[i], dist)
            w[i], m[i], v[i] = adam_update(w[i], g, m[i], v[i], t, lr, beta1, beta2, eps)
    return w, losses, m, v
