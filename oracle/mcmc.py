"""FP64 CPU oracle for the MCMC dimension reduction of the trained ensemble.

TEST INFRASTRUCTURE ONLY: imported by the tests -- never by the product path.
It shares no code with the CUDA library; the random numbers come from the
oracle's own Philox4x32-10 / Box-Muller (``oracle.philox``, ``oracle.normals``).

What it computes (Sec. "Dimension reduction phase"; Introduction, automatic
PMF calculation): W walkers run Metropolis Monte Carlo in CV space on the
ensemble-mean free energy Abar(s) = (1/M) sum_i A_i(s) at temperature kT, and
the visited CVs are projected onto one histogram per CV and one 2-D histogram
of a chosen CV pair (bins per dimension over [-pi, pi)); the projected PMF is
-kT ln(count / total), shifted to a zero minimum.

Readings (the paper names the parameters, not the move):
  proposal  s'_c = wrap(s_c + step_size * xi_c), xi from Philox counter
            (c // 3, walker, step, 2), normal c % 3 of the three Box-Muller
            normals of that counter (the MD noise mapping);
  accept    iff kT ln u + (Abar(s') - Abar(s)) < 0, u = (x + 1/2) 2^-32 from
            word 0 of counter (0, walker, step, 3);
  counting  after every step t >= n_burn, every walker's current state;
  bins      floor((s + pi) / (2 pi) * bins), clamped to [0, bins - 1];
  wrap      d - 2 pi floor(d / (2 pi) + 1/2).
Distance CVs (Sec. "CV selection"; the dimension reduction's cv_type "dis"
with cv_lower_bound / cv_upper_bound): a distance CV is not wrapped, its
proposal s' = s + step_size xi is refused when any distance CV leaves its
range [lo, hi] (the walk then samples exp(-Abar/kT) restricted to the box),
its bins are floor((s - lo) / (hi - lo) * bins) clamped, its MLP input is
(s, 0), and path differences over it are plain.
The "path" projection maps a state onto the path collective variables of
Branduardi, Gervasio and Parrinello (2007) for nodes p_1..p_P over a subset of
the CVs (wrapped differences): with d_i = |s - p_i|^2,
  s_path = sum_i i exp(-lambda d_i) / sum_i exp(-lambda d_i)  in [1, P],
  z_path = -(1/lambda) ln sum_i exp(-lambda d_i),
evaluated with the smallest d_i factored out; the (s_path, z_path) histogram
has bins over [1, P] and over a given [z_lo, z_hi], values clamped.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from oracle import train as T


def wrap(d):
    return d - 2.0 * math.pi * np.floor(d / (2.0 * math.pi) + 0.5)


def ensemble_mean_value(weights, D, L, H, resnet, s, dist=None):
    """Abar at points s [W][C] (float64), members' forward passes as matmuls."""
    u = T.features(s, dist)
    tot = np.zeros(s.shape[0])
    for w in np.asarray(weights, dtype=np.float64):
        layers, w_out, b_out = T.unpack(w, D, L, H)
        h = u
        for l, (W, b) in enumerate(layers):
            t = np.tanh(h @ W.T + b)
            h = t + h if (resnet and l >= 1) else t
        tot += h @ w_out + b_out[0]
    return tot / len(weights)


def proposal_normals(W, C, step, seed):
    nk = (C + 2) // 3
    ctr = np.array([[k, w, step, 2] for w in range(W) for k in range(nk)], dtype=np.uint32)
    return oracle.normals(ctr, seed).reshape(W, 3 * nk)[:, :C]


def accept_log_u(W, step, seed):
    ctr = np.array([[0, w, step, 3] for w in range(W)], dtype=np.uint32)
    x = oracle.philox(ctr, seed)[:, 0].astype(np.float64)
    return np.log((x + 0.5) * 2.0 ** -32)


def bin_index(s, bins, dist=None, lo=None, hi=None):
    s = np.asarray(s, dtype=np.float64)
    b = np.floor((s + math.pi) / (2.0 * math.pi) * bins)
    if dist is not None and np.any(dist):
        d = np.asarray(dist, dtype=bool)
        b[..., d] = np.floor((s[..., d] - np.asarray(lo)[d]) / (np.asarray(hi)[d] - np.asarray(lo)[d]) * bins)
    return np.clip(b.astype(np.int64), 0, bins - 1)


def path_cv(s, nodes, cvs, lam, dist=None):
    """(s_path, z_path) of points s [W][C] for path nodes [P][Cp] over the CVs `cvs`."""
    nodes = np.asarray(nodes, dtype=np.float64)
    d = np.asarray(s, dtype=np.float64)[:, None, list(cvs)] - nodes[None]
    per = np.ones(len(cvs), dtype=bool) if dist is None else ~np.asarray(dist, dtype=bool)[list(cvs)]
    d[..., per] = wrap(d[..., per])
    d2 = (d * d).sum(axis=-1)                          # [W][P]
    m = d2.min(axis=1)
    e = np.exp(-lam * (d2 - m[:, None]))
    se = e.sum(axis=1)
    sp = (e * np.arange(1, nodes.shape[0] + 1)).sum(axis=1) / se
    return sp, m - np.log(se) / lam


def path_bins(sp, z, n_nodes, z_lo, z_hi, bins):
    bs = np.floor((np.asarray(sp) - 1.0) / (n_nodes - 1) * bins).astype(np.int64)
    bz = np.floor((np.asarray(z) - z_lo) / (z_hi - z_lo) * bins).astype(np.int64)
    return np.clip(bs, 0, bins - 1), np.clip(bz, 0, bins - 1)


def run(weights, C, L, H, resnet, s0, n_steps, n_burn, kT, step_size, seed, bins, pair, path=None,
        dist=None, lo=None, hi=None):
    """Returns dict(s, A, n_accepted, hist1 [C][bins], hist2 [bins][bins],
    hist_path [bins][bins] (when path = (nodes, cvs, lam, z_lo, z_hi)),
    min_margin [W]): min_margin is each walker's smallest |kT ln u + dA| over
    the run (how close its closest accept decision came to the threshold),
    and with distance CVs (dist [C] bool, ranges lo / hi [C]) also the closest
    approach of a proposal to a range edge."""
    D = 2 * C
    s = np.array(s0, dtype=np.float64)
    W = s.shape[0]
    dmask = np.zeros(C, dtype=bool) if dist is None else np.asarray(dist, dtype=bool)
    lo = np.zeros(C) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.zeros(C) if hi is None else np.asarray(hi, dtype=np.float64)
    A = ensemble_mean_value(weights, D, L, H, resnet, s, dmask)
    hist1 = np.zeros((C, bins), dtype=np.int64)
    hist2 = np.zeros((bins, bins), dtype=np.int64)
    histp = np.zeros((bins, bins), dtype=np.int64)
    n_acc = 0
    min_margin = np.full(W, np.inf)
    for t in range(n_steps):
        sp = s + step_size * proposal_normals(W, C, t, seed)
        sp[:, ~dmask] = wrap(sp[:, ~dmask])
        inside = np.all((sp[:, dmask] >= lo[dmask]) & (sp[:, dmask] <= hi[dmask]), axis=1)
        if dmask.any():
            edge = np.minimum(np.abs(sp[:, dmask] - lo[dmask]), np.abs(sp[:, dmask] - hi[dmask])).min(axis=1)
            min_margin = np.minimum(min_margin, edge)
        Ap = ensemble_mean_value(weights, D, L, H, resnet, sp, dmask)
        margin = kT * accept_log_u(W, t, seed) + (Ap - A)
        acc = (margin < 0.0) & inside
        min_margin = np.minimum(min_margin, np.where(inside, np.abs(margin), np.inf))
        s[acc] = sp[acc]
        A[acc] = Ap[acc]
        n_acc += int(acc.sum())
        if t >= n_burn:
            b = bin_index(s, bins, dmask, lo, hi)
            for c in range(C):
                hist1[c] += np.bincount(b[:, c], minlength=bins)
            np.add.at(hist2, (b[:, pair[0]], b[:, pair[1]]), 1)
            if path is not None:
                nodes, cvs, lam, z_lo, z_hi = path
                sp_, z_ = path_cv(s, nodes, cvs, lam, dmask)
                bs, bz = path_bins(sp_, z_, len(nodes), z_lo, z_hi, bins)
                np.add.at(histp, (bs, bz), 1)
    return dict(s=s, A=A, n_accepted=n_acc, hist1=hist1, hist2=hist2, hist_path=histp, min_margin=min_margin)


def projected_pmf(hist, kT):
    """-kT ln(count / total) shifted to a zero minimum; +inf for empty bins."""
    h = np.asarray(hist, dtype=np.float64)
    with np.errstate(divide="ignore"):
        f = -kT * np.log(h / h.sum())
    return f - f[np.isfinite(f)].min()
