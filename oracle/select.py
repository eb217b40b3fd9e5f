"""CPU oracle for the selection phase: candidate frames by model deviation,
threshold clustering of their CVs, representatives.

TEST INFRASTRUCTURE ONLY: imported by the tests -- never by the product path.
It shares no code with the CUDA library.

What it computes (Sec. "Selection phase": cluster_threshold,
numb_cluster_lower / numb_cluster_upper, max_selection; Sec. "Selection":
the explored CVs are clustered, and values with high model deviation are
collected by the trust levels; Sec. "CV selection": per-CV clustering weights
and the angular mask).  Readings (the paper names the parameters, not the
algorithm):
  candidates   frames with trust_lo <= eps < trust_hi (FP32), in frame order;
  distance     d(a, b)^2 = sum_c w_c delta_c^2, delta = a_c - b_c, wrapped onto
               [-pi, pi) for periodic CVs;
  clustering   the leader algorithm in candidate order: a candidate joins the
               first leader within the threshold (d^2 <= t^2), else it becomes
               a leader; each leader is its cluster's representative;
  adaptation   (when asked) the threshold is searched until the cluster count
               falls in [lower, upper]: doubled / halved until the count is
               bracketed, then geometric bisection, at most 64 trials;
  selection    the first max_selection leaders.
The distance test decides an integer (which cluster), so it is taken in FP32
with the operations, and their order, of the kernel:
  delta = a - b; periodic: delta = delta - 2 pi floor(delta * (1 / 2 pi) + 1/2);
  acc = acc + w * (delta * delta), c = 0, 1, ...; compare acc <= float32(t^2).
Every other quantity (the threshold search) is float64.
"""
from __future__ import annotations

import math

import numpy as np

F = np.float32
TWO_PI = F(6.28318530717959)
INV_2PI = F(0.159154943091895)


def dist2(a, b, w, periodic):
    """FP32 weighted squared distances between rows of a [n][C] and one point b [C]."""
    a = np.asarray(a, dtype=F)
    b = np.asarray(b, dtype=F)
    acc = np.zeros(a.shape[0], dtype=F)
    for c in range(a.shape[1]):
        d = (a[:, c] - b[c]).astype(F)
        if periodic[c]:
            k = np.floor((d * INV_2PI).astype(F) + F(0.5)).astype(F)
            d = (d - (TWO_PI * k).astype(F)).astype(F)
        acc = (acc + (F(w[c]) * (d * d).astype(F)).astype(F)).astype(F)
    return acc


def candidates(eps, trust_lo, trust_hi):
    """Frames with trust_lo <= eps < trust_hi, compared in FP32 (the model
    deviations are FP32 and the window decides which frames count)."""
    eps = np.asarray(eps, dtype=F)
    return np.nonzero((eps >= F(trust_lo)) & (eps < F(trust_hi)))[0]


def leaders(cv, w, periodic, t):
    """Leader clustering of the rows of cv in order; returns the leader row
    indices and each row's cluster (index into the leader list)."""
    t2 = F(t * t)
    lead = []
    assign = np.empty(cv.shape[0], dtype=np.int64)
    for k in range(cv.shape[0]):
        j = -1
        if lead:
            d2 = dist2(cv[lead], cv[k], w, periodic)
            hit = np.nonzero(d2 <= t2)[0]
            if hit.size:
                j = int(hit[0])
        if j < 0:
            lead.append(k)
            j = len(lead) - 1
        assign[k] = j
    return np.array(lead, dtype=np.int64), assign


def select(cv, eps, trust_lo, trust_hi, threshold, lower, upper, adapt, max_selection, w=None, periodic=None):
    """Returns dict(selected: frame indices, n_clusters, threshold)."""
    cv = np.asarray(cv, dtype=F)
    C = cv.shape[1]
    w = np.ones(C) if w is None else np.asarray(w)
    periodic = np.ones(C, dtype=bool) if periodic is None else np.asarray(periodic, dtype=bool)
    cand = candidates(eps, trust_lo, trust_hi)
    x = cv[cand]
    t = float(threshold)
    lead, _ = leaders(x, w, periodic, t)
    if adapt and x.shape[0] > 0:
        lo, hi = 0.0, math.inf
        for _ in range(63):
            n = lead.size
            if lower <= n <= upper:
                break
            if n > upper:
                lo = t
                t = 2.0 * t if hi == math.inf else math.sqrt(t * hi)
            else:
                hi = t
                t = 0.5 * t if lo == 0.0 else math.sqrt(lo * t)
            lead, _ = leaders(x, w, periodic, t)
    sel = cand[lead[:max_selection]]
    return dict(selected=sel, n_clusters=int(lead.size), threshold=t)
