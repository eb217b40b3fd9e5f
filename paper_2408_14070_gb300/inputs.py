"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the method itself (no forces, CVs, network
passes or integrator): it only draws parameters and starting geometries from a
seed, so that the GPU path and the FP64 oracle see byte-identical inputs.

The paper's workloads (solvated chignolin with 18 backbone torsions, a 4 x
[300]^4 residual ensemble, 12 walkers; the HfO2 Deep-Potential system) are not
available, so bead chains in implicit solvent stand in for them:

* force field (reduced units, kT = 1, mass = 1): harmonic bonds k = 100,
  r0 = 1; harmonic angles k = 20, theta0 = 110 deg; three-term dihedrals
  sum_n k_n (1 + cos(n phi - delta_n)) with k_n ~ U(0, 2), delta_n ~ U(0, 2 pi)
  per dihedral; Lennard-Jones eps = 1, sigma = 1, cutoff 2.5, 1-2 and 1-3
  pairs excluded;
* CVs: C evenly spaced backbone-like torsions i_j = floor((j + 1/2)(N - 3)/C)
  over beads (i_j, i_j+1, i_j+2, i_j+3) -- the stand-in for the phi/psi
  torsions of "torsion" mode (Sec. "CV selection", Table 2);
* ensemble: M tanh MLPs D -> H x L -> 1 (Sec. "Training phase": numb_models,
  neurons), Glorot-uniform weights; biases are drawn U(-0.2, 0.2) rather than
  zero so that a dropped bias term shows up in every parity test;
* starting chains: self-avoiding random chains built bead by bead from the
  bond length, bond angle and a uniform random dihedral, rejecting placements
  closer than 0.9 to any non-excluded earlier bead.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "SystemParams", "EnsembleParams", "make_system", "cv_is_distance", "make_chains",
    "make_ensemble", "make_label_targets", "ensemble_param_count",
    "WORKLOADS", "workload", "chain_length_buckets", "label_batch_jobs", "serving_requests",
]

_TAG_SYSTEM, _TAG_CHAIN, _TAG_ENS, _TAG_LABEL, _TAG_MIX = 11, 23, 37, 41, 53


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(tag)])


@dataclass
class SystemParams:
    n_beads: int
    n_cv: int
    seed: int
    mass: float = 1.0
    kT: float = 1.0
    dt: float = 0.005
    gamma: float = 1.0
    bond_k: float = 100.0
    bond_r0: float = 1.0
    angle_k: float = 20.0
    angle_theta0: float = math.radians(110.0)
    lj_eps: float = 1.0
    lj_sigma: float = 1.0
    lj_rc: float = 2.5
    output_freq: int = 50
    dihedral_k: np.ndarray = field(default=None, repr=False)      # [N-3][3] f64
    dihedral_delta: np.ndarray = field(default=None, repr=False)  # [N-3][3] f64
    cv_atoms: np.ndarray = field(default=None, repr=False)        # [C][4] int32


@dataclass
class EnsembleParams:
    n_models: int
    n_in: int
    n_layers: int
    width: int
    resnet: bool
    weights: np.ndarray = field(repr=False)  # [M][P] float32, packed per model
    trust_lo: float = 2.0
    trust_hi: float = 3.0


def evenly_spaced_cvs(n_beads: int, n_cv: int) -> np.ndarray:
    """C torsion quadruples spread evenly along the chain."""
    if n_beads < 4 or n_cv < 1:
        raise ValueError("need n_beads >= 4 and n_cv >= 1")
    nd = n_beads - 3
    first = np.floor((np.arange(n_cv) + 0.5) * nd / n_cv).astype(np.int64)
    return (first[:, None] + np.arange(4)[None, :]).astype(np.int32)


def make_system(n_beads: int, n_cv: int, seed: int, n_dist: int = 0, dist_span: int = 5,
                **overrides) -> SystemParams:
    """A chain with n_cv CVs: n_cv - n_dist evenly spaced torsions, then
    n_dist distance CVs between beads (a, a + dist_span), their first beads
    spread evenly along the chain (rows (a, a + span, -1, -1))."""
    sp = SystemParams(n_beads=n_beads, n_cv=n_cv, seed=seed, **overrides)
    g = _rng(seed, _TAG_SYSTEM)
    nd = n_beads - 3
    sp.dihedral_k = g.uniform(0.0, 2.0, size=(nd, 3))
    sp.dihedral_delta = g.uniform(0.0, 2.0 * math.pi, size=(nd, 3))
    nt = n_cv - n_dist
    if n_dist < 0 or nt < 0 or (n_dist and n_beads <= dist_span):
        raise ValueError("need 0 <= n_dist <= n_cv and n_beads > dist_span")
    rows = [evenly_spaced_cvs(n_beads, nt)] if nt else []
    if n_dist:
        first = np.floor((np.arange(n_dist) + 0.5) * (n_beads - dist_span) / n_dist).astype(np.int32)
        rows.append(np.stack([first, first + dist_span, -np.ones_like(first), -np.ones_like(first)], axis=1))
    sp.cv_atoms = np.ascontiguousarray(np.concatenate(rows).astype(np.int32))
    return sp


def cv_is_distance(sp: SystemParams) -> np.ndarray:
    """Boolean [C]: which CVs are distances (rows ending in -1, -1)."""
    return np.asarray(sp.cv_atoms)[:, 2] < 0


def _place_next(a, b, c, bond, theta, phi):
    """Place a bead at distance `bond` from c, angle `theta` at c (b-c-new)
    and dihedral `phi` for (a, b, c, new).  Vectorised over rows."""
    bc = c - b
    bc /= np.linalg.norm(bc, axis=-1, keepdims=True)
    n = np.cross(b - a, bc)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    m = np.cross(n, bc)
    d2 = np.stack([-bond * np.cos(theta) * np.ones_like(phi),
                   bond * np.sin(theta) * np.cos(phi),
                   bond * np.sin(theta) * np.sin(phi)], axis=-1)
    return c + d2[:, :1] * bc + d2[:, 1:2] * m + d2[:, 2:3] * n


def _grow(n, N, r0, th, g, min_dist, max_tries):
    """Grow n chains; returns positions and a mask of chains that got trapped."""
    x = np.zeros((n, N, 3), dtype=np.float64)
    x[:, 1, 0] = r0
    if N > 2:
        x[:, 2, 0] = r0 - r0 * math.cos(th)
        x[:, 2, 1] = r0 * math.sin(th)
    alive = np.ones(n, dtype=bool)
    for i in range(3, N):
        todo = np.flatnonzero(alive)
        for _ in range(max_tries):
            phi = g.uniform(-math.pi, math.pi, size=todo.size)
            cand = _place_next(x[todo, i - 3], x[todo, i - 2], x[todo, i - 1], r0, th, phi)
            d = np.linalg.norm(x[todo, : i - 2] - cand[:, None, :], axis=-1)
            ok = (d >= min_dist).all(axis=1)
            x[todo[ok], i] = cand[ok]
            todo = todo[~ok]
            if todo.size == 0:
                break
        alive[todo] = False
    return x, alive


def make_chains(n_walkers: int, sp: SystemParams, seed: int,
                min_dist: float = 0.9, max_tries: int = 200) -> np.ndarray:
    """Self-avoiding starting chains, float32 [W][N][3], centred at the origin.

    Chains that get trapped while growing are regrown from scratch."""
    N = sp.n_beads
    g = _rng(seed, _TAG_CHAIN)
    x = np.zeros((n_walkers, N, 3), dtype=np.float64)
    need = np.arange(n_walkers)
    for _ in range(100):
        xs, ok = _grow(need.size, N, sp.bond_r0, sp.angle_theta0, g, min_dist, max_tries)
        x[need[ok]] = xs[ok]
        need = need[~ok]
        if need.size == 0:
            break
    if need.size:
        raise RuntimeError("chain growth kept getting trapped")
    # a random overall orientation per walker (QR of a Gaussian matrix), centred
    q, r = np.linalg.qr(g.standard_normal((n_walkers, 3, 3)))
    q = q * np.sign(np.diagonal(r, axis1=1, axis2=2))[:, None, :]
    x = np.einsum("wij,wnj->wni", q, x)
    x -= x.mean(axis=1, keepdims=True)
    return np.ascontiguousarray(x.astype(np.float32))


def ensemble_param_count(n_in: int, n_layers: int, width: int) -> int:
    """Floats per packed model: W1[H][D], b1[H], (W_l[H][H], b_l[H]) for
    l = 2..L, w_out[H], b_out."""
    H = width
    return H * n_in + H + (n_layers - 1) * (H * H + H) + H + 1


def make_ensemble(n_models: int, n_in: int, n_layers: int, width: int, seed: int,
                  resnet: bool = False, trust_lo: float = 2.0,
                  trust_hi: float = 3.0, bias_scale: float = 0.2) -> EnsembleParams:
    g = _rng(seed, _TAG_ENS)
    P = ensemble_param_count(n_in, n_layers, width)
    out = np.empty((n_models, P), dtype=np.float32)
    for m in range(n_models):
        parts = []
        fan_in = n_in
        for _ in range(n_layers):
            a = math.sqrt(6.0 / (fan_in + width))
            parts.append(g.uniform(-a, a, size=(width, fan_in)).ravel())
            parts.append(g.uniform(-bias_scale, bias_scale, size=width))
            fan_in = width
        a = math.sqrt(6.0 / (width + 1))
        parts.append(g.uniform(-a, a, size=width))
        parts.append(g.uniform(-bias_scale, bias_scale, size=1))
        out[m] = np.concatenate(parts).astype(np.float32)
    return EnsembleParams(n_models, n_in, n_layers, width, resnet, out, trust_lo, trust_hi)


def make_label_targets(n_runs: int, n_cv: int, seed: int) -> np.ndarray:
    """Restraint centres s0, uniform on the torus [-pi, pi)^C, float64 [R][C]."""
    g = _rng(seed, _TAG_LABEL)
    return g.uniform(-math.pi, math.pi, size=(n_runs, n_cv))


# Workload recipes (chain length, CV count, ensemble shape, batch) -------------
WORKLOADS = {
    "tiny_n22": dict(n_beads=22, n_cv=2, n_models=4, n_layers=3, width=64,
                     n_walkers=16, n_steps=2000, n_label_runs=16,
                     label_steps=1000, kappa=50.0),
    "chain_n200_w1024": dict(n_beads=200, n_cv=20, n_models=4, n_layers=4,
                             width=256, n_walkers=1024, n_steps=10000),
    "chain_n100_w8192": dict(n_beads=100, n_cv=32, n_models=8, n_layers=4,
                             width=512, n_walkers=8192, n_steps=10000),
}


def workload(name: str) -> dict:
    return dict(WORKLOADS[name])


# --------------------------------------------------------------------------
# Job mixes for batched labeling and for the request stream.  Chain lengths
# are drawn log-uniformly and snapped to a fixed set of bucket lengths, so that
# starting chains can be grown once per bucket for many jobs.

def chain_length_buckets(lo: int, hi: int, n: int = 24) -> np.ndarray:
    return np.unique(np.round(np.geomspace(lo, hi, n)).astype(int))


def _snap(x: np.ndarray, buckets: np.ndarray) -> np.ndarray:
    lx, lb = np.log(x), np.log(buckets.astype(np.float64))
    return buckets[np.abs(lx[:, None] - lb[None, :]).argmin(axis=1)]


def label_batch_jobs(n_jobs: int, seed: int, n_lo: int = 50, n_hi: int = 500, cv_lo: int = 4, cv_hi: int = 40,
                     kappa_lo: float = 50.0, kappa_hi: float = 500.0, width_lo: int = 128, width_hi: int = 512,
                     n_steps: int = 2000) -> list:
    """Uneven restrained labeling jobs, one run each: chain length log-uniform
    in [n_lo, n_hi] (snapped to buckets), CV count uniform in [cv_lo, cv_hi],
    per-CV kappa uniform in [kappa_lo, kappa_hi], an ensemble width uniform in
    [width_lo, width_hi] (multiples of 32; labeling runs do not use it)."""
    g = _rng(seed, _TAG_MIX)
    b = chain_length_buckets(n_lo, n_hi)
    N = _snap(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), size=n_jobs)), b)
    out = []
    for k in range(n_jobs):
        C = int(min(g.integers(cv_lo, cv_hi + 1), N[k] - 3))
        out.append(dict(n_beads=int(N[k]), n_cv=C, seed=int(g.integers(1, 2 ** 31)),
                        kappa=g.uniform(kappa_lo, kappa_hi, size=C),
                        width=int(32 * g.integers(width_lo // 32, width_hi // 32 + 1)), n_steps=n_steps))
    return out


def serving_requests(n_req: int, rate: float, seed: int, p_label: float = 0.7, n_lo: int = 20, n_hi: int = 2000,
                     cv_lo: int = 2, cv_hi: int = 64, steps_lo: int = 500, steps_hi: int = 5000,
                     width_lo: int = 64, width_hi: int = 512, explore_walkers: int = 12,
                     kappa_lo: float = 50.0, kappa_hi: float = 500.0) -> list:
    """A Poisson stream of mixed requests: arrival times with exponential gaps
    of mean 1/rate; a labeling request (one run) with probability p_label,
    else an exploration request with `explore_walkers` walkers; chain length
    log-uniform in [n_lo, n_hi] (snapped to buckets), CV count uniform in
    [cv_lo, cv_hi], step count uniform in [steps_lo, steps_hi], ensemble of
    4 members of width uniform in [width_lo, width_hi] (multiples of 32) with
    4 hidden layers."""
    g = _rng(seed, _TAG_MIX + 1)
    t = np.cumsum(g.exponential(1.0 / rate, size=n_req))
    b = chain_length_buckets(n_lo, n_hi)
    N = _snap(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), size=n_req)), b)
    out = []
    for k in range(n_req):
        label = bool(g.uniform() < p_label)
        C = int(min(g.integers(cv_lo, cv_hi + 1), N[k] - 3))
        out.append(dict(t=float(t[k]), kind="label" if label else "explore", n_beads=int(N[k]), n_cv=C,
                        walkers=1 if label else explore_walkers, n_steps=int(g.integers(steps_lo, steps_hi + 1)),
                        width=int(32 * g.integers(width_lo // 32, width_hi // 32 + 1)), n_layers=4, n_models=4,
                        kappa=g.uniform(kappa_lo, kappa_hi, size=C), seed=int(g.integers(1, 2 ** 31))))
    return out
