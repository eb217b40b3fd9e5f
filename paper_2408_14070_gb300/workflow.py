"""The RiD cycle driven from one configuration (Sec. "Overall Automatic
Workflow"): each iteration explores with the current ensemble, selects frames
by model deviation and clustering, labels them with restrained MD, filters
the labels by their standard deviation, and retrains the ensemble on every
label so far.  Every phase is a call of this library; this module only moves
arrays between them.

Readings, where the paper leaves the cycle to its workflow engine:
  * exploration runs in chunks of `chunk` steps (a multiple of the system's
    output_freq); the configuration at the end of every chunk is a frame,
    with the CVs and model deviation of that step;
  * a first iteration without a model (no `weights` given) explores
    unbiased and takes every frame as a selection candidate (the trust window
    is unbounded); with `weights` given, the first iteration already explores
    with that ensemble's bias and its trust window;
  * a label is kept when the standard deviation of each of its mean-force
    components (kappa times the CV offset from the restraint centre) is at
    most std_threshold (LabelMDConfig; a mean-force threshold);
  * labeling runs n_steps with the first tenth as equilibration and 20
    blocks for the standard error (the restrained-label readings);
  * each iteration trains from the current weights with fresh Adam moments,
    for `epochs` passes over all labels in batches of batch_size (Train),
    each member drawing its own batches;
  * the MD settings (dt, kT, friction) are the system's; the configuration
    supplies the counts, trust levels, restraints, selection and training.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import config as K
from . import inputs as I
from . import rid


@dataclass
class RidResult:
    weights: np.ndarray                 # [M][P] float32, the ensemble after the last iteration
    s: np.ndarray                       # [n][C] float32, restraint centres of the kept labels
    mf: np.ndarray                      # [n][C] float32, their mean forces
    se: np.ndarray                      # [n][C] float64, their standard errors
    x: np.ndarray                       # [W][N][3] float32, the walkers at the end
    iterations: list = field(default_factory=list)   # per-iteration counts and losses


def run(cfg, sp: I.SystemParams, x0: np.ndarray, weights: np.ndarray | None = None, n_iters: int | None = None,
        chunk: int | None = None, precision: int = rid.RID_PREC_FP32, seed: int = 0) -> RidResult:
    """Run the cycle.  cfg: a RidConfig or anything config.load accepts;
    x0 [W][N][3] the starting walkers (W = numb_walkers); weights the initial
    ensemble [M][P] (None: a seeded random one of the Train section's shape)."""
    c = cfg if isinstance(cfg, K.RidConfig) else K.load(cfg)
    if c.cv_mode != "torsion" or c.label["method"] != "restrained":
        raise ValueError("the cycle runs torsion CVs with restrained labels")
    if sp.n_cv != c.n_cv:
        raise ValueError(f"the system has {sp.n_cv} CVs, the configuration {c.n_cv}")
    W, N, C = int(x0.shape[0]), sp.n_beads, sp.n_cv
    if W != c.n_walkers:
        raise ValueError(f"x0 holds {W} walkers, numb_walkers is {c.n_walkers}")
    t = c.train
    D, L, H, M = 2 * C, t["n_layers"], t["width"], t["n_models"]
    biased_first = weights is not None        # a given ensemble biases the first iteration too
    if weights is None:
        weights = I.make_ensemble(M, D, L, H, seed, resnet=t["resnet"]).weights
    weights = np.ascontiguousarray(weights, dtype=np.float32)
    of = sp.output_freq
    chunk = chunk or of * max(1, c.explore["n_steps"] // (of * 10))
    if chunk % of:
        raise ValueError("chunk must be a multiple of the system's output_freq")
    n_chunks = max(1, c.explore["n_steps"] // chunk)
    lab_steps = c.label["n_steps"]
    n_equil, n_blocks = lab_steps // 10, 20
    rng = np.random.default_rng(seed)
    s_all, mf_all, se_all, its = [], [], [], []
    x, v = np.ascontiguousarray(x0, dtype=np.float32), None
    step = 0
    with rid.System(sp) as s:
        for it in range(n_iters if n_iters is not None else c.n_iters):
            rec = {"iteration": it}
            have_model = it > 0 or biased_first
            if have_model:
                s.set_ensemble(I.EnsembleParams(M, D, L, H, t["resnet"], weights, c.trust_lo, c.trust_hi),
                               precision=precision)
            # ---- exploration: one frame per chunk and walker
            fx, fcv, feps = [], [], []
            T = chunk // of
            for _ in range(n_chunks):
                cv = np.zeros((W, T, C), np.float32)
                eps = np.zeros((W, T), np.float32)
                xo, vo = np.zeros_like(x), np.zeros_like(x)
                s.explore(x, chunk, v0=v, step0=step, cv_out=cv, eps_out=eps, x_out=xo, v_out=vo)
                step += chunk
                fx.append(xo)
                fcv.append(cv[:, -1])
                feps.append(eps[:, -1])
                x, v = xo, vo
            fx = np.concatenate(fx)
            fcv = np.ascontiguousarray(np.concatenate(fcv))
            feps = np.ascontiguousarray(np.concatenate(feps))
            rec.update(frames=int(fx.shape[0]), eps_mean=float(feps.mean()))
            # ---- selection
            sc = c.select
            lo, hi = (sc["trust_lo"], sc["trust_hi"]) if have_model else (-1e30, 1e30)
            sel, nc, thr = rid.select(fcv, feps, lo, hi, sc["threshold"], sc["lower"], sc["upper"], sc["adapt"],
                                      sc["max_selection"], weights=sc["weights"], periodic=sc["periodic"])
            rec.update(clusters=int(nc), threshold=float(thr), selected=int(sel.size))
            # ---- restrained labels at the selected frames, centred on their CVs
            if sel.size:
                R = sel.size
                s0 = fcv[sel].astype(np.float64)
                kappa = np.ascontiguousarray(np.broadcast_to(c.label["kappa"], (R, C)))
                mf, se, sd = (np.zeros((R, C)) for _ in range(3))
                s.label(np.ascontiguousarray(fx[sel]), s0, kappa, lab_steps, n_equil, n_blocks, mf, se, sd,
                        step0=step)
                step += lab_steps   # later runs draw fresh noise counters
                keep = np.all(sd <= c.label["std_threshold"], axis=1) & np.all(np.isfinite(mf), axis=1)
                s_all.append(s0[keep].astype(np.float32))
                mf_all.append(mf[keep].astype(np.float32))
                se_all.append(se[keep])
                rec["labels_kept"] = int(keep.sum())
            else:
                rec["labels_kept"] = 0
            # ---- training on every label so far
            n_lab = int(sum(a.shape[0] for a in s_all))
            rec["labels_total"] = n_lab
            if n_lab:
                B = t["batch_size"]
                steps = c.train_steps(n_lab)
                idx = rng.integers(0, n_lab, size=(steps, M, B)).astype(np.int32)
                losses = np.zeros((steps, M), np.float32)
                with rid.Trainer(M, C, L, H, weights, batch_size=B, resnet=t["resnet"], init_lr=t["init_lr"],
                                 decay_rate=t["decay_rate"], decay_steps=t["decay_steps"],
                                 dropout_rate=t["dropout_rate"], dropout_seed=seed + it) as tr:
                    tr.set_data(np.concatenate(s_all), np.concatenate(mf_all))
                    tr.run(idx, losses)
                    weights, _ = tr.weights()
                rec.update(train_steps=steps, loss_first=float(losses[0].mean()), loss_last=float(losses[-1].mean()))
            its.append(rec)
    C0 = np.zeros((0, C), np.float32)
    return RidResult(weights, np.concatenate(s_all) if s_all else C0, np.concatenate(mf_all) if mf_all else C0,
                     np.concatenate(se_all) if se_all else C0.astype(np.float64), x, its)
