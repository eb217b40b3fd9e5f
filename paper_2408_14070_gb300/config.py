"""Run settings from a RiD-style JSON configuration.

The paper drives every phase of the workflow from one JSON document (Sec.
"Overall workflow setting", "CV selection" and the Exploration, Selection,
Labeling, Training and Dimension reduction phases).  This module reads the
keys those sections define and returns the arguments of this library's
calls, so a configuration written for the paper's workflow carries over:

  top level          numb_walkers, numb_iters, trust_lvl_1, trust_lvl_2
  "CV"               mode ("torsion" | "distance"), selected_resid (torsion:
                     2 n - 2 CVs for n residues), selected_atomid (distance:
                     pairs of 1-based atom ids), angular_mask, weights
  "ExploreMDConfig"  nsteps, dt, temperature, output_freq
  "LabelMDConfig"    method ("restrained" | "constrained"), nsteps, kappas,
                     std_threshold, dt, temperature, output_freq
  "SelectorConfig"   cluster_threshold, numb_cluster_lower,
                     numb_cluster_upper, max_selection
  "Train"            numb_models, neurons, resnet, batch_size, epochs,
                     init_lr, decay_steps, decay_rate, drop_out_rate
  "MCMC_Config"      numb_steps, numb_walkers, temperature, bins, cv_type
                     ("dih" | "dis"), cv_lower_bound, cv_upper_bound,
                     proj_info {proj_mode, proj_cv_index, path_list, path_lm}

Units: energies (trust levels, kappas, std_threshold) are passed through in
the configuration's own unit (kJ/mol in the paper), and kT = kB * temperature
with kB in that unit per kelvin (the molar gas constant in kJ/(mol K) by
default).  With reduced=True, kT = 1 and every value is kept as given (the
reduced units of the bead chains).  Keys that configure the paper's external
engines and files (GROMACS / LAMMPS / PLUMED settings, cv_file, init_models,
dp_model, numb_threads, name) are ignored.  Host logic only: nothing here
touches a device.
"""
from __future__ import annotations

import json
import math
from dataclasses import dataclass, field

import numpy as np

KB_KJ_PER_MOL_K = 8.31446261815324e-3   # molar gas constant, kJ / (mol K)


@dataclass
class RidConfig:
    n_walkers: int
    n_iters: int
    trust_lo: float
    trust_hi: float
    cv_mode: str                        # "torsion" | "distance"
    n_cv: int
    periodic: np.ndarray                # [C] int32, 1 = periodic over 2 pi
    cv_weights: np.ndarray              # [C] float32 (selection distance)
    distance_pairs: np.ndarray | None   # [C][2] int32, 0-based (distance mode)
    explore: dict = field(default_factory=dict)
    label: dict = field(default_factory=dict)
    select: dict = field(default_factory=dict)
    train: dict = field(default_factory=dict)
    mcmc: dict = field(default_factory=dict)

    def train_steps(self, n_labels: int) -> int:
        """Adam steps of `epochs` passes over n_labels labels in batches of batch_size."""
        t = self.train
        return int(math.ceil(t["epochs"] * n_labels / t["batch_size"]))


def _per_cv(values, n_cv: int, name: str, dtype) -> np.ndarray:
    a = np.asarray(values, dtype=dtype).reshape(-1)
    if a.size == 1:
        return np.full(n_cv, a[0], dtype=dtype)
    if a.size != n_cv:
        raise ValueError(f"{name} has {a.size} entries for {n_cv} CVs")
    return a


def _kT(temperature, reduced: bool, kb: float) -> float:
    return 1.0 if reduced else kb * float(temperature)


def cv_atoms(c: "RidConfig", torsion_atoms: np.ndarray | None = None) -> np.ndarray:
    """cv_atoms rows of rid_create_system for the configuration's CVs: the
    given torsion quadruples in torsion mode, rows (a, b, -1, -1) (0-based)
    for the distance pairs in distance mode."""
    if c.cv_mode == "distance":
        p = np.asarray(c.distance_pairs, dtype=np.int32)
        return np.ascontiguousarray(np.concatenate([p, -np.ones_like(p)], axis=1))
    if torsion_atoms is None:
        raise ValueError("torsion mode: the torsion quadruples come from the system")
    return np.ascontiguousarray(torsion_atoms, dtype=np.int32)


def load(cfg, reduced: bool = False, kb: float = KB_KJ_PER_MOL_K) -> RidConfig:
    """Parse a RiD-style configuration: a dict, a JSON string or a path."""
    if isinstance(cfg, str):
        cfg = json.loads(cfg) if cfg.lstrip().startswith("{") else json.load(open(cfg))
    cv = cfg.get("CV", {})
    mode = cv.get("mode", "torsion")
    pairs = None
    if mode == "torsion":
        resid = cv.get("selected_resid", [])
        if len(resid) < 2:
            raise ValueError("torsion CVs need at least two selected residues")
        n_cv = 2 * len(resid) - 2                      # no phi on the first residue, no psi on the last
    elif mode == "distance":
        ids = np.asarray(cv.get("selected_atomid", []), dtype=np.int64)
        if ids.ndim != 2 or ids.shape[1] != 2 or ids.shape[0] < 1 or (ids < 1).any():
            raise ValueError("selected_atomid must be pairs of 1-based atom ids")
        pairs = (ids - 1).astype(np.int32)
        n_cv = pairs.shape[0]
    else:
        raise ValueError(f"CV mode {mode!r}: only 'torsion' and 'distance' run in this library")
    periodic = _per_cv(cv.get("angular_mask", 1 if mode == "torsion" else 0), n_cv, "angular_mask", np.int32)
    weights = _per_cv(cv.get("weights", 1.0), n_cv, "weights", np.float32)
    tlo, thi = float(cfg.get("trust_lvl_1", 2.0)), float(cfg.get("trust_lvl_2", 3.0))
    if not thi > tlo:
        raise ValueError("trust_lvl_2 must exceed trust_lvl_1")

    ex = cfg.get("ExploreMDConfig", {})
    explore = {"n_steps": int(ex.get("nsteps", 0)), "dt": float(ex.get("dt", 0.005)),
               "kT": _kT(ex.get("temperature", 300.0), reduced, kb), "output_freq": int(ex.get("output_freq", 1))}

    lb = cfg.get("LabelMDConfig", {})
    method = lb.get("method", "restrained")
    if method not in ("restrained", "constrained"):
        raise ValueError(f"label method {method!r}")
    if method == "constrained" and mode != "distance":
        raise ValueError("constrained labels need distance CVs")
    label = {"method": method, "n_steps": int(lb.get("nsteps", 0)), "dt": float(lb.get("dt", explore["dt"])),
             "kT": _kT(lb.get("temperature", ex.get("temperature", 300.0)), reduced, kb),
             "output_freq": int(lb.get("output_freq", explore["output_freq"]))}
    if method == "restrained":
        label["kappa"] = _per_cv(lb.get("kappas", 500.0), n_cv, "kappas", np.float64)
        label["std_threshold"] = float(lb.get("std_threshold", 5.0))

    sc = cfg.get("SelectorConfig", {})
    select = {"trust_lo": tlo, "trust_hi": thi, "threshold": float(sc.get("cluster_threshold", 1.0)),
              "lower": int(sc.get("numb_cluster_lower", 1)), "upper": int(sc.get("numb_cluster_upper", 1 << 30)),
              "adapt": "numb_cluster_lower" in sc or "numb_cluster_upper" in sc,
              "max_selection": int(sc.get("max_selection", 50)), "weights": weights, "periodic": periodic}

    tr = cfg.get("Train", {})
    neurons = list(tr.get("neurons", [256, 256, 256, 256]))
    if not neurons or len(set(neurons)) != 1:
        raise ValueError("neurons must list one width for every hidden layer")
    train = {"n_models": int(tr.get("numb_models", 4)), "n_layers": len(neurons), "width": int(neurons[0]),
             "resnet": bool(tr.get("resnet", False)), "batch_size": int(tr.get("batch_size", 128)),
             "epochs": int(tr.get("epochs", 1)), "init_lr": float(tr.get("init_lr", 8e-4)),
             "decay_steps": int(tr.get("decay_steps", 120)), "decay_rate": float(tr.get("decay_rate", 0.96)),
             "dropout_rate": float(tr.get("drop_out_rate", 0.0))}
    if train["n_models"] < 1:
        raise ValueError("numb_models must be at least 1")

    mc = cfg.get("MCMC_Config", {})
    mcmc = {}
    if mc:
        cv_type = mc.get("cv_type", "dih")
        if cv_type not in ("dih", "dis"):
            raise ValueError(f"MCMC cv_type {cv_type!r}: 'dih' (torsions) or 'dis' (distances)")
        if (cv_type == "dis") != (mode == "distance"):
            raise ValueError(f"MCMC cv_type {cv_type!r} does not match the CV mode {mode!r}")
        proj = mc.get("proj_info", {"proj_mode": "cv", "proj_cv_index": [0, 1]})
        idx = [int(i) for i in proj.get("proj_cv_index", [0, 1])]
        if any(i < 0 or i >= n_cv for i in idx):
            raise ValueError("proj_cv_index outside the CVs")
        mcmc = {"n_walkers": int(mc.get("numb_walkers", 2000)), "n_steps": int(mc.get("numb_steps", 0)),
                "kT": _kT(mc.get("temperature", 300.0), reduced, kb), "bins": int(mc.get("bins", 101)),
                "pair": (0, min(1, n_cv - 1)), "path": None, "cv_dist": np.zeros(n_cv, dtype=bool),
                "cv_range": None}
        if cv_type == "dis":
            # reading: cv_lower_bound / cv_upper_bound (the paper's range of the
            # initial values, "usually set for distance CVs") bound the walk of
            # each distance CV; the library needs a range, so they are required
            if "cv_lower_bound" not in mc or "cv_upper_bound" not in mc:
                raise ValueError("distance CVs in MCMC need cv_lower_bound and cv_upper_bound")
            lo = _per_cv(mc["cv_lower_bound"], n_cv, "cv_lower_bound", np.float64)
            hi = _per_cv(mc["cv_upper_bound"], n_cv, "cv_upper_bound", np.float64)
            if not np.all(hi > lo):
                raise ValueError("cv_upper_bound must exceed cv_lower_bound")
            mcmc["cv_dist"] = np.ones(n_cv, dtype=bool)
            mcmc["cv_range"] = (lo, hi)
        if proj.get("proj_mode", "cv") == "cv":
            if len(idx) != 2:
                raise ValueError("the 'cv' projection takes two CV indices")
            mcmc["pair"] = (idx[0], idx[1])
        elif proj["proj_mode"] == "path":
            nodes = np.asarray(proj.get("path_list", []), dtype=np.float32)
            if nodes.ndim != 2 or nodes.shape[1] != len(idx) or nodes.shape[0] < 2:
                raise ValueError("path_list must hold at least two nodes over the proj_cv_index CVs")
            lam = float(proj.get("path_lm", 1.0))
            if not lam > 0:
                raise ValueError("path_lm must be positive")
            # z_path spans [-ln(P) / lambda, max d]: d <= Cp pi^2 for wrapped
            # differences, d <= sum (hi - lo)^2 over the path's distance CVs
            z_lo = -math.log(nodes.shape[0]) / lam
            if cv_type == "dis":
                lo, hi = mcmc["cv_range"]
                z_hi = float(sum((hi[i] - lo[i]) ** 2 for i in idx))
            else:
                z_hi = len(idx) * math.pi ** 2
            mcmc["path"] = (nodes, idx, lam, z_lo, z_hi)
        else:
            raise ValueError(f"proj_mode {proj['proj_mode']!r}")
    return RidConfig(int(cfg.get("numb_walkers", 12)), int(cfg.get("numb_iters", 1)), tlo, thi, mode, n_cv,
                     periodic, weights, pairs, explore, label, select, train, mcmc)
