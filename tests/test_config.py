"""The RiD-style JSON configuration loader (paper_2408_14070_gb300.config):
key names of the paper's workflow sections mapped onto this library's
arguments, the CV counts the paper states (2 n - 2 torsions for n residues,
one distance per atom pair), unit handling, the path projection's z range,
errors, and that every mapped dict binds to the binding's signatures.  CPU
only; the values below are this test's own."""
import inspect
import json
import math

import numpy as np
import pytest

from paper_2408_14070_gb300 import config as K
from paper_2408_14070_gb300 import rid

TORSION = {
    "numb_walkers": 8, "numb_iters": 5, "trust_lvl_1": 1.5, "trust_lvl_2": 4.0,
    "CV": {"mode": "torsion", "selected_resid": [1, 2, 3, 4], "angular_mask": [1, 1, 1, 1, 1, 1],
           "weights": [1, 2, 1, 2, 1, 2], "cv_file": [""]},
    "ExploreMDConfig": {"nsteps": 4000, "dt": 0.002, "temperature": 310, "output_freq": 20, "ntmpi": 1},
    "LabelMDConfig": {"method": "restrained", "nsteps": 6000, "kappas": [300, 300, 300, 400, 400, 400],
                      "std_threshold": 2.5, "output_freq": 10},
    "SelectorConfig": {"cluster_threshold": 1.7, "numb_cluster_lower": 6, "numb_cluster_upper": 9,
                       "max_selection": 7, "numb_cluster_threshold": 3},
    "Train": {"numb_models": 3, "neurons": [64, 64, 64], "resnet": True, "batch_size": 32, "epochs": 10,
              "init_lr": 1e-3, "decay_steps": 50, "decay_rate": 0.9, "drop_out_rate": 0.2, "numb_threads": 4},
    "MCMC_Config": {"cv_dimension": 6, "numb_steps": 300, "numb_walkers": 64, "temperature": 310,
                    "proj_info": {"proj_mode": "cv", "proj_cv_index": [2, 5]}, "cv_type": "dih", "bins": 31},
}


def test_torsion_configuration_maps_onto_the_calls():
    c = K.load(TORSION)
    assert (c.n_walkers, c.n_iters, c.trust_lo, c.trust_hi) == (8, 5, 1.5, 4.0)
    assert c.cv_mode == "torsion" and c.n_cv == 6 and c.distance_pairs is None     # 2 x 4 - 2 torsions
    assert np.array_equal(c.periodic, np.ones(6)) and np.array_equal(c.cv_weights, [1, 2, 1, 2, 1, 2])
    kT = K.KB_KJ_PER_MOL_K * 310
    assert c.explore == {"n_steps": 4000, "dt": 0.002, "kT": pytest.approx(kT), "output_freq": 20}
    assert c.label["method"] == "restrained" and c.label["n_steps"] == 6000 and c.label["dt"] == 0.002
    assert np.array_equal(c.label["kappa"], [300, 300, 300, 400, 400, 400]) and c.label["std_threshold"] == 2.5
    s = c.select
    assert (s["threshold"], s["lower"], s["upper"], s["max_selection"], s["adapt"]) == (1.7, 6, 9, 7, True)
    assert (s["trust_lo"], s["trust_hi"]) == (1.5, 4.0)
    t = c.train
    assert (t["n_models"], t["n_layers"], t["width"], t["resnet"], t["batch_size"]) == (3, 3, 64, True, 32)
    assert (t["init_lr"], t["decay_steps"], t["decay_rate"], t["dropout_rate"]) == (1e-3, 50, 0.9, 0.2)
    assert c.train_steps(100) == math.ceil(10 * 100 / 32)
    m = c.mcmc
    assert (m["n_walkers"], m["n_steps"], m["bins"], m["pair"], m["path"]) == (64, 300, 31, (2, 5), None)
    assert m["kT"] == pytest.approx(kT)


def test_json_text_and_reduced_units():
    c = K.load(json.dumps(TORSION), reduced=True)
    assert c.explore["kT"] == 1.0 and c.label["kT"] == 1.0 and c.mcmc["kT"] == 1.0
    assert c.trust_lo == 1.5        # energies are kept as given


def test_distance_cvs_and_constrained_labels():
    cfg = {"CV": {"mode": "distance", "selected_atomid": [[2, 5], [5, 7], [9, 12]], "angular_mask": [0, 0, 0]},
           "LabelMDConfig": {"method": "constrained", "nsteps": 1000}, "Train": {"neurons": [32, 32]}}
    c = K.load(cfg, reduced=True)
    assert c.cv_mode == "distance" and c.n_cv == 3
    assert np.array_equal(c.distance_pairs, [[1, 4], [4, 6], [8, 11]])       # 0-based
    assert np.array_equal(c.periodic, [0, 0, 0])
    assert c.label["method"] == "constrained" and "kappa" not in c.label
    assert c.mcmc == {}


def test_path_projection_and_its_z_range():
    from oracle import mcmc as MC
    cfg = dict(TORSION)
    nodes = [[-2.0, 1.0], [-1.0, 0.5], [0.0, 0.0], [1.0, -0.5], [2.0, -1.0]]
    cfg["MCMC_Config"] = dict(TORSION["MCMC_Config"],
                              proj_info={"proj_mode": "path", "proj_cv_index": [0, 3], "path_list": nodes,
                                         "path_lm": 1.5})
    c = K.load(cfg)
    nd, cvs, lam, z_lo, z_hi = c.mcmc["path"]
    assert np.array_equal(nd, np.asarray(nodes, np.float32)) and cvs == [0, 3] and lam == 1.5
    # every state's z_path lies inside the range (so the histogram never clamps)
    s = np.random.default_rng(1).uniform(-math.pi, math.pi, size=(20000, 6))
    sp, z = MC.path_cv(s, nd, cvs, lam)
    assert z.min() >= z_lo and z.max() <= z_hi
    # the bounds are reached: z -> -ln(P) / lambda for P coincident nodes, and
    # z -> max d = Cp pi^2 far from a single node
    one = np.zeros((3, 2))
    _, z1 = MC.path_cv(np.zeros((1, 6)), one, [0, 3], lam)
    assert z1[0] == pytest.approx(-math.log(3) / lam)
    _, z2 = MC.path_cv(np.full((1, 6), math.pi), np.zeros((1, 2)), [0, 3], lam)
    assert z2[0] == pytest.approx(2 * math.pi ** 2)


@pytest.mark.parametrize("patch,msg", [
    ({"CV": {"mode": "custom", "selected_atomid": [[1, 2]]}}, "only"),
    ({"CV": {"mode": "torsion", "selected_resid": [3]}}, "two selected residues"),
    ({"CV": {"mode": "distance", "selected_atomid": [[0, 2]]}}, "1-based"),
    ({"CV": {"mode": "torsion", "selected_resid": [1, 2, 3], "angular_mask": [1, 1, 1]}}, "angular_mask"),
    ({"LabelMDConfig": {"method": "restrained", "kappas": [1, 2, 3]}}, "kappas"),
    ({"LabelMDConfig": {"method": "constrained"}}, "distance CVs"),
    ({"Train": {"neurons": [64, 32]}}, "one width"),
    ({"trust_lvl_1": 3, "trust_lvl_2": 3}, "trust_lvl_2"),
    ({"MCMC_Config": {"cv_type": "dis"}}, "does not match"),
    ({"MCMC_Config": {"cv_type": "xyz"}}, "'dih'"),
    ({"MCMC_Config": {"proj_info": {"proj_mode": "cv", "proj_cv_index": [0, 9]}}}, "outside"),
])
def test_errors(patch, msg):
    cfg = {**TORSION, **patch}
    with pytest.raises(ValueError, match=msg):
        K.load(cfg)


def test_mapped_arguments_bind_to_the_binding():
    c = K.load(TORSION)
    s = c.select
    inspect.signature(rid.select).bind(np.zeros((1, c.n_cv), np.float32), np.zeros(1, np.float32), s["trust_lo"],
                                       s["trust_hi"], s["threshold"], s["lower"], s["upper"], s["adapt"],
                                       s["max_selection"], weights=s["weights"], periodic=s["periodic"])
    t = c.train
    inspect.signature(rid.Trainer.__init__).bind(None, t["n_models"], c.n_cv, t["n_layers"], t["width"], None,
                                                  batch_size=t["batch_size"], resnet=t["resnet"],
                                                  init_lr=t["init_lr"], decay_rate=t["decay_rate"],
                                                  decay_steps=t["decay_steps"], dropout_rate=t["dropout_rate"])
    m = c.mcmc
    inspect.signature(rid.System.mcmc).bind(None, None, m["n_steps"], 0, m["kT"], 0.3, 1, bins=m["bins"],
                                            pair=m["pair"], path=m["path"])


def test_distance_mcmc_ranges_and_cv_rows():
    """cv_type "dis" with the paper's cv_lower_bound / cv_upper_bound: the
    walk's ranges, the path's z range from them, and the system's CV rows."""
    cfg = {"CV": {"mode": "distance", "selected_atomid": [[2, 5], [5, 7], [9, 12]], "angular_mask": [0, 0, 0]},
           "LabelMDConfig": {"method": "restrained", "kappas": [500, 500, 500]},
           "MCMC_Config": {"numb_walkers": 64, "numb_steps": 100, "temperature": 300, "bins": 41,
                           "cv_type": "dis", "cv_lower_bound": [1.0, 2.0, 0.5], "cv_upper_bound": [4.5, 5.0, 3.5],
                           "proj_info": {"proj_mode": "path", "proj_cv_index": [0, 2],
                                         "path_list": [[1.5, 1.0], [3.0, 2.0], [4.0, 3.0]], "path_lm": 2.0}}}
    c = K.load(cfg, reduced=True)
    assert np.array_equal(c.mcmc["cv_dist"], [True, True, True])
    lo, hi = c.mcmc["cv_range"]
    assert np.array_equal(lo, [1.0, 2.0, 0.5]) and np.array_equal(hi, [4.5, 5.0, 3.5])
    nodes, idx, lam, z_lo, z_hi = c.mcmc["path"]
    assert z_lo == pytest.approx(-np.log(3) / 2.0) and z_hi == pytest.approx(3.5 ** 2 + 3.0 ** 2)
    assert np.array_equal(K.cv_atoms(c), [[1, 4, -1, -1], [4, 6, -1, -1], [8, 11, -1, -1]])
    bad = dict(cfg["MCMC_Config"])
    del bad["cv_lower_bound"]
    with pytest.raises(ValueError, match="cv_lower_bound"):
        K.load(dict(cfg, MCMC_Config=bad), reduced=True)
    bad = dict(cfg["MCMC_Config"], cv_upper_bound=[1.0, 2.0, 0.5])
    with pytest.raises(ValueError, match="exceed"):
        K.load(dict(cfg, MCMC_Config=bad), reduced=True)
