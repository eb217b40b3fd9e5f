"""Two iterations of the RiD cycle through workflow.run from a RiD-style
configuration: the first iteration explores without a model (none given) and
takes every frame as a candidate, the labels it keeps train the ensemble, and the second
explores with the trained ensemble.  Checked against each phase's
definition: frame counts, selections within max_selection, labels kept by
the std threshold, the training loss falling, and the trained weights
differing from the initial ones."""
import numpy as np
import pytest

from paper_2408_14070_gb300 import config as K
from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CFG = {
    "numb_walkers": 16, "numb_iters": 2, "trust_lvl_1": 0.0, "trust_lvl_2": 1e9,
    "CV": {"mode": "torsion", "selected_resid": [1, 2], "angular_mask": [1, 1], "weights": [1, 1]},
    "ExploreMDConfig": {"nsteps": 400, "output_freq": 50},
    "LabelMDConfig": {"method": "restrained", "nsteps": 1000, "kappas": [100, 100], "std_threshold": 1e9},
    "SelectorConfig": {"cluster_threshold": 0.5, "numb_cluster_lower": 4, "numb_cluster_upper": 12,
                       "max_selection": 8},
    "Train": {"numb_models": 3, "neurons": [32, 32], "resnet": False, "batch_size": 16, "epochs": 200,
              "init_lr": 3e-3, "decay_steps": 100, "decay_rate": 0.96, "drop_out_rate": 0.0},
}


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def test_two_iterations_of_the_cycle(R):
    from paper_2408_14070_gb300 import workflow
    c = K.load(CFG, reduced=True)
    sp = I.make_system(22, c.n_cv, 3, output_freq=50)
    x0 = I.make_chains(16, sp, 3)
    w0 = I.make_ensemble(3, 4, 2, 32, 1).weights        # the seeded start run() draws with seed = 1
    res = workflow.run(c, sp, x0, seed=1)
    it0, it1 = res.iterations
    assert it0["frames"] == it1["frames"] == 16 * 8            # one frame per 50-step chunk and walker
    assert it0["eps_mean"] == 0.0 and it1["eps_mean"] > 0.0    # no model first, the trained ensemble next
    assert 1 <= it0["selected"] <= 8 and it0["labels_kept"] == it0["selected"]
    assert it1["labels_total"] == it0["labels_kept"] + it1["labels_kept"] == res.s.shape[0]
    assert res.mf.shape == res.s.shape and np.all(np.isfinite(res.mf)) and np.all(res.se > 0)
    assert it0["loss_last"] < 0.5 * it0["loss_first"]
    assert not np.array_equal(res.weights, w0) and np.all(np.isfinite(res.weights))
    assert np.all(np.isfinite(res.x))


def test_a_given_ensemble_biases_the_first_iteration(R):
    """Restarting from a trained ensemble: the first iteration explores with
    its bias and trust window instead of unbiased."""
    from paper_2408_14070_gb300 import workflow
    c = K.load(CFG, reduced=True)
    sp = I.make_system(22, c.n_cv, 3, output_freq=50)
    x0 = I.make_chains(16, sp, 3)
    w0 = I.make_ensemble(3, 4, 2, 32, 5).weights
    res = workflow.run(c, sp, x0, weights=w0, n_iters=1, seed=2)
    assert res.iterations[0]["eps_mean"] > 0.0
