"""Change control of the FP64 oracle: its outputs on the small seeded cases
stored in tests/golden/oracle_small.json (inputs included, so the input
generators do not enter) are reproduced.  Forces, CVs, the ensemble, biased
and restrained forces, a 20-step biased trajectory with energies, restrained
labels, three training steps with dropout, a selection with threshold
adaptation and an MCMC run, at non-unit physics with a torsion + distance CV
set.  Integer results (Philox words, selected frames, histograms) are exact;
floating-point ones within a few ulps of accumulated rounding, which allows a
different libm but no change of arithmetic.  CPU only."""
import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import oracle_cases as G  # noqa: E402


@pytest.fixture(scope="module")
def stored():
    import oracle
    oracle.build()
    doc = json.load(open(os.path.join(HERE, "golden", "oracle_small.json")))
    inp, want = G.decode(doc["inputs"]), G.decode(doc["outputs"])
    return want, G.run(inp)


def _compare(path, want, got):
    if isinstance(want, dict):
        assert set(want) == set(got), path
        for k in want:
            _compare(f"{path}.{k}", want[k], got[k])
        return
    w, g = np.asarray(want), np.asarray(got)
    assert w.shape == g.shape, path
    if w.dtype.kind in "iub" or g.dtype.kind in "iub":
        assert np.array_equal(w, g), path
    elif g.dtype == np.float32:
        np.testing.assert_allclose(g, w, rtol=2e-6, atol=1e-6, err_msg=path)
    else:
        np.testing.assert_allclose(g, w, rtol=1e-9, atol=1e-11, err_msg=path)


@pytest.mark.parametrize("part", ["philox", "walker0", "walker1", "explore", "label", "train", "select", "mcmc"])
def test_oracle_reproduces_its_stored_outputs(stored, part):
    want, got = stored
    _compare(part, want[part], got[part])


def test_the_cases_reach_every_branch_they_are_for(stored):
    want, _ = stored
    # the switch strictly between its limits, so sigma and its scaling enter
    for w in ("walker0", "walker1"):
        assert 0.0 < want[w]["sigma"] < 1.0
    # the selection adapted its threshold into [lower, upper]
    assert 6 <= want["select"]["n_clusters"] <= 9
    # the MCMC run accepted and refused moves
    assert 0 < want["mcmc"]["n_accepted"] < 8 * 60


def test_a_changed_parameter_fails_the_comparison(stored):
    """Planted on the CPU: the friction off by one part in 10^6 changes the
    trajectory, one ensemble weight off by 10^-6 the member gradients."""
    want, _ = stored
    doc = json.load(open(os.path.join(HERE, "golden", "oracle_small.json")))
    inp = G.decode(doc["inputs"])
    inp["system"]["gamma"] *= 1.0 + 1e-6
    inp["ensemble"]["weights"] = inp["ensemble"]["weights"].copy()
    inp["ensemble"]["weights"][1, 2] += np.float32(1e-6)   # W_1[0][2], on cos s_1
    got = G.run(inp)
    with pytest.raises(AssertionError):
        _compare("explore", want["explore"], got["explore"])
    with pytest.raises(AssertionError):
        _compare("walker0", want["walker0"], got["walker0"])
    _compare("philox", want["philox"], got["philox"])
