"""Selection (rid_select) against the selection oracle.  Every output is an
integer or the threshold search's float64 sequence, and the oracle takes the
kernel's FP32 distance and window decisions, so the results must be equal
exactly: selected frame indices, cluster count and the threshold used.
"""
import math

import numpy as np
import pytest

from oracle import select as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def _frames(n, C, seed, walkers=8):
    # CV traces of a few walkers (random walks on the torus), eps in [0, 4)
    rng = np.random.default_rng(seed)
    steps = rng.normal(0.0, 0.15, size=(walkers, n // walkers, C))
    cv = np.cumsum(steps, axis=1) + rng.uniform(-math.pi, math.pi, size=(walkers, 1, C))
    cv = (cv + math.pi) % (2 * math.pi) - math.pi
    cv = cv.reshape(-1, C)
    eps = rng.uniform(0.0, 4.0, size=cv.shape[0])
    return cv.astype(np.float32), eps.astype(np.float32)


@pytest.mark.parametrize("n,C,thr,lower,upper,adapt,maxsel", [
    (8000, 20, 2.6, 30, 45, True, 50),      # the paper's selection config on 20 torsions
    (6000, 4, 0.3, 1, 1 << 30, False, 100000),   # hundreds of leaders, many per chunk
    (3000, 2, 5.0, 10, 12, True, 5),        # threshold search downwards, truncation
])
def test_selection_matches_the_oracle(R, n, C, thr, lower, upper, adapt, maxsel):
    cv, eps = _frames(n, C, n + C)
    sel, nc, t = R.select(cv, eps, 2.0, 3.0, thr, lower, upper, adapt, maxsel)
    ref = S.select(cv, eps, 2.0, 3.0, thr, lower, upper, adapt, maxsel)
    print(f"\n[{n}x{C}] clusters {nc} (oracle {ref['n_clusters']}), threshold {t:.4f}")
    assert nc == ref["n_clusters"]
    assert t == ref["threshold"]
    np.testing.assert_array_equal(sel, ref["selected"])
    if adapt and upper < (1 << 30):
        assert lower <= nc <= upper


def test_weights_and_angular_mask(R):
    cv, eps = _frames(4000, 5, 9)
    cv[:, 3] *= 0.4                            # a non-periodic CV in a bounded range
    w = [1.0, 0.5, 2.0, 1.0, 0.0]
    per = [1, 1, 1, 0, 1]
    sel, nc, t = R.select(cv, eps, 1.0, 3.5, 1.1, 1, 1 << 30, False, 1000, weights=w, periodic=per)
    ref = S.select(cv, eps, 1.0, 3.5, 1.1, 1, 1 << 30, False, 1000, w=w, periodic=per)
    assert nc == ref["n_clusters"]
    np.testing.assert_array_equal(sel, ref["selected"])


def test_edge_cases(R):
    cv, eps = _frames(500, 3, 4)
    sel, nc, _ = R.select(cv, eps, 10.0, 11.0, 1.0, 1, 5, True, 10)     # no candidate frames
    assert nc == 0 and sel.size == 0
    same = np.repeat(cv[:1], cv.shape[0], axis=0)
    sel, nc, _ = R.select(same, eps, 0.0, 5.0, 0.01, 1, 1 << 30, False, 10)
    assert nc == 1 and list(sel) == [0]
    sel, nc, _ = R.select(cv, eps, 0.0, 5.0, 0.5, 1, 1 << 30, False, 0)
    assert sel.size == 0 and nc > 0
    with pytest.raises(R.RidError) as e:
        R.select(cv, eps, 0.0, 5.0, -1.0)
    assert e.value.code == R.RID_ERR_ARG


def test_device_arguments_match_host_arguments(R):
    import torch
    cv, eps = _frames(5000, 6, 5)
    sel_h, nc_h, t_h = R.select(cv, eps, 2.0, 3.0, 1.5, 8, 12, True, 20)
    out = torch.zeros(20, dtype=torch.int32, device="cuda")
    sel_d, nc_d, t_d = R.select(torch.from_numpy(cv).cuda(), torch.from_numpy(eps).cuda(), 2.0, 3.0, 1.5, 8, 12,
                                True, 20, selected=out)
    assert nc_h == nc_d and t_h == t_d
    np.testing.assert_array_equal(sel_h, sel_d.cpu().numpy())
