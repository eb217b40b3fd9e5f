"""Constrained-MD labels on distance CVs (rid_label_constrained) against the
exact free-energy derivative of a bonded chain and against the FP64 oracle.

Tolerances: a 20-step trajectory from the same state and noise stays within
1e-4 of the oracle's (FP32 against FP64, the bound of the unconstrained
step); constraints hold to FP32 rounding of the distance (1e-5 relative);
mean forces are statistical estimates and are compared within combined
standard errors (at least 90% of the entries within 2, none beyond 4, the
rule of the restrained labels), the exact derivative within 3.5.
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KB, R0, KT = 20.0, 1.0, 1.0


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def _exact_mean_force(d0):
    # the end-to-middle distance of three bonded beads: see tests/test_oracle_constrained.py
    r = np.linspace(0.05, 3.0, 200001)
    dr = r[1] - r[0]
    g = r ** 2 * np.exp(-KB * (r - R0) ** 2 / (2 * KT))
    g /= np.trapezoid(g, r)
    h = g / r
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (h[1:] + h[:-1]) * dr)])

    def P(Rr):
        inner = np.interp(Rr + r, r, cum) - np.interp(np.abs(Rr - r), r, cum)
        return 0.5 * Rr * np.trapezoid(h * inner, r)

    e = 1e-3
    return -KT * (np.log(P(d0 + e)) - np.log(P(d0 - e))) / (2 * e)


def _bonded_chain(runs):
    sp = I.make_system(4, 1, 3, lj_eps=0.0, angle_k=0.0, bond_k=KB, bond_r0=R0, kT=KT)
    sp.dihedral_k[:] = 0.0
    x0 = np.zeros((runs, 4, 3), np.float32)
    x0[:, :, 0] = np.arange(4)
    x0[:, 2, 1] = 0.5
    return sp, x0


@pytest.mark.parametrize("d0", [1.2, 1.5, 1.8])
def test_mean_force_matches_the_exact_marginal(R, d0):
    runs = 64
    sp, x0 = _bonded_chain(runs)
    mf, se, sd = (np.zeros((runs, 1)) for _ in range(3))
    xo = np.zeros_like(x0)
    with R.System(sp) as s:
        s.label_constrained(x0, [[0, 2]], np.full((runs, 1), d0), 60000, 5000, 20, mf, se, sd, x_out=xo)
    m, e = mf.mean(), np.sqrt((se ** 2).sum()) / runs
    exact = _exact_mean_force(d0)
    print(f"\nd0 {d0}: GPU {m:.4f} +- {e:.4f}, exact {exact:.4f}")
    assert abs(m - exact) < 3.5 * e
    r = np.linalg.norm(xo[:, 0] - xo[:, 2], axis=-1)
    assert np.max(np.abs(r - d0)) < 1e-5 * d0


def _chain_problem(runs, seed=5):
    sp = I.make_system(60, 4, seed)
    x0 = I.make_chains(runs, sp, seed)
    pairs = np.array([[3, 9], [15, 27], [30, 34], [40, 55]], np.int32)
    cur = np.linalg.norm(x0[:, pairs[:, 0]] - x0[:, pairs[:, 1]], axis=-1)
    d0 = np.ascontiguousarray(cur * np.random.default_rng(seed).uniform(0.95, 1.05, size=cur.shape), dtype=np.float64)
    return sp, x0, pairs, d0


def test_short_trajectory_follows_the_oracle(R, orc):
    runs = 4
    sp, x0, pairs, d0 = _chain_problem(runs)
    v0 = (0.5 * np.random.default_rng(1).standard_normal(x0.shape)).astype(np.float32)
    mf, se, sd = (np.zeros((runs, 4)) for _ in range(3))
    xo, vo = np.zeros_like(x0), np.zeros_like(x0)
    with R.System(sp) as s:
        s.label_constrained(x0, pairs, d0, 20, 0, 2, mf, se, sd, v0=v0, x_out=xo, v_out=vo)
    ref = orc.label_constrained(sp, x0, pairs, d0, 20, 0, 2, v0=v0)
    assert np.max(np.abs(xo - ref["x"])) < 1e-4
    assert np.max(np.abs(vo - ref["v"])) < 1e-3
    np.testing.assert_allclose(mf, ref["mf"], rtol=1e-3, atol=1e-3)
    r = np.linalg.norm(xo[:, pairs[:, 0]] - xo[:, pairs[:, 1]], axis=-1)
    assert np.max(np.abs(r - d0) / d0) < 1e-5


def test_labels_within_standard_errors_of_the_oracle(R, orc):
    runs = 6
    sp, x0, pairs, d0 = _chain_problem(runs, seed=7)
    mf, se, sd = (np.zeros((runs, 4)) for _ in range(3))
    with R.System(sp) as s:
        s.label_constrained(x0, pairs, d0, 4000, 400, 10, mf, se, sd)
    ref = orc.label_constrained(sp, x0, pairs, d0, 4000, 400, 10)
    z = np.abs(mf - ref["mf"]) / np.sqrt(se ** 2 + ref["se"] ** 2)
    print(f"\nz: mean {z.mean():.2f}, max {z.max():.2f}")
    assert np.mean(z < 2.0) >= 0.9 and z.max() < 4.0, z


def test_device_arguments_match_host_arguments(R):
    import torch
    runs = 3
    sp, x0, pairs, d0 = _chain_problem(runs, seed=9)
    out_h = [np.zeros((runs, 4)) for _ in range(3)]
    with R.System(sp) as s:
        s.label_constrained(x0, pairs, d0, 300, 30, 5, *out_h)
        out_d = [torch.zeros((runs, 4), dtype=torch.float64, device="cuda") for _ in range(3)]
        s.label_constrained(torch.from_numpy(x0).cuda(), pairs, torch.from_numpy(d0).cuda(), 300, 30, 5, *out_d)
    for a, b in zip(out_h, out_d):
        assert np.array_equal(a, b.cpu().numpy())


def test_errors(R):
    sp, x0, pairs, d0 = _chain_problem(1, seed=11)
    z = [np.zeros((1, 2)) for _ in range(3)]
    with R.System(sp) as s:
        for bad in ([[3, 9], [9, 20]], [[4, 4], [5, 6]], [[3, 70], [5, 6]]):
            with pytest.raises(R.RidError) as e:
                s.label_constrained(x0, bad, np.ones((1, 2)), 100, 10, 5, *z)
            assert e.value.code == R.RID_ERR_ARG
        with pytest.raises(R.RidError) as e:
            s.label_constrained(x0, [[3, 9], [12, 20]], np.array([[1.0, -1.0]]), 100, 10, 5, *z)
        assert e.value.code == R.RID_ERR_ARG
