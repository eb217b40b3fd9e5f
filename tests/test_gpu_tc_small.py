"""The small-batch tensor-core ensemble kernel (k_mlp_tc_small: up to 16
walkers, BF16, the GEMMs transposed so that the outputs fill the MMA's rows,
the 128-output tiles split over the CTAs of a cluster).

Against the FP64 oracle at the BF16 bounds of the other tensor-core tests
(mean CV gradient normwise 3e-2, member values and model deviation likewise),
on walker counts 1 to 16 (ragged and full), residual networks, the paper's
width 300 at its 12 walkers and width 512 (four M-tiles), 128 inputs;
determinism (repeated evaluations and trajectories are the same bits); the
same bits with the tiles split over 1, 2, 3 or 4 CTAs; and agreement with the
128-row kernel, which evaluates the same walkers inside a larger batch.
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GRAD_TOL = 3e-2


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def normwise(a, b):
    b = np.asarray(b, np.float64)
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


def evaluate(R, sp, ens, x):
    W, C, M = x.shape[0], sp.n_cv, ens.n_models
    f = np.zeros((W, sp.n_beads, 3), np.float32)
    eps = np.zeros(W, np.float32)
    abar = np.zeros(W, np.float32)
    g = np.zeros((M, W, C), np.float32)
    with R.System(sp) as sysobj:
        sysobj.set_ensemble(ens, precision=R.RID_PREC_BF16)
        sysobj.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=f, eps_out=eps, abar_out=abar, grad_out=g)
    return f, eps, abar, g


SMALL_CASES = [
    (30, 4, 1, 4, 3, 64, False, 1),       # one walker
    (200, 18, 12, 4, 4, 300, True, 2),    # the paper's network at its 12 walkers
    (60, 9, 16, 3, 2, 96, False, 3),      # 16 columns, full
    (60, 9, 7, 3, 3, 128, True, 4),       # ragged, residual
    (120, 20, 13, 4, 2, 512, False, 5),   # width 512: four M-tiles
    (80, 64, 16, 2, 2, 64, True, 6),      # 128 inputs
]


@pytest.mark.parametrize("n,C,W,M,L,H,resnet,seed", SMALL_CASES)
def test_small_batch_matches_the_oracle(R, orc, n, C, W, M, L, H, resnet, seed):
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, resnet=resnet, trust_lo=1e9, trust_hi=2e9)
    f, eps, abar, g = evaluate(R, sp, ens, x)
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(abar)) and np.all(np.isfinite(f))
    for w in sorted({0, W // 2, W - 1}):
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])
        assert normwise(g[:, w].mean(axis=0), e["gradA"].mean(axis=0)) < GRAD_TOL, w
        for m in range(M):
            assert normwise(g[m, w], e["gradA"][m]) < 2 * GRAD_TOL, (w, m)
        assert abs(abar[w] - e["Abar"]) <= GRAD_TOL * (abs(e["Abar"]) + 0.1), w
        assert abs(eps[w] - e["eps"]) <= 2 * GRAD_TOL * (abs(e["eps"]) + 0.05), w


def test_small_batch_is_deterministic(R):
    sp = I.make_system(200, 18, 7, output_freq=5)
    x = I.make_chains(12, sp, 7)
    ens = I.make_ensemble(4, 36, 4, 300, 7, resnet=True)
    a = evaluate(R, sp, ens, x)
    b = evaluate(R, sp, ens, x)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    runs = []
    for _ in range(2):
        xo = np.zeros_like(x)
        cv = np.zeros((12, 6, 18), np.float32)
        with R.System(sp) as sysobj:
            sysobj.set_ensemble(ens, precision=R.RID_PREC_BF16)
            sysobj.explore(x, 30, cv_out=cv, x_out=xo)
        runs.append((xo, cv))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


SPLIT_CASES = [
    (200, 18, 12, 4, 4, 300, True, 11),    # the paper's network: 3 tiles
    (60, 9, 16, 3, 3, 160, False, 12),     # 2 tiles, 16 walkers
    (120, 20, 5, 2, 2, 512, True, 13),     # 4 tiles, ragged walkers
    (80, 64, 1, 2, 3, 416, False, 14),     # 4 tiles (the last ragged), 128 inputs, one walker
]


@pytest.mark.parametrize("n,C,W,M,L,H,resnet,seed", SPLIT_CASES)
def test_tile_split_gives_identical_bits(R, orc, n, C, W, M, L, H, resnet, seed):
    """The 128-output tiles split over 1, 2, up to 4 CTAs of a cluster: every
    split accumulates each tile by the same MMAs and adds the member value in
    the same order, so forces, member gradients, values and a short
    trajectory are the same bits; the default splits one CTA per tile."""
    sp = I.make_system(n, C, seed)
    x = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, resnet=resnet, trust_lo=1e9, trust_hi=2e9)
    tiles = -(-max(H, -(-2 * C // 64) * 64) // 128)
    outs = {}
    for cs in (1, 2, 4, 0):
        f = np.zeros((W, n, 3), np.float32)
        eps = np.zeros(W, np.float32)
        abar = np.zeros(W, np.float32)
        g = np.zeros((M, W, C), np.float32)
        with R.System(sp) as sysobj:
            sysobj.set_ensemble(ens, precision=R.RID_PREC_BF16)
            sysobj.set_mlp_cluster(cs)
            sysobj.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=f, eps_out=eps, abar_out=abar, grad_out=g)
            assert sysobj.mlp_cluster() == (min(cs, tiles) if cs else tiles), cs
            xo = np.zeros_like(x)
            sysobj.explore(x, 8, x_out=xo)
        outs[cs] = (f, eps, abar, g, xo)
    for cs in (2, 4, 0):
        for a, b in zip(outs[cs], outs[1]):
            assert np.array_equal(a, b), cs
    f, eps, abar, g, _ = outs[0]
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(outs[0][4]))
    for w in sorted({0, W - 1}):
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])
        assert normwise(g[:, w].mean(axis=0), e["gradA"].mean(axis=0)) < GRAD_TOL, w
        assert abs(abar[w] - e["Abar"]) <= GRAD_TOL * (abs(e["Abar"]) + 0.1), w


@pytest.mark.parametrize("W", [1, 12, 16])
def test_small_batch_agrees_with_the_row_kernel(R, W):
    """The first W walkers alone (small-batch kernel) against the same walkers
    inside a batch of 200 (128-row tiles): the same BF16 network, rounded in a
    different MMA order, so within the BF16 bound, not bit for bit."""
    sp = I.make_system(150, 16, 8)
    x = I.make_chains(200, sp, 8)
    ens = I.make_ensemble(4, 32, 4, 256, 8, trust_lo=1e9, trust_hi=2e9)
    _, _, abar_s, g_s = evaluate(R, sp, ens, np.ascontiguousarray(x[:W]))
    _, _, abar_b, g_b = evaluate(R, sp, ens, x)
    for w in range(W):
        assert normwise(g_s[:, w], g_b[:, w]) < GRAD_TOL, w
    assert np.allclose(abar_s, abar_b[:W], rtol=GRAD_TOL, atol=GRAD_TOL * 0.1)
