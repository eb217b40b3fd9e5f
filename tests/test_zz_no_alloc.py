"""rid_ensemble_grad_noalloc (member gradients with static scratch, no device
allocation): checked against the FP64 oracle directly (member gradients and
member values at every point, 1e-5 relative, the FP32 parity tolerance of the
force tests) and against the FP32 ensemble path of rid_eval_forces, on two
calls in a row.
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2408_14070_gb300 import build, rid
    build.build()
    torch.cuda.init()
    return rid, torch


def reference(rid, sp, ens, x):
    """CVs and member gradients through the existing entry point."""
    W = x.shape[0]
    s = np.zeros((W, sp.n_cv), np.float32)
    g = np.zeros((ens.n_models, W, sp.n_cv), np.float32)
    abar = np.zeros(W, np.float32)
    with rid.System(sp) as sys:
        sys.set_ensemble(ens, precision=rid.RID_PREC_FP32)
        sys.eval_forces(x, rid.RID_BIAS_ENSEMBLE, s_out=s, grad_out=g, abar_out=abar)
    return s, g, abar


def normwise(a, b):
    return np.linalg.norm(a.astype(np.float64) - b) / max(np.linalg.norm(b.astype(np.float64)), 1e-30)


def run_noalloc(rid, torch, ens, s):
    dev = torch.device("cuda:0")
    P, C = s.shape
    sd = torch.from_numpy(s).to(dev)
    wd = torch.from_numpy(np.ascontiguousarray(ens.weights, np.float32)).to(dev)
    g = torch.full((ens.n_models, P, C), float("nan"), device=dev)
    v = torch.full((ens.n_models, P), float("nan"), device=dev)
    stream = torch.cuda.current_stream()
    rid.ensemble_grad_noalloc(sd, wd, ens.n_models, ens.n_layers, ens.width, g, v, resnet=ens.resnet,
                              stream=stream)
    torch.cuda.synchronize()
    return g.cpu().numpy(), v.cpu().numpy()


def check(ref_s, ref_g, ref_abar, g, v):
    M, P, _ = ref_g.shape
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(v))
    for p in range(P):
        for m in range(M):
            assert normwise(g[m, p], ref_g[m, p]) < TOL, (p, m)
    np.testing.assert_allclose(v.mean(axis=0), ref_abar, rtol=TOL, atol=TOL)


def check_oracle(orc, ens, s, g, v):
    """Every point against the FP64 oracle at the same (FP32) CV values:
    dA_i/ds normwise within 1e-5, A_i within 1e-5 (|A_i| + 1)."""
    sd = s.astype(np.float64)
    for p in range(s.shape[0]):
        e = orc.ensemble(ens, sd[p])
        u = np.stack([np.cos(sd[p]), np.sin(sd[p])], axis=1).ravel()
        for m in range(ens.n_models):
            assert normwise(g[m, p], e["gradA"][m]) < TOL, (p, m)
            A, _ = orc.mlp(ens, m, u)
            assert abs(v[m, p] - A) <= TOL * (abs(A) + 1.0), (p, m)


def test_two_calls_in_a_row_match_the_oracle_and_eval_forces(env, orc):
    rid, torch = env
    sp = I.make_system(200, 20, 11)
    ens = I.make_ensemble(4, 40, 4, 256, 11)
    xa = I.make_chains(300, sp, 11)          # ragged: 300 = 9 tiles of 32 + 12
    xb = I.make_chains(480, sp, 12)
    ra = reference(rid, sp, ens, xa)
    rb = reference(rid, sp, ens, xb)
    ga, va = run_noalloc(rid, torch, ens, ra[0])
    gb, vb = run_noalloc(rid, torch, ens, rb[0])
    check_oracle(orc, ens, ra[0], ga, va)
    check_oracle(orc, ens, rb[0], gb, vb)
    check(*ra, ga, va)
    check(*rb, gb, vb)
    # the scratch keeps the second call's contents: repeating the first call
    # must give the same answer bit for bit
    ga2, va2 = run_noalloc(rid, torch, ens, ra[0])
    assert np.array_equal(ga, ga2) and np.array_equal(va, va2)


def test_residual_net_and_narrow_shape(env, orc):
    rid, torch = env
    sp = I.make_system(60, 9, 13)
    ens = I.make_ensemble(3, 18, 3, 96, 13, resnet=True)
    x = I.make_chains(70, sp, 13)
    r = reference(rid, sp, ens, x)
    g, v = run_noalloc(rid, torch, ens, r[0])
    check_oracle(orc, ens, r[0], g, v)
    check(*r, g, v)


def test_rejects_requests_beyond_the_static_scratch(env):
    rid, torch = env
    ens = I.make_ensemble(4, 40, 4, 256, 11)
    P = 513                                  # 4 * 17 * 32 * 4 * 256 > 2^21 floats
    s = torch.zeros((P, 20), device="cuda:0")
    wd = torch.from_numpy(np.ascontiguousarray(ens.weights, np.float32)).to("cuda:0")
    g = torch.zeros((4, P, 20), device="cuda:0")
    with pytest.raises(rid.RidError) as e:
        rid.ensemble_grad_noalloc(s, wd, 4, 4, 256, g)
    assert e.value.code == rid.RID_ERR_ARG
    assert "scratch" in str(e.value)
    # 512 points fit exactly
    s2 = s[:512].contiguous()
    g2 = torch.zeros((4, 512, 20), device="cuda:0")
    rid.ensemble_grad_noalloc(s2, wd, 4, 4, 256, g2)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(g2).all())
