"""Distance CVs as a system CV type (Sec. "CV selection": torsion and distance
CVs), on the GPU against the FP64 oracle: a system mixing torsions and
distances (rows (a, b, -1, -1) of cv_atoms) for the ensemble bias (FP32, BF16
and FP8 ensembles, every cluster size of the tensor-core kernel), the
restraint, 20-step trajectories, labels, and the batched / served label
kernels bit-equal to rid_label.

Tolerances are those of the torsion-only tests: forces and member gradients
1e-5 relative (FP32), 3e-2 / 6e-2 normwise (BF16 / FP8), trajectories 1e-4,
labels within 2 combined standard errors.
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORCE_RTOL = 1e-5


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def close_rel(got, ref):
    ref = np.asarray(ref, np.float64)
    return (np.abs(np.asarray(got, np.float64) - ref) / (np.abs(ref) + np.sqrt(np.mean(ref ** 2)))).max()


def normwise(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


def mixed(n=60, C=8, n_dist=3, W=24, seed=71, **kw):
    sp = I.make_system(n, C, seed, n_dist=n_dist, **kw)
    x = I.make_chains(W, sp, seed)
    return sp, x


def centres(orc, sp, x, seed):
    """Restraint centres: torsions uniform on the torus, distances 0.3 around
    the start's distances."""
    rng = np.random.default_rng(seed)
    s0 = I.make_label_targets(x.shape[0], sp.n_cv, seed)
    dist = I.cv_is_distance(sp)
    for w in range(x.shape[0]):
        s = orc.cvs(sp, x[w].astype(np.float64))[0]
        s0[w, dist] = s[dist] + rng.uniform(-0.3, 0.3, size=dist.sum())
    return s0


def test_mixed_cvs_values_forces_and_member_gradients(R, orc):
    sp, x = mixed()
    W, n, C = x.shape[0], sp.n_beads, sp.n_cv
    ens = I.make_ensemble(4, 2 * C, 3, 64, 71)
    eps_all = np.array([orc.ensemble(ens, orc.cvs(sp, xi.astype(np.float64))[0], sp.cv_atoms)["eps"] for xi in x])
    ens.trust_lo, ens.trust_hi = float(np.percentile(eps_all, 25)), float(np.percentile(eps_all, 75))
    f = np.zeros((W, n, 3), np.float32)
    s = np.zeros((W, C), np.float32)
    eps = np.zeros(W, np.float32)
    g = np.zeros((4, W, C), np.float32)
    fr = np.zeros_like(f)
    s0 = centres(orc, sp, x, 71)
    kap = np.random.default_rng(1).uniform(50, 500, size=(W, C))
    with R.System(sp) as sysm:
        sysm.set_ensemble(ens)
        sysm.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=f, s_out=s, eps_out=eps, grad_out=g)
        sysm.eval_forces(x, R.RID_BIAS_RESTRAINT, s0=s0, kappa=kap, f_out=fr)
    dist = I.cv_is_distance(sp)
    for w in range(W):
        xd = x[w].astype(np.float64)
        r = orc.total(sp, xd, ens=ens, mode=1)
        e = orc.ensemble(ens, r["s"], sp.cv_atoms)
        assert np.all(np.abs(s[w, dist] - r["s"][dist]) <= FORCE_RTOL * r["s"][dist])
        assert close_rel(g[:, w], e["gradA"]) < FORCE_RTOL, w
        assert abs(eps[w] - e["eps"]) <= FORCE_RTOL * (abs(e["eps"]) + 1e-3)
        slope = np.pi / 2 / (ens.trust_hi - ens.trust_lo)
        assert close_rel(f[w], r["f"]) < FORCE_RTOL + slope * abs(eps[w] - e["eps"]), w
        rr = orc.total(sp, xd, mode=2, s0=s0[w], kappa=kap[w])
        assert close_rel(fr[w], rr["f"]) < FORCE_RTOL, w


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_mixed_cvs_on_the_tensor_cores_every_cluster_size(R, orc, prec):
    sp, x = mixed(n=120, C=18, n_dist=6, W=200, seed=72)
    ens = I.make_ensemble(4, 36, 4, 128, 72, resnet=True, trust_lo=1e9, trust_hi=2e9)
    p = R.RID_PREC_BF16 if prec == "bf16" else R.RID_PREC_FP8
    outs = []
    for cs in (1, 2, 4):
        g = np.zeros((4, 200, 18), np.float32)
        with R.System(sp) as sysm:
            sysm.set_ensemble(ens, precision=p)
            sysm.set_mlp_cluster(cs)
            sysm.eval_forces(x, R.RID_BIAS_ENSEMBLE, grad_out=g)
        outs.append(g)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    tol = 3e-2 if prec == "bf16" else 6e-2
    for w in (0, 77, 199):
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0], sp.cv_atoms)
        assert normwise(outs[0][:, w].mean(axis=0), e["gradA"].mean(axis=0)) < tol, w


def test_mixed_cvs_twenty_step_trajectories(R, orc):
    sp, x0 = mixed(n=45, C=6, n_dist=2, W=16, seed=73, output_freq=1)
    ens = I.make_ensemble(4, 12, 3, 64, 73)
    eps_all = np.array([orc.ensemble(ens, orc.cvs(sp, xi.astype(np.float64))[0], sp.cv_atoms)["eps"] for xi in x0])
    ens.trust_lo, ens.trust_hi = float(np.percentile(eps_all, 25)), float(np.percentile(eps_all, 75))
    steps = 20
    cv = np.zeros((16, steps, 6), np.float32)
    eps = np.zeros((16, steps), np.float32)
    xo, vo = np.zeros_like(x0), np.zeros_like(x0)
    with R.System(sp) as sysm:
        sysm.set_ensemble(ens)
        sysm.explore(x0, steps, cv_out=cv, eps_out=eps, x_out=xo, v_out=vo)
    ref = orc.explore(sp, x0, steps, ens=ens)
    tol = 1e-4
    assert np.all(np.abs(xo - ref["x"]) <= tol * (np.abs(ref["x"]) + 1))
    assert np.all(np.abs(vo - ref["v"]) <= tol * (np.abs(ref["v"]) + 1))
    d = cv - ref["cv"]
    d[..., :4] -= 2 * np.pi * np.floor(d[..., :4] / (2 * np.pi) + 0.5)
    assert np.all(np.abs(d) <= tol * (np.abs(ref["cv"]) + 1))
    assert np.all(np.abs(eps - ref["eps"]) <= tol * (np.abs(ref["eps"]) + 1))


def test_mixed_cvs_labels_within_two_standard_errors(R, orc):
    sp, x0 = mixed(n=22, C=4, n_dist=2, W=16, seed=74, dist_span=4)
    s0 = centres(orc, sp, x0, 74)
    kap = np.full((16, 4), 50.0)
    n_steps, n_equil, B = 4000, 400, 20
    mf, se, sd = (np.zeros((16, 4)) for _ in range(3))
    with R.System(sp) as sysm:
        sysm.label(x0, s0, kap, n_steps, n_equil, B, mf, se, sd)
    ref = orc.label(sp, x0, s0, kap, n_steps, n_equil, B)
    z = (mf - ref["mf"]) / np.sqrt(se ** 2 + ref["se"] ** 2)
    assert np.mean(np.abs(z) <= 2) >= 0.9 and np.all(np.abs(z) < 4), z
    # the spread of kappa d: per CV the median ratio over the runs near 1, no run off by 2x
    ratio = sd / ref["std"]
    assert np.all(np.abs(np.median(ratio, axis=0) - 1) < 0.2), ratio
    assert np.all((ratio > 0.5) & (ratio < 2.0)), ratio


def test_mixed_cvs_label_statistics_exact_on_first_steps(R, orc):
    sp, x0 = mixed(n=30, C=5, n_dist=2, W=6, seed=75)
    s0 = centres(orc, sp, x0, 75)
    kap = np.full((6, 5), 200.0)
    mf, se, sd = (np.zeros((6, 5)) for _ in range(3))
    with R.System(sp) as sysm:
        sysm.label(x0, s0, kap, 23, 0, 7, mf, se, sd)
    ref = orc.label(sp, x0, s0, kap, 23, 0, 7)
    assert np.allclose(mf, ref["mf"], rtol=1e-4, atol=1e-3)
    assert np.allclose(sd, ref["std"], rtol=1e-2, atol=1e-3)


def test_mixed_cvs_batched_and_served_labels_bit_equal_to_rid_label(R, orc):
    jobs = []
    for n, C, nd, runs, steps, seed, mb in [(22, 3, 1, 3, 300, 76, True), (61, 9, 4, 2, 240, 77, False),
                                             (130, 20, 10, 1, 200, 78, True)]:
        sp = I.make_system(n, C, seed, n_dist=nd)
        x0 = I.make_chains(runs, sp, seed)
        rng = np.random.default_rng(seed)
        v0 = None if mb else (0.3 * rng.standard_normal(x0.shape)).astype(np.float32)
        jobs.append(dict(system=R.System(sp), x0=x0, v0=v0, s0=centres(orc, sp, x0, seed),
                         kappa=rng.uniform(50, 150, size=(runs, C)), step0=0, n_steps=steps,
                         n_equil=steps // 10, n_blocks=5))

    def outs(j):
        runs, C = j["s0"].shape
        return dict(mf=np.zeros((runs, C)), se=np.zeros((runs, C)), std=np.zeros((runs, C)),
                    x_out=np.zeros_like(j["x0"]), v_out=np.zeros_like(j["x0"]))

    ref = []
    for j in jobs:
        o = outs(j)
        j["system"].label(j["x0"], j["s0"], j["kappa"], j["n_steps"], j["n_equil"], j["n_blocks"], o["mf"], o["se"],
                          o["std"], v0=j["v0"], x_out=o["x_out"], v_out=o["v_out"])
        ref.append(o)
    batch = [dict(j, **outs(j)) for j in jobs]
    served = [outs(j) for j in jobs]
    with R.Server(256 << 20) as srv:
        srv.label_batch(batch)
        ids = [srv.submit_label(j["system"], j["x0"], j["s0"], j["kappa"], j["n_steps"], j["n_equil"],
                                j["n_blocks"], o["mf"], o["se"], o["std"], v0=j["v0"], x_out=o["x_out"],
                                v_out=o["v_out"]) for j, o in zip(jobs, served)]
        res = srv.wait(ids)
        assert all(res[i][0] == R.RID_OK for i in ids)
    for r, b, s in zip(ref, batch, served):
        for k in ("mf", "se", "std", "x_out", "v_out"):
            assert np.array_equal(b[k], r[k]), k
            assert np.array_equal(s[k], r[k]), k
    for j in jobs:
        j["system"].close()


def test_distance_cv_argument_errors(R):
    sp = I.make_system(20, 3, 79, n_dist=1)
    sp.cv_atoms[2] = [5, 5, -1, -1]                 # a distance of a bead to itself
    with pytest.raises(R.RidError) as e:
        R.System(sp)
    assert e.value.code == R.RID_ERR_ARG
    sp.cv_atoms[2] = [5, 25, -1, -1]                # a bead past the chain
    with pytest.raises(R.RidError) as e:
        R.System(sp)
    assert e.value.code == R.RID_ERR_ARG
    sp.cv_atoms[2] = [5, 9, -1, 3]                  # half a distance
    with pytest.raises(R.RidError) as e:
        R.System(sp)
    assert e.value.code == R.RID_ERR_ARG
