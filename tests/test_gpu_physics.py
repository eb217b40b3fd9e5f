"""GPU parity with every physical parameter off 1: bead mass, kT, time step,
friction and the LJ sigma and epsilon.

Sec. "Exploration phase" sets the temperature and the time step of the
walkers; the configuration loader turns 300 K into kT = R T = 2.49 kJ/mol.
Two parameter sets run: the first has kT/m close to 1 (m = 2.5), the second
puts kT/m far from 1 (m = 3, kT = 0.6), so that kT/m written where sqrt(kT/m) belongs,
a dropped 1/m, or m and kT swapped move the results of one of them.

Tolerances are those of the unit-parameter parity tests: forces and member
gradients 1e-5 relative, 20-step trajectories 1e-4, labels within 2 combined
standard errors, and bit-identity between the batched / served label kernels
and rid_label.
"""
import math

import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORCE_RTOL = 1e-5
TRAJ_RTOL = 1e-4
PHYS = [dict(mass=2.5, kT=2.49, dt=0.004, gamma=0.5, lj_sigma=1.1, lj_eps=0.7),
        dict(mass=3.0, kT=0.6, dt=0.004, gamma=0.5, lj_sigma=1.1, lj_eps=0.7)]
IDS = ["m2.5_kT2.49", "m3_kT0.6"]


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def close_rel(got, ref):
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    return (np.abs(got - ref) / (np.abs(ref) + np.sqrt(np.mean(ref ** 2)))).max()


def wrapd(d):
    return d - 2 * np.pi * np.floor(d / (2 * np.pi) + 0.5)


def system(n, C, seed, phys, **kw):
    sp = I.make_system(n, C, seed, **phys, **kw)
    return sp


def chains(W, sp, seed):
    # starting chains keep non-excluded beads 1.0 apart (sigma = 1.1)
    return I.make_chains(W, sp, seed, min_dist=1.0)


@pytest.mark.parametrize("phys", PHYS, ids=IDS)
def test_forces_biased_and_restrained(R, orc, phys):
    n, C, W = 60, 6, 24
    sp = system(n, C, 51, phys)
    x = chains(W, sp, 51)
    ens = I.make_ensemble(4, 2 * C, 3, 64, 51)
    eps_all = np.array([orc.ensemble(ens, orc.cvs(sp, xi.astype(np.float64))[0])["eps"] for xi in x])
    ens.trust_lo, ens.trust_hi = float(np.percentile(eps_all, 25)), float(np.percentile(eps_all, 75))
    f = np.zeros((W, n, 3), np.float32)
    fr = np.zeros((W, n, 3), np.float32)
    eps = np.zeros(W, np.float32)
    g = np.zeros((4, W, C), np.float32)
    s0 = I.make_label_targets(W, C, 51)
    kap = np.random.default_rng(5).uniform(50, 500, size=(W, C))
    with R.System(sp) as sysm:
        sysm.set_ensemble(ens)
        sysm.eval_forces(x, R.RID_BIAS_ENSEMBLE, f_out=f, eps_out=eps, grad_out=g)
        sysm.eval_forces(x, R.RID_BIAS_RESTRAINT, s0=s0, kappa=kap, f_out=fr)
    for w in range(W):
        xd = x[w].astype(np.float64)
        r = orc.total(sp, xd, ens=ens, mode=1)
        e = orc.ensemble(ens, r["s"])
        assert close_rel(g[:, w], e["gradA"]) < FORCE_RTOL
        slope = math.pi / 2 / (ens.trust_hi - ens.trust_lo)
        assert close_rel(f[w], r["f"]) < FORCE_RTOL + slope * abs(eps[w] - e["eps"]), w
        rr = orc.total(sp, xd, mode=2, s0=s0[w], kappa=kap[w])
        assert close_rel(fr[w], rr["f"]) < FORCE_RTOL, w


@pytest.mark.parametrize("phys", PHYS, ids=IDS)
def test_maxwell_boltzmann_start_matches_the_oracle(R, orc, phys):
    """Zero steps: the velocities returned are the drawn start, element by
    element (FP32 Box-Muller against FP64)."""
    sp = system(45, 4, 52, phys)
    x0 = chains(9, sp, 52)
    vo = np.zeros_like(x0)
    with R.System(sp) as sysm:
        sysm.explore(x0, 0, v_out=vo)
    ref = orc.explore(sp, x0, 0)["v"]
    sd = math.sqrt(sp.kT / sp.mass)
    assert np.all(np.abs(vo - ref) <= 2e-6 * (np.abs(ref) + 2 * sd))


@pytest.mark.parametrize("phys", PHYS, ids=IDS)
@pytest.mark.parametrize("mb", [True, False], ids=["mb_start", "given_v0"])
def test_twenty_step_biased_trajectories(R, orc, phys, mb):
    n, C, W = 45, 6, 20
    sp = system(n, C, 53, phys, output_freq=1)
    x0 = chains(W, sp, 53)
    v0 = None if mb else (math.sqrt(sp.kT / sp.mass) * np.random.default_rng(3).standard_normal(x0.shape)).astype(np.float32)
    ens = I.make_ensemble(4, 2 * C, 3, 64, 53)
    eps_all = np.array([orc.ensemble(ens, orc.cvs(sp, xi.astype(np.float64))[0])["eps"] for xi in x0])
    ens.trust_lo, ens.trust_hi = float(np.percentile(eps_all, 25)), float(np.percentile(eps_all, 75))
    steps = 20
    cv = np.zeros((W, steps, C), np.float32)
    eps = np.zeros((W, steps), np.float32)
    xo, vo = np.zeros_like(x0), np.zeros_like(x0)
    with R.System(sp) as sysm:
        sysm.set_ensemble(ens)
        sysm.explore(x0, steps, v0=v0, cv_out=cv, eps_out=eps, x_out=xo, v_out=vo)
    ref = orc.explore(sp, x0, steps, ens=ens, v0=v0)
    assert np.all(np.abs(xo - ref["x"]) <= TRAJ_RTOL * (np.abs(ref["x"]) + 1))
    assert np.all(np.abs(vo - ref["v"]) <= TRAJ_RTOL * (np.abs(ref["v"]) + 1))
    assert np.all(np.abs(wrapd(cv - ref["cv"])) <= TRAJ_RTOL * (np.abs(ref["cv"]) + 1))
    assert np.all(np.abs(eps - ref["eps"]) <= TRAJ_RTOL * (np.abs(ref["eps"]) + 1))


@pytest.mark.parametrize("phys", PHYS, ids=IDS)
def test_nve_energy_terms_and_drift(R, orc, phys):
    """gamma = 0: the FP64 energy trace (U_ff, -Abar, kinetic 1/2 m v^2) of the
    first frame equals the oracle's, and the drift over 10 k steps stays within
    twice the oracle's walker mean."""
    ph = dict(phys, gamma=0.0)
    sp = system(22, 2, 54, ph, output_freq=50)
    x0 = chains(8, sp, 54)
    ens = I.make_ensemble(4, 4, 3, 64, 54, trust_lo=1e9, trust_hi=2e9)
    steps = 10000
    en = np.zeros((8, steps // 50, 3))
    with R.System(sp) as sysm:
        sysm.set_ensemble(ens)
        sysm.explore(x0, steps, energy_out=en)
    ref = orc.explore(sp, x0, steps, ens=ens, energy=True)
    assert np.allclose(en[:, 0], ref["energy"][:, 0], rtol=1e-3, atol=1e-3 * sp.kT)

    def drift(e):
        E = e.sum(-1)
        return np.abs(E - E[:, :1]).max(axis=1) / (3 * sp.n_beads * sp.kT)
    dg, do = drift(en), drift(ref["energy"])
    assert dg.mean() <= 2 * do.mean() + 1e-6, (dg, do)
    assert dg.max() < 2e-3


@pytest.mark.parametrize("phys", PHYS, ids=IDS)
def test_labels_within_two_standard_errors(R, orc, phys):
    sp = system(22, 2, 55, phys)
    Rn = 16
    x0 = chains(Rn, sp, 55)
    s0 = I.make_label_targets(Rn, 2, 55)
    kap = np.full((Rn, 2), 50.0)
    n_steps, n_equil, B = 5000, 500, 20
    mf, se, sd = (np.zeros((Rn, 2)) for _ in range(3))
    with R.System(sp) as sysm:
        sysm.label(x0, s0, kap, n_steps, n_equil, B, mf, se, sd)
    ref = orc.label(sp, x0, s0, kap, n_steps, n_equil, B)
    z = (mf - ref["mf"]) / np.sqrt(se ** 2 + ref["se"] ** 2)
    assert np.mean(np.abs(z) <= 2) >= 0.9 and np.all(np.abs(z) < 4), z
    assert np.allclose(sd, ref["std"], rtol=0.3)


@pytest.mark.parametrize("phys", PHYS, ids=IDS)
def test_batched_and_served_labels_bit_equal_to_rid_label(R, phys):
    """The persistent label kernel (rid_label_batch and the request loop's
    label ticks) applies the mass, temperature and LJ parameters exactly as
    the per-step kernels do."""
    specs = [(22, 2, 3, 300, 61, True), (61, 9, 2, 240, 62, False), (130, 20, 1, 200, 63, True)]
    jobs = []
    for n, C, runs, steps, seed, mb in specs:
        sp = system(n, C, seed, phys)
        x0 = chains(runs, sp, seed)
        rng = np.random.default_rng(seed)
        v0 = None if mb else (math.sqrt(sp.kT / sp.mass) * rng.standard_normal(x0.shape)).astype(np.float32)
        jobs.append(dict(system=R.System(sp), x0=x0, v0=v0, s0=rng.uniform(-np.pi, np.pi, size=(runs, C)),
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
