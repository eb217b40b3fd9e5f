"""Batched restrained labeling (rid_label_batch: every run of every job in one
persistent launch) against the per-job path (rid_label) and the FP64 oracle.

The persistent kernel applies the per-step kernels' arithmetic in the same
order, so each job's outputs must be bit-identical to rid_label on the same
inputs; the oracle comparison uses the label tolerance of the per-step path
(within 2 combined standard errors).
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


def make_job(R, n, C, runs, steps, seed, n_equil=None, blocks=8, mb=False, step0=0, kappa=(50.0, 500.0)):
    sp = I.make_system(n, C, seed)
    x0 = I.make_chains(runs, sp, seed)
    rng = np.random.default_rng(seed + 100)
    s0 = rng.uniform(-np.pi, np.pi, size=(runs, C))
    kappa = rng.uniform(kappa[0], kappa[1], size=(runs, C))
    v0 = None if mb else (0.3 * rng.standard_normal(x0.shape)).astype(np.float32)
    sysobj = R.System(sp)
    j = dict(system=sysobj, x0=x0, v0=v0, s0=s0, kappa=kappa, step0=step0, n_steps=steps,
             n_equil=steps // 10 if n_equil is None else n_equil, n_blocks=blocks,
             mf=np.zeros((runs, C)), se=np.zeros((runs, C)), std=np.zeros((runs, C)),
             x_out=np.zeros_like(x0), v_out=np.zeros_like(x0))
    return j


def alone(j):
    runs, C = j["s0"].shape
    out = dict(mf=np.zeros((runs, C)), se=np.zeros((runs, C)), std=np.zeros((runs, C)),
               x_out=np.zeros_like(j["x0"]), v_out=np.zeros_like(j["x0"]))
    j["system"].label(j["x0"], j["s0"], j["kappa"], j["n_steps"], j["n_equil"], j["n_blocks"], out["mf"], out["se"],
                      out["std"], v0=j["v0"], step0=j["step0"], x_out=out["x_out"], v_out=out["v_out"])
    return out


def uneven_jobs(R):
    return [make_job(R, 22, 2, 3, 120, 1),
            make_job(R, 61, 9, 2, 90, 2, mb=True, step0=1000),
            make_job(R, 200, 20, 1, 60, 3, blocks=4),
            make_job(R, 130, 40, 2, 75, 4, n_equil=0),
            make_job(R, 257, 12, 1, 40, 5, blocks=2),
            make_job(R, 51, 7, 1, 60, 9, mb=True)]       # odd bead count, no v0: staging offsets not multiples of 8


@pytest.mark.parametrize("threads", [128, 256, 512, 0])
def test_batch_is_bit_identical_to_per_job_label(R, threads):
    jobs = uneven_jobs(R)
    with R.Server(256 << 20) as srv:
        st = srv.label_batch(jobs, threads=threads)
    assert st == [R.RID_OK] * len(jobs)
    for j in jobs:
        ref = alone(j)
        for k in ("mf", "se", "std", "x_out", "v_out"):
            assert np.array_equal(j[k], ref[k]), (j["system"].N, k)
        j["system"].close()


def test_batch_on_device_pointers_matches_host(R):
    import torch
    jobs = uneven_jobs(R)[:3]
    with R.Server(128 << 20) as srv:
        srv.label_batch(jobs, threads=256)
        dj = []
        for j in jobs:
            d = dict(j)
            for k in ("x0", "s0", "kappa"):
                d[k] = torch.from_numpy(np.ascontiguousarray(j[k])).cuda()
            d["v0"] = None if j["v0"] is None else torch.from_numpy(j["v0"]).cuda()
            for k in ("mf", "se", "std"):
                d[k] = torch.zeros(j[k].shape, dtype=torch.float64, device="cuda")
            for k in ("x_out", "v_out"):
                d[k] = torch.zeros(j[k].shape, dtype=torch.float32, device="cuda")
            dj.append(d)
        srv.label_batch(dj, threads=256)
        torch.cuda.synchronize()
    for j, d in zip(jobs, dj):
        for k in ("mf", "se", "std", "x_out", "v_out"):
            assert np.array_equal(j[k], d[k].cpu().numpy()), k
        j["system"].close()


def test_batch_labels_within_two_standard_errors_of_the_oracle(R, orc):
    jobs = [make_job(R, 22, 2, 6, 3000, 11, n_equil=300, blocks=10, kappa=(50.0, 100.0)),
            make_job(R, 40, 4, 4, 3000, 12, n_equil=300, blocks=10, kappa=(50.0, 100.0))]
    with R.Server(64 << 20) as srv:
        srv.label_batch(jobs)
    z = []
    for j in jobs:
        ref = orc.label(j["system"].sp, j["x0"], j["s0"], j["kappa"], j["n_steps"], j["n_equil"], j["n_blocks"],
                        v0=j["v0"])
        se = np.sqrt(j["se"] ** 2 + ref["se"] ** 2)
        z.append(np.abs(j["mf"] - ref["mf"]) / se)
        j["system"].close()
    z = np.concatenate([a.ravel() for a in z])
    assert np.mean(z < 2.0) >= 0.9 and z.max() < 4.0, z


def test_large_chain_without_shared_bonded_slots(R):
    # beyond 1024 beads the force field takes the per-bead bonded path
    jobs = [make_job(R, 1500, 16, 1, 12, 21, blocks=2), make_job(R, 90, 6, 2, 30, 22)]
    with R.Server(64 << 20) as srv:
        srv.label_batch(jobs, threads=512)
    for j in jobs:
        ref = alone(j)
        for k in ("mf", "se", "std", "x_out", "v_out"):
            assert np.array_equal(j[k], ref[k]), (j["system"].N, k)
        j["system"].close()


def test_budget_and_argument_errors(R):
    j = make_job(R, 200, 20, 64, 40, 31)
    with R.Server(1 << 20) as srv:
        with pytest.raises(R.RidError) as e:
            srv.label_batch([j])
        assert e.value.code == R.RID_ERR_OOM
    bad = dict(j, n_blocks=1)
    with R.Server(64 << 20) as srv:
        with pytest.raises(R.RidError) as e:
            srv.label_batch([bad])
        assert e.value.code == R.RID_ERR_ARG
        with pytest.raises(R.RidError) as e:
            srv.label_batch([j], threads=96)
        assert e.value.code == R.RID_ERR_ARG
    j["system"].close()


def test_nonfinite_job_is_reported_per_job(R):
    good = make_job(R, 40, 4, 1, 30, 41)
    badj = make_job(R, 40, 4, 1, 30, 42)
    badj["x0"][0, 5] = badj["x0"][0, 9]          # two beads on top of each other
    with R.Server(64 << 20) as srv:
        st = srv.label_batch([good, badj], raise_nonfinite=False)
    assert st == [R.RID_OK, R.RID_ERR_NONFINITE]
    ref = alone(good)
    assert np.array_equal(good["mf"], ref["mf"])
    good["system"].close()
    badj["system"].close()
