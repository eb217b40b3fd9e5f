"""The request loop (rid_submit / rid_poll): label and exploration jobs of
different chain lengths, CV counts and ensembles arriving over time, admitted
by device footprint and run concurrently (label jobs in ticks of the
persistent kernel, exploration jobs as replayed CUDA graphs).

Each job's results must be the same bits as the per-job path (rid_label,
rid_explore) on the same inputs, and the same bits alone in the server as in
any mix.  (BF16 exploration jobs of up to 16 walkers run the small-batch
ensemble kernel's lean variant in the server, 8 epilogue warps and 3 weight
stages, and the full variant per job; label runs of long chains run as
thread-block clusters of the persistent kernel in the server and through the
per-step kernels per job: the same bits.)
"""
import time

import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


class Spec:
    """One request and the arrays it writes."""

    def __init__(self, R, kind, n, C, W, steps, seed, prec=None, H=64, sysobj=None, of=10):
        self.kind, self.steps = kind, steps
        if sysobj is None:
            sp = I.make_system(n, C, seed, output_freq=of)
            sysobj = R.System(sp)
            if kind == "explore" and prec is not None:
                ens = I.make_ensemble(4, 2 * C, 3, H, seed)
                sysobj.set_ensemble(ens, precision=prec)
        self.sys = sysobj
        sp = sysobj.sp
        self.x0 = I.make_chains(W, sp, seed)
        rng = np.random.default_rng(seed + 7)
        self.v0 = (0.4 * rng.standard_normal(self.x0.shape)).astype(np.float32) if seed % 2 else None
        if kind == "label":
            self.s0 = rng.uniform(-np.pi, np.pi, size=(W, sp.n_cv))
            self.kappa = rng.uniform(50.0, 500.0, size=(W, sp.n_cv))
            self.n_equil, self.blocks = steps // 10, 5
        self.fresh()

    def fresh(self):
        W, N, C = self.x0.shape[0], self.sys.N, self.sys.C
        self.x_out, self.v_out = np.zeros_like(self.x0), np.zeros_like(self.x0)
        if self.kind == "label":
            self.mf, self.se, self.std = (np.zeros((W, C)) for _ in range(3))
        else:
            T = self.steps // self.sys.sp.output_freq
            self.cv, self.eps = np.zeros((W, T, C), np.float32), np.zeros((W, T), np.float32)

    def submit(self, srv):
        if self.kind == "label":
            return srv.submit_label(self.sys, self.x0, self.s0, self.kappa, self.steps, self.n_equil, self.blocks,
                                    self.mf, self.se, self.std, v0=self.v0, x_out=self.x_out, v_out=self.v_out)
        return srv.submit_explore(self.sys, self.x0, self.steps, v0=self.v0, cv_out=self.cv, eps_out=self.eps,
                                  x_out=self.x_out, v_out=self.v_out)

    def outputs(self):
        if self.kind == "label":
            return [self.mf, self.se, self.std, self.x_out, self.v_out]
        return [self.cv, self.eps, self.x_out, self.v_out]

    def per_job(self):
        """The same job through rid_label / rid_explore."""
        W, N, C = self.x0.shape[0], self.sys.N, self.sys.C
        xo, vo = np.zeros_like(self.x0), np.zeros_like(self.x0)
        if self.kind == "label":
            mf, se, sd = (np.zeros((W, C)) for _ in range(3))
            self.sys.label(self.x0, self.s0, self.kappa, self.steps, self.n_equil, self.blocks, mf, se, sd,
                           v0=self.v0, x_out=xo, v_out=vo)
            return [mf, se, sd, xo, vo]
        T = self.steps // self.sys.sp.output_freq
        cv, eps = np.zeros((W, T, C), np.float32), np.zeros((W, T), np.float32)
        self.sys.explore(self.x0, self.steps, v0=self.v0, cv_out=cv, eps_out=eps, x_out=xo, v_out=vo)
        return [cv, eps, xo, vo]


def mixed_specs(R):
    shared = Spec(R, "explore", 61, 9, 5, 600, 13, prec=R.RID_PREC_FP32)
    return [
        Spec(R, "label", 22, 2, 3, 400, 1),
        Spec(R, "explore", 200, 20, 12, 520, 2, prec=R.RID_PREC_BF16, H=128),
        Spec(R, "explore", 150, 18, 12, 530, 9, prec=R.RID_PREC_BF16, H=300),  # small-batch kernel, 3 tiles
        Spec(R, "label", 200, 20, 1, 300, 3),
        Spec(R, "label", 130, 40, 2, 250, 4),
        shared,
        Spec(R, "explore", 61, 9, 4, 260, 14, sysobj=shared.sys),      # same system: runs after the other
        Spec(R, "label", 61, 9, 2, 900, 5),
        Spec(R, "explore", 22, 2, 16, 333, 6, prec=R.RID_PREC_FP32),  # graph chunks + a remainder chunk
        Spec(R, "label", 300, 12, 1, 120, 7),
        Spec(R, "label", 51, 7, 1, 100, 8),                            # odd bead count, no v0
        Spec(R, "label", 900, 16, 2, 150, 10),                         # long chain: clusters of CTAs
        Spec(R, "label", 1777, 30, 1, 90, 11),                         # long chain, ragged last slice
    ]


def test_mixed_stream_matches_per_job_path_and_alone(R):
    specs = mixed_specs(R)
    with R.Server(512 << 20) as srv:
        ids = []
        for k, sp in enumerate(specs):
            ids.append(sp.submit(srv))
            if k % 3 == 2:
                time.sleep(0.01)                   # later arrivals join running work
        res = srv.wait(ids)
        mixed = [[a.copy() for a in sp.outputs()] for sp in specs]
        for jid in ids:
            st, info = res[jid]
            assert st == R.RID_OK
            assert info["t_submit_ms"] <= info["t_start_ms"] <= info["t_end_ms"]
        # each job alone in the server
        for sp, out in zip(specs, mixed):
            sp.fresh()
            jid = sp.submit(srv)
            st, _ = srv.wait([jid])[jid]
            assert st == R.RID_OK
            for a, b in zip(sp.outputs(), out):
                assert np.array_equal(a, b), sp.kind
    for sp, out in zip(specs, mixed):
        ref = sp.per_job()
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), (sp.kind, sp.sys.N)
    for sp in specs:
        sp.sys.close()


def test_admission_by_footprint_keeps_within_the_budget(R):
    specs = [Spec(R, "label", 200, 20, 8, 200, 20 + k) for k in range(12)]
    budget = 1 << 20
    with R.Server(budget) as srv:
        ids = [sp.submit(srv) for sp in specs]
        seen_queue, peak = 0, 0
        while True:
            q, r, b = srv.load()
            seen_queue = max(seen_queue, q)
            peak = max(peak, b)
            if q == 0 and r == 0:
                break
            time.sleep(0.001)
        res = srv.wait(ids)
    assert peak <= budget
    assert seen_queue > 0                          # the budget held some jobs back
    # statuses and results as through rid_label (a stiff restraint can make a
    # run non-finite on both paths)
    for sp, jid in zip(specs, ids):
        out = [a.copy() for a in sp.outputs()]
        try:
            ref, st_ref = sp.per_job(), R.RID_OK
        except R.RidError as e:
            ref, st_ref = None, e.code
        assert res[jid][0] == st_ref
        if ref is not None:
            for a, b in zip(out, ref):
                assert np.array_equal(a, b)
    for sp in specs:
        sp.sys.close()


def test_cancel_withdraws_queued_jobs_only(R):
    """A 1 MiB budget holds most of twelve label jobs back; the last four are
    withdrawn right after submission, while the first ones still run (2000
    steps each).  A withdrawn job's outputs stay untouched and it polls as
    cancelled, never started; the others give the per-job results.  A job
    that is final but not yet polled cannot be withdrawn; an id that was
    polled or never given is unknown."""
    specs = [Spec(R, "label", 200, 20, 8, 2000, 40 + k) for k in range(12)]
    with R.Server(1 << 20) as srv:
        ids = [sp.submit(srv) for sp in specs]
        withdrawn = [jid for jid in ids[8:] if srv.cancel(jid)]
        assert withdrawn                               # queued behind the budget
        while srv.load()[:2] != (0, 0):
            time.sleep(0.001)
        assert not srv.cancel(ids[0])                  # final, not yet polled
        res = srv.wait(ids)
        with pytest.raises(R.RidError) as e:
            srv.cancel(ids[0])                         # polled: forgotten
        assert e.value.code == R.RID_ERR_ARG
        with pytest.raises(R.RidError) as e:
            srv.cancel(987654)
        assert e.value.code == R.RID_ERR_ARG
    for sp, jid in zip(specs, ids):
        st, info = res[jid]
        if jid in withdrawn:
            assert st == R.RID_ERR_CANCELLED and info["t_start_ms"] == -1
            assert all(not a.any() for a in sp.outputs())
            continue
        out = [a.copy() for a in sp.outputs()]
        try:
            ref, st_ref = sp.per_job(), R.RID_OK
        except R.RidError as err:
            ref, st_ref = None, err.code
        assert st == st_ref
        if ref is not None:
            for a, b in zip(out, ref):
                assert np.array_equal(a, b)
    for sp in specs:
        sp.sys.close()


def test_request_errors(R):
    big = Spec(R, "label", 400, 20, 256, 40, 31)
    with R.Server(2 << 20) as srv:
        with pytest.raises(R.RidError) as e:
            big.submit(srv)
        assert e.value.code == R.RID_ERR_OOM
        with pytest.raises(R.RidError) as e:
            srv.poll(12345)
        assert e.value.code == R.RID_ERR_ARG
        small = Spec(R, "label", 22, 2, 1, 40, 32)
        jid = small.submit(srv)
        st, _ = srv.wait([jid])[jid]
        assert st == R.RID_OK
        with pytest.raises(R.RidError):
            srv.poll(jid)                          # forgotten after the final status
        small.sys.close()
    big.sys.close()
