"""Benchmark of the RiD biased Langevin step (walker-steps/s).

Workload: 1024 walkers of a 200-bead chain, 20 torsion CVs, ensemble of
4 MLPs 40 -> 256 x 4 -> 1 (tanh), BAOAB dt = 0.005, gamma = 1, kT = 1;
synthetic seeded inputs.  One bench step = one MD step of every walker
(force field + CVs + ensemble forward / input gradient + switched bias +
chain rule + BAOAB).  The walker state (~30 MB) fits in L2, so L2 is flushed
(256 MiB write) before every timed step and each step is timed on its own
with CUDA events on the stream the kernels run on.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16]
                  [--impl ours|reference]

More legs on rank 0 (N = 1) go into the same JSON line: "fp32_plain" (the
same step with the FP32 SIMT ensemble), "paper_network" (the paper's own
4 x [300]^4 residual ensemble on 18 torsions: FP32 / BF16 / FP8 and the
ensemble kernel's roofline at that shape), "tiny" (the 22-bead
configuration through rid_explore and rid_label), "precision" (the
8192-walker sweep: FP32 / BF16 / FP8 throughput, ensemble roofline,
deviation from FP32, NVE drift), "batching" (512 uneven restrained labeling
jobs in one persistent launch against the per-job path), "training",
"constrained", "selection", "mcmc", "serving" (a Poisson stream of mixed
requests through rid_submit / rid_poll at 200/s against the plain FP32
per-job path) and "serving_sustained" (the same mix at a rate the GPU
clears).  "cpu_baseline" times the FP64 oracle on the host cores (the
headline workload, the small configuration, a sample of the precision
sweep) and gives the precision sweep's errors against the oracle.  The line
ends with "legs", a short summary of every leg's headline figures.

--impl reference times the FP64 CPU oracle on the host cores (a bounded
sample of the same workload per step).  Under torchrun every rank runs its
own 1024 walkers (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# 32 hardware work queues for the request loop's 16 exploration streams (the
# runtime's default of 8 makes streams wait on one another); read when the
# CUDA context is created, so set before torch starts CUDA.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from paper_2408_14070_gb300 import inputs as I  # noqa: E402

WORKLOAD = "chain_n200_w1024"
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
_FP32_MEASURED = None


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def fp32_peak(torch):
    """(peak TFLOP/s, source) for FP32 ALU-bound kernels: dense FP32 throughput
    measured on this GPU with a library GEMM (cuBLAS SGEMM 8192^3, TF32 off),
    as the BF16 peak is measured with cuBLAS; the derived figure if that fails."""
    global _FP32_MEASURED
    if _FP32_MEASURED is None:
        try:
            prev_tf32, prev_prec = torch.backends.cuda.matmul.allow_tf32, torch.get_float32_matmul_precision()
            torch.backends.cuda.matmul.allow_tf32 = False
            torch.set_float32_matmul_precision("highest")
            n = 8192
            g = torch.Generator(device="cuda").manual_seed(0)
            a = torch.randn(n, n, device="cuda", generator=g)
            b = torch.randn(n, n, device="cuda", generator=g)
            for _ in range(3):
                a @ b
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                a @ b
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 10
            torch.backends.cuda.matmul.allow_tf32 = prev_tf32
            torch.set_float32_matmul_precision(prev_prec)
            del a, b
            _FP32_MEASURED = (2.0 * n ** 3 / (ms * 1e-3) / 1e12,
                              "measured: cuBLAS FP32 SGEMM 8192^3, TF32 off, in this run "
                              f"(derived {FP32_PEAK_TFLOPS:.1f} TFLOP/s = {FP32_PEAK_NOTE})")
        except Exception as e:   # measurement unavailable: the derived peak
            _FP32_MEASURED = (FP32_PEAK_TFLOPS, f"derived: {FP32_PEAK_NOTE} ({type(e).__name__})")
    return _FP32_MEASURED


def workload_desc(wl):
    return (f"{wl['n_walkers']} walkers, {wl['n_beads']}-bead chain, {wl['n_cv']} torsion CVs, "
            f"{wl['n_models']} x MLP {2 * wl['n_cv']}-{wl['width']}x{wl['n_layers']}-1")


def make_inputs(wl, seed=1):
    sp = I.make_system(wl["n_beads"], wl["n_cv"], seed, output_freq=10)
    x0 = I.make_chains(wl["n_walkers"], sp, seed)
    ens = I.make_ensemble(wl["n_models"], 2 * wl["n_cv"], wl["n_layers"], wl["width"], seed)
    return sp, x0, ens


def mlp_flops_per_walker_step(wl):
    D, H, L, M = 2 * wl["n_cv"], wl["width"], wl["n_layers"], wl["n_models"]
    return M * 4 * (D * H + (L - 1) * H * H)


def pair_flops_per_walker_step(wl):
    N = wl["n_beads"]
    return 20 * (N - 2) * (N - 3) // 2


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.lines = []

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def wait_first(self, timeout=5.0):
        t0 = time.monotonic()
        while self.p and not self.lines and time.monotonic() - t0 < timeout:
            time.sleep(0.02)

    def mark(self, start, end):
        self.window = (start, end)

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo, hi = getattr(self, "window", (-1e30, 1e30))
        def parsed(ln):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                return None
            try:
                return float(f[0]), float(f[1]), f
            except ValueError:
                return None
        good = [(t, parsed(ln)) for t, ln in self.lines]
        good = [(t, p) for t, p in good if p is not None]
        inside = [p for t, p in good if lo - 0.1 <= t <= hi + 0.1]
        if not inside and good:             # region shorter than the sampling period
            inside = [min(good, key=lambda tp: abs(tp[0] - 0.5 * (lo + hi)))[1]]
        for s_mhz, m_mhz, f in inside:
            sm.append(s_mhz)
            mx.append(m_mhz)
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash(name):
    path = os.path.join(ROOT, "paper_2408_14070_gb300", "csrc", name)
    try:
        return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None


def traffic_for(kernel, src_file, workload):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source
    is unchanged since it was taken; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        rec = json.load(open(path)).get(f"{kernel}@{workload}")
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha256_16") != kernel_source_hash(src_file):
        return None
    return rec.get("bytes_per_launch")


def cpu_baseline(sp, x0, ens, walkers, steps):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.explore(sp, x0[:walkers], steps, ens=ens)
    dt = time.perf_counter() - t0
    return {"value": walkers * steps / dt, "unit": "walker-steps/s", "cores": int(r["threads"]),
            "kind": "oracle",
            "sample": f"{walkers} walkers x {steps} steps of the same workload (FP64, plus one initial "
                      f"force evaluation per walker), {dt:.1f} s"}


def chain_pools(lengths, walkers, seed):
    """Starting chains grown once per chain length: {N: [walkers][N][3]}."""
    pools = {}
    for N in sorted(set(int(n) for n in lengths)):
        pools[N] = I.make_chains(walkers, I.make_system(N, 1, seed + N), seed + N)
    return pools


def targets_near_start(rid, system, x0, rng, spread=0.3):
    """Restraint centres near the CVs of the starting configuration (labeling
    restrains selected configurations at their own CV values), perturbed."""
    s = np.zeros((x0.shape[0], system.C), np.float32)
    system.eval_forces(x0, rid.RID_BIAS_NONE, s_out=s)
    return s.astype(np.float64) + rng.uniform(-spread, spread, size=s.shape)


def run_batching(rid, n_jobs, n_steps, plain_jobs, seed=3):
    """Uneven restrained labeling jobs (one run each) in one persistent launch
    (rid_label_batch, CTA size autotuned), against the plain FP32 per-job path
    (rid_label, one job after another) on an evenly spaced sample of the jobs."""
    specs = I.label_batch_jobs(n_jobs, seed, n_steps=n_steps)
    rng = np.random.default_rng(seed)
    pools = chain_pools([j["n_beads"] for j in specs], max(1, max(
        sum(1 for j in specs if j["n_beads"] == n) for n in set(j["n_beads"] for j in specs))), seed)
    used = {}
    jobs = []
    for j in specs:
        sp = I.make_system(j["n_beads"], j["n_cv"], j["seed"])
        system = rid.System(sp)
        k = used.get(j["n_beads"], 0)
        used[j["n_beads"]] = k + 1
        x0 = np.ascontiguousarray(pools[j["n_beads"]][k:k + 1])
        s0 = targets_near_start(rid, system, x0, rng)
        C = j["n_cv"]
        jobs.append(dict(system=system, x0=x0, s0=s0, kappa=np.ascontiguousarray(j["kappa"][None, :]),
                         n_steps=j["n_steps"], n_equil=j["n_steps"] // 10, n_blocks=20,
                         mf=np.zeros((1, C)), se=np.zeros((1, C)), std=np.zeros((1, C))))
    wsteps = sum(j["n_steps"] for j in jobs)
    srv = rid.Server(8 << 30)
    srv.label_batch(jobs, threads=0, raise_nonfinite=False)              # autotune + warm
    t0 = time.perf_counter()
    st = srv.label_batch(jobs, threads=0, raise_nonfinite=False)
    dt = time.perf_counter() - t0
    srv.close()
    order = sorted(range(len(jobs)), key=lambda k: jobs[k]["system"].N)
    sample = [order[int(i)] for i in np.linspace(0, len(order) - 1, min(plain_jobs, len(order)))]
    t_plain, ws_plain = 0.0, 0
    for k in sample:
        j = jobs[k]
        C = j["system"].C
        j["system"].set_fused_steps(False)   # the plain path: per-step kernels
        mf, se, sd = np.zeros((1, C)), np.zeros((1, C)), np.zeros((1, C))
        t1 = time.perf_counter()
        try:
            j["system"].label(j["x0"], j["s0"], j["kappa"], j["n_steps"], j["n_equil"], j["n_blocks"], mf, se, sd)
        except rid.RidError:
            pass
        t_plain += time.perf_counter() - t1
        ws_plain += j["n_steps"]
    for j in jobs:
        j["system"].close()
    Ns = [j["system"].N for j in jobs]
    return {"workload": f"{n_jobs} restrained labeling jobs, 1 run x {n_steps} steps each, chain length "
                        f"log-uniform {min(Ns)}-{max(Ns)} beads, 4-40 torsion CVs, kappa 50-500, "
                        f"restraint centres near the starting CVs",
            "value": wsteps / dt, "unit": "walker-steps/s", "wall_s": dt, "kernel_launches": 1,
            "timed": "one rid_label_batch call from host arrays (uploads, the persistent kernel, downloads); "
                     "a first call picked the CTA size",
            "nonfinite_jobs": int(sum(1 for x in st if x != rid.RID_OK)),
            "plain_per_job": {"value": ws_plain / t_plain, "unit": "walker-steps/s", "jobs": len(sample),
                              "path": "rid_label per job (per-step kernels, FP32), jobs run one after another"},
            "speedup_vs_plain": (wsteps / dt) / (ws_plain / t_plain)}


def train_flops_per_sample(D, L, H):
    """Algorithmic FP32 flops of one training sample of one member: forward,
    input gradient and its adjoint 2F each, the pass back through the forward
    layers 2 (L - 1) H^2, and the two outer products of the weight gradient 4F,
    with F = D H + (L - 1) H^2 multiply-adds per pass."""
    F = D * H + (L - 1) * H * H
    return 10 * F + 2 * (L - 1) * H * H


def run_training(rid, torch, steps, seed=11):
    """Ensemble training on mean-force labels (rid_trainer_run) for the
    exploration model of the 200-bead workload: 4 members 40-256x4-1, batch
    128 per member, the training section's learning-rate schedule and dropout
    rate 0.1, labels = the CV gradient of a teacher network at points on the CV
    torus."""
    wl = I.workload(WORKLOAD)
    M, C, L, H, B = wl["n_models"], wl["n_cv"], wl["n_layers"], wl["width"], 128
    D = 2 * C
    n = 16384
    student = I.make_ensemble(M, D, L, H, seed)
    teacher = I.make_ensemble(1, D, L, H, seed + 1)
    rng = np.random.default_rng(seed)
    s = torch.from_numpy(rng.uniform(-np.pi, np.pi, size=(n, C)).astype(np.float32)).cuda()
    mf = torch.zeros((1, n, C), dtype=torch.float32, device="cuda")
    tw = torch.from_numpy(teacher.weights).cuda()
    for c0 in range(0, n, 1024):
        rid.ensemble_grad_noalloc(s[c0:c0 + 1024], tw, 1, L, H, mf[:, c0:c0 + 1024])
    mf = mf[0].contiguous()
    warm = 5
    idx = torch.from_numpy(rng.integers(0, n, size=(warm + steps, M, B)).astype(np.int32)).cuda()
    loss = torch.zeros((warm + steps, M), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    with rid.Trainer(M, C, L, H, student.weights, batch_size=B, dropout_rate=0.1, dropout_seed=seed) as tr:
        tr.set_data(s, mf, stream=stream)
        tr.run(idx[:warm], loss[:warm], stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tr.run(idx[warm:], loss[warm:], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lo = loss.cpu().numpy()
    fl = train_flops_per_sample(D, L, H) * M * B
    achieved = fl * steps / (ms * 1e-3) / 1e12
    return {"workload": f"{M} members {D}-{H}x{L}-1, batch {B} per member, dropout 0.1, {n} labels "
                        "(teacher CV gradients)",
            "value": M * B * steps / (ms * 1e-3), "unit": "member-samples/s", "steps": steps,
            "ms_per_step": ms / steps, "kernel_launches_per_step": 4 * L + 4,
            "loss_first": float(lo[:warm].mean()), "loss_last": float(lo[-20:].mean()),
            "algorithmic_gflop_per_step": fl / 1e9,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak(torch)[0], "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak(torch)[0], "peak_source": fp32_peak(torch)[1]},
            "timed": "one rid_trainer_run call of all steps (device-resident labels and batch indices), "
                     "CUDA events on the launching stream"}


def run_mcmc(rid, torch, steps, seed=13):
    """MCMC dimension reduction (rid_mcmc) with the exploration model of the
    200-bead workload: 2000 walkers (the paper's numb_walkers), 101 bins."""
    wl = I.workload(WORKLOAD)
    M, C, L, H = wl["n_models"], wl["n_cv"], wl["n_layers"], wl["width"]
    D = 2 * C
    W, bins, burn = 2000, 101, steps // 10
    ens = I.make_ensemble(M, D, L, H, seed)
    rng = np.random.default_rng(seed)
    w = torch.from_numpy(ens.weights).cuda()
    s0 = torch.from_numpy(rng.uniform(-np.pi, np.pi, size=(W, C)).astype(np.float32)).cuda()
    h1 = torch.zeros((C, bins), dtype=torch.uint64, device="cuda")
    f2 = torch.zeros((bins, bins), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rid.mcmc(w, M, C, L, H, s0, 20, 0, 1.0, 0.3, seed, bins=bins, hist1=h1, pmf2=f2, stream=stream)   # warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    acc = rid.mcmc(w, M, C, L, H, s0, steps, burn, 1.0, 0.3, seed, bins=bins, hist1=h1, pmf2=f2, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    fl = M * 2 * (D * H + (L - 1) * H * H + H) * W        # forward GEMMs and the output layer, per step
    achieved = fl * steps / (ms * 1e-3) / 1e12
    # the same chain with the system's BF16 ensemble on the tensor cores (rid_mcmc_system)
    sp = I.make_system(wl["n_beads"], C, seed)
    with rid.System(sp) as system:
        system.set_ensemble(ens, precision=rid.RID_PREC_BF16)
        system.mcmc(s0, 20, 0, 1.0, 0.3, seed, bins=bins, hist1=h1, pmf2=f2, stream=stream)   # warm, tunes
        torch.cuda.synchronize()
        e0.record(stream)
        acc16 = system.mcmc(s0, steps, burn, 1.0, 0.3, seed, bins=bins, hist1=h1, pmf2=f2, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms16 = e0.elapsed_time(e1)
    bf16 = _peaks().get("bf16_tflops") or 1900.0
    ach16 = fl * steps / (ms16 * 1e-3) / 1e12
    return {"workload": f"{W} walkers, {M} members {D}-{H}x{L}-1, {steps} Metropolis steps ({burn} burn-in), "
                        f"{bins} bins per CV, 2-D projection on CVs (0, 1)",
            "value": W * steps / (ms * 1e-3), "unit": "walker-steps/s", "ms_per_step": ms / steps,
            "acceptance": acc / (W * steps), "kernel_launches_per_step": L + 2,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak(torch)[0], "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak(torch)[0], "peak_source": fp32_peak(torch)[1]},
            "timed": "one rid_mcmc call (device-resident weights and starting CVs; includes the call's "
                     "allocation, the initial evaluation and the PMF projection), CUDA events",
            "bf16_tensor_cores": {
                "value": W * steps / (ms16 * 1e-3), "unit": "walker-steps/s", "ms_per_step": ms16 / steps,
                "acceptance": acc16 / (W * steps),
                "path": "rid_mcmc_system: the system's BF16 ensemble kernel (tcgen05) in its forward-only "
                        "mode (the L forward GEMMs and the member values; no input gradient)",
                "roofline": {"bound": "tensor", "achieved": ach16, "peak": bf16, "unit": "TFLOP/s",
                             "frac": ach16 / bf16, "work": "forward flops only (what the Metropolis test needs)",
                             "peak_source": "measured bf16_tflops (burst)" if _peaks().get("bf16_tflops")
                             else "fallback 1.9 PFLOP/s bf16"}}}


def run_selection(rid, torch, seed=17):
    """Selection (rid_select) with the paper's selector config (threshold 2.6,
    30-45 clusters, 50 selections) on the CV / model-deviation traces of
    exploration: 1024 walkers x 100 output frames of the 200-bead system's 20
    torsions (synthetic torus random walks of that shape), trust window [2, 3)."""
    wl = I.workload(WORKLOAD)
    C, W, T = wl["n_cv"], wl["n_walkers"], 100
    rng = np.random.default_rng(seed)
    cv = np.cumsum(rng.normal(0.0, 0.15, size=(W, T, C)), axis=1) + rng.uniform(-np.pi, np.pi, size=(W, 1, C))
    cv = ((cv + np.pi) % (2 * np.pi) - np.pi).reshape(-1, C).astype(np.float32)
    eps = rng.uniform(0.0, 4.0, size=W * T).astype(np.float32)
    dcv, deps = torch.from_numpy(cv).cuda(), torch.from_numpy(eps).cuda()
    out = torch.zeros(50, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rid.select(dcv, deps, 2.0, 3.0, 2.6, 30, 45, True, 50, selected=out, stream=stream)     # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sel, nc, thr = rid.select(dcv, deps, 2.0, 3.0, 2.6, 30, 45, True, 50, selected=out, stream=stream)
    dt = time.perf_counter() - t0
    return {"workload": f"{W * T} frames ({W} walkers x {T}) of {C} torsion CVs, trust window [2, 3), "
                        f"threshold 2.6 adapted into [30, 45] clusters, max_selection 50",
            "value": W * T / dt, "unit": "frames/s", "wall_ms": 1e3 * dt, "clusters": nc, "threshold": thr,
            "selected": int(sel.numel()),
            "timed": "one rid_select call on device-resident traces (candidate compaction and every "
                     "clustering trial of the threshold search)"}


def run_constrained(rid, torch, runs=1024, steps=1000, seed=19):
    """Constrained-MD labelling (rid_label_constrained) on the 200-bead chain:
    `runs` runs, 10 distance CVs between beads 10 apart, each held at its
    starting length."""
    wl = I.workload(WORKLOAD)
    sp = I.make_system(wl["n_beads"], wl["n_cv"], seed)
    x0 = I.make_chains(runs, sp, seed)
    pairs = np.array([[20 * k, 20 * k + 10] for k in range(10)], np.int32)
    d0 = np.ascontiguousarray(np.linalg.norm(x0[:, pairs[:, 0]] - x0[:, pairs[:, 1]], axis=-1), dtype=np.float64)
    xd, d0d = torch.from_numpy(x0).cuda(), torch.from_numpy(d0).cuda()
    out = [torch.zeros((runs, 10), dtype=torch.float64, device="cuda") for _ in range(3)]
    stream = torch.cuda.current_stream()
    with rid.System(sp) as system:
        system.label_constrained(xd[:8], pairs, d0d[:8], 50, 10, 4, *[o[:8] for o in out], stream=stream)   # warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        system.label_constrained(xd, pairs, d0d, steps, steps // 10, 20, *out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"workload": f"{runs} constrained runs x {steps} steps, {wl['n_beads']}-bead chain, 10 distance CVs "
                        f"(beads 10 apart) held at their starting lengths",
            "value": runs * steps / (ms * 1e-3), "unit": "walker-steps/s", "wall_ms": ms, "kernel_launches": 1,
            "mean_abs_mean_force": float(out[0].abs().mean()),
            "timed": "one rid_label_constrained call on device arrays (staging, the chain-resident kernel, "
                     "statistics), CUDA events"}


def run_serving(rid, n_req, rate, plain_req, seed=5):
    """Poisson stream of mixed labeling / exploration requests through the
    request loop (BF16 ensembles), and the first plain_req requests of the
    same stream through the plain FP32 per-job path in arrival order."""
    reqs = I.serving_requests(n_req, rate, seed)
    pools = chain_pools([r["n_beads"] for r in reqs], 12, seed)
    rng = np.random.default_rng(seed)

    def build_req(r, prec):
        sp = I.make_system(r["n_beads"], r["n_cv"], r["seed"], output_freq=10)
        system = rid.System(sp)
        W, N, C = r["walkers"], r["n_beads"], r["n_cv"]
        d = dict(r, system=system)
        if r["kind"] == "label":
            k = r["seed"] % pools[N].shape[0]
            d["x0"] = np.ascontiguousarray(pools[N][k:k + 1])
            d["s0"] = targets_near_start(rid, system, d["x0"], rng)
            d["kappa_a"] = np.ascontiguousarray(r["kappa"][None, :])
            d["mf"], d["se"], d["std"] = (np.zeros((1, C)) for _ in range(3))
        else:
            ens = I.make_ensemble(r["n_models"], 2 * C, r["n_layers"], r["width"], r["seed"])
            system.set_ensemble(ens, precision=prec)
            d["x0"] = np.ascontiguousarray(pools[N][:W])
            T = r["n_steps"] // 10
            d["cv"], d["eps"] = np.zeros((W, T, C), np.float32), np.zeros((W, T), np.float32)
        return d

    served = [build_req(r, rid.RID_PREC_BF16) for r in reqs]
    srv = rid.Server(16 << 30)
    out, pending = {}, {}
    t0 = time.perf_counter()
    k = 0
    while k < len(served) or pending:
        now = time.perf_counter() - t0
        while k < len(served) and served[k]["t"] <= now:
            d = served[k]
            if d["kind"] == "label":
                jid = srv.submit_label(d["system"], d["x0"], d["s0"], d["kappa_a"], d["n_steps"], d["n_steps"] // 10,
                                       20, d["mf"], d["se"], d["std"])
            else:
                jid = srv.submit_explore(d["system"], d["x0"], d["n_steps"], cv_out=d["cv"], eps_out=d["eps"])
            pending[jid] = k
            k += 1
        for jid in list(pending):
            st, info = srv.poll(jid)
            if st != rid.RID_NOT_READY:
                out[pending.pop(jid)] = (st, info)
        time.sleep(0.0002)
    srv.close()
    lat = {"label": [], "explore": []}
    wsteps = 0
    t_first = min(i["t_submit_ms"] for _, i in out.values())
    t_last = max(i["t_end_ms"] for _, i in out.values())
    for idx, (st, info) in out.items():
        r = served[idx]
        lat[r["kind"]].append(info["t_end_ms"] - info["t_submit_ms"])
        wsteps += r["walkers"] * r["n_steps"]
    for d in served:
        d["system"].close()

    # plain FP32 per-job path on the first plain_req requests, in arrival order (per-step
    # kernels: the fused steps off)
    plain = [build_req(r, rid.RID_PREC_FP32) for r in reqs[:plain_req]]
    for d in plain:
        d["system"].set_fused_steps(False)
    lat_p = {"label": [], "explore": []}
    t0 = time.perf_counter()
    busy_until = 0.0
    for d in plain:
        now = time.perf_counter() - t0
        if now < d["t"]:
            time.sleep(d["t"] - now)
        try:
            if d["kind"] == "label":
                d["system"].label(d["x0"], d["s0"], d["kappa_a"], d["n_steps"], d["n_steps"] // 10, 20, d["mf"],
                                  d["se"], d["std"])
            else:
                d["system"].explore(d["x0"], d["n_steps"], cv_out=d["cv"], eps_out=d["eps"])
        except rid.RidError:
            pass
        lat_p[d["kind"]].append(1e3 * (time.perf_counter() - t0 - d["t"]))
    for d in plain:
        d["system"].close()
    served_first = {"label": [], "explore": []}
    for idx in range(min(plain_req, len(served))) if plain else []:
        st, info = out[idx]
        served_first[served[idx]["kind"]].append(info["t_end_ms"] - info["t_submit_ms"])

    def pct(v, q):
        return float(np.percentile(v, q)) if v else None

    return {"workload": f"{n_req} requests, Poisson arrivals at {rate:g}/s, 70% labeling (1 run) / 30% exploration "
                        f"(12 walkers), chains log-uniform 20-2000 beads, 2-64 torsion CVs, 500-5000 steps, "
                        f"ensembles 4 x (64-512 wide, 4 layers)",
            "throughput": wsteps / ((t_last - t_first) / 1e3), "unit": "walker-steps/s",
            "requests_per_s": len(out) / ((t_last - t_first) / 1e3),
            "label_latency_ms": {"p50": pct(lat["label"], 50), "p99": pct(lat["label"], 99), "n": len(lat["label"])},
            "explore_latency_ms": {"p50": pct(lat["explore"], 50), "p99": pct(lat["explore"], 99),
                                   "n": len(lat["explore"])},
            "nonfinite": int(sum(1 for st, _ in out.values() if st == rid.RID_ERR_NONFINITE)),
            "failed": int(sum(1 for st, _ in out.values() if st not in (rid.RID_OK, rid.RID_ERR_NONFINITE))),
            "mlp_precision": "bf16",
            "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
            "plain_per_job": {"requests": len(plain), "path": "rid_label / rid_explore per request in arrival "
                                                              "order, FP32 ensembles, per-step kernels, one at "
                                                              "a time",
                              "label_latency_ms": {"p50": pct(lat_p["label"], 50), "p99": pct(lat_p["label"], 99)},
                              "explore_latency_ms": {"p50": pct(lat_p["explore"], 50),
                                                     "p99": pct(lat_p["explore"], 99)},
                              "served_same_requests_label_latency_ms": {"p50": pct(served_first["label"], 50),
                                                                        "p99": pct(served_first["label"], 99)},
                              "served_same_requests_explore_latency_ms": {"p50": pct(served_first["explore"], 50),
                                                                          "p99": pct(served_first["explore"], 99)}}}


def run_fp32_plain(rid, torch, steps, seed=1):
    """The headline workload (1024 walkers, 200-bead chain, 4 x 40-256x4-1)
    with the FP32 ensemble (SIMT kernels) against the BF16 tensor-core
    ensemble: walker-steps/s of both, timed like the headline (each step alone
    between CUDA events, L2 flushed before it), and the BF16 path's deviation
    from FP32 in the mean CV force and in epsilon on the same positions."""
    wl = I.workload(WORKLOAD)
    sp, x0, ens = make_inputs(wl, seed)
    W, C = wl["n_walkers"], wl["n_cv"]
    stream = torch.cuda.current_stream()
    xd = torch.from_numpy(x0).cuda()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    res, grads, eps = {}, {}, {}
    for name, prec in (("fp32", rid.RID_PREC_FP32), ("bf16", rid.RID_PREC_BF16)):
        with rid.System(sp) as system:
            system.set_ensemble(ens, precision=prec)
            g = torch.zeros((wl["n_models"], W, C), dtype=torch.float32, device="cuda")
            e = torch.zeros(W, dtype=torch.float32, device="cuda")
            system.eval_forces(xd, rid.RID_BIAS_ENSEMBLE, grad_out=g, eps_out=e, stream=stream)
            grads[name], eps[name] = g.mean(dim=0).double(), e.double()
            system.walkers_load(xd, stream=stream)
            system.walkers_advance(3, stream=stream)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for k in range(steps):
                flush.zero_()
                ev[k][0].record(stream)
                system.walkers_advance(1, stream=stream)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev)
            system.walkers_read()
        res[name] = {"value": W * steps / (ms / 1e3), "unit": "walker-steps/s", "ms_per_step": ms / steps}
    d = (grads["bf16"] - grads["fp32"]).norm(dim=1) / grads["fp32"].norm(dim=1).clamp_min(1e-30)
    de = (eps["bf16"] - eps["fp32"]).abs() / eps["fp32"].abs().clamp_min(1e-30)
    res["bf16"]["mean_force_rel_dev_from_fp32"] = {"median": float(d.median()), "max": float(d.max())}
    res["bf16"]["eps_rel_dev_from_fp32"] = {"median": float(de.median()), "max": float(de.max())}
    res["bf16_speedup_vs_fp32"] = res["bf16"]["value"] / res["fp32"]["value"]
    res["workload"] = f"{WORKLOAD}: the headline step with each ensemble precision, {steps} steps"
    return res


def run_precision(rid, torch, steps=10, nve_walkers=64, nve_steps=10000, seed=4):
    """Precision sweep: 8192 walkers of a 100-bead chain, 32 torsion CVs,
    8 x MLP 64 -> 512 x 4 -> 1.  Per ensemble precision: throughput of full
    steps, the CV force's deviation from the FP32 path on the same positions,
    and the NVE (gamma = 0, sigma = 1) energy drift over nve_steps steps of
    nve_walkers walkers."""
    wl = I.workload("chain_n100_w8192")
    sp, x0, ens = make_inputs(wl, seed)
    W = wl["n_walkers"]
    ens.trust_lo, ens.trust_hi = 1e9, 2e9
    res = {"workload": f"{W} walkers, {wl['n_beads']}-bead chain, {wl['n_cv']} torsion CVs, {wl['n_models']} x MLP "
                       f"{2 * wl['n_cv']}-{wl['width']}x{wl['n_layers']}-1; state and MLP scratch exceed L2"}
    xd = torch.from_numpy(x0).cuda()
    stream = torch.cuda.current_stream()
    grads = {}
    sample = {"seed": seed, "walkers": 16, "gpu": {}}
    flops = mlp_flops_per_walker_step(wl) * W
    mlp_ms = {}
    for name, prec in (("fp32", rid.RID_PREC_FP32), ("bf16", rid.RID_PREC_BF16), ("fp8", rid.RID_PREC_FP8)):
        with rid.System(sp) as system:
            system.set_ensemble(ens, precision=prec)
            g = torch.zeros((wl["n_models"], W, wl["n_cv"]), dtype=torch.float32, device="cuda")
            ee = torch.zeros(W, dtype=torch.float32, device="cuda")
            system.eval_forces(xd, rid.RID_BIAS_ENSEMBLE, grad_out=g, eps_out=ee, stream=stream)
            grads[name] = g.mean(dim=0).double()
            sample["gpu"][name] = (grads[name][:16].cpu().numpy(), ee[:16].double().cpu().numpy())
            system.walkers_load(xd, stream=stream)
            system.walkers_advance(3, stream=stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            system.walkers_advance(steps, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            system.profile_enable(True)
            system.walkers_advance(steps, stream=stream)
            torch.cuda.synchronize()
            prof = system.profile_read()
            system.profile_enable(False)
            mlp = "k_mlp_tc" if prec != rid.RID_PREC_FP32 else "k_mlp_fp32"
            mlp_ms[name] = prof[mlp][0] / prof[mlp][1]
            system.walkers_read()
        # NVE drift: gamma = 0, bias on with sigma = 1 (a conservative force)
        spn = I.make_system(wl["n_beads"], wl["n_cv"], seed, output_freq=nve_steps // 100, gamma=0.0)
        with rid.System(spn) as system:
            system.set_ensemble(ens, precision=prec)
            T = nve_steps // spn.output_freq
            en = np.zeros((nve_walkers, T, 3))
            v0 = np.zeros((nve_walkers, wl["n_beads"], 3), np.float32)
            system.explore(x0[:nve_walkers], nve_steps, v0=v0, energy_out=en)
            e = en.sum(axis=2)
            drift = np.abs(e - e[:, :1]).max(axis=1) / (3 * wl["n_beads"] * spn.kT)
        res[name] = {"value": W * steps / (ms / 1e3), "unit": "walker-steps/s", "ms_per_step": ms / steps,
                     "nve_drift_max_over_3NkT": float(drift.max()), "nve_drift_mean_over_3NkT": float(drift.mean()),
                     "nve": f"{nve_walkers} walkers x {nve_steps} steps, dt = {spn.dt}, energy sampled every "
                            f"{spn.output_freq} steps"}
    for name in ("bf16", "fp8"):
        d = (grads[name] - grads["fp32"]).norm(dim=1) / grads["fp32"].norm(dim=1).clamp_min(1e-30)
        res[name]["mean_force_rel_dev_from_fp32"] = {"median": float(d.median()), "max": float(d.max())}
        res[name]["roofline"] = tensor_roofline(flops, mlp_ms[name], fp8_forward=name == "fp8")
    fp = fp32_peak(torch)[0]
    res["fp32"]["roofline"] = {"bound": "alu", "kernel": "k_mlp_fp32", "achieved": flops / (mlp_ms["fp32"] / 1e3) / 1e12,
                               "peak": fp, "unit": "TFLOP/s", "frac": flops / (mlp_ms["fp32"] / 1e3) / 1e12 / fp,
                               "avg_launch_ms": mlp_ms["fp32"]}
    res["fp8"]["arithmetic"] = "forward GEMMs e4m3 (weights / (amax/448) per matrix), input-gradient GEMMs BF16"
    res["_sample"] = sample
    return res


def _timed_steps(torch, system, xd, stream, steps, flush):
    """Walker-steps timing of `steps` full steps (each alone between CUDA
    events, L2 flushed before it) and the per-kernel live times."""
    system.walkers_load(xd, stream=stream)
    system.walkers_advance(3, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        system.walkers_advance(1, stream=stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    system.profile_enable(True)
    for k in range(steps):
        flush.zero_()
        system.walkers_advance(1, stream=stream)
    torch.cuda.synchronize()
    prof = system.profile_read()
    system.profile_enable(False)
    system.walkers_read()
    return ms, {k: v[0] / v[1] for k, v in prof.items()}


def tensor_roofline(flops, ms, fp8_forward=False):
    """Ensemble kernel against its tensor peak.  FP8 mode: the forward GEMMs
    (half the work) run e4m3 at twice the BF16 rate (the nominal 4.5 : 2.25
    PFLOP/s ratio applied to the measured BF16 peak), the input-gradient GEMMs
    BF16, so the peak is flops / (flops/2 / (2 P) + flops/2 / P) = 4/3 P."""
    p16 = _peaks().get("bf16_tflops") or 1900.0
    src = "measured bf16_tflops (burst)" if _peaks().get("bf16_tflops") else "fallback 1.9 PFLOP/s"
    peak = p16 * 4.0 / 3.0 if fp8_forward else p16
    if fp8_forward:
        src += " x 4/3 (forward half at 2x for e4m3, nominal ratio)"
    ach = flops / (ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "k_mlp_tc", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "avg_launch_ms": ms, "peak_source": src}


def run_paper_network(rid, torch, steps, seed=21):
    """The paper's own ensemble (Sec. "Training phase": four models, neurons
    [300, 300, 300, 300], resnet) on 18 torsion CVs (its chignolin example's
    count) of the 200-bead chain: 1024 walkers, FP32 / BF16 / FP8 steps timed
    like the headline, the ensemble kernel's roofline at this shape, the
    deviation of BF16 / FP8 from FP32, and the step time at the paper's 12
    walkers."""
    C, M, L, H = 18, 4, 4, 300
    sp = I.make_system(200, C, seed, output_freq=10)
    W = 1024
    x0 = I.make_chains(W, sp, seed)
    ens = I.make_ensemble(M, 2 * C, L, H, seed, resnet=True)
    stream = torch.cuda.current_stream()
    xd = torch.from_numpy(x0).cuda()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    flops = M * 4 * (2 * C * H + (L - 1) * H * H) * W
    res = {"workload": f"{W} walkers, 200-bead chain, {C} torsion CVs, {M} x MLP {2 * C}-{H}x{L}-1 with residual "
                       f"connections (the paper's network)"}
    grads = {}
    for name, prec in (("fp32", rid.RID_PREC_FP32), ("bf16", rid.RID_PREC_BF16), ("fp8", rid.RID_PREC_FP8)):
        with rid.System(sp) as system:
            system.set_ensemble(ens, precision=prec)
            g = torch.zeros((M, W, C), dtype=torch.float32, device="cuda")
            system.eval_forces(xd, rid.RID_BIAS_ENSEMBLE, grad_out=g, stream=stream)
            grads[name] = g.mean(dim=0).double()
            ms, kern = _timed_steps(torch, system, xd, stream, steps, flush)
            r = {"value": W * steps / (ms / 1e3), "unit": "walker-steps/s", "ms_per_step": ms / steps,
                 "kernels_ms": kern}
            if name != "fp32":
                r["roofline"] = tensor_roofline(flops, kern["k_mlp_tc"], fp8_forward=name == "fp8")
                r["mlp_kernel"] = mlp_kernel_desc(system)
            res[name] = r
        if name == "bf16":
            # the paper's walker count: step latency
            with rid.System(sp) as system:
                system.set_ensemble(ens, precision=prec)
                x12 = xd[:12].contiguous()
                ms12, kern12 = _timed_steps(torch, system, x12, stream, steps, flush)
                res["bf16_12_walkers"] = {"ms_per_step": ms12 / steps, "kernels_ms": kern12,
                                          "mlp_kernel": mlp_kernel_desc(system, 12)}
            res["bf16_12_walkers_ms_per_step"] = ms12 / steps
    for name in ("bf16", "fp8"):
        d = (grads[name] - grads["fp32"]).norm(dim=1) / grads["fp32"].norm(dim=1).clamp_min(1e-30)
        res[name]["mean_force_rel_dev_from_fp32"] = {"median": float(d.median()), "max": float(d.max())}
    res["bf16_speedup_vs_fp32"] = res["bf16"]["value"] / res["fp32"]["value"]
    return res


def mlp_kernel_desc(system, walkers=None, bf16=True):
    """The tensor-core ensemble kernel variant of the system's last launch
    (BF16 ensembles at up to 16 walkers run the small-batch kernel)."""
    cs = system.mlp_cluster()
    if cs == 0:
        return "FP32 SIMT (k_mlp_fp32)"
    if walkers is not None and walkers <= 16 and bf16:
        return f"k_mlp_tc_small: GEMMs transposed, 128-output tiles over clusters of {cs} CTAs per member"
    if cs == 1:
        return "k_mlp_tc: one CTA per 128-walker tile and member"
    return f"k_mlp_tc_cluster: clusters of {cs} CTAs per 128-walker tile and member"


def run_tiny(rid, torch, seed=1):
    """The small configuration (22-bead chain, 2 torsion CVs, 4 x MLP
    4-64x3-1, FP32): 16 biased walkers x 2000 steps through one rid_explore
    call and 16 restrained runs (kappa 50) x 1000 steps through one rid_label
    call, device buffers, timed with CUDA events around each call."""
    wl = I.workload("tiny_n22")
    sp = I.make_system(wl["n_beads"], wl["n_cv"], seed, output_freq=10)
    W = 16
    x0 = torch.from_numpy(I.make_chains(W, sp, seed)).cuda()
    ens = I.make_ensemble(wl["n_models"], 2 * wl["n_cv"], wl["n_layers"], wl["width"], seed)
    stream = torch.cuda.current_stream()
    out = {"workload": "tiny_n22: 22-bead chain, 2 torsion CVs, 4 x MLP 4-64x3-1 (FP32); 16 walkers x 2000 "
                       "biased steps and 16 restrained runs x 1000 steps"}
    with rid.System(sp) as system:
        system.set_ensemble(ens, precision=rid.RID_PREC_FP32)
        T = 2000 // sp.output_freq
        cv = torch.zeros((W, T, wl["n_cv"]), device="cuda")
        eps = torch.zeros((W, T), device="cuda")
        s0 = torch.from_numpy(I.make_label_targets(W, wl["n_cv"], seed)).cuda()
        kap = torch.full((W, wl["n_cv"]), 50.0, dtype=torch.float64, device="cuda")
        mf, se, sd = (torch.zeros((W, wl["n_cv"]), dtype=torch.float64, device="cuda") for _ in range(3))
        for rep in range(2):          # the first call of each kind warms up
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            system.explore(x0, 2000, cv_out=cv, eps_out=eps, stream=stream)
            e1.record(stream)
            system.label(x0, s0, kap, 1000, 100, 20, mf, se, sd, stream=stream)
            e2.record(stream)
            torch.cuda.synchronize()
        out["explore"] = {"value": W * 2000 / (e0.elapsed_time(e1) / 1e3), "unit": "walker-steps/s",
                          "ms_per_call": e0.elapsed_time(e1)}
        out["label"] = {"value": W * 1000 / (e1.elapsed_time(e2) / 1e3), "unit": "walker-steps/s",
                        "ms_per_call": e1.elapsed_time(e2)}
    return out


def cpu_configs(precision_sample):
    """The oracle on the host cores for the small configuration (all of it) and
    on a sample of the precision sweep's workload, plus the precision sweep's
    errors against the oracle on that sample (the GPU mean forces and model
    deviations of its first walkers, passed in)."""
    import oracle
    oracle.build()
    out = {}
    wl = I.workload("tiny_n22")
    sp = I.make_system(wl["n_beads"], wl["n_cv"], 1, output_freq=10)
    x0 = I.make_chains(16, sp, 1)
    ens = I.make_ensemble(wl["n_models"], 2 * wl["n_cv"], wl["n_layers"], wl["width"], 1)
    t0 = time.perf_counter()
    r = oracle.explore(sp, x0, 2000, ens=ens)
    t1 = time.perf_counter()
    oracle.label(sp, x0, I.make_label_targets(16, wl["n_cv"], 1), 50.0, 1000, 100, 20)
    t2 = time.perf_counter()
    out["tiny_n22"] = {"explore": {"value": 16 * 2000 / (t1 - t0), "unit": "walker-steps/s"},
                       "label": {"value": 16 * 1000 / (t2 - t1), "unit": "walker-steps/s"},
                       "cores": int(r["threads"]), "sample": "all of it: 16 walkers x 2000 steps, 16 runs x 1000"}
    if precision_sample is not None:
        wl4 = I.workload("chain_n100_w8192")
        sp4, x4, ens4 = make_inputs(wl4, precision_sample["seed"])
        ens4.trust_lo, ens4.trust_hi = 1e9, 2e9
        n = precision_sample["walkers"]
        t0 = time.perf_counter()
        r = oracle.explore(sp4, x4[:64], 4, ens=ens4)
        dt = time.perf_counter() - t0
        out["chain_n100_w8192"] = {"value": 64 * 4 / dt, "unit": "walker-steps/s", "cores": int(r["threads"]),
                                   "sample": "64 walkers x 4 steps"}
        errs = {}
        ref_f, ref_e = [], []
        for w in range(n):
            e = oracle.ensemble(ens4, oracle.cvs(sp4, x4[w].astype(np.float64))[0])
            ref_f.append(e["gradA"].mean(axis=0))
            ref_e.append(e["eps"])
        ref_f, ref_e = np.array(ref_f), np.array(ref_e)
        for name, (fbar, eps) in precision_sample["gpu"].items():
            d = np.linalg.norm(fbar - ref_f, axis=1) / np.linalg.norm(ref_f, axis=1)
            de = np.abs(eps - ref_e) / np.abs(ref_e)
            errs[name] = {"mean_force_rel_err": {"median": float(np.median(d)), "max": float(d.max())},
                          "eps_rel_err": {"median": float(np.median(de)), "max": float(de.max())}}
        out["precision_errors_vs_oracle"] = dict(errs, sample=f"the first {n} walkers of the precision sweep, "
                                                                "FP64 oracle at the same positions")
    return out


def rank_seed(rank):
    """Every rank runs its own walkers: seed of the inputs of `rank`."""
    return 1 + rank


def max_over_ranks(pg, x, device):
    """Largest x over all ranks (the job's time is its slowest rank's)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(walkers_per_rank, world, steps, seconds):
    """Walker-steps of all ranks per second of the slowest rank."""
    return walkers_per_rank * world * steps / seconds


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return
    wl = I.workload(WORKLOAD)
    sp, x0, ens = make_inputs(wl)
    import oracle
    oracle.build()
    walkers, md = 64, 4
    for _ in range(args.warmup):
        oracle.explore(sp, x0[:walkers], 1, ens=ens)
    times = []
    threads = 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.explore(sp, x0[walkers * (k % 8):walkers * (k % 8 + 1)], md, ens=ens)
        times.append(time.perf_counter() - t0)
        threads = r["threads"]
    tot = sum(times)
    value = walkers * md * len(times) / tot
    sample = (f"{walkers} walkers x {md} MD steps per bench step (plus one initial force evaluation "
              f"each), FP64 oracle")
    out = {"metric": "biased MD walker-steps/s", "value": value, "unit": "walker-steps/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "description": workload_desc(wl)},
           "cpu_baseline": {"value": value, "unit": "walker-steps/s", "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "walker-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def legs_summary(out):
    """One short object at the end of the line with each leg's headline
    figures (the full legs precede it)."""
    def g(*path):
        v = out
        for k in path:
            if not isinstance(v, dict) or k not in v:
                return None
            v = v[k]
        return round(v, 4) if isinstance(v, float) and abs(v) < 10 else (round(v) if isinstance(v, float) else v)
    return {
        "headline": {"value": g("value"), "e2e": g("e2e", "value"), "ms_per_step": g("ms_per_step"),
                     "roofline": [g("roofline", "kernel"), g("roofline", "frac")]},
        "fp32_plain": {"fp32": g("fp32_plain", "fp32", "value"), "bf16": g("fp32_plain", "bf16", "value"),
                       "speedup": g("fp32_plain", "bf16_speedup_vs_fp32")},
        "paper_network": {p: [g("paper_network", p, "value"), g("paper_network", p, "roofline", "frac")]
                          for p in ("fp32", "bf16", "fp8")} | {"bf16_12_walkers_ms": g("paper_network",
                                                                                            "bf16_12_walkers_ms_per_step")},
        "precision": {p: [g("precision", p, "value"), g("precision", p, "roofline", "frac"),
                          g("cpu_baseline", "configs", "precision_errors_vs_oracle", p, "mean_force_rel_err", "max")]
                      for p in ("fp32", "bf16", "fp8")},
        "tiny": [g("tiny", "explore", "value"), g("tiny", "label", "value")],
        "batching": g("batching", "value"),
        "training": g("training", "value"),
        "mcmc": [g("mcmc", "value"), g("mcmc", "bf16_tensor_cores", "value")],
        "constrained": g("constrained", "value"),
        "selection_ms": g("selection", "wall_ms"),
        "serving": {"tput": g("serving", "throughput"), "label_p99_ms": g("serving", "label_latency_ms", "p99"),
                    "plain_label_p99_ms": g("serving", "plain_per_job", "label_latency_ms", "p99")},
        "serving_sustained": {"tput": g("serving_sustained", "throughput"),
                              "req_s": g("serving_sustained", "requests_per_s"),
                              "label_p50_ms": g("serving_sustained", "label_latency_ms", "p50"),
                              "label_p99_ms": g("serving_sustained", "label_latency_ms", "p99")},
        "cpu": [g("cpu_baseline", "value"), g("cpu_baseline", "cores")],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--e2e-calls", type=int, default=20)
    ap.add_argument("--e2e-md-steps", type=int, default=20)
    ap.add_argument("--cpu-walkers", type=int, default=1024)
    ap.add_argument("--cpu-steps", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-jobs", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=2000)
    ap.add_argument("--batch-plain-jobs", type=int, default=24)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-plain-requests", type=int, default=24)
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-fp32-plain", action="store_true")
    ap.add_argument("--no-training", action="store_true")
    ap.add_argument("--train-steps", type=int, default=400)
    ap.add_argument("--no-mcmc", action="store_true")
    ap.add_argument("--no-selection", action="store_true")
    ap.add_argument("--no-constrained", action="store_true")
    ap.add_argument("--cons-runs", type=int, default=1024)
    ap.add_argument("--cons-steps", type=int, default=1000)
    ap.add_argument("--mcmc-steps", type=int, default=500)
    ap.add_argument("--mlp-cluster", type=int, default=0,
                    help="cluster size of the tensor-core ensemble kernel (0: tuned by the library)")
    ap.add_argument("--ff-threads", type=int, default=0,
                    help="CTA size of the force-field kernel (0: tuned by the library)")
    ap.add_argument("--no-paper-net", action="store_true")
    ap.add_argument("--no-tiny", action="store_true")
    ap.add_argument("--serve-sustained-rate", type=float, default=50.0)
    ap.add_argument("--serve-sustained-requests", type=int, default=200)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    from paper_2408_14070_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if pg:
        pg.barrier()
    from paper_2408_14070_gb300 import rid

    wl = I.workload(WORKLOAD)
    W = wl["n_walkers"]
    sp, x0, ens = make_inputs(wl, seed=rank_seed(rank))
    prec = rid.RID_PREC_BF16 if args.precision == "bf16" else rid.RID_PREC_FP32
    stream = torch.cuda.current_stream()
    system = rid.System(sp)
    system.set_ensemble(ens, precision=prec)
    system.set_mlp_cluster(args.mlp_cluster)
    system.set_ff_threads(args.ff_threads)
    xd = torch.from_numpy(x0).cuda()
    system.walkers_load(xd, stream=stream)
    system.walkers_advance(args.warmup, stream=stream)
    torch.cuda.synchronize()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2

    # ---- timed region: K steps, each bracketed by events, L2 flushed before each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    l0 = system.launch_count()
    with ClockSampler(local) as clk:
        clk.wait_first()
        t_start = time.monotonic()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            system.walkers_advance(1, stream=stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clk.mark(t_start, time.monotonic())
    launches = system.launch_count() - l0
    if pg:
        pg.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = max_over_ranks(pg, sum(step_ms), "cuda")
    system.walkers_read()   # raises on non-finite state
    value = whole_job_rate(W, world, args.steps, tot_ms / 1e3)

    # ---- per-kernel timing over the same kind of region (dominant kernel roofline)
    system.profile_enable(True)
    for k in range(args.steps):
        flush.zero_()
        system.walkers_advance(1, stream=stream)
    torch.cuda.synchronize()
    prof = system.profile_read()
    system.profile_enable(False)
    top = max(prof, key=lambda k: prof[k][0])
    avg_ms = prof[top][0] / prof[top][1]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    tkey = top
    if top == "k_mlp_tc":
        # the variant the tuner kept names the source and the traffic record
        tkey = "k_mlp_tc" if system.mlp_cluster() == 1 else "k_mlp_tc_cluster"
        work, src = mlp_flops_per_walker_step(wl) * W, tkey + ".cu"
        peak = peaks.get("bf16_tflops")
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": peak if peak else 1900.0,
                "peak_source": "measured bf16_tflops (burst)" if peak else "fallback 1.9 PFLOP/s bf16"}
        achieved = work / (avg_ms / 1e3) / 1e12
    elif top == "k_mlp_fp32":
        work, src = mlp_flops_per_walker_step(wl) * W, "k_mlp_fp32.cu"
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": fp32_peak(torch)[0], "peak_source": fp32_peak(torch)[1]}
        achieved = work / (avg_ms / 1e3) / 1e12
    elif top == "k_head":
        # integrator: read x, v, f and write x, v (12 B each) per bead
        work, src = 60 * wl["n_beads"] * W, "k_step.cu"
        peak = peaks.get("hbm_gbs")
        roof = {"bound": "hbm", "unit": "GB/s", "peak": peak if peak else 6800.0,
                "peak_source": "measured hbm_gbs" if peak else "fallback 6.8 TB/s"}
        achieved = work / (avg_ms / 1e3) / 1e9
    else:
        work, src = pair_flops_per_walker_step(wl) * W, "k_step.cu"
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": fp32_peak(torch)[0], "peak_source": fp32_peak(torch)[1]}
        achieved = work / (avg_ms / 1e3) / 1e12
    roofline = {"kernel": top, "bound": roof["bound"], "achieved": achieved, "peak": roof["peak"],
                "unit": roof["unit"], "frac": achieved / roof["peak"] if roof["peak"] else None,
                "traffic": traffic_for(tkey, src, WORKLOAD), "work_per_launch": work, "source": src,
                "avg_launch_ms": avg_ms, "peak_source": roof["peak_source"],
                "kernels": {k: {"total_ms": v[0], "launches": v[1], "share": v[0] / sum(x[0] for x in prof.values())}
                            for k, v in prof.items()}}

    # ---- end to end through the public C ABI with pinned host buffers
    md = args.e2e_md_steps
    T = md // sp.output_freq
    hx = torch.from_numpy(x0).pin_memory()
    hv = torch.zeros_like(hx).pin_memory()
    system.walkers_load(xd, stream=stream)
    system.walkers_advance(5, stream=stream)
    system.walkers_read(x_out=hx.numpy(), v_out=hv.numpy())
    ocv = torch.zeros((W, T, sp.n_cv), dtype=torch.float32).pin_memory()
    oeps = torch.zeros((W, T), dtype=torch.float32).pin_memory()
    ox = torch.zeros_like(hx).pin_memory()
    ov = torch.zeros_like(hx).pin_memory()
    h2d = hx.numel() * 4 * 2
    d2h = (ox.numel() + ov.numel() + ocv.numel() + oeps.numel()) * 4
    system.explore(hx, md, v0=hv, cv_out=ocv, eps_out=oeps, x_out=ox, v_out=ov, stream=stream)   # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(args.e2e_calls):
        system.explore(hx, md, v0=hv, step0=md * (c + 1), cv_out=ocv, eps_out=oeps, x_out=ox, v_out=ov,
                       stream=stream)
        hx, ox = ox, hx
        hv, ov = ov, hv
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(pg, time.perf_counter() - t0, "cuda")
    e2e = {"value": whole_job_rate(W, world, md * args.e2e_calls, e2e_s), "unit": "walker-steps/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "step": f"one rid_explore call from pinned host buffers: {md} MD steps of all walkers, "
                   f"initial force evaluation, CV/eps trace every {sp.output_freq} steps, final x and v"}

    out = {"metric": "biased MD walker-steps/s", "value": value, "unit": "walker-steps/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16" if prec == rid.RID_PREC_BF16 else "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "description": workload_desc(wl), "walkers_per_gpu": W,
                      "n_beads": wl["n_beads"], "n_cv": wl["n_cv"], "ensemble": f"{wl['n_models']}x"
                      f"[{2 * wl['n_cv']}-{wl['width']}x{wl['n_layers']}-1]",
                      "mlp_precision": args.precision, "forces_integrator": "f32",
                      "mlp_kernel": mlp_kernel_desc(system), "ff_cta_threads": system.ff_threads(),
                      "l2": "flushed (256 MiB write) before every timed step; each step timed alone",
                      "parallelism": f"walkers sharded, {world} independent rank(s)"},
           "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(),
           "fp32_peak": {"value": fp32_peak(torch)[0], "unit": "TFLOP/s", "source": fp32_peak(torch)[1]}}
    if rank == 0 and world == 1 and not args.no_fp32_plain:
        out["fp32_plain"] = run_fp32_plain(rid, torch, args.steps)
    if rank == 0 and world == 1 and not args.no_paper_net:
        out["paper_network"] = run_paper_network(rid, torch, args.steps)
    if rank == 0 and world == 1 and not args.no_tiny:
        out["tiny"] = run_tiny(rid, torch)
    if rank == 0 and world == 1 and not args.no_batching:
        out["batching"] = run_batching(rid, args.batch_jobs, args.batch_steps, args.batch_plain_jobs)
    if rank == 0 and world == 1 and not args.no_precision:
        out["precision"] = run_precision(rid, torch)
    if rank == 0 and world == 1 and not args.no_training:
        out["training"] = run_training(rid, torch, args.train_steps)
    if rank == 0 and world == 1 and not args.no_constrained:
        out["constrained"] = run_constrained(rid, torch, args.cons_runs, args.cons_steps)
    if rank == 0 and world == 1 and not args.no_selection:
        out["selection"] = run_selection(rid, torch)
    if rank == 0 and world == 1 and not args.no_mcmc:
        out["mcmc"] = run_mcmc(rid, torch, args.mcmc_steps)
    if rank == 0 and world == 1 and not args.no_serving:
        out["serving"] = run_serving(rid, args.serve_requests, args.serve_rate, args.serve_plain_requests)
        if args.serve_sustained_rate > 0:
            out["serving_sustained"] = run_serving(rid, args.serve_sustained_requests, args.serve_sustained_rate, 0,
                                                   seed=7)
    sample = out["precision"].pop("_sample", None) if "precision" in out else None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sp, x0, ens, args.cpu_walkers, args.cpu_steps)
        out["cpu_baseline"]["configs"] = cpu_configs(sample)
    if rank == 0:
        out["legs"] = legs_summary(out)
        print(json.dumps(out))
    system.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
