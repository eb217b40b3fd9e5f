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

from paper_2408_14070_gb300 import inputs as I  # noqa: E402

WORKLOAD = "chain_n200_w1024"
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


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
        inside = [ln for t, ln in self.lines if lo - 0.1 <= t <= hi + 0.1]
        if not inside and self.lines:       # region shorter than the sampling period
            inside = [min(self.lines, key=lambda tl: abs(tl[0] - 0.5 * (lo + hi)))[1]]
        for ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
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
    sp, x0, ens = make_inputs(wl, seed=1 + rank)
    prec = rid.RID_PREC_BF16 if args.precision == "bf16" else rid.RID_PREC_FP32
    stream = torch.cuda.current_stream()
    system = rid.System(sp)
    system.set_ensemble(ens, precision=prec)
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
    tot_ms = sum(step_ms)
    if pg:
        t = torch.tensor([tot_ms], device="cuda", dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        tot_ms = float(t.item())
    system.walkers_read()   # raises on non-finite state
    value = W * world * args.steps / (tot_ms / 1e3)

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
    if top == "k_mlp_tc":
        work, src = mlp_flops_per_walker_step(wl) * W, "k_mlp_tc.cu"
        peak = peaks.get("bf16_tflops")
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": peak if peak else 1900.0,
                "peak_source": "measured bf16_tflops (burst)" if peak else "fallback 1.9 PFLOP/s bf16"}
        achieved = work / (avg_ms / 1e3) / 1e12
    elif top == "k_mlp_fp32":
        work, src = mlp_flops_per_walker_step(wl) * W, "k_mlp_fp32.cu"
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": FP32_PEAK_TFLOPS, "peak_source": f"derived: {FP32_PEAK_NOTE}"}
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
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": FP32_PEAK_TFLOPS, "peak_source": f"derived: {FP32_PEAK_NOTE}"}
        achieved = work / (avg_ms / 1e3) / 1e12
    roofline = {"kernel": top, "bound": roof["bound"], "achieved": achieved, "peak": roof["peak"],
                "unit": roof["unit"], "frac": achieved / roof["peak"] if roof["peak"] else None,
                "traffic": traffic_for(top, src, WORKLOAD), "work_per_launch": work,
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
    e2e_s = time.perf_counter() - t0
    if pg:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": W * world * md * args.e2e_calls / e2e_s, "unit": "walker-steps/s",
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
                      "l2": "flushed (256 MiB write) before every timed step; each step timed alone",
                      "parallelism": f"walkers sharded, {world} independent rank(s)"},
           "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sp, x0, ens, args.cpu_walkers, args.cpu_steps)
    if rank == 0:
        print(json.dumps(out))
    system.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
