"""Host logic of bench.py on CPU: the algorithmic work per unit behind the
roofline figures (against the counts written out from their definitions), the
roofline arithmetic, the clock record taken during the timed region, the DRAM
traffic lookup keyed by kernel source, and the summary at the end of the line."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def B():
    import bench
    return bench


def test_pair_work_counts_every_unique_non_excluded_pair(B):
    # pairs (i, j), i < j, with |i - j| > 2, counted one by one; 20 flop each
    for N in (4, 5, 22, 200):
        pairs = sum(1 for i in range(N) for j in range(i + 3, N))
        assert B.pair_flops_per_walker_step({"n_beads": N}) == 20 * pairs
    # 399.4 MFLOP per launch at 1024 walkers of the 200-bead chain
    assert 1024 * B.pair_flops_per_walker_step({"n_beads": 200}) == pytest.approx(399.4e6, rel=1e-4)


def test_ensemble_work_counts_forward_and_input_gradient_gemms(B):
    # per member: forward D*H + (L-1)*H^2 multiply-adds, the input gradient
    # the same again; 2 flop each
    for D, H, L, M in ((40, 256, 4, 4), (36, 300, 4, 4), (4, 64, 3, 4), (64, 512, 4, 8)):
        layers = [D] + [H] * L
        macs = sum(layers[k] * layers[k + 1] for k in range(L))
        wl = {"n_cv": D // 2, "width": H, "n_layers": L, "n_models": M}
        assert B.mlp_flops_per_walker_step(wl) == M * 2 * 2 * macs
    wl = {"n_cv": 20, "width": 256, "n_layers": 4, "n_models": 4}
    assert 1024 * B.mlp_flops_per_walker_step(wl) == pytest.approx(3.389e9, rel=1e-3)


def test_training_work_per_sample(B):
    # 2.46 MFLOP per sample and member for 40-256x4-1
    assert B.train_flops_per_sample(40, 4, 256) == 2461696
    # one hidden layer: no pass back through hidden-to-hidden layers
    assert B.train_flops_per_sample(8, 1, 16) == 10 * 8 * 16


def test_tensor_roofline_arithmetic(B, monkeypatch):
    monkeypatch.setattr(B, "_peaks", lambda: {"bf16_tflops": 2000.0})
    r = B.tensor_roofline(3.0e9, 0.0015)          # 3 GFLOP in 1.5 ms = 2 PFLOP/s
    assert r["achieved"] == pytest.approx(2000.0) and r["frac"] == pytest.approx(1.0)
    assert r["peak_source"].startswith("measured")
    f = B.tensor_roofline(3.0e9, 0.0015, fp8_forward=True)
    # half the work at twice the rate: time-weighted peak 4/3 of BF16's
    assert f["peak"] == pytest.approx(2000.0 * 4 / 3)
    assert 1.5e9 / (2 * 2000e12) + 1.5e9 / 2000e12 == pytest.approx(3.0e9 / (f["peak"] * 1e12))
    monkeypatch.setattr(B, "_peaks", lambda: {})
    assert B.tensor_roofline(1.9e9, 1.0)["peak_source"].startswith("fallback")


def _sampler(B, lines, window):
    s = B.ClockSampler(0)
    s.lines = lines
    if window is not None:
        s.mark(*window)
    return s


def test_clock_record_keeps_samples_of_the_timed_region(B):
    row = "{sm}, 2070, 900.5, {hw}, Not Active, Not Active, {pc}"
    lines = [(0.0, row.format(sm=1000, hw="Active", pc="Not Active")),      # before the region
             (1.0, row.format(sm=2070, hw="Not Active", pc="Not Active")),
             (1.1, row.format(sm=2040, hw="Not Active", pc="Active")),
             (1.2, row.format(sm=2055, hw="Not Active", pc="Not Active")),
             (1.25, "garbled"),
             (1.3, "[N/A], 2070, 1, Not Active, Not Active, Not Active, Not Active"),
             (3.0, row.format(sm=500, hw="Active", pc="Not Active"))]        # after it
    s = _sampler(B, lines, (1.0, 1.2)).summary()
    assert s == {"sm_mhz": 2055, "sm_max_mhz": 2070, "reasons": ["sw_power_cap"], "samples": 3}
    # a region shorter than the sampling period takes the sample nearest its middle
    s = _sampler(B, lines, (2.8, 2.81)).summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 500 and s["reasons"] == ["hw_slowdown"]
    # ... the nearest sample that parses: not the unreadable one at 1.3
    s = _sampler(B, lines, (1.6, 1.61)).summary()
    assert s == {"sm_mhz": 2055, "sm_max_mhz": 2070, "reasons": [], "samples": 1}
    assert _sampler(B, [], (0, 1)).summary()["sm_mhz"] is None


def test_traffic_is_reported_only_for_the_source_it_was_taken_on(B, monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    key = next(k for k in rec if k.startswith("k_mlp_tc@"))
    kernel, workload = key.split("@")
    src = "k_mlp_tc.cu"
    monkeypatch.setattr(B, "kernel_source_hash", lambda name: rec[key]["source_sha256_16"])
    assert B.traffic_for(kernel, src, workload) == rec[key]["bytes_per_launch"]
    monkeypatch.setattr(B, "kernel_source_hash", lambda name: "0" * 16)
    assert B.traffic_for(kernel, src, workload) is None
    assert B.traffic_for("no_such_kernel", src, workload) is None


def test_every_traffic_record_names_its_summary_and_source(B):
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    for key, r in rec.items():
        kernel, workload = key.split("@")
        assert os.path.isfile(os.path.join(ROOT, r["from"])), key
        assert kernel in open(os.path.join(ROOT, r["from"])).read(), key
        assert len(r["source_sha256_16"]) == 16 and r["bytes_per_launch"] > 0, key


def test_rate_over_ranks_and_summary_of_the_line(B):
    assert B.whole_job_rate(1024, 4, 20, 0.5) == 1024 * 4 * 20 / 0.5
    out = {"value": 19155310.2, "e2e": {"value": 17342928.0}, "ms_per_step": 0.0535,
           "roofline": {"kernel": "k_mlp_tc", "frac": 0.042712},
           "serving": {"throughput": 2046016.0, "label_latency_ms": {"p99": 676.2}},
           "cpu_baseline": {"value": 11031.8, "cores": 16}}
    s = B.legs_summary(out)
    assert s["headline"] == {"value": 19155310, "e2e": 17342928, "ms_per_step": 0.0535,
                             "roofline": ["k_mlp_tc", 0.0427]}
    assert s["serving"]["tput"] == 2046016 and s["serving"]["label_p99_ms"] == 676
    assert s["serving"]["plain_label_p99_ms"] is None and s["batching"] is None
    assert s["cpu"] == [11032, 16]


def test_reference_arm_line_on_rank_zero(B, monkeypatch, capsys):
    """The reference arm times the oracle on the host cores and prints one
    JSON line with the primary arm's metric, unit and config."""
    for k, v in (("RANK", "0"), ("WORLD_SIZE", "1"), ("LOCAL_RANK", "0")):
        monkeypatch.setenv(k, v)

    class A:
        steps, warmup, gpus = 1, 0, 1
    B.run_reference(A())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "biased MD walker-steps/s"
    assert line["unit"] == "walker-steps/s" and line["higher_is_better"] is True
    assert line["config"]["workload"] == B.WORKLOAD and line["dtype"] == "f64"
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "walker-steps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
