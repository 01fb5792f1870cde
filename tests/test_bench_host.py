"""Host-side checks of the benchmark's roofline arithmetic (no GPU).

The bench line reports, for each timed kernel, algorithmic work per launch over its
measured duration against a peak, and, from counters of ncu captures kept in bench.py,
the issued instructions and DRAM traffic.  These tests pin that arithmetic and check that
the kept counters belong to the kernel sources as they stand (a kernel changed after its
capture must report no counters rather than stale ones).
"""
import bench
import workloads


def test_counters_belong_to_the_current_kernel_sources():
    fp = bench._kernel_fingerprint()
    assert bench.COUNTERS, "no counters kept"
    for key, (stamp, traffic, inst) in bench.COUNTERS.items():
        assert stamp == fp, f"counters of {key} were taken on other kernel sources"
        assert inst > 0 and (traffic is None or traffic > 0)


def test_stale_counters_are_not_reported(monkeypatch):
    monkeypatch.setattr(bench, "_kernel_fingerprint", lambda: "not-the-captured-sources")
    assert bench._counter("double_well", "fwd_pair", "inst") is None
    assert bench._counter("double_well", "adj_stored", "traffic") is None


def test_stored_adjoint_hbm_roofline_arithmetic():
    p = workloads.double_well(M=1 << 20, Nt=1000)
    peaks = {"hbm_gbs": 6785.2, "sm_max_mhz": 2070.0}
    ms = 2.66
    r = bench.kernel_roofline("adj_stored", (3, 3 * ms), p, peaks, "measured")
    # states (4 d bytes), one flag bit, and the jump log (lambda dt records of 2 + d words)
    per = 4 * p.d + 0.125 + p.lam * p.dt * (2 + p.d) * 4
    assert abs(r["algorithmic_bytes_per_path_step"] - per) < 1e-12
    achieved = per * p.M * p.Nt / (ms * 1e-3) / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - achieved) < 1e-6 * achieved
    assert abs(r["frac"] - achieved / 6785.2) < 1e-12
    inst = bench._counter("double_well", "adj_stored", "inst")
    if inst is not None:   # issue fraction: warp-instructions per second against the issue peak
        iss = r["issue"]
        assert abs(iss["achieved_warp_inst_per_s"] - inst * p.M * p.Nt / 32 / (ms * 1e-3)) < 1.0
        assert abs(iss["frac"] - iss["achieved_warp_inst_per_s"] / iss["peak_warp_inst_per_s"]) < 1e-12


def test_forward_lane_operation_model():
    p = workloads.double_well(M=1 << 20, Nt=1000)
    # d = 2 double well, one control: draws 40 (one Philox block) + 6 (two uniforms) + 7
    # (one Box-Muller pair) + 1 (Poisson test) = 54; arithmetic 14 (A x, B u, cubic term) +
    # 4 (Euler update) + 6 + 4 (running cost) = 28; a jump, at lambda dt = 0.01, costs
    # 80 (two slot blocks) + 12 + 14 + 2 x 10 = 126: 54 + 28 + 1.26 = 83.26
    single = bench.forward_ops(p)
    pair = bench.forward_ops(p, controls=2)
    assert abs(single - 83.26) < 1e-9
    assert abs(pair - 111.46) < 1e-9
    # the second control adds its own arithmetic but shares the draws
    assert single < pair < 2 * single


def test_forward_roofline_reports_the_issue_fraction_only_for_captured_kernels():
    peaks = {"hbm_gbs": 6785.2, "sm_max_mhz": 2070.0}
    p = workloads.double_well(M=1 << 20, Nt=1000)
    r = bench.kernel_roofline("fwd_pair", (1, 11.68), p, peaks, "measured", 0, "stored")
    assert r["bound"] == "alu" and r["frac"] < 1.0
    if bench._counter("double_well", "fwd_pair", "inst") is not None:
        assert "issue" in r and r["traffic"] > 0
    # the paired sweep of the recompute plan is a different kernel (checkpoint mode): no counters
    r2 = bench.kernel_roofline("fwd_pair", (1, 9.78), p, peaks, "measured", 0, "recompute")
    assert "issue" not in r2 and r2["traffic"] is None
