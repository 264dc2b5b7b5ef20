"""Host logic of bench.py's roofline accounting (no GPU): the work counted
per sample for the one- and two-stage screens, and the binding resource."""
import bench


def _two_stage(nx, nt):
    """The rule the compiled kernels use for the split (integrand_kernels.cuh)."""
    d = nx * nt
    nq = (d + 3) // 4
    bp = (3 * nq + 4) // 5
    mc = min(4 * bp // nt, nx)
    return nq >= 3 and mc < nx and 20 * (mc - 2) >= 7 * nx


def test_screen_work_per_sample_10x2():
    # full screen: 5 Philox blocks x 10 rounds x 4, 20 points x 2, 20 residuals x 8
    assert bench.screen_ops(10, 2) == 200 + 40 + 160
    # stage 1: 3 blocks, the 12 coordinates of sites 0..5, the residuals of sites 1..4 over both slices
    assert bench.partial_ops(10, 2) == 120 + 24 + 64


def test_partial_work_is_a_fraction_of_the_full_screen_where_the_split_is_compiled():
    shapes = [(8, 2), (10, 2), (16, 2), (32, 2), (8, 4), (10, 4), (16, 4)]
    assert [s for s in [(2, 1), (3, 1), (4, 1), (2, 2), (3, 2), (4, 2), (6, 2), (8, 2), (10, 2), (16, 2), (32, 2),
                        (4, 4), (6, 4), (8, 4), (10, 4), (16, 4)] if _two_stage(*s)] == shapes
    for nx, nt in shapes:
        assert 0.4 < bench.partial_ops(nx, nt) / bench.screen_ops(nx, nt) < 0.75


def test_roofline_counts_stage_one_for_all_and_the_rest_for_survivors():
    n, n_eval, ms = 1 << 30, 1_750_000, 14.0
    one = bench.roofline(bench.one_stage_work(n, n_eval), ms, "fp64", 10, 2)
    two_w = {"samples": n, "stage1": n, "survivors": n // 5, "full_screen": 0, "evaluated": n_eval, "rest_screen": 1}
    two = bench.roofline(two_w, ms, "fp64", 10, 2)
    t = ms * 1e-3
    integer = bench.eval_ops_fp64(10, 2)[1]
    assert abs(one["achieved"] * 1e9 * t - (n * 400 + n_eval * integer)) < 1e3
    # a survivor draws blocks 0, 2, 3, 4 again: 160 + 32 points + the 12 residuals of sites 0 and 5..9
    assert bench.rest_ops(10, 2) == 160 + 32 + 96
    assert abs(two["achieved"] * 1e9 * t - (n * 208 + (n // 5) * 288 + n_eval * integer)) < 1e3
    assert two["survivors"] == n // 5 and one["full_screened"] == n and two["full_screened"] == 0
    assert one["bound"] == "alu" and one["resource"] == "FP32/INT issue"
    assert 0 < two["frac"] < one["frac"]


def test_roofline_of_mixed_chunks_and_full_survivor_screens():
    # a job whose last chunks are too short for stage 1, and survivors screened in full (mass2 != 0)
    w = {"samples": 1000, "stage1": 700, "survivors": 100, "full_screen": 300, "evaluated": 0, "rest_screen": 0}
    assert bench.screen_work(w, 10, 2) == 700 * 208 + 300 * 400 + 100 * 400
    w["rest_screen"] = 1
    assert bench.screen_work(w, 10, 2) == 700 * 208 + 300 * 400 + 100 * 288


def test_fp32_roofline_has_no_fp64_work():
    w = {"samples": 1 << 34, "stage1": 1 << 34, "survivors": 3_300_000_000, "full_screen": 0,
         "evaluated": 3_000_000, "rest_screen": 1}
    r = bench.roofline(w, 216.0, "fp32", 10, 2)
    assert r["fp64_frac"] == 0 and r["resource"] == "FP32/INT issue"


def test_traffic_is_reported_only_for_the_kernel_sources_it_was_measured_on(tmp_path, monkeypatch):
    f = tmp_path / "t.txt"
    f.write_text("# a summary\ndram_bytes_per_launch: 12345\nkernel_sources_sha256: " + bench.kernel_sources_sha256() +
                 "\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic()[0] == 12345
    f.write_text("dram_bytes_per_launch: 12345\nkernel_sources_sha256: 0000\n")
    assert bench.measured_traffic()[0] is None
    # keyed to the chunk size of the capture as well
    f.write_text("dram_bytes_per_launch: 12345\nchunk_samples: 262144\nkernel_sources_sha256: " +
                 bench.kernel_sources_sha256() + "\n")
    assert bench.measured_traffic(262144)[0] == 12345
    assert bench.measured_traffic(131072)[0] is None


def test_summary_is_short_and_last():
    roof = {"frac": 0.5}
    fp32 = {"value": 8e10, "roofline": {"frac": 0.53}, "vs_fp64_mode": {"Z_rel": 1e-6, "C_rel_to_C0": [1e-7, -2e-7]},
            "err_bound": {"Z_rel": 4e-7, "C_rel_to_C0": [5e-7, 6e-7]}}
    batch = {"value": 3e10, "roofline": {"frac": 0.4}, "ms_per_launch": 340.0}
    serving = {"rate": 200.0, "jobs": 2000, "p50_ms": 4000.0, "p99_ms": 8000.0, "samples_per_s": 1.6e10, "failed": 0,
               "roofline": {"frac": 0.3}}
    tte = {"samples_to_target_C_err_over_C0_max": 1.5e14, "seconds_to_target_C_err_over_C0_max": 1850.0}
    s = bench.summary(7.7e10, roof, {"value": 7.6e10}, fp32, batch, serving, tte)
    import json
    assert len(json.dumps({"summary": s})) < 1000
    assert s["fp32_err_bound_C"] == 6e-7 and s["fp32_vs_fp64_C_rel_max"] == 2e-7 and s["serving_frac"] == 0.3


def test_kernel_hash_follows_code_not_comments():
    src = {name: "// a\nint f(int x) { return x + 1; } /* b */\n" for name in bench.KERNEL_SOURCES}
    base = bench.kernel_sources_sha256(lambda n: src[n])
    commented = {n: t.replace("// a", "// another comment") + "\n\n// more\n" for n, t in src.items()}
    assert bench.kernel_sources_sha256(lambda n: commented[n]) == base
    changed = dict(src)
    changed[bench.KERNEL_SOURCES[0]] = src[bench.KERNEL_SOURCES[0]].replace("x + 1", "x + 2")
    assert bench.kernel_sources_sha256(lambda n: changed[n]) != base


def test_bench_jobs_have_one_box_per_budget_for_every_lattice(monkeypatch):
    """The bench's job for --lattice NXxNT: 1024 subvolumes whatever d is (the
    bisection cycles over the coordinates when d < 10), which partition
    [-5, 5]^d; the plan reads one box per budget."""
    import numpy as np
    for nx, nt in [(4, 2), (3, 1), (10, 2), (32, 4)]:
        monkeypatch.setattr(bench, "NX", nx)
        monkeypatch.setattr(bench, "NT", nt)
        monkeypatch.setattr(bench, "D", nx * nt)
        job = bench.make_job(0, 1, 1 << 10)
        d = nx * nt
        assert job.lo.shape == job.hi.shape == (1024, d) and job.samples.shape == (1024,)
        assert np.all(job.hi > job.lo) and np.all(job.lo >= -5.0) and np.all(job.hi <= 5.0)
        vol = np.prod(job.hi - job.lo, axis=1)
        assert abs(vol.sum() / 10.0 ** d - 1.0) < 1e-12 and len({tuple(r) for r in job.lo}) == 1024
        # disjoint: in every pair of boxes some coordinate's intervals do not overlap
        rng = np.random.default_rng(d)
        for a, b in rng.integers(0, 1024, (200, 2)):
            if a != b:
                assert np.any((job.hi[a] <= job.lo[b]) | (job.hi[b] <= job.lo[a]))


def test_clock_record_keeps_the_samples_inside_the_timed_region():
    """nvidia-smi lines (timestamp first): the record's median clock and
    throttle reasons come from the samples inside the timed region only, and
    fall back to all samples, flagged, when none falls inside."""
    import datetime
    t0 = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)

    def line(ds, mhz, thermal="Not Active"):
        ts = (t0 + datetime.timedelta(seconds=ds)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 900.5, 0x0000000000000000, Not Active, {thermal}, Not Active, Active"

    lines = [line(0.0, 1500, "Active"), line(0.1, 2070), line(0.2, 2070), line(0.3, 2055), line(0.9, 1400)]
    base = t0.timestamp()
    rec = bench.parse_clock_samples(lines, (base + 0.05, base + 0.35))
    assert rec["samples"] == 3 and rec["samples_total"] == 5 and rec["in_region"]
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]          # the thermal flag at t = 0 lies outside
    rec = bench.parse_clock_samples(lines, (base + 5.0, base + 6.0))
    assert rec["samples"] == 0 and not rec["in_region"] and rec["samples_total"] == 5
    assert "hw_thermal_slowdown" in rec["reasons"]     # all samples, so the rejection rule still sees it
    assert bench.parse_clock_samples(["garbage", ""], None)["sm_mhz"] is None
