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
    one = bench.roofline(n, n_eval, ms, "fp64", 10, 2)
    two = bench.roofline(n, n_eval, ms, "fp64", 10, 2, screened=n // 5)
    t = ms * 1e-3
    integer = bench.eval_ops_fp64(10, 2)[1]
    assert abs(one["achieved"] * 1e9 * t - (n * 400 + n_eval * integer)) < 1e3
    # a survivor draws blocks 0, 2, 3, 4 again: 160 + 32 points + the 12 residuals of sites 0 and 5..9
    assert bench.rest_ops(10, 2) == 160 + 32 + 96
    assert abs(two["achieved"] * 1e9 * t - (n * 208 + (n // 5) * 288 + n_eval * integer)) < 1e3
    assert two["full_screened"] == n // 5 and one["full_screened"] == n
    assert two["partial_ops_per_sample"] == 208 and one["partial_ops_per_sample"] is None
    assert one["bound"] == "alu" and one["resource"] == "FP32/INT issue"
    assert 0 < two["frac"] < one["frac"]


def test_fp32_roofline_has_no_fp64_work():
    r = bench.roofline(1 << 34, 3_000_000, 216.0, "fp32", 10, 2, screened=3_300_000_000)
    assert r["fp64_frac"] == 0 and r["resource"] == "FP32/INT issue"
