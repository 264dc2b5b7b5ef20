"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances.  FP64 mode: every per-subvolume sum within 1e-12 relative of the
oracle, first order (w, w P_r) and second order (w^2, w^2 P_r, w^2 P_r^2)
alike, where sums with P_r (|P_r| <= P_0 per sample, so their terms are
bounded by their r = 0 member's) are measured against their P_0 counterpart;
C(r) within 1e-12 of C(0).  FP32 mode is compared with the oracle's
FP32-points mode (the identical float points evaluated in FP64), every sum
within FP32_RTOL = 1e-6, the bound the FP32 path states.  The records of the
two sides use different shifts m_s (the device starts from a hint), so sums
are compared after moving them to the oracle's shift.  The stated statistical
errors are square roots of differences of sums (n sum w^2 - (sum w)^2, and the
delta-method combination for C(r)) that cancel when the weights are nearly
equal or one sample dominates C(r)'s variance, so they carry the rounding of
those sums magnified: they are compared at 1e-9 relative or FP64_ERR_ATOL C(0)
(FP64) and 1e-4 or FP32_ERR_ATOL C(0) (FP32).  For lattices whose smallest
action S is large, exp(-S) cannot be reproduced to better than ~eps S relative
by any FP64 evaluation: the FP64 bound is max(1e-12, 16 eps S).
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-12
FP32_RTOL = 1e-6
FP32_ERR_ATOL = 1e-3
FP64_ERR_ATOL = 1e-7
# compiled thread-per-sample shapes, and shapes that run on the generic warp-per-sample kernel
SHAPES = [(2, 1), (3, 1), (4, 1), (2, 2), (3, 2), (4, 2), (6, 2), (8, 2), (10, 2), (16, 2), (32, 2),
          (4, 4), (6, 4), (8, 4), (10, 4), (16, 4)]
GENERIC = [(5, 3), (7, 1), (12, 3), (32, 4), (64, 8)]


def budget(nx, nt, base):
    """Smaller budgets for big lattices, where the oracle is slow."""
    d = nx * nt
    return base if d <= 64 else max(3000, base // (d // 16))


@pytest.fixture(scope="module")
def dev(bfi):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def lat_of(mod, job, **kw):
    return mod.lattice(job.nx, job.nt, job.nu, job.D, job.a, job.tau, **kw)


def run_gpu(bfi, dev, job, precision, nonlinear=1.0, mass2=0.0):
    lat = lat_of(bfi, job, nonlinear=nonlinear, mass2=mass2)
    plan = bfi.Plan(lat, job.samples, precision)
    lo = torch.tensor(job.lo, dtype=torch.float64, device=dev)
    hi = torch.tensor(job.hi, dtype=torch.float64, device=dev)
    sid = None if job.sub_id is None else torch.tensor(job.sub_id.astype(np.int32), device=dev)
    slots, totals = plan.execute(lo, hi, job.seed, job.job_id, sub_id=sid)
    torch.cuda.synchronize()
    return slots.cpu().numpy(), totals.cpu().numpy(), plan


def run_oracle(job, fp32_points=False, nonlinear=1.0, mass2=0.0):
    lat = lat_of(oracle, job, nonlinear=nonlinear, mass2=mass2)
    return oracle.integrate(lat, job.lo, job.hi, job.samples, job.seed, job.job_id,
                            sub_id=job.sub_id, fp32_points=fp32_points)


def cond_rtol(rtol, m, eps):
    """exp(-S) has relative error at least the absolute error of S, ~eps S:
    for big lattices (S in the thousands) no two FP64 evaluations agree to
    1e-12, so the bound grows to 16 eps S there."""
    return np.maximum(rtol, 16.0 * eps * np.abs(m))


def slot_deviations(g, o, R, eps=2.0 ** -52):
    """Largest deviation of each group of sums from the oracle's, after moving
    the GPU sums to the oracle's shift, relative to the group's scale: the sum
    itself for sum w and sum w^2 (non-negative terms), the r = 0 member for the
    sums with P_r (|P_r| <= P_0 per sample, so sum |w^k P_r| <= sum w^k P_0 and
    sum w^2 P_r^2 <= sum w^2 P_0^2).  Also returns the conditioning bound
    max(1, 16 eps S_min / rtol) factor per subvolume (see cond_rtol)."""
    used = o[:, 0] > 0
    g, o = g[used], o[used]
    dm = g[:, 1] - o[:, 1]
    f1, f2 = np.exp(-dm)[:, None], np.exp(-2 * dm)[:, None]
    sc = lambda x: np.where(x > 0, x, 1.0)
    dev = {
        "sw": np.abs(g[:, 3:4] * f1 - o[:, 3:4]) / sc(o[:, 3:4]),
        "sw2": np.abs(g[:, 4:5] * f2 - o[:, 4:5]) / sc(o[:, 4:5]),
        "swp": np.abs(g[:, 5:5 + R] * f1 - o[:, 5:5 + R]) / sc(o[:, 5:6]),
        "sw2p": np.abs(g[:, 5 + R:5 + 2 * R] * f2 - o[:, 5 + R:5 + 2 * R]) / sc(o[:, 5 + R:5 + R + 1]),
        "sw2p2": np.abs(g[:, 5 + 2 * R:] * f2 - o[:, 5 + 2 * R:]) / sc(o[:, 5 + 2 * R:5 + 2 * R + 1]),
    }
    return dev, o[:, 1]


def assert_slots_close(g, o, R, rtol, rtol_var=None, eps=2.0 ** -52):
    """Every sum within rtol of the oracle's (scaled as in slot_deviations),
    widened only by the conditioning of exp(-S) for large actions.  The
    first-order sums (w, w P_r) and the second-order ones (w^2, w^2 P_r,
    w^2 P_r^2) are all sums of terms bounded by their group's scale, so one
    tolerance holds for all of them; rtol_var, if given, applies to the
    second-order sums instead.""" 
    assert np.array_equal(g[:, 0], o[:, 0]), "sample counts differ"
    used = o[:, 0] > 0
    # the device shift starts at a hint (an FP32 action, rounded by up to ~4 d 2^-24 S, d <= 512) and moves
    # down only when beaten by more than 16: to the action in FP64, by whole multiples of ln 2 to within ln 2
    # below it in FP32; so it lies within [min S - ln 2 - slack, min S + 16 + slack] (the oracle's is min S)
    gu, ou = g[used], o[used]
    slack = 1e-3 + 1.2e-4 * np.abs(ou[:, 1])
    assert np.all(gu[:, 1] >= ou[:, 1] - np.log(2.0) - slack) and np.all(gu[:, 1] <= ou[:, 1] + 16.0 + slack)
    np.testing.assert_allclose(gu[:, 2], ou[:, 2], rtol=1e-14, atol=1e-14)    # log V_s
    dev, m = slot_deviations(g, o, R, eps)
    rt = cond_rtol(rtol, m, eps)[:, None]
    rv = rt if rtol_var is None else np.maximum(rt, rtol_var)
    for key, tol in (("sw", rt), ("swp", rt), ("sw2", rv), ("sw2p", rv), ("sw2p2", rv)):
        bad = dev[key] > tol
        assert not np.any(bad), f"{key}: deviation {dev[key].max():.3e} > tolerance {np.min(tol):.1e}"


def assert_totals_close(g, o, R, rtol, rtol_var, err_atol=None, m=0.0, eps=2.0 ** -52):
    rtol = float(cond_rtol(rtol, m, eps))
    assert g[2] == o[2] and g[3] == o[3]
    assert abs(g[0] - o[0]) <= rtol * max(1.0, abs(o[0])) + rtol            # log Z  ->  Z within rtol
    assert np.all(np.abs(g[4:4 + R] - o[4:4 + R]) <= rtol * o[4])          # C(r), |C(r)| <= C(0)
    np.testing.assert_allclose(g[1], o[1], rtol=max(rtol_var, rtol))
    atol = (FP64_ERR_ATOL if err_atol is None else err_atol) * o[4]
    np.testing.assert_allclose(g[4 + R:], o[4 + R:], rtol=max(rtol_var, rtol), atol=atol)


# ---------------------------------------------------------------------------
# step 1: points
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("d,first", [(8, 0), (20, 12345), (21, (3 << 32) - 5), (512, 7)])
def test_points_bit_exact(bfi, dev, precision, d, first):
    rng = np.random.default_rng(d)
    lo = rng.uniform(-5, 0, d)
    hi = lo + rng.uniform(0.1, 5, d)
    count = 3000 if d < 100 else 200
    y = bfi.points(d, torch.tensor(lo, device=dev), torch.tensor(hi, device=dev), 77, 9, 4, first,
                   count, precision).cpu().numpy()
    yo = oracle.points(d, lo, hi, 77, 9, 4, first, count, fp32_points=bool(precision))
    assert np.array_equal(y, yo)


# ---------------------------------------------------------------------------
# steps 2 and 4: action and products at given points
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,nt", SHAPES + GENERIC)
@pytest.mark.parametrize("params", [dict(), dict(nu=0.3, D=2.0, a=0.7, tau=0.5, nonlinear=1.0, mass2=0.4),
                                    dict(nonlinear=0.0, mass2=1.0)])
def test_eval_matches_oracle(bfi, dev, nx, nt, params):
    d = nx * nt
    rng = np.random.default_rng(nx * 10 + nt)
    y = rng.uniform(-5, 5, (4096 if d <= 64 else 512, d))
    S_o, P_o = oracle.eval_points(oracle.lattice(nx, nt, **params), y)
    S, P = bfi.evaluate(bfi.lattice(nx, nt, **params), torch.tensor(y, device=dev), 0)
    np.testing.assert_allclose(S.cpu().numpy(), S_o, rtol=1e-13)
    assert np.all(np.abs(P.cpu().numpy() - P_o) <= 1e-13 * P_o[:, :1])
    # FP32: the same device code on float points, against FP64 on the same points
    y32 = y.astype(np.float32).astype(np.float64)
    S_o32, P_o32 = oracle.eval_points(oracle.lattice(nx, nt, **params), y32)
    S32, P32 = bfi.evaluate(bfi.lattice(nx, nt, **params), torch.tensor(y32, device=dev), 1)
    np.testing.assert_allclose(S32.cpu().numpy(), S_o32, rtol=2e-5 * max(1, d // 32))
    assert np.all(np.abs(P32.cpu().numpy() - P_o32) <= 2e-6 * P_o32[:, :1])
    # the compensated FP32 action used near the minimum: ~2^-44 relative to the terms
    Sc, _ = bfi.evaluate(bfi.lattice(nx, nt, **params), torch.tensor(y32, device=dev), 2)
    np.testing.assert_allclose(Sc.cpu().numpy(), S_o32, rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------------------
# the whole path
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,nt", SHAPES + GENERIC)
def test_integrate_fp64_ragged(bfi, dev, nx, nt):
    job = workloads.small_ragged(nx, nt, seed=5 + nx, nsub=3, base=budget(nx, nt, 30_000))
    g_s, g_t, plan = run_gpu(bfi, dev, job, 0)
    info = plan.info()
    assert info.chunks >= 3 * 2  # several chunks per subvolume, ragged last ones
    assert info.kernel == (1 if (nx, nt) in GENERIC else 0)
    # the two-stage screen is compiled for shapes with >= 3 Philox blocks whose first ~60% complete the
    # neighbourhoods of at least 35% of the sites, but not all; these jobs' chunks hold fewer than 256 rows per
    # thread, so stage 1 does not run and every sample is screened in one stage (the two-stage runs are
    # test_two_stage_screen_and_a_flat_action and test_parity_params_gpu.py)
    n_eval, _ = plan.stats()
    full, two = plan.screen_stats()
    work = plan.work()
    d = nx * nt
    bp = (3 * ((d + 3) // 4) + 4) // 5
    mc = min(4 * bp // nt, nx)
    assert work.two_stage_shape == ((nx, nt) not in GENERIC and (d + 3) // 4 >= 3 and mc < nx and
                                    20 * (mc - 2) >= 7 * nx)
    assert not two and full == job.total_samples
    assert (work.samples, work.stage1, work.survivors, work.full_screen, work.evaluated) == \
        (job.total_samples, 0, 0, job.total_samples, n_eval)
    assert n_eval <= job.total_samples
    o_s, o_t = run_oracle(job)
    R = nx // 2 + 1
    assert_slots_close(g_s, o_s, R, FP64_RTOL)
    assert_totals_close(g_t, o_t, R, FP64_RTOL, 1e-9, m=o_s[:, 1].max())


@pytest.mark.parametrize("nonlinear,mass2,params", [(0.0, 1.0, {}), (1.0, 0.5, dict(nu=0.4, a=0.8, tau=0.6, D=1.7))])
def test_integrate_fp64_parameters(bfi, dev, nonlinear, mass2, params):
    job = workloads.small_ragged(4, 2, seed=11, nsub=2, base=20_000)
    for k, v in params.items():
        setattr(job, k, v)
    job.job_id = 3
    job.sub_id = np.array([17, 4_000_000_000], dtype=np.uint32)
    g_s, g_t, _ = run_gpu(bfi, dev, job, 0, nonlinear, mass2)
    o_s, o_t = run_oracle(job, False, nonlinear, mass2)
    assert_slots_close(g_s, o_s, 3, FP64_RTOL)
    assert_totals_close(g_t, o_t, 3, FP64_RTOL, 1e-9)


@pytest.mark.parametrize("nx,nt", [(3, 1), (4, 2), (10, 2), (16, 4), (32, 2), (5, 3), (32, 4), (64, 8)])
def test_integrate_fp32_against_fp32_points(bfi, dev, nx, nt):
    job = workloads.small_ragged(nx, nt, seed=21 + nx, nsub=3, base=budget(nx, nt, 30_000))
    g_s, g_t, _ = run_gpu(bfi, dev, job, 1)
    o_s, o_t = run_oracle(job, fp32_points=True)
    R = nx // 2 + 1
    assert_slots_close(g_s, o_s, R, FP32_RTOL)
    assert_totals_close(g_t, o_t, R, FP32_RTOL, 1e-4, FP32_ERR_ATOL)


def test_edge_cases_empty_single_and_tiny(bfi, dev):
    job = workloads.small_ragged(4, 2, seed=3, nsub=4, base=100)
    job.samples = np.array([0, 1, 37, 1000], dtype=np.uint64)
    g_s, g_t, _ = run_gpu(bfi, dev, job, 0)
    o_s, o_t = run_oracle(job)
    assert g_s[0, 0] == 0 and g_s[0, 3] == 0
    assert np.isinf(g_t[1]) and np.isinf(o_t[1])
    assert_slots_close(g_s, o_s, 3, FP64_RTOL)
    assert g_t[0] == pytest.approx(o_t[0], rel=1e-12)
    # without the one-sample subvolume the errors are finite again
    sub = job.subset([0, 2, 3])
    g_s2, g_t2, _ = run_gpu(bfi, dev, sub, 0)
    o_s2, o_t2 = run_oracle(sub)
    assert_totals_close(g_t2, o_t2, 3, FP64_RTOL, 1e-9)


def test_binding_checks_array_sizes_before_any_launch(bfi, dev):
    """The library reads and writes device arrays by the sizes the plan fixes;
    the binding refuses tensors of another size before calling it."""
    lat = bfi.lattice(4, 2)
    plan = bfi.Plan(lat, [1000, 1000])
    lo, hi = torch.zeros((2, 8), dtype=torch.float64, device=dev), torch.ones((2, 8), dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        plan.execute(lo[:1], hi[:1], 1)
    with pytest.raises(ValueError):
        plan.execute(lo, hi, 1, sub_id=torch.zeros(3, dtype=torch.int32, device=dev))
    with pytest.raises(ValueError):
        plan.execute(lo, hi, 1, slots=torch.empty((1, bfi.slot_len(4)), dtype=torch.float64, device=dev))
    with pytest.raises(ValueError):
        bfi.integrate_static_scratch(lat, [1000, 1000, 1000], lo, hi, 1)
    with pytest.raises(ValueError):
        bfi.Batch([dict(lattice=lat, samples=[10, 10, 10], lo=lo, hi=hi)], autotune=False)
    s, t = plan.execute(lo, hi, 1)   # the right sizes still run
    torch.cuda.synchronize()
    assert np.isfinite(t.cpu().numpy()[0])
    plan.close()


def test_device_merge_equals_host_merge_and_is_deterministic(bfi, dev):
    job = workloads.small_ragged(10, 2, seed=2, nsub=5, base=20_000)
    g_s, g_t, _ = run_gpu(bfi, dev, job, 0)
    g_s2, g_t2, _ = run_gpu(bfi, dev, job, 0)
    assert np.array_equal(g_s, g_s2) and np.array_equal(g_t, g_t2)
    h_t = bfi.merge_host(10, g_s)
    R = 6
    np.testing.assert_allclose(h_t[:4 + R], g_t[:4 + R], rtol=1e-13, atol=1e-13 * abs(g_t[4]))
    # the stated C(r) errors are square roots of variances that cancel when one
    # sample dominates: summed in different orders they agree to ~sqrt(eps) C(0)
    np.testing.assert_allclose(h_t[4 + R:], g_t[4 + R:], rtol=1e-9, atol=FP64_ERR_ATOL * g_t[4])


def test_host_buffer_path_equals_device_path(bfi, dev):
    job = workloads.small_ragged(4, 2, seed=8, nsub=3, base=25_000)
    g_s, g_t, _ = run_gpu(bfi, dev, job, 1)
    ctx = bfi.Context(0)
    h_s, h_t = ctx.integrate(lat_of(bfi, job), job.lo, job.hi, job.samples, job.seed, job.job_id,
                             precision=1)
    assert np.array_equal(g_s, h_s) and np.array_equal(g_t, h_t)
    h_s2, h_t2 = ctx.integrate(lat_of(bfi, job), job.lo, job.hi, job.samples, job.seed, job.job_id,
                               precision=1)
    assert np.array_equal(h_t, h_t2)
    ctx.close()


def test_every_shape_up_to_512_sites_is_supported(bfi, dev):
    for nx, nt in [(5, 5), (2, 256), (512, 1), (3, 170)]:
        assert bfi.Plan(bfi.lattice(nx, nt), [100]).info().kernel == 1
    with pytest.raises(bfi.BfiError) as e:
        bfi.Plan(bfi.lattice(33, 16), [100])
    assert e.value.status == 1


# ---------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark uses
# ---------------------------------------------------------------------------
def test_plain_4x2_full_size(bfi, dev):
    job = workloads.plain_4x2()
    g_s, g_t, _ = run_gpu(bfi, dev, job, 0)
    o_s, o_t = run_oracle(job)
    assert_slots_close(g_s, o_s, 3, FP64_RTOL)
    assert_totals_close(g_t, o_t, 3, FP64_RTOL, 1e-9)


@pytest.mark.parametrize("total,rows", [(1 << 12, 4), (1 << 20, 4), (1 << 24, 32), (1 << 27, 256), (1 << 28, 512),
                                        (1 << 29, 512), ((1 << 30) - 256, 512), (1 << 30, 1024),
                                        ((1 << 31) - 256, 1024), (1 << 31, 2048), (1 << 36, 2048)])
def test_chunk_size_follows_the_job_alone(bfi, dev, total, rows):
    """Rows per thread in a chunk: at least 2048 chunks, up to 512 rows, then
    doubling up to 2048 while 4096 chunks remain; the same for either
    precision and for any split of the job into subvolumes."""
    lat = bfi.lattice(10, 2)
    for precision in (0, 1):
        for nsub in (1, 64):
            smp = np.full(nsub, total // nsub, dtype=np.uint64)
            smp[0] += total - int(smp.sum())
            plan = bfi.Plan(lat, smp, precision)
            info = plan.info()
            plan.close()
            assert info.chunk_samples == rows * 256 and info.total_samples == total
            # the plan cuts the job as the host rule says, tail included
            ch = bfi.chunking(smp)
            assert (info.chunk_samples, info.tail_subvolume, info.tail_chunk_samples, info.chunks) == \
                (ch.chunk_samples, ch.tail_subvolume, ch.tail_chunk_samples, ch.chunks)


@pytest.mark.parametrize("nx,nt,precision,sampler,log2n", [(10, 2, 0, 0, 21), (10, 2, 1, 0, 21), (6, 4, 0, 0, 21),
                                                             (32, 4, 1, 0, 21), (64, 8, 0, 0, 21), (4, 2, 0, 1, 21),
                                                             (4, 2, 0, 2, 21), (5, 3, 0, 2, 21), (10, 2, 0, 0, 28),
                                                             (10, 2, 1, 0, 28)])
def test_results_do_not_depend_on_which_cta_takes_a_chunk(bfi, dev, nx, nt, precision, sampler, log2n):
    """After its first chunk a CTA takes the next chunk not yet taken, so the
    chunk-to-CTA map changes from run to run and with the grid.  A chunk's
    record depends on the chunk alone: every grid (1 CTA per SM up to the
    occupancy limit) and a repeat give bitwise the same slots, totals and work
    counts.  Jobs of 2^21 samples have 2048 chunks, so each CTA takes several
    (thread-per-sample, warp-per-sample, range-map and Gaussian kernels); the
    2^28-sample jobs have chunks of 512 rows and, in their last two
    subvolumes, tail chunks of 256 rows."""
    d = nx * nt
    nsub = 16
    lo = np.full((nsub, d), -3.0 if sampler != 1 else -0.9)
    hi = np.full((nsub, d), 3.0 if sampler != 1 else 0.9)
    lo[:, 0] = np.linspace(lo[0, 0], hi[0, 0], nsub + 1)[:-1]
    hi[:, 0] = np.linspace(lo[0, 0], hi[0, 0], nsub + 1)[1:]
    samples = np.full(nsub, (1 << log2n) // nsub, dtype=np.uint64)
    samples[3] += 777
    if log2n == 28:
        samples[5] += 1000   # 2^28 + 1777 in all: chunks of 512 rows
    else:
        samples[5] -= 1000
    lat = bfi.lattice(nx, nt)
    plan = bfi.Plan(lat, samples, precision)
    if sampler:
        plan.set_sampler(sampler, mean=np.zeros(d) if sampler == 2 else None,
                         factor=np.eye(d) * 0.8 if sampler == 2 else None)
    assert plan.info().chunks >= 2048
    if log2n == 28:
        assert plan.info().tail_subvolume == 14 and plan.info().tail_chunk_samples == 256 * 256
    lo_t, hi_t = torch.tensor(lo, device=dev), torch.tensor(hi, device=dev)

    def run():
        s, t = plan.execute(lo_t, hi_t, 5, 3)
        torch.cuda.synchronize()
        return s.cpu().numpy(), t.cpu().numpy(), plan.work().as_dict()

    ref = run()
    assert ref[2]["samples"] == int(samples.sum())
    for g in sorted({1, 2, plan.info().ctas_per_sm_max}):
        if g > plan.info().ctas_per_sm_max:
            continue
        plan.set_grid(g)
        for _ in range(2):
            out = run()
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]) and out[2] == ref[2], g
    plan.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_paper_10x2_full_size_sampled(bfi, dev, precision):
    job = workloads.paper_10x2()
    g_s, g_t, plan = run_gpu(bfi, dev, job, precision)
    # 1024 rows per thread; the last 128 subvolumes in chunks of 256 rows, handed out last
    info = plan.info()
    assert info.chunk_samples == 1024 * 256 and info.tail_subvolume == 896 and info.tail_chunk_samples == 256 * 256
    # a fixed random subset of 64 of the 1024 subvolumes (subvolumes are independent, so subset parity is exact)
    pick = np.sort(np.random.default_rng(64).choice(1024, 64, replace=False))
    assert (pick >= 896).sum() >= 4 and (pick < 896).sum() >= 4
    o_s, _ = run_oracle(job.subset(pick), fp32_points=bool(precision))
    tol = FP64_RTOL if precision == 0 else FP32_RTOL
    assert_slots_close(g_s[pick], o_s, 6, tol)
    # totals: the device merge of all 1024 records equals the oracle's merge of them
    o_t = oracle.merge(10, g_s)
    assert_totals_close(g_t, o_t, 6, 1e-13, 1e-9)
    assert g_t[2] == 1024 * (1 << 20) and g_t[3] == 1024
    # invariants: Z > 0 (finite log), C(0) > 0, |C(r)| <= C(0)
    assert np.isfinite(g_t[0]) and g_t[4] > 0 and np.all(np.abs(g_t[4:10]) <= g_t[4])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("D,mass2", [(20.0, 0.0), (1.0, 0.0), (1.0, 0.5)])
def test_two_stage_screen_and_a_flat_action(bfi, dev, D, mass2, precision):
    """10x2 with 16 subvolumes of about 2^23 samples: chunks of 256 rows per
    thread, so the two-stage screen runs.  With the force variance D = 20
    the action is 20 times flatter and over 99% of the samples survive the
    partial action: the survivor queue carries nearly the whole chunk.  At
    D = 1 about a seventh survive.  With mass2 = 0 stage 2 adds the rest of the
    action to the survivor's partial one; the mass term needs every coordinate,
    so with mass2 = 0.5 stage 2 screens in full.  In every case the records of
    the first and last subvolumes match the oracle's, and the totals are the
    oracle's merge of all records."""
    lo, hi = workloads.bisected_boxes(20, 4)
    # 2^23 + 65436 samples per subvolume: 128 full chunks and a ragged one of 65436 (256 rows, the last short by
    # 100 samples), which still runs in two stages
    job = workloads.Job(10, 2, lo, hi, np.full(16, (1 << 23) + 65436, dtype=np.uint64), seed=9, D=D)
    g_s, g_t, plan = run_gpu(bfi, dev, job, precision, mass2=mass2)
    assert plan.info().chunk_samples == 256 * 256
    n_eval, _ = plan.stats()
    full, two = plan.screen_stats()
    assert two and n_eval <= full <= job.total_samples
    # every chunk holds 256 rows, so every sample runs stage 1 and 'full' counts the survivors
    work = plan.work()
    assert (work.stage1, work.full_screen, work.survivors, work.evaluated) == (job.total_samples, 0, full, n_eval)
    assert work.two_stage_shape == 1 and work.rest_screen == (1 if mass2 == 0.0 else 0)
    if D > 1.0:
        assert full > 0.9 * job.total_samples
    elif mass2 == 0.0:  # the mass term, left out of P, lets more samples through
        assert full < 0.35 * job.total_samples
    pick = [0, 15]
    o_s, _ = run_oracle(job.subset(pick), fp32_points=bool(precision), mass2=mass2)
    tol = FP64_RTOL if precision == 0 else FP32_RTOL
    assert_slots_close(g_s[pick], o_s, 6, tol)
    assert_totals_close(g_t, oracle.merge(10, g_s), 6, 1e-13, 1e-9)
