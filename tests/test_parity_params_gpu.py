"""Whole-path parity over the parameter space of the batching and serving
workloads, against the FP64 CPU oracle, through the C ABI.

Sec. 2 states the problem for any viscosity nu, force variance D and lattice
spacings a, tau (Eq. (Gen2)); the batching workload draws nu log-uniform in
[0.1, 10] with D = 1 and the serving workload adds 64x8 lattices.  Each case
here runs a lattice at the ends of that nu range, with unit and with
non-unit (D, a, tau), on each kind of kernel the workloads reach:

* 10x2 with 2^27 samples (64 subvolumes of 2^21): chunks of 256 rows per
  thread, so the two-stage screen runs, with the survivor's partial action
  carried through the queue;
* 6x4 and 4x2 (thread-per-sample, one-stage screen), 32x2 (two-stage shape,
  one-stage at this budget);
* 32x4 and 64x8 (warp-per-sample kernel with the register-resident screen).

FP64: every sum within 1e-12 of the oracle (widened only by the conditioning
of exp(-S) at large actions, see cond_rtol).  FP32: within the stated 1e-6 of
the oracle evaluating the identical float points.  Then the batching workload
itself: the 256 jobs of seed 3 in one CUDA graph, with the oracle on one or two
subvolumes of every job whose subvolume budget times d stays below 2^25.
"""
import concurrent.futures
import os

import numpy as np
import pytest

import oracle
import workloads
from test_parity_gpu import (FP32_ERR_ATOL, FP32_RTOL, FP64_RTOL, assert_slots_close, assert_totals_close, budget,
                             cond_rtol, dev, run_gpu, run_oracle)  # noqa: F401 (dev is a fixture)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PARAMS = [dict(nu=0.1), dict(nu=10.0), dict(nu=0.1, D=1.7, a=0.8, tau=0.6), dict(nu=10.0, D=1.7, a=0.8, tau=0.6)]
PARAM_IDS = ["nu0.1", "nu10", "nu0.1-Dat", "nu10-Dat"]
SHAPES = [(4, 2), (6, 4), (32, 2), (32, 4), (64, 8)]


def _with(job, params):
    for k, v in params.items():
        setattr(job, k, v)
    return job


def _compare(g_s, g_t, o_s, o_t, R, precision):
    if precision == 0:
        assert_slots_close(g_s, o_s, R, FP64_RTOL)
        assert_totals_close(g_t, o_t, R, FP64_RTOL, 1e-9, m=o_s[:, 1].max())
    else:
        assert_slots_close(g_s, o_s, R, FP32_RTOL)
        assert_totals_close(g_t, o_t, R, FP32_RTOL, 1e-4, FP32_ERR_ATOL)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("params", PARAMS, ids=PARAM_IDS)
@pytest.mark.parametrize("nx,nt", SHAPES)
def test_parameter_range_small_jobs(bfi, dev, nx, nt, params, precision):
    job = _with(workloads.small_ragged(nx, nt, seed=90 + nx + nt, nsub=3, base=budget(nx, nt, 30_000)), params)
    job.job_id = 7
    g_s, g_t, _ = run_gpu(bfi, dev, job, precision)
    o_s, o_t = run_oracle(job, fp32_points=bool(precision))
    _compare(g_s, g_t, o_s, o_t, nx // 2 + 1, precision)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("params", PARAMS, ids=PARAM_IDS)
def test_parameter_range_two_stage_10x2(bfi, dev, params, precision):
    """10x2, [-5,5]^20 bisected into 64 subvolumes of 2^21 samples (2^27 in
    all): 256 rows per thread, so stage 1 of the screen runs on every chunk.
    Eight subvolumes (a fixed random pick) against the oracle; the totals are
    the oracle's merge of all 64 records."""
    lo, hi = workloads.bisected_boxes(20, 6)
    job = _with(workloads.Job(10, 2, lo, hi, np.full(64, 1 << 21, dtype=np.uint64), seed=4, job_id=11), params)
    g_s, g_t, plan = run_gpu(bfi, dev, job, precision)
    assert plan.info().chunk_samples == 256 * 256
    n_eval, _ = plan.stats()
    full, two = plan.screen_stats()
    assert two and n_eval <= full < job.total_samples
    pick = np.sort(np.random.default_rng(8).choice(64, 8, replace=False))
    o_s, _ = run_oracle(job.subset(pick), fp32_points=bool(precision))
    if precision == 0:
        assert_slots_close(g_s[pick], o_s, 6, FP64_RTOL)
    else:
        assert_slots_close(g_s[pick], o_s, 6, FP32_RTOL)
    assert_totals_close(g_t, oracle.merge(10, g_s), 6, 1e-13, 1e-9)


def _batch_checks(jobs, cap_two=1 << 22, cap_one=1 << 25):
    """(job index, subvolume) pairs the oracle checks: the first and last
    subvolume of jobs with budget x d <= cap_two, the last of those up to cap_one."""
    picks = []
    for k, j in enumerate(jobs):
        cost = int(j.samples[0]) * j.d
        if cost <= cap_two:
            picks += [(k, 0), (k, j.nsub - 1)]
        elif cost <= cap_one:
            picks.append((k, j.nsub - 1))
    return picks


@pytest.mark.parametrize("precision", [0, 1])
def test_batching_workload_sampled(bfi, dev, precision):
    """The batching workload as the benchmark runs it (256 jobs of seed 3,
    one CUDA graph, autotuned grids) in both precisions; every job's record of
    the checked subvolumes against the oracle, and every job's totals against
    the oracle's merge of its records."""
    jobs = workloads.batch_jobs(256, seed=3)
    descs = []
    for j in jobs:
        descs.append(dict(lattice=bfi.lattice(j.nx, j.nt, j.nu, j.D, j.a, j.tau), samples=j.samples,
                          lo=torch.tensor(j.lo, device=dev), hi=torch.tensor(j.hi, device=dev), seed=j.seed,
                          job_id=j.job_id))
    batch = bfi.Batch(descs, precision=precision, nstreams=8, autotune=True)
    batch.launch()
    torch.cuda.synchronize()
    slots = [s.cpu().numpy() for s in batch.slots]
    totals = [t.cpu().numpy() for t in batch.totals]
    batch.close()
    picks = _batch_checks(jobs)
    assert len({k for k, _ in picks}) >= 230 and {(jobs[k].nx, jobs[k].nt) for k, _ in picks} == \
        {(j.nx, j.nt) for j in jobs}

    def one(pick):
        k, s = pick
        j = jobs[k].subset([s])
        lat = oracle.lattice(j.nx, j.nt, j.nu, j.D, j.a, j.tau)
        return oracle.integrate(lat, j.lo, j.hi, j.samples, j.seed, j.job_id, sub_id=j.sub_id,
                                fp32_points=bool(precision), nthreads=1)[0]

    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        oracle_slots = list(ex.map(one, picks))
    for (k, s), o_s in zip(picks, oracle_slots):
        j = jobs[k]
        R = j.nx // 2 + 1
        try:
            if precision == 0:
                assert_slots_close(slots[k][[s]], o_s, R, FP64_RTOL)
            else:
                assert_slots_close(slots[k][[s]], o_s, R, FP32_RTOL)
        except AssertionError as e:
            raise AssertionError(f"job {k} ({j.name}), subvolume {s}: {e}") from None
    for k, j in enumerate(jobs):
        R = j.nx // 2 + 1
        assert_totals_close(totals[k], oracle.merge(j.nx, slots[k]), R, 1e-13, 1e-9)
        assert np.isfinite(totals[k][0]) and totals[k][4] > 0


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nx,nt,params", [(4, 2, {}), (10, 2, {}), (10, 2, dict(nu=10.0)),
                                          (10, 2, dict(nu=0.1, D=1.7, a=0.8, tau=0.6)), (6, 4, dict(nu=0.1)),
                                          (16, 4, {}), (32, 4, dict(nu=10.0)), (64, 8, {})])
def test_stated_error_bound_holds(bfi, dev, nx, nt, params, precision):
    """Each result's stated arithmetic error (bfi_error_bound on its own
    records) bounds its measured distance from the oracle evaluating the same
    points: Z relative, C(r) relative to C(0).  In FP32 the oracle runs the
    identical float points in FP64, so the difference is the FP32 path's
    arithmetic alone."""
    job = _with(workloads.small_ragged(nx, nt, seed=120 + nx + nt, nsub=3, base=budget(nx, nt, 40_000)), params)
    g_s, g_t, _ = run_gpu(bfi, dev, job, precision)
    o_s, o_t = run_oracle(job, fp32_points=bool(precision))
    R = nx // 2 + 1
    lat = bfi.lattice(nx, nt, job.nu, job.D, job.a, job.tau)
    bound = bfi.error_bound(lat, precision, g_s, 5.0)
    z_err = abs(np.expm1(g_t[0] - o_t[0]))
    c_err = np.abs(g_t[4:4 + R] - o_t[4:4 + R]) / o_t[4]
    assert z_err <= bound[0], (z_err, bound[0])
    assert np.all(c_err <= bound[1:]), (c_err, bound[1:])
    if precision == 1 and (nx, nt) in [(4, 2), (10, 2)]:
        assert bound.max() < 1e-6
