"""The server: jobs admitted as they arrive, overlapping on the device, with
adaptive splitting.  A job's result must not depend on what else runs (same
bits alone, in a mix, and through a plan); split jobs must agree with the
oracle on their leaf subvolumes; waits are bounded; cancellation and the
memory budget work."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev(bfi):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _lat(mod, j):
    return mod.lattice(j.nx, j.nt, j.nu, j.D, j.a, j.tau)


def _mix(n=20):
    jobs = workloads.batch_jobs(n, seed=11)
    for j in jobs:
        j.samples = np.minimum(j.samples, max(1, (1 << 18) // j.nsub)).astype(np.uint64)
    return jobs


@pytest.mark.parametrize("precision", [0, 1])
def test_result_is_the_same_alone_in_a_mix_and_through_a_plan(bfi, dev, precision):
    target = workloads.small_ragged(10, 2, seed=2, nsub=6, base=40_000)
    target.job_id = 77
    srv = bfi.Server(slots=4, precision=precision)
    alone = srv.submit(_lat(bfi, target), target.lo, target.hi, target.samples, target.seed, target.job_id)
    alone.wait(60_000)
    t_alone, s_alone, *_ = alone.result(leaves=True)
    reqs = []
    for k, j in enumerate(_mix()):
        reqs.append(srv.submit(_lat(bfi, j), j.lo, j.hi, j.samples, j.seed, j.job_id))
        if k == 10:
            mixed = srv.submit(_lat(bfi, target), target.lo, target.hi, target.samples, target.seed, target.job_id)
    for r in reqs:
        r.wait(120_000)
    mixed.wait(120_000)
    t_mix, s_mix, *_ = mixed.result(leaves=True)
    assert np.array_equal(t_alone, t_mix) and np.array_equal(s_alone, s_mix)
    st = srv.stats()
    assert st.completed == 22 and st.failed == 0 and st.running == 0 and st.queued == 0
    srv.close()
    plan = bfi.Plan(_lat(bfi, target), target.samples, precision)
    p_slots, p_tot = plan.execute(torch.tensor(target.lo, device=dev), torch.tensor(target.hi, device=dev),
                                  target.seed, target.job_id)
    torch.cuda.synchronize()
    # the records are the plan's, bit for bit; the server merges them on the host
    assert np.array_equal(p_slots.cpu().numpy(), s_alone)
    assert np.array_equal(bfi.merge_host(10, p_slots.cpu().numpy()), t_alone)
    np.testing.assert_allclose(p_tot.cpu().numpy()[:10], t_alone[:10], rtol=1e-13)


def test_adaptive_splitting_agrees_with_the_oracle_on_the_leaves(bfi, dev):
    job = workloads.small_ragged(3, 2, seed=9, nsub=2, base=3000, half=3.0)
    job.job_id = 5
    srv = bfi.Server(slots=2, precision=0, split_rel_var=1e-2, max_split_rounds=2)
    req = srv.submit(_lat(bfi, job), job.lo, job.hi, job.samples, job.seed, job.job_id)
    req.wait(60_000)
    info = req.info()
    work = req.work()
    totals, slots, lo, hi, sid = req.result(leaves=True)
    srv.close()
    # the counted work covers every pass, split parents included
    assert work.samples == info.samples and work.full_screen == work.samples and 0 < work.evaluated <= work.samples
    assert info.passes >= 2 and info.nsub_final > job.nsub  # something was split
    # the leaves tile the original boxes
    vol = lambda a, b: np.prod(b - a, axis=1)
    assert np.isclose(vol(lo, hi).sum(), vol(job.lo, job.hi).sum(), rtol=1e-14)
    assert len(set(sid.tolist())) == len(sid)
    # every leaf, evaluated by the oracle with its own box, budget and sub_id
    o_slots, o_tot = oracle.integrate(oracle.lattice(job.nx, job.nt), lo, hi, slots[:, 0].astype(np.uint64),
                                      job.seed, job.job_id, sub_id=sid)
    assert np.array_equal(slots[:, 0], o_slots[:, 0])
    dm = slots[:, 1] - o_slots[:, 1]
    np.testing.assert_allclose(slots[:, 3] * np.exp(-dm), o_slots[:, 3], rtol=1e-12)
    np.testing.assert_allclose(totals[0], o_tot[0], rtol=1e-12, atol=1e-12)
    R = 2
    assert np.all(np.abs(totals[4:4 + R] - o_tot[4:4 + R]) <= 1e-12 * o_tot[4])
    assert info.samples >= int(slots[:, 0].sum())  # leaves plus the split parents


def test_bounded_wait_and_cancel(bfi, dev):
    big = workloads.paper_10x2(1 << 16)
    srv = bfi.Server(slots=1, precision=1)
    a = srv.submit(bfi.lattice(10, 2), big.lo, big.hi, big.samples, big.seed, 1)
    b = srv.submit(bfi.lattice(10, 2), big.lo, big.hi, big.samples, big.seed, 2)
    with pytest.raises(bfi.BfiError) as e:
        b.wait(0)
    assert e.value.status == 4  # BFI_E_TIMEOUT
    b.cancel()
    with pytest.raises(bfi.BfiError) as e:
        b.wait(60_000)
    assert e.value.status == 5  # BFI_E_CANCELLED
    a.wait(60_000)
    assert a.info().state == 2 and b.info().state == 3
    assert srv.stats().cancelled >= 1
    srv.close()


def test_memory_budget(bfi, dev):
    jobs = _mix(6)
    srv = bfi.Server(slots=4, precision=1, memory_budget=6 << 20)
    reqs = [srv.submit(_lat(bfi, j), j.lo, j.hi, j.samples, j.seed, j.job_id) for j in jobs]
    for r in reqs:
        r.wait(120_000)
    st = srv.stats()
    assert st.completed == len(jobs) and st.bytes_peak <= 6 << 20 and st.bytes_in_use == 0
    srv.close()
    tiny = bfi.Server(slots=1, precision=1, memory_budget=4096)
    r = tiny.submit(_lat(bfi, jobs[0]), jobs[0].lo, jobs[0].hi, jobs[0].samples, 1, 0)
    with pytest.raises(bfi.BfiError) as e:
        r.wait(60_000)
    assert e.value.status == 2  # BFI_E_NOMEM: can never be admitted
    tiny.close()


def _run_all(bfi, srv, jobs, timeout_ms=120_000):
    """Submits every job, waits for each: {job_id: (totals, leaf slots)} of
    the jobs that completed and {job_id: status} of those that failed."""
    reqs = [(j.job_id, srv.submit(_lat(bfi, j), j.lo, j.hi, j.samples, j.seed, j.job_id)) for j in jobs]
    done, failed = {}, {}
    for jid, r in reqs:
        try:
            r.wait(timeout_ms)
        except bfi.BfiError as e:
            failed[jid] = e.status
            continue
        t, s, *_ = r.result(leaves=True)
        done[jid] = (t, s)
    return done, failed


@pytest.mark.parametrize("point,status", [(1, 2), (2, 3), (3, 3)])
def test_injected_pass_failure_fails_its_job_alone(bfi, dev, point, status):
    """A pass that fails after admission (its pool allocation, a launch, or the
    stream status when it completes; the fault is made on the host) fails its
    own job with a status; every other job completes with the same bits as in
    a server without the fault; the memory goes back to the budget; shutdown
    returns within its bound."""
    import time
    jobs = _mix(8)
    ref_srv = bfi.Server(slots=4, precision=1)
    ref, ref_failed = _run_all(bfi, ref_srv, jobs)
    ref_srv.close()
    assert not ref_failed
    srv = bfi.Server(slots=4, precision=1)
    srv.inject_fault(point, 3)  # the fourth pass to reach the point fails there
    done, failed = _run_all(bfi, srv, jobs)
    assert list(failed.values()) == [status]
    for jid, (t, s) in done.items():
        assert np.array_equal(t, ref[jid][0]) and np.array_equal(s, ref[jid][1]), jid
    st = srv.stats()
    assert (st.completed, st.failed, st.running, st.queued, st.bytes_in_use) == (len(jobs) - 1, 1, 0, 0, 0)
    t0 = time.perf_counter()
    srv.shutdown(10_000)
    assert time.perf_counter() - t0 < 10.0
    srv.close()


def test_scheduler_failure_ends_every_pending_job(bfi, dev):
    """If the scheduler thread stops on an error (injected after the third
    completed pass), the jobs it finished keep their results, every other job
    fails with BFI_E_NOMEM (no wait is left without an end), new submissions
    are refused with BFI_E_BUSY, and shutdown returns within its bound."""
    import time
    jobs = _mix(12)
    srv = bfi.Server(slots=2, precision=1)
    srv.inject_fault(bfi.FAULT_SCHEDULER, 2)
    done, failed = _run_all(bfi, srv, jobs)
    assert len(done) == 2 and len(failed) == len(jobs) - 2 and set(failed.values()) == {2}
    st = srv.stats()
    assert st.completed == 2 and st.failed == len(jobs) - 2
    with pytest.raises(bfi.BfiError) as e:
        srv.submit(_lat(bfi, jobs[0]), jobs[0].lo, jobs[0].hi, jobs[0].samples, 1, 0)
    assert e.value.status == 6  # BFI_E_BUSY
    t0 = time.perf_counter()
    srv.shutdown(10_000)
    assert time.perf_counter() - t0 < 10.0
    srv.close()


def test_shutdown_is_bounded_while_passes_run(bfi, dev):
    """shutdown with a short limit while a long pass runs returns BFI_E_TIMEOUT
    in time; the queued job is cancelled; a later shutdown completes."""
    import time
    big = workloads.paper_10x2(1 << 22)  # 2^32 samples in FP64: tens of milliseconds on the device
    srv = bfi.Server(slots=1, precision=0)
    a = srv.submit(bfi.lattice(10, 2), big.lo, big.hi, big.samples, big.seed, 1)
    b = srv.submit(bfi.lattice(10, 2), big.lo, big.hi, big.samples, big.seed, 2)
    while a.info().state == 0:  # until the first pass is admitted
        time.sleep(0.001)
    t0 = time.perf_counter()
    with pytest.raises(bfi.BfiError) as e:
        srv.shutdown(1)
    assert e.value.status == 4 and time.perf_counter() - t0 < 1.0  # BFI_E_TIMEOUT
    srv.shutdown(60_000)
    assert a.info().state == 2 and b.info().state == 3
    srv.close()
