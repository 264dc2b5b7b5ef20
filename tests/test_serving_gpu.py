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
    totals, slots, lo, hi, sid = req.result(leaves=True)
    srv.close()
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
