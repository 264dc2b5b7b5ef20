"""Batches: many uneven jobs in one CUDA graph.  Each job's result must be the
one its own plan gives alone (bitwise: same chunking, same kernels), on every
replay of the graph, and the grid autotuner must return a valid grid."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev(bfi):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _small_jobs(seed=7):
    rng = np.random.default_rng(seed)
    jobs = workloads.batch_jobs(10, seed=3, rng=rng)
    for j in jobs:  # keep the test quick: at most 2^16 points per job
        j.samples = np.minimum(j.samples, max(1, (1 << 16) // j.nsub)).astype(np.uint64)
    jobs.append(workloads.small_ragged(5, 3, seed=3, nsub=3, base=5000))     # generic kernel
    jobs.append(workloads.small_ragged(32, 4, seed=3, nsub=2, base=4000))    # generic kernel
    for k, j in enumerate(jobs):
        j.job_id = 100 + k
    return jobs


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_jobs_alone(bfi, dev, precision):
    jobs = _small_jobs()
    descs, alone = [], []
    for j in jobs:
        lat = bfi.lattice(j.nx, j.nt, j.nu, j.D, j.a, j.tau)
        lo = torch.tensor(j.lo, device=dev)
        hi = torch.tensor(j.hi, device=dev)
        descs.append(dict(lattice=lat, samples=j.samples, lo=lo, hi=hi, seed=j.seed, job_id=j.job_id))
        s, t = bfi.Plan(lat, j.samples, precision).execute(lo, hi, j.seed, j.job_id)
        torch.cuda.synchronize()
        alone.append((s.cpu().numpy(), t.cpu().numpy()))
    batch = bfi.Batch(descs, precision=precision, nstreams=4, autotune=True)
    for rep in range(2):
        for t in batch.totals:
            t.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        for k in range(len(jobs)):
            assert np.array_equal(batch.slots[k].cpu().numpy(), alone[k][0]), (rep, k)
            assert np.array_equal(batch.totals[k].cpu().numpy(), alone[k][1]), (rep, k)
    batch.close()


def test_autotuned_grid_is_valid_and_does_not_change_results(bfi, dev):
    job = workloads.small_ragged(10, 2, seed=2, nsub=4, base=50_000)
    lat = bfi.lattice(10, 2)
    c = bfi.autotune_grid(lat, 1)
    plan = bfi.Plan(lat, job.samples, 1)
    assert 1 <= c <= plan.info().ctas_per_sm_max
    lo = torch.tensor(job.lo, device=dev)
    hi = torch.tensor(job.hi, device=dev)
    ref = [x.cpu().numpy() for x in plan.execute(lo, hi, job.seed)]
    for g in range(1, plan.info().ctas_per_sm_max + 1):
        plan.set_grid(g)
        assert plan.info().ctas_per_sm == g
        out = [x.cpu().numpy() for x in plan.execute(lo, hi, job.seed)]
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
    with pytest.raises(bfi.BfiError):
        plan.set_grid(plan.info().ctas_per_sm_max + 1)
