"""bfi_integrate_static_scratch, the entry point that allocates nothing.

Some callers cannot allocate device memory (a plugin whose host application
owns the device heap, a loop where allocating is not allowed after start-up).
This entry point keeps its scratch in one fixed device array inside the
library.  Here it is called through the C ABI, twice in a row (the second call
finds the first call's leftovers in the shared array), and each result is
compared with the plan path's on the same job, with the tolerances of the
parity tests.  A job too big for the array must be refused with a clear
message.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-12
FP32_RTOL = 1e-6


@pytest.fixture(scope="module")
def dev(bfi):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _close(a, b, rtol, R):
    # totals: log Z, counts and C(r) at the parity tolerance (C(r) against C(0))
    assert a[2] == b[2] and a[3] == b[3]
    assert abs(a[0] - b[0]) <= rtol * max(1.0, abs(b[0]))
    assert np.all(np.abs(a[4:4 + R] - b[4:4 + R]) <= rtol * abs(b[4]))


@pytest.mark.parametrize("precision", [0, 1])
def test_static_scratch_matches_plan_twice(bfi, dev, precision):
    rtol = FP64_RTOL if precision == 0 else FP32_RTOL
    jobs = [workloads.small_ragged(10, 2, seed=4, nsub=5, base=60_000),
            workloads.small_ragged(4, 2, seed=9, nsub=3, base=20_000)]
    for job in jobs:
        lat = bfi.lattice(job.nx, job.nt)
        R = job.nx // 2 + 1
        lo = torch.tensor(job.lo, device=dev)
        hi = torch.tensor(job.hi, device=dev)
        plan = bfi.Plan(lat, job.samples, precision)
        p_slots, p_tot = plan.execute(lo, hi, job.seed, job.job_id)
        torch.cuda.synchronize()
        p_tot = p_tot.cpu().numpy()
        p_slots = p_slots.cpu().numpy()
        for _ in range(2):
            s_slots, s_tot = bfi.integrate_static_scratch(lat, job.samples, lo, hi, job.seed, job.job_id,
                                                          precision=precision)
            torch.cuda.synchronize()
            s_tot = s_tot.cpu().numpy()
            _close(s_tot, p_tot, rtol, R)
            np.testing.assert_array_equal(s_slots.cpu().numpy()[:, 0], p_slots[:, 0])
            np.testing.assert_allclose(s_slots.cpu().numpy()[:, 3], p_slots[:, 3], rtol=rtol)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("log2n", [23, 24])
def test_static_scratch_two_stage_screen(bfi, dev, precision, log2n):
    """10x2 with 16 subvolumes of 2^23 samples (2^27 in all, 2048 chunk
    records, well inside the array): chunks of 256 rows per thread, so the
    two-stage screen and its survivor queue run on the static scratch's hint
    and counter layout.  With 2^24 per subvolume the chunks hold 512 rows and
    the last two subvolumes are cut into tail chunks of 256 rows, the table
    the static scratch builds on the device.  Two calls in a row, each against
    the plan path."""
    rtol = FP64_RTOL if precision == 0 else FP32_RTOL
    lo_np, hi_np = workloads.bisected_boxes(20, 4)
    samples = np.full(16, 1 << log2n, dtype=np.uint64)
    lat = bfi.lattice(10, 2)
    lo = torch.tensor(lo_np, device=dev)
    hi = torch.tensor(hi_np, device=dev)
    plan = bfi.Plan(lat, samples, precision)
    p_slots, p_tot = plan.execute(lo, hi, 6)
    torch.cuda.synchronize()
    info = plan.info()
    assert plan.screen_stats()[1] and info.chunk_samples == (256 << (log2n - 23)) * 256
    assert info.tail_subvolume == (16 if log2n == 23 else 14)
    p_slots, p_tot = p_slots.cpu().numpy(), p_tot.cpu().numpy()
    for _ in range(2):
        s_slots, s_tot = bfi.integrate_static_scratch(lat, samples, lo, hi, 6, precision=precision)
        torch.cuda.synchronize()
        s_slots, s_tot = s_slots.cpu().numpy(), s_tot.cpu().numpy()
        _close(s_tot, p_tot, rtol, 6)
        # the same kernels on the same chunks: the records agree bit for bit
        np.testing.assert_array_equal(s_slots, p_slots)


def test_static_scratch_refuses_jobs_beyond_its_size(bfi, dev):
    job = workloads.paper_10x2(1 << 26)   # 2^36 samples: ~131k chunk records, more than 16 MiB
    lat = bfi.lattice(job.nx, job.nt)
    lo = torch.tensor(job.lo, device=dev)
    hi = torch.tensor(job.hi, device=dev)
    with pytest.raises(bfi.BfiError) as e:
        bfi.integrate_static_scratch(lat, job.samples, lo, hi, job.seed)
    assert e.value.status == 1 and "static scratch holds" in str(e.value)
