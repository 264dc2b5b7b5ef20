"""The multi-rank path without GPUs: two gloo ranks on the CPU each integrate a
contiguous shard of a job's subvolumes (with the oracle, since no GPU is
here), all-gather the records with the library's gather and merge them with
the library's FP64 merge; the result must equal the single-process merge."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _job():
    lo, hi = workloads.bisected_boxes(8, 3)
    return workloads.Job(4, 2, lo, hi, np.array([2000, 3000, 1000, 0, 2500, 1500, 3500, 500], dtype=np.uint64),
                         seed=4, job_id=2)


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1803_07560_gb300 import shard
        job = _job()
        a, b = shard.shard_range(job.nsub, world, rank)
        sid = np.arange(a, b, dtype=np.uint32)
        slots, _ = oracle.integrate(oracle.lattice(4, 2), job.lo[a:b], job.hi[a:b], job.samples[a:b], job.seed,
                                    job.job_id, sub_id=sid, nthreads=1)
        totals = shard.merge_across_ranks(4, torch.tensor(slots))
        np.save(os.path.join(out, f"rank{rank}.npy"), totals)
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_every_subvolume_once():
    from paper_1803_07560_gb300 import shard
    for n in (1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, b = shard.shard_range(n, world, r)
                seen += list(range(a, b))
            assert seen == list(range(n))


def test_two_gloo_ranks_merge_to_the_single_process_result(tmp_path, bfi):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    job = _job()
    slots, totals = oracle.integrate(oracle.lattice(4, 2), job.lo, job.hi, job.samples, job.seed, job.job_id)
    ref = bfi.merge_host(4, slots)
    np.testing.assert_allclose(ref, totals, rtol=1e-13)
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npy")
        assert np.array_equal(got, ref)
