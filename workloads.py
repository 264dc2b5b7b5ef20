"""Seeded synthetic workloads shaped like the paper's (Sec. 4: a 10x2 lattice,
nu = D = a = tau = 1, the integration volume split into subvolumes, 1e6-2e6
samples per subvolume).  Input recipes only: box bounds, budgets, seeds and
lattice parameters.  None of the method's arithmetic lives here, so the CUDA
path and the CPU oracle can both be fed from it.

The paper maps the infinite range to +-1 with a transform it does not state;
these workloads integrate over the truncated box [-5, 5]^d instead.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Job:
    nx: int
    nt: int
    lo: np.ndarray            # [nsub, d]
    hi: np.ndarray            # [nsub, d]
    samples: np.ndarray       # [nsub] uint64
    seed: int
    job_id: int = 0
    sub_id: np.ndarray | None = None
    nu: float = 1.0
    D: float = 1.0
    a: float = 1.0
    tau: float = 1.0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.nx * self.nt

    @property
    def nsub(self) -> int:
        return int(self.lo.shape[0])

    @property
    def total_samples(self) -> int:
        return int(np.sum(self.samples, dtype=np.uint64))

    def subset(self, idx) -> "Job":
        """The same job restricted to some subvolumes (their sub_ids kept)."""
        idx = np.asarray(idx)
        sid = np.arange(self.nsub, dtype=np.uint32) if self.sub_id is None else self.sub_id
        return Job(self.nx, self.nt, self.lo[idx], self.hi[idx], self.samples[idx], self.seed,
                   self.job_id, sid[idx].astype(np.uint32), self.nu, self.D, self.a, self.tau,
                   self.name + f"[{len(idx)} subvolumes]", dict(self.meta))


def bisected_boxes(d: int, k: int, half: float = 5.0):
    """2^k subvolumes of [-half, half]^d.  With k <= d, coordinate j < k is
    bisected once: subvolume s takes the upper half [0, half] of coordinate j
    iff bit j of s is set, and the full range in coordinates j >= k.  With
    k > d the bisection cycles over the coordinates: bit b of s splits
    coordinate b mod d once more, the bits of a coordinate read from its first
    split (most significant) on, so every subvolume is one of 2^(levels)
    equal intervals in each coordinate."""
    nsub = 1 << k
    lo = np.full((nsub, d), -half)
    hi = np.full((nsub, d), half)
    s = np.arange(nsub)
    for j in range(min(d, k)):
        bits = list(range(j, k, d))   # the bits of s that split coordinate j, first split first
        idx = np.zeros(nsub, dtype=np.int64)
        for b in bits:
            idx = 2 * idx + ((s >> b) & 1)
        width = 2.0 * half / (1 << len(bits))
        lo[:, j] = -half + idx * width
        hi[:, j] = -half + (idx + 1) * width
    return lo, hi


def plain_4x2(samples: int = 1 << 20) -> Job:
    """4x2 lattice (8 dimensions), box [-5,5]^8 as one volume, seed 1."""
    lo, hi = bisected_boxes(8, 0)
    return Job(4, 2, lo, hi, np.array([samples], dtype=np.uint64), seed=1, name="4x2 one volume")


def paper_10x2(samples_per_sub: int = 1 << 20) -> Job:
    """10x2 lattice (20 dimensions), [-5,5]^20 bisected along coordinates 0..9
    into 1024 equal subvolumes, seed 2."""
    lo, hi = bisected_boxes(20, 10)
    return Job(10, 2, lo, hi, np.full(1024, samples_per_sub, dtype=np.uint64), seed=2,
               name=f"10x2 1024 subvolumes x {samples_per_sub}")


def small_ragged(nx: int, nt: int, seed: int = 5, nsub: int = 3, base: int = 40_000,
                 half: float = 5.0) -> Job:
    """A few subvolumes with budgets that are not multiples of any chunk size."""
    d = nx * nt
    k = int(np.ceil(np.log2(max(nsub, 1))))
    lo, hi = bisected_boxes(d, min(k, d), half)
    lo, hi = lo[:nsub], hi[:nsub]
    samples = np.array([base + 1237 * s + 3 for s in range(nsub)], dtype=np.uint64)
    return Job(nx, nt, lo, hi, samples, seed=seed, name=f"{nx}x{nt} ragged")


def batch_jobs(njobs: int = 256, seed: int = 3, extra_64x8: float = 0.0, rng=None):
    """Uneven jobs: Nx from {4,6,8,10,16,32}, Nt from {2,4}, nu log-uniform in
    [0.1,10], D = 1, box [-5,5]^d bisected along its first coordinates into
    2^k subvolumes with k uniform in 6..10 (64-1024), a total budget
    log-uniform in [2^20, 2^28] points split evenly; job k has job_id k and
    Philox seed 'seed'.  A fraction extra_64x8 of the jobs are 64x8 lattices
    instead.  The parameters are drawn with numpy's PCG64 seeded by 'seed'."""
    rng = np.random.default_rng(seed) if rng is None else rng
    jobs = []
    for k in range(njobs):
        if extra_64x8 > 0 and rng.uniform() < extra_64x8:
            nx, nt = 64, 8
        else:
            nx = int(rng.choice([4, 6, 8, 10, 16, 32]))
            nt = int(rng.choice([2, 4]))
        nu = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        kk = int(rng.integers(6, 11))
        total = float(np.exp(rng.uniform(20 * np.log(2), 28 * np.log(2))))
        d = nx * nt
        lo, hi = bisected_boxes(d, min(kk, d))
        nsub = lo.shape[0]
        per = max(1, int(total) // nsub)
        jobs.append(Job(nx, nt, lo, hi, np.full(nsub, per, dtype=np.uint64), seed=seed, job_id=k, nu=nu,
                        name=f"batch job {k}: {nx}x{nt}, nu={nu:.3g}, {nsub} x {per}"))
    return jobs
