"""The register-resident screen of the generic kernel (Nx = G SPL, each lane
of a G-lane group owning whole sites and Philox blocks; half-warp groups, two
samples per warp, for 32x4, 64x2 and 128x1) on every shape it is compiled
for, against the oracle: FP64 records at the FP64 parity bound, FP32 records
against the oracle on the same float points, and general parameters with the
mass term (the screen's second group sum) on the half-warp shapes."""
import numpy as np
import pytest

import oracle
import workloads
from test_parity_gpu import (FP32_ERR_ATOL, FP32_RTOL, FP64_RTOL, assert_slots_close, assert_totals_close, budget,
                             dev, run_gpu, run_oracle)  # noqa: F401 (dev is a fixture)

# Nx = G SPL with SPL Nt in {4, 8, 16}: odd Nt (scalar residuals), Nt = 2 (the
# packed pair's seam on every slice), and up to 16 coordinates per lane
LANES = [(32, 4), (32, 8), (32, 16), (64, 2), (64, 4), (64, 8), (128, 1), (128, 2), (128, 4), (256, 1),
         (256, 2), (512, 1)]


@pytest.mark.gpu
@pytest.mark.parametrize("nx,nt", LANES)
def test_lane_screen_fp64(bfi, dev, nx, nt):
    job = workloads.small_ragged(nx, nt, seed=40 + nx + nt, nsub=3, base=budget(nx, nt, 30_000))
    g_s, g_t, plan = run_gpu(bfi, dev, job, 0)
    assert plan.info().kernel == 1
    o_s, o_t = run_oracle(job)
    R = nx // 2 + 1
    assert_slots_close(g_s, o_s, R, FP64_RTOL)
    assert_totals_close(g_t, o_t, R, FP64_RTOL, 1e-9, m=o_s[:, 1].max())


@pytest.mark.gpu
@pytest.mark.parametrize("nx,nt", LANES)
def test_lane_screen_fp32(bfi, dev, nx, nt):
    job = workloads.small_ragged(nx, nt, seed=60 + nx + nt, nsub=3, base=budget(nx, nt, 30_000))
    g_s, g_t, _ = run_gpu(bfi, dev, job, 1)
    o_s, o_t = run_oracle(job, fp32_points=True)
    R = nx // 2 + 1
    assert_slots_close(g_s, o_s, R, FP32_RTOL)
    assert_totals_close(g_t, o_t, R, FP32_RTOL, 1e-4, FP32_ERR_ATOL)


@pytest.mark.gpu
@pytest.mark.parametrize("nx,nt", [(32, 4), (64, 2), (128, 1)])
def test_lane_screen_general_parameters(bfi, dev, nx, nt):
    job = workloads.small_ragged(nx, nt, seed=80 + nx, nsub=2, base=budget(nx, nt, 20_000), half=2.0)
    job.nu, job.D, job.a, job.tau = 0.4, 1.7, 0.8, 0.6
    g_s, g_t, _ = run_gpu(bfi, dev, job, 0, nonlinear=1.0, mass2=0.5)
    o_s, o_t = run_oracle(job, nonlinear=1.0, mass2=0.5)
    R = nx // 2 + 1
    assert_slots_close(g_s, o_s, R, FP64_RTOL)
    assert_totals_close(g_t, o_t, R, FP64_RTOL, 1e-9, m=o_s[:, 1].max())
