"""Adaptive subdivision with the convergence test of Sec. 3 on the GPU
against the oracle's driver: the same decisions (checked to lie well away from
their thresholds, so rounding cannot flip them), the same leaves in the same
order, and results within the FP64 parity bounds."""
import math

import numpy as np
import pytest

import oracle
from oracle.adaptive import Convergence, adaptive_integrate, adaptive_nsphere
from test_parity_gpu import FP64_RTOL, assert_slots_close, assert_totals_close

SAFE_MARGIN = 1e-8  # decisions closer than this to a threshold could flip under rounding

NSPHERE = [  # dims, n, seed, conv, lo, hi
    (3, 100_000, 1, Convergence(2.0, 0.003, 0.0, 0.0, 8, 1 << 16), -1.0, 1.0),     # Listing 1
    (2, 4_000, 2, Convergence(2.0, 0.0, 0.0, 1e-300, 3, 1 << 10), 0.5, 1.3),
    (5, 20_000, 3, Convergence(2.0, 0.01, 0.0, 0.0, 6, 256), -1.0, 1.0),
    (2, 256, 1, Convergence(2.0, 0.0, 0.0, 0.0, 6, 5), -1.0, 1.0),
    (4, 30_001, 4, Convergence(1.5, 0.02, 1e-3, 0.0, 5, 64), -0.9, 1.0),
]


def _conv(bfi, c):
    return bfi.convergence(c.factor, c.rel_tol, c.abs_tol, c.small, c.max_depth, c.max_leaves)


@pytest.mark.gpu
@pytest.mark.parametrize("dims,n,seed,conv,lo,hi", NSPHERE)
def test_adaptive_nsphere_matches_oracle(bfi, dims, n, seed, conv, lo, hi):
    ores, oerr, out = adaptive_nsphere(dims, n, seed, conv, lo=lo, hi=hi)
    assert min(out.margins, default=math.inf) > SAFE_MARGIN, "a decision lies at its threshold: pick other inputs"
    res, err, stats = bfi.adaptive_nsphere(dims, n, seed, _conv(bfi, conv), lo=lo, hi=hi)
    assert stats.as_dict() == out.stats
    assert res == pytest.approx(ores, rel=1e-12, abs=1e-300)
    assert err == pytest.approx(oerr, rel=1e-10, abs=1e-300)


@pytest.mark.gpu
def test_adaptive_listing1(bfi):
    # Sec. 3, Listing 1: half the volume of the unit 4-ball, pi^2/4
    res, err, stats = bfi.adaptive_nsphere(3, 100_000, 1, bfi.convergence(2.0, 0.003, 0.0, 0.0, 8, 1 << 16))
    assert err < 0.01 and abs(res - math.pi ** 2 / 4) < 4 * err
    assert stats.leaves == stats.converged


LATTICE = [  # nx, nt, n, seed, conv, half
    (4, 2, 20_000, 3, Convergence(2.0, 0.05, 0.0, 0.0, 4, 1 << 10), 5.0),
    (3, 1, 20_000, 11, Convergence(2.0, 0.02, 0.0, 0.0, 5, 64), 5.0),
    (4, 2, 512, 7, Convergence(2.0, 0.0, 0.0, 0.0, 3, 1 << 10), 5.0),
    (10, 2, 4_096, 2, Convergence(2.0, 0.2, 0.0, 0.0, 3, 8), 5.0),
    (5, 3, 3_001, 5, Convergence(1.25, 0.1, 0.0, 0.0, 4, 6), 4.0),
]


@pytest.mark.gpu
@pytest.mark.parametrize("nx,nt,n,seed,conv,half", LATTICE)
def test_adaptive_lattice_matches_oracle(bfi, nx, nt, n, seed, conv, half):
    lat_o = oracle.lattice(nx, nt)
    o_tot, out = adaptive_integrate(lat_o, -half, half, n, seed, conv, job_id=1)
    assert min(out.margins, default=math.inf) > SAFE_MARGIN, "a decision lies at its threshold: pick other inputs"
    ctx = bfi.Context(0)
    try:
        g_tot, stats, llo, lhi, lsl = ctx.adaptive_integrate(bfi.lattice(nx, nt), -half, half, n, seed,
                                                             _conv(bfi, conv), job_id=1, leaf_capacity=4096)
    finally:
        ctx.close()
    assert stats.as_dict() == out.stats
    assert np.array_equal(llo, np.array(out.leaves_lo)) and np.array_equal(lhi, np.array(out.leaves_hi))
    o_sl = np.array(out.kept)
    R = nx // 2 + 1
    assert_slots_close(lsl, o_sl, R, FP64_RTOL)
    assert_totals_close(g_tot, o_tot, R, FP64_RTOL, 1e-9, m=o_sl[:, 1].max())


@pytest.mark.gpu
def test_adaptive_lattice_leaf_capacity_and_fp32(bfi):
    lat = bfi.lattice(4, 2)
    conv = bfi.convergence(2.0, 0.05, 0.0, 0.0, 4, 1 << 10)
    ctx = bfi.Context(0)
    try:
        t64, s64 = ctx.adaptive_integrate(lat, -5.0, 5.0, 20_000, 3, conv, job_id=1)
        t64b, s64b, llo, lhi, lsl = ctx.adaptive_integrate(lat, -5.0, 5.0, 20_000, 3, conv, job_id=1,
                                                           leaf_capacity=2)
        t32, s32 = ctx.adaptive_integrate(lat, -5.0, 5.0, 20_000, 3, conv, job_id=1, precision=bfi.FP32)
    finally:
        ctx.close()
    # deterministic, and the capacity only limits what is copied out
    assert np.array_equal(t64, t64b) and s64.as_dict() == s64b.as_dict()
    assert s64.leaves > 2 and llo.shape == (2, 8) and lsl.shape == (2, bfi.slot_len(4))
    # FP32 decides on its own results: a valid run whose Z agrees within the errors
    assert s32.leaves == s32.converged + s32.kept_depth + s32.kept_budget
    z64, z32 = math.exp(t64[0]), math.exp(t32[0])
    assert abs(z64 - z32) < 5 * math.hypot(z64 * t64[1], z32 * t32[1])


@pytest.mark.parametrize("conv", [
    Convergence(0.5, 0.1, 0.0, 0.0, 4, 16),
    Convergence(2.0, 0.1, 0.0, 0.0, 31, 16),
    Convergence(2.0, 0.1, 0.0, 0.0, -1, 16),
    Convergence(2.0, 0.1, 0.0, 0.0, 4, 0),
    Convergence(2.0, float("nan"), 0.0, 0.0, 4, 16),
])
def test_adaptive_rejects_bad_settings_before_the_device(bfi, conv):
    with pytest.raises(bfi.BfiError):
        bfi.adaptive_nsphere(2, 1000, 1, _conv(bfi, conv))


def test_adaptive_rejects_bad_boxes_before_the_device(bfi):
    conv = bfi.convergence(2.0, 0.1)
    with pytest.raises(bfi.BfiError):
        bfi.adaptive_nsphere(2, 1000, 1, conv, lo=[0, 1], hi=[1, 1])
    with pytest.raises(bfi.BfiError):
        bfi.adaptive_nsphere(2, 1, 1, conv)
    with pytest.raises(bfi.BfiError):
        bfi.adaptive_nsphere(2, 1 << 47, 1, bfi.convergence(4.0, 0.1))
