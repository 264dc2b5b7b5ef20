"""The transform and Gaussian samplers on the GPU against the oracle's
(oracle/maps.py): records and totals within the FP64 parity bounds, the
zero-variance case, empty boxes, the context path, and argument checks.  The
linear-limit proposal is host code and is checked on the CPU."""
import math

import numpy as np
import pytest

import oracle
from oracle.maps import GAUSSIAN, TRANSFORM, integrate_mapped, proposal_covariance
from test_parity_gpu import FP64_RTOL, assert_slots_close, assert_totals_close
from gl_reference import linear_limit


@pytest.mark.parametrize("nx,nt,sigma,mass2", [(4, 2, 4.0, 0.0), (10, 2, 5.0, 0.0), (5, 3, math.inf, 0.5),
                                               (3, 1, 2.0, 0.0), (8, 8, 3.0, 0.0)])
def test_gaussian_proposal_covariance(bfi, nx, nt, sigma, mass2):
    F = bfi.gaussian_proposal(bfi.lattice(nx, nt, mass2=mass2), sigma)
    assert np.allclose(np.tril(F, -1), 0.0)  # upper triangular
    cov = proposal_covariance(oracle.lattice(nx, nt, mass2=mass2), sigma)
    np.testing.assert_allclose(F @ F.T, cov, rtol=1e-9, atol=1e-11 * np.abs(cov).max())


def test_gaussian_proposal_needs_a_regulator(bfi):
    with pytest.raises(bfi.BfiError):
        bfi.gaussian_proposal(bfi.lattice(4, 2), math.inf)       # constant mode unregulated
    with pytest.raises(bfi.BfiError):
        bfi.gaussian_proposal(bfi.lattice(16, 8), 1.0)           # d = 128 > 64


def _boxes_in_unit_cube(d, nsub, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, (nsub, d))
    b = rng.uniform(-1.0, 1.0, (nsub, d))
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    lo[0], hi[0] = -1.0, 1.0  # the whole range: all of R^d
    return lo, hi


def _run_plan(bfi, lat, lo, hi, samples, seed, sub_id, kind, mean=None, factor=None):
    import torch
    plan = bfi.Plan(lat, samples)
    plan.set_sampler(kind, mean=mean, factor=factor)
    dev = torch.device("cuda:0")
    slots = torch.empty((lo.shape[0], bfi.slot_len(lat.nx)), dtype=torch.float64, device=dev)
    totals = torch.empty(bfi.totals_len(lat.nx), dtype=torch.float64, device=dev)
    plan.execute(torch.from_numpy(lo).to(dev), torch.from_numpy(hi).to(dev), seed,
                 sub_id=None if sub_id is None else torch.from_numpy(sub_id.astype(np.int32)).to(dev), slots=slots,
                 totals=totals)
    torch.cuda.synchronize()
    out = slots.cpu().numpy(), totals.cpu().numpy()
    plan.close()
    return out


# (5, 3) and (7, 2) run on the warp-per-sample kernel; the other shapes have a
# compiled thread-per-sample kernel (both translation units of shapes)
@pytest.mark.gpu
@pytest.mark.parametrize("nx,nt,mass2,nonlinear", [(4, 2, 0.0, 1.0), (10, 2, 0.0, 1.0), (5, 3, 0.3, 1.0),
                                                   (3, 1, 1.0, 0.0), (2, 2, 0.0, 1.0), (7, 2, 0.0, 1.0),
                                                   (6, 4, 0.0, 1.0), (16, 2, 0.2, 1.0), (16, 4, 0.0, 1.0)])
def test_transform_matches_oracle(bfi, nx, nt, mass2, nonlinear):
    d = nx * nt
    lo, hi = _boxes_in_unit_cube(d, 3, seed=nx * 10 + nt)
    samples = np.array([20_011, 3_000, 9_999], dtype=np.uint64)
    sid = np.array([5, 1, 9], dtype=np.uint32)
    g_s, g_t = _run_plan(bfi, bfi.lattice(nx, nt, nonlinear=nonlinear, mass2=mass2), lo, hi, samples, 7, sid,
                         bfi.SAMPLE_TRANSFORM)
    o_s, o_t = integrate_mapped(oracle.lattice(nx, nt, nonlinear=nonlinear, mass2=mass2), lo, hi, samples, 7,
                                sub_id=sid, kind=TRANSFORM)
    R = nx // 2 + 1
    assert_slots_close(g_s, o_s, R, FP64_RTOL)
    assert_totals_close(g_t, o_t, R, FP64_RTOL, 1e-9, m=np.abs(o_s[:, 1]).max())


@pytest.mark.gpu
@pytest.mark.parametrize("nx,nt", [(10, 2), (5, 3)])
def test_transform_ragged_counts_and_edge_boxes(bfi, nx, nt):
    """Sample counts of 0, 1, one short of a CTA row, a row and a few chunks,
    and boxes near the ends of the range: a slab in every coordinate near
    y = 1 (v between 128 and 256) and one near y = -1, the whole range, and a
    box of width 2^-20 around 0.  (Slabs closer to +-1 put S far beyond 1e9,
    where two FP64 evaluations of exp(-S) share no digits.)"""
    d = nx * nt
    lo = np.stack([np.full(d, -1.0), np.full(d, 1.0 - 2.0 ** -8), np.full(d, -1.0 + 2.0 ** -9), np.full(d, -1.0),
                   np.full(d, -2.0 ** -21), np.full(d, -0.5), np.full(d, -1.0)])
    hi = np.stack([np.full(d, 1.0), np.full(d, 1.0 - 2.0 ** -9), np.full(d, -1.0 + 2.0 ** -8), np.full(d, 1.0),
                   np.full(d, 2.0 ** -21), np.full(d, 0.25), np.full(d, 1.0)])
    samples = np.array([0, 4097, 3001, 1, 255, 256, 70_001], dtype=np.uint64)
    g_s, g_t = _run_plan(bfi, bfi.lattice(nx, nt), lo, hi, samples, 11, None, bfi.SAMPLE_TRANSFORM)
    o_s, o_t = integrate_mapped(oracle.lattice(nx, nt), lo, hi, samples, 11, kind=TRANSFORM)
    R = nx // 2 + 1
    assert g_s[0, 0] == 0 and g_s[0, 1] == math.inf and np.all(g_s[0, 3:] == 0.0)
    assert_slots_close(g_s, o_s, R, FP64_RTOL)
    assert_totals_close(g_t, o_t, R, FP64_RTOL, 1e-9, m=np.abs(o_s[1:, 1]).max())


# factor: "lower" (Cholesky factor of the covariance), "upper" (the inverse
# transpose of the precision's Cholesky factor, the form of
# bfi_gaussian_proposal) or "dense" (lower times an orthogonal matrix).
# Shapes with d <= 40 in the compiled tables run on the thread-per-sample
# kernel (upper: its triangular form); (5, 3), (8, 8) and (32, 2) on the
# warp-per-sample kernel.
@pytest.mark.gpu
@pytest.mark.parametrize("nx,nt,sigma,with_mean,factor", [(4, 2, 4.0, False, "lower"), (10, 2, 5.0, False, "lower"),
                                                          (3, 1, 2.0, True, "lower"), (5, 3, 3.0, True, "dense"),
                                                          (8, 8, 3.0, False, "lower"), (10, 2, 5.0, True, "upper"),
                                                          (6, 4, 3.0, False, "upper"), (8, 4, 3.0, True, "dense"),
                                                          (10, 4, 4.0, False, "upper"), (2, 1, 2.0, False, "upper"),
                                                          (32, 2, 3.0, False, "upper")])
def test_gaussian_matches_oracle(bfi, nx, nt, sigma, with_mean, factor):
    d = nx * nt
    lat_o = oracle.lattice(nx, nt)
    cov = proposal_covariance(lat_o, sigma)
    F = np.linalg.cholesky(cov)
    rng = np.random.default_rng(d)
    if factor == "dense":  # any non-singular factor, not only a triangular one
        Q, _ = np.linalg.qr(rng.normal(size=(d, d)))
        F = F @ Q
    elif factor == "upper":
        F = np.linalg.inv(np.linalg.cholesky(np.linalg.inv(cov))).T
        assert np.allclose(np.tril(F, -1), 0.0) and np.allclose(F @ F.T, cov)
        F = np.triu(F)
    mean = rng.normal(scale=0.3, size=d) if with_mean else None
    lo = np.stack([np.full(d, -5.0), np.full(d, -2.0), np.full(d, 0.0)])
    hi = np.stack([np.full(d, 5.0), np.full(d, 3.0), np.full(d, 5.0)])
    samples = np.array([30_001, 8_000, 12_345], dtype=np.uint64)
    g_s, g_t = _run_plan(bfi, bfi.lattice(nx, nt), lo, hi, samples, 3, None, bfi.SAMPLE_GAUSSIAN, mean=mean,
                         factor=F)
    o_s, o_t = integrate_mapped(lat_o, lo, hi, samples, 3, kind=GAUSSIAN, mean=mean, factor=F)
    R = nx // 2 + 1
    used = np.isfinite(o_s[:, 1])
    assert np.array_equal(used, np.isfinite(g_s[:, 1]))
    assert np.array_equal(g_s[~used], o_s[~used])
    assert_slots_close(g_s[used], o_s[used], R, FP64_RTOL)
    assert_totals_close(g_t, o_t, R, FP64_RTOL, 1e-9, m=np.abs(o_s[used, 1]).max())


@pytest.mark.gpu
def test_gaussian_zero_variance_and_closed_form(bfi):
    lat = bfi.lattice(4, 2, nonlinear=0.0, mass2=1.0)
    F = bfi.gaussian_proposal(lat, math.inf)   # the target itself
    lo, hi = np.full((1, 8), -1e3), np.full((1, 8), 1e3)
    _, t = _run_plan(bfi, lat, lo, hi, np.array([1 << 20], dtype=np.uint64), 5, None, bfi.SAMPLE_GAUSSIAN, factor=F)
    Z_exact, C_exact, _ = linear_limit(4, 2, mass2=1.0)
    assert math.exp(t[0]) == pytest.approx(Z_exact, rel=1e-10)
    assert t[1] < 1e-6
    for r in range(3):
        assert abs(t[4 + r] - C_exact[r]) < 5 * t[4 + 3 + r]


@pytest.mark.gpu
def test_gaussian_box_no_sample_hits(bfi):
    lat = bfi.lattice(3, 1)
    F = np.eye(3) * 1e-3
    s, t = _run_plan(bfi, lat, np.full((1, 3), 4.0), np.full((1, 3), 5.0), np.array([1000], dtype=np.uint64), 1,
                     None, bfi.SAMPLE_GAUSSIAN, factor=F)
    assert s[0, 0] == 1000 and s[0, 1] == math.inf and s[0, 3] == 0.0
    assert t[0] == -math.inf


@pytest.mark.gpu
def test_context_sampler_path_and_checks(bfi):
    lat = bfi.lattice(4, 2)
    lo, hi = _boxes_in_unit_cube(8, 2, seed=1)
    samples = np.array([5000, 7000], dtype=np.uint64)
    ctx = bfi.Context(0)
    try:
        ctx.set_sampler(bfi.SAMPLE_TRANSFORM)
        c_s, c_t = ctx.integrate(lat, lo, hi, samples, 4)
        ctx.set_sampler(bfi.SAMPLE_BOX)
        b_s, _ = ctx.integrate(lat, lo, hi, samples, 4)
        with pytest.raises(bfi.BfiError):
            ctx.set_sampler(bfi.SAMPLE_TRANSFORM)
            ctx.integrate(lat, lo, hi, samples, 4, precision=bfi.FP32)   # FP64 only
    finally:
        ctx.close()
    p_s, p_t = _run_plan(bfi, lat, lo, hi, samples, 4, None, bfi.SAMPLE_TRANSFORM)
    assert np.array_equal(c_s, p_s) and np.array_equal(c_t, p_t)
    assert not np.array_equal(b_s, c_s)
    plan = bfi.Plan(bfi.lattice(16, 8), [1000])
    try:
        with pytest.raises(bfi.BfiError):
            plan.set_sampler(bfi.SAMPLE_GAUSSIAN, factor=np.eye(128))   # d > 64
        with pytest.raises(bfi.BfiError):
            plan.set_sampler(7)
    finally:
        plan.close()
    plan = bfi.Plan(bfi.lattice(3, 1), [1000])
    try:
        with pytest.raises(bfi.BfiError):
            plan.set_sampler(bfi.SAMPLE_GAUSSIAN, factor=np.zeros((3, 3)))   # singular
    finally:
        plan.close()
