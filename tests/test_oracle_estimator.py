"""Pins of the oracle's estimator (steps a3, a5, a6): the paper's worked Monte
Carlo example, Gauss-Legendre quadrature on tiny lattices, the closed form of
the regulated linear limit, calibration of the stated errors, subvolume
additivity, merge invariants and edge cases."""
import os

import numpy as np
import pytest

import oracle
from gl_reference import gl_box, linear_limit

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "listing2_nsphere.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _box(d, half):
    return np.full((1, d), -half), np.full((1, d), half)


def test_listing2_nsphere_example():
    # Sec. 3, Listing 2: 1e7 plain-MC samples of sqrt(1-|x|^2) over [-1,1]^2.
    g = _golden()
    n, dims = int(g["samples"]), int(g["dims"])
    exact = 2 * np.pi / 3
    vol = (g["hi"] - g["lo"]) ** dims
    sigma_exact = vol * np.sqrt(np.pi / 8 - (np.pi / 6) ** 2) / np.sqrt(n)
    # the paper's printed error is the plain-MC V sigma / sqrt(n) of its run
    assert g["printed_abs_error"] == pytest.approx(sigma_exact, rel=2e-4)
    assert abs(g["printed_result"] - exact) < 4 * g["printed_abs_error"]
    res, err = oracle.nsphere(dims, n, seed=1)
    assert err == pytest.approx(g["printed_abs_error"], rel=0.01)
    assert abs(res - exact) < 4 * err


@pytest.mark.parametrize("nx,nt,half,gl", [(3, 1, 5.0, (16, 8)), (4, 1, 5.0, (6, 8)),
                                           (2, 2, 5.0, (6, 8))])
def test_mc_agrees_with_gauss_legendre(nx, nt, half, gl):
    d = nx * nt
    R = nx // 2 + 1
    Zq, Nq = gl_box(nx, nt, -half, half, panels=gl[0], order=gl[1])
    lat = oracle.lattice(nx, nt)
    lo, hi = _box(d, half)
    _, tot = oracle.integrate(lat, lo, hi, 2 ** 18, seed=11)
    Z = np.exp(tot[0])
    assert abs(Z - Zq) < 4 * Z * tot[1]
    C = tot[4:4 + R]
    assert np.all(np.abs(C - Nq / Zq) < 4 * tot[4 + R:])


def test_gauss_legendre_is_converged():
    Z1, N1 = gl_box(3, 1, -5, 5, panels=16, order=8)
    Z2, N2 = gl_box(3, 1, -5, 5, panels=24, order=8)
    assert Z1 == pytest.approx(Z2, rel=1e-9)
    np.testing.assert_allclose(N1, N2, rtol=1e-9)


@pytest.mark.parametrize("nx,nt", [(2, 1), (3, 1)])
def test_linear_limit_closed_form(nx, nt):
    # Nonlinear term off, mass2 = 1: Gaussian with the Fourier-diagonal precision.
    # The box half-width 8 is >= 8 sigma_max (sigma_max = 1/sqrt(mass2)).
    d = nx * nt
    R = nx // 2 + 1
    Zc, Cc, lam = linear_limit(nx, nt, mass2=1.0)
    assert 8.0 >= 8.0 / np.sqrt(lam.min())
    Zq, Nq = gl_box(nx, nt, -8, 8, panels=16, order=8, nonlinear=0.0, mass2=1.0)
    assert Zq == pytest.approx(Zc, rel=1e-10)
    np.testing.assert_allclose(Nq / Zq, Cc, rtol=1e-10, atol=1e-12)
    lat = oracle.lattice(nx, nt, nonlinear=0.0, mass2=1.0)
    lo, hi = _box(d, 8.0)
    _, tot = oracle.integrate(lat, lo, hi, 2 ** 19, seed=4)
    assert abs(np.exp(tot[0]) - Zc) < 4 * np.exp(tot[0]) * tot[1]
    assert np.all(np.abs(tot[4:4 + R] - Cc) < 4 * tot[4 + R:])


def test_linear_limit_without_regulator_grows_with_box():
    # Without mass2 the constant mode has zero action: Z grows with the box.
    lat = oracle.lattice(3, 1, nonlinear=0.0, mass2=0.0)
    z = []
    for half in (2.0, 4.0, 8.0):
        lo, hi = _box(3, half)
        _, tot = oracle.integrate(lat, lo, hi, 2 ** 16, seed=1)
        z.append(tot[0])
    assert z[0] < z[1] < z[2]


def test_stated_errors_are_calibrated():
    # z-scores of 96 independent runs against quadrature: mean ~ 0, spread ~ 1.
    nx, nt, half = 3, 1, 5.0
    R = nx // 2 + 1
    Zq, Nq = gl_box(nx, nt, -half, half, panels=16, order=8)
    lat = oracle.lattice(nx, nt)
    lo, hi = _box(3, half)
    zs_Z, zs_C = [], []
    for seed in range(100, 196):
        _, tot = oracle.integrate(lat, lo, hi, 4096, seed=seed, nthreads=1)
        Z = np.exp(tot[0])
        zs_Z.append((Z - Zq) / (Z * tot[1]))
        zs_C.append((tot[4:4 + R] - Nq / Zq) / tot[4 + R:])
    zs_Z = np.array(zs_Z)
    zs_C = np.array(zs_C)
    assert abs(zs_Z.mean()) < 0.45 and 0.7 < zs_Z.std() < 1.3
    for r in range(R):
        assert abs(zs_C[:, r].mean()) < 0.45 and 0.7 < zs_C[:, r].std() < 1.3


def test_subvolume_additivity():
    # Sec. 1/3: the integral over a region is the sum over its parts.  Quadrature
    # over a 2x2x2 split matches the whole box; MC over the split agrees within sigma.
    nx, nt, half = 3, 1, 5.0
    R = nx // 2 + 1
    Zw, Nw = gl_box(nx, nt, -half, half, panels=16, order=8)
    Zs, Ns = 0.0, np.zeros(R)
    los, his = [], []
    for s in range(8):
        lo = np.array([0.0 if (s >> j) & 1 else -half for j in range(3)])
        hi = np.array([half if (s >> j) & 1 else 0.0 for j in range(3)])
        z, n = gl_box(nx, nt, lo, hi, panels=8, order=8)
        Zs, Ns = Zs + z, Ns + n
        los.append(lo)
        his.append(hi)
    assert Zs == pytest.approx(Zw, rel=1e-9)
    np.testing.assert_allclose(Ns, Nw, rtol=1e-9)
    lat = oracle.lattice(nx, nt)
    _, tot = oracle.integrate(lat, np.array(los), np.array(his), 2 ** 15, seed=21)
    assert abs(np.exp(tot[0]) - Zw) < 4 * np.exp(tot[0]) * tot[1]
    assert np.all(np.abs(tot[4:4 + R] - Nw / Zw) < 4 * tot[4 + R:])


def test_slot_contents_and_shift():
    # The slot's sums are those of w = exp(-(S - m_s)) with m_s the smallest
    # action; Z_s = V/n e^{-m_s} sum w.  Recompute one subvolume from the points.
    nx, nt = 4, 2
    d, R = 8, 3
    lat = oracle.lattice(nx, nt, nu=0.8)
    lo, hi = np.full(d, -2.0), np.full(d, 3.0)
    n = 500
    slots, tot = oracle.integrate(lat, lo[None], hi[None], n, seed=3, job_id=5, sub_id=[9])
    y = oracle.points(d, lo, hi, sid=9, seed=3, job_id=5, first=0, count=n)
    S, P = oracle.eval_points(lat, y)
    m = S.min()
    w = np.exp(-(S - m))
    q = slots[0]
    assert q[0] == n and q[1] == m
    assert q[2] == pytest.approx(d * np.log(5.0), rel=1e-15)
    np.testing.assert_allclose(q[3:5], [w.sum(), (w * w).sum()], rtol=1e-13)
    np.testing.assert_allclose(q[5:5 + R], (w[:, None] * P).sum(0), rtol=1e-12)
    np.testing.assert_allclose(q[5 + R:5 + 2 * R], (w[:, None] ** 2 * P).sum(0), rtol=1e-12)
    np.testing.assert_allclose(q[5 + 2 * R:], ((w[:, None] * P) ** 2).sum(0), rtol=1e-12)
    logZ = np.log(5.0 ** d / n * w.sum()) - m
    assert tot[0] == pytest.approx(logZ, rel=1e-13)
    np.testing.assert_allclose(tot[4:4 + R], (w[:, None] * P).sum(0) / w.sum(), rtol=1e-12)
    f = 5.0 ** d * np.exp(-m) * w
    assert tot[1] == pytest.approx(f.std(ddof=1) / np.sqrt(n) / f.mean(), rel=1e-10)
    # one subvolume: the delta-method error of C = sum wP / sum w is the textbook
    # ratio-estimator standard error sqrt(n/(n-1) sum w^2 (P - C)^2) / sum w
    C = tot[4:4 + R]
    se = np.sqrt(n / (n - 1) * ((w[:, None] * (P - C)) ** 2).sum(0)) / w.sum()
    np.testing.assert_allclose(tot[4 + R:], se, rtol=1e-8)


def test_merge_invariants():
    nx = 6
    R = 4
    lat = oracle.lattice(nx, 2)
    d = 12
    lo = np.stack([np.full(d, -3.0), np.full(d, -1.0), np.full(d, 0.0)])
    hi = np.stack([np.full(d, 3.0), np.full(d, 1.0), np.full(d, 0.5)])
    slots, tot = oracle.integrate(lat, lo, hi, [1000, 3000, 2000], seed=8)
    # order of subvolumes does not matter
    tot_p = oracle.merge(nx, slots[[2, 0, 1]])
    np.testing.assert_allclose(tot_p, tot, rtol=1e-13)
    # a different shift with rescaled sums is the same record
    sh = slots.copy()
    delta = 1.7
    sh[:, 1] -= delta
    sh[:, 3] *= np.exp(-delta)
    sh[:, 4] *= np.exp(-2 * delta)
    sh[:, 5:5 + R] *= np.exp(-delta)
    sh[:, 5 + R:] *= np.exp(-2 * delta)
    m2 = oracle.merge(nx, sh)
    vals = [0, 2, 3] + list(range(4, 4 + R))
    errs = [1] + list(range(4 + R, 4 + 2 * R))
    np.testing.assert_allclose(m2[vals], tot[vals], rtol=1e-12)
    np.testing.assert_allclose(m2[errs], tot[errs], rtol=1e-9)  # variances cancel
    assert np.isfinite(tot).all() and tot[2] == 6000 and tot[3] == 3


def test_deterministic_and_thread_independent():
    lat = oracle.lattice(4, 2)
    lo = np.full((5, 8), -5.0)
    hi = np.full((5, 8), 5.0)
    a = oracle.integrate(lat, lo, hi, 3000, seed=1, nthreads=1)
    b = oracle.integrate(lat, lo, hi, 3000, seed=1, nthreads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_edge_cases_empty_and_single_sample():
    lat = oracle.lattice(4, 2)
    lo = np.full((2, 8), -5.0)
    hi = np.full((2, 8), 5.0)
    slots, tot = oracle.integrate(lat, lo, hi, [0, 4000], seed=1)
    _, tot1 = oracle.integrate(lat, lo[1:], hi[1:], [4000], seed=1, sub_id=[1])
    # an empty subvolume contributes nothing
    assert slots[0, 0] == 0 and slots[0, 3] == 0
    np.testing.assert_array_equal(tot[[0, 1, 2] + list(range(4, 10))], tot1[[0, 1, 2] + list(range(4, 10))])
    # one sample: a value but no variance estimate
    _, t1 = oracle.integrate(lat, lo[:1], hi[:1], [1], seed=1)
    assert np.isfinite(t1[0]) and np.isinf(t1[1])


def test_nsphere_split_suggestion():
    # The split suggestion is the coordinate across which the integrand is least
    # even.  On [-1,1]^2 x [0,1] the ball's density falls along the third
    # coordinate only; on a box symmetric in every coordinate no coordinate is
    # preferred beyond noise, so a box lopsided in the first one picks it.
    _, _, sd = oracle.nsphere(3, 200_000, 1, lo=[-1, -1, 0], hi=[1, 1, 1], split=True)
    assert sd == 2
    _, _, sd = oracle.nsphere(3, 200_000, 2, lo=[-0.2, -1, -1], hi=[1, 1, 1], split=True)
    assert sd == 0
