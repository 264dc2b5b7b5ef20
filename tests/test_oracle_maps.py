"""Pins of the oracle's samplers (the transform of Sec. 4 and Gaussian
importance sampling): the numpy record against the C integrator, the map and
its Jacobian against quadrature, closed forms of the regulated linear limit on
all of R^d, a zero-variance case, and Gauss-Legendre quadrature of a box."""
import math

import numpy as np
import pytest
from scipy import integrate as sint

import oracle
from oracle.maps import (BOX, GAUSSIAN, TRANSFORM, integrate_mapped, linear_limit_eigen, log_jacobian,
                         proposal_covariance, sincospi, standard_normals, transform)
from gl_reference import action_np, gl_box, linear_limit


def test_box_record_matches_the_c_integrator():
    lat = oracle.lattice(4, 2)
    rng = np.random.default_rng(3)
    lo = -rng.uniform(1, 3, (3, 8))
    hi = rng.uniform(1, 3, (3, 8))
    s_np, t_np = integrate_mapped(lat, lo, hi, [5000, 7, 12345], seed=9, job_id=2, kind=BOX)
    s_c, t_c = oracle.integrate(lat, lo, hi, np.array([5000, 7, 12345], dtype=np.uint64), seed=9, job_id=2)
    np.testing.assert_allclose(s_np, s_c, rtol=1e-13, atol=0)
    np.testing.assert_allclose(t_np, t_c, rtol=1e-12, atol=1e-15)


def test_transform_and_its_jacobian():
    from fractions import Fraction
    y = np.array([-0.9, -0.5, 0.0, 0.25, 0.999])
    exact = [float(Fraction(t) / (1 - Fraction(t) ** 2)) for t in y]
    np.testing.assert_allclose(transform(y), exact, rtol=4e-16)
    # dv/dy: by central differences where they are accurate, and exactly
    h = 1e-6
    num = (transform(y[:4] + h) - transform(y[:4] - h)) / (2 * h)
    np.testing.assert_allclose(np.exp(log_jacobian(y[:4])), num, rtol=1e-8)
    jac = [float((1 + Fraction(t) ** 2) / (1 - Fraction(t) ** 2) ** 2) for t in y]
    np.testing.assert_allclose(np.exp(log_jacobian(y)), jac, rtol=1e-13)
    # change of variables: int_{-1}^{1} exp(-T(y)^2/2) T'(y) dy = sqrt(2 pi)
    val, _ = sint.quad(lambda t: math.exp(-transform(t) ** 2 / 2 + log_jacobian(t)), -1, 1, limit=200)
    assert val == pytest.approx(math.sqrt(2 * math.pi), rel=1e-10)


@pytest.mark.parametrize("nx,nt", [(3, 1), (4, 1), (2, 2)])
def test_transform_linear_limit_closed_form(nx, nt):
    # regulated linear limit on all of R^d: (-1,1)^d maps onto R^d
    lat = oracle.lattice(nx, nt, nonlinear=0.0, mass2=1.0)
    Z_exact, C_exact, _ = linear_limit(nx, nt, mass2=1.0)
    d = nx * nt
    _, tot = integrate_mapped(lat, -np.ones(d), np.ones(d), 1 << 18, seed=4, kind=TRANSFORM)
    Z = math.exp(tot[0])
    assert abs(Z - Z_exact) < 4 * Z * tot[1]
    R = nx // 2 + 1
    for r in range(R):
        assert abs(tot[4 + r] - C_exact[r]) < 4 * tot[4 + R + r]


def test_transform_nonlinear_against_quadrature():
    # 2x1 lattice (d = 2) with the advection term and a mass: Z on R^2 by
    # adaptive 2-D quadrature of exp(-S) (the action written out in numpy)
    lat = oracle.lattice(2, 1, mass2=0.5)
    f = lambda a, b: math.exp(-float(action_np(np.array([[a], [b]]), mass2=0.5)))
    Zq, _ = sint.dblquad(lambda b, a: f(a, b), -12, 12, -12, 12, epsabs=1e-11, epsrel=1e-10)
    _, tot = integrate_mapped(lat, -np.ones(2), np.ones(2), 1 << 18, seed=8, kind=TRANSFORM)
    Z = math.exp(tot[0])
    assert abs(Z - Zq) < 4 * Z * tot[1]


def test_proposal_covariance_inverts_the_linear_action():
    # v^T A v / 2 is the linear-limit action: compare with the numpy action
    lat = oracle.lattice(5, 2, nonlinear=0.0, mass2=0.3)
    cov = proposal_covariance(lat, zero_mode_sigma=1e9)
    A = np.linalg.inv(cov)
    rng = np.random.default_rng(0)
    for _ in range(5):
        v = rng.normal(size=10)
        S = float(action_np(v.reshape(5, 2), nonlinear=0.0, mass2=0.3))
        assert 0.5 * v @ A @ v == pytest.approx(S, rel=1e-7)
    # eigenvalues: the Fourier symbol, and the zero mode of mass2 = 0
    lam = np.sort(linear_limit_eigen(oracle.lattice(10, 2)).ravel())
    assert lam[0] == pytest.approx(0.0, abs=1e-14) and lam[1] > 1e-3


def test_gaussian_from_the_target_has_zero_variance():
    # importance sampling of the regulated linear limit from its own Gaussian
    # on a box that holds every sample: every weight is Z, so the estimate is
    # exact up to rounding and the stated error vanishes
    lat = oracle.lattice(4, 2, nonlinear=0.0, mass2=1.0)
    cov = proposal_covariance(lat, zero_mode_sigma=math.inf)
    F = np.linalg.cholesky(cov)
    Z_exact, C_exact, _ = linear_limit(4, 2, mass2=1.0)
    slots, tot = integrate_mapped(lat, -1e3 * np.ones(8), 1e3 * np.ones(8), 4096, seed=2, kind=GAUSSIAN, factor=F)
    assert math.exp(tot[0]) == pytest.approx(Z_exact, rel=1e-10)
    assert tot[1] < 1e-6
    # C(r) is then a plain average of P_r over the Gaussian: within its error
    R = 3
    for r in range(R):
        assert abs(tot[4 + r] - C_exact[r]) < 4 * tot[4 + R + r]


def test_gaussian_on_a_box_against_quadrature():
    # the paper's action (mass2 = 0, nonlinear) on the box [-5,5]^3 of a 3x1
    # lattice: importance sampling from the regulated linear-limit Gaussian
    # and Gauss-Legendre quadrature estimate the same Z and C(r)
    lat = oracle.lattice(3, 1)
    Zq, Nq = gl_box(3, 1, -5.0, 5.0, panels=16, order=8)
    F = np.linalg.cholesky(proposal_covariance(lat, zero_mode_sigma=4.0))
    _, tot = integrate_mapped(lat, -5 * np.ones(3), 5 * np.ones(3), 1 << 17, seed=6, kind=GAUSSIAN, factor=F)
    Z = math.exp(tot[0])
    assert abs(Z - Zq) < 4 * Z * tot[1]
    for r in range(2):
        assert abs(tot[4 + r] - Nq[r] / Zq) < 4 * tot[4 + 2 + r] + 1e-9
    # and with fewer samples it is more precise than the uniform box estimate
    _, tb = oracle.integrate(lat, -5 * np.ones((1, 3)), 5 * np.ones((1, 3)), 1 << 17, seed=6)
    assert tot[1] < tb[1]


def test_gaussian_with_no_sample_in_the_box():
    lat = oracle.lattice(3, 1)
    F = np.eye(3) * 1e-3
    slots, tot = integrate_mapped(lat, 4 * np.ones(3), 5 * np.ones(3), 100, seed=1, kind=GAUSSIAN, factor=F)
    assert slots[0, 0] == 100 and slots[0, 1] == math.inf and slots[0, 3] == 0.0
    assert tot[0] == -math.inf


def test_normal_pairs_at_closed_form_points():
    """Box-Muller at points where it has exact values: u_{2p} = e^-2 gives
    r = 2; angles of 2 pi u in eighths and quarters of a turn, with cos on the
    even coordinate and sin on the odd one."""
    u = np.array([[math.exp(-2.0), 0.125, math.exp(-0.5), 0.25, math.exp(-2.0), 0.75]])
    z = standard_normals(u, 5)    # d = 5: the sixth word completes the last pair and is dropped
    assert z.shape == (1, 5)
    np.testing.assert_allclose(z[0], [math.sqrt(2.0), math.sqrt(2.0), 0.0, 1.0, 0.0], atol=1e-15)
    s, c = sincospi(np.array([0.0, 0.5, 1.0, 1.5, 1.0 / 6.0, 1.75]))
    np.testing.assert_allclose(s, [0.0, 1.0, 0.0, -1.0, 0.5, -math.sqrt(0.5)], atol=1e-16)
    np.testing.assert_allclose(c, [1.0, 0.0, -1.0, 0.0, math.sqrt(0.75), math.sqrt(0.5)], atol=1e-16)


def test_normals_from_philox_points_are_standard_and_independent():
    """z from 2^16 oracle unit points (d = 5, six words): each coordinate passes
    a Kolmogorov-Smirnov test against N(0, 1), its variance is 1 within four
    standard errors, and the two members of a pair are uncorrelated."""
    from scipy import stats
    n, d = 1 << 16, 5
    u = oracle.points(d + 1, np.zeros(d + 1), np.ones(d + 1), 4, 11, 2, 0, n)
    z = standard_normals(u, d)
    for j in range(d):
        assert stats.kstest(z[:, j], "norm").pvalue > 1e-3, j
        assert abs(np.mean(z[:, j] ** 2) - 1.0) < 4.0 * math.sqrt(2.0 / n)
    for j in (0, 2):
        assert abs(np.corrcoef(z[:, j], z[:, j + 1])[0, 1]) < 4.0 / math.sqrt(n)
