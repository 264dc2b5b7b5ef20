"""Pins of the oracle's action S[u] (step a2, Eq. (Gen2)) and correlation
products P_r (step a4), against hand-derived values, the Fourier symbol of the
linear part and the lattice symmetries."""
import numpy as np
import pytest

import oracle

SHAPES = [(3, 2), (4, 2), (6, 4), (10, 2), (5, 3), (16, 4)]


def _u(nx, nt, sites):
    """Configuration with v(t_l, x_m) = value at the given (l, m), zero elsewhere."""
    u = np.zeros(nx * nt)
    for (l, m), val in sites.items():
        u[m * nt + l] = val  # coordinate j = m*Nt + l
    return u


@pytest.mark.parametrize("nx,nt", SHAPES)
def test_constant_field_has_zero_action(nx, nt):
    lat = oracle.lattice(nx, nt, nu=0.7, D=1.3, a=0.9, tau=0.4)
    assert abs(oracle.action(lat, np.full(nx * nt, 2.5))) < 1e-24
    lat_m = oracle.lattice(nx, nt, mass2=0.6)
    assert oracle.action(lat_m, np.full(nx * nt, 2.0)) == pytest.approx(0.5 * 0.6 * 4.0 * nx * nt)


@pytest.mark.parametrize("nx,nt", [s for s in SHAPES if s[0] >= 3 and s[1] >= 2])
@pytest.mark.parametrize("nu,D,a,tau", [(1, 1, 1, 1), (0.3, 2.0, 0.7, 0.5), (3.0, 0.5, 1.5, 0.2)])
def test_single_site(nx, nt, nu, D, a, tau):
    # One site v = h.  Residuals of Eq. (Gen2) that see it (c = nu tau / a^2):
    #   (l0, m0):     -h + 2 c h         (time step and the diagonal of the Laplacian)
    #   (l0-1, m0):   +h                 (it is the "next time" value there)
    #   (l0, m0+-1):  -c h each          (off-diagonal Laplacian; advection vanishes)
    # S = h^2 / (2 D tau) [ (2c - 1)^2 + 1 + 2 c^2 ]
    h = 0.83
    lat = oracle.lattice(nx, nt, nu, D, a, tau)
    c = nu * tau / a ** 2
    expect = h * h / (2 * D * tau) * ((2 * c - 1) ** 2 + 1 + 2 * c * c)
    for (l0, m0) in [(0, 0), (nt - 1, nx - 1), (1, 2)]:
        assert oracle.action(lat, _u(nx, nt, {(l0, m0): h})) == pytest.approx(expect, rel=1e-14)


@pytest.mark.parametrize("nx,nt", [s for s in SHAPES if s[0] >= 4 and s[1] >= 2])
@pytest.mark.parametrize("nu,D,a,tau", [(1, 1, 1, 1), (0.3, 2.0, 0.7, 0.5), (3.0, 0.5, 1.5, 0.2)])
def test_two_adjacent_sites(nx, nt, nu, D, a, tau):
    # v(l0, m0) = p and v(l0, m0+1) = q; c = nu tau / a^2, b = tau / (2a).
    #   (l0, m0):    -p + b p q - c (q - 2p)
    #   (l0, m0+1):  -q - b p q - c (p - 2q)
    #   (l0-1, m0): p, (l0-1, m0+1): q, (l0, m0-1): -c p, (l0, m0+2): -c q
    # With unit parameters this is S = (p - q + pq/2)^2 + p^2 + q^2.
    p, q = 0.37, -1.21
    lat = oracle.lattice(nx, nt, nu, D, a, tau)
    c, b = nu * tau / a ** 2, tau / (2 * a)
    r1 = -p + b * p * q - c * (q - 2 * p)
    r2 = -q - b * p * q - c * (p - 2 * q)
    expect = (r1 ** 2 + r2 ** 2 + p ** 2 + q ** 2 + c * c * (p * p + q * q)) / (2 * D * tau)
    u = _u(nx, nt, {(1, 2): p, (1, 3): q})
    assert oracle.action(lat, u) == pytest.approx(expect, rel=1e-14)
    if (nu, D, a, tau) == (1, 1, 1, 1):
        assert oracle.action(lat, u) == pytest.approx((p - q + p * q / 2) ** 2 + p * p + q * q,
                                                      rel=1e-14)


@pytest.mark.parametrize("nx,nt", [s for s in SHAPES if s[0] >= 4 and s[1] >= 3])
def test_three_sites_fix_the_time_direction(nx, nt):
    # v(l0, m0) = p, v(l0, m0+1) = q, v(l0+1, m0) = s, unit parameters.  The
    # advection at t_l0 pairs with the forward difference v(t_{l0+1}) - v(t_l0)
    # (explicit step of Eq. (Gen2)); the residuals that see the three sites are
    #   (l0-1, m0): p          (l0-1, m0+1): q
    #   (l0, m0):   s - p + pq/2 - (q - 2p) = s + p - q + pq/2
    #   (l0, m0+1): -q - pq/2 - (p - 2q)    = q - p - pq/2
    #   (l0, m0-1): -p         (l0, m0+2): -q
    #   (l0+1, m0): -s + 2s = s   (l0+1, m0+-1): -s each
    p, q, s = 0.9, -0.4, 1.3
    lat = oracle.lattice(nx, nt)
    u = _u(nx, nt, {(1, 1): p, (1, 2): q, (2, 1): s})
    expect = 0.5 * (p * p + q * q + (s + p - q + p * q / 2) ** 2 + (q - p - p * q / 2) ** 2
                    + p * p + q * q + s * s + 2 * s * s)
    assert oracle.action(lat, u) == pytest.approx(expect, rel=1e-14)


@pytest.mark.parametrize("nx,nt", SHAPES)
@pytest.mark.parametrize("nu,D,a,tau,mass2", [(1, 1, 1, 1, 0.0), (0.3, 2.0, 0.7, 0.5, 1.5)])
def test_linear_part_matches_fourier_symbol(nx, nt, nu, D, a, tau, mass2):
    # Without advection S = 1/(2 D tau) sum |R|^2 + mass2/2 |v|^2 is diagonal in
    # Fourier space: R^(k,w) = mu(k,w) v^(k,w), mu = e^{iw} - 1 + 4 nu tau/a^2 sin^2(k/2).
    rng = np.random.default_rng(nx * 100 + nt)
    lat = oracle.lattice(nx, nt, nu, D, a, tau, nonlinear=0.0, mass2=mass2)
    k = 2 * np.pi * np.arange(nx)[:, None] / nx
    w = 2 * np.pi * np.arange(nt)[None, :] / nt
    mu2 = np.abs(np.exp(1j * w) - 1 + 4 * nu * tau / a ** 2 * np.sin(k / 2) ** 2) ** 2
    for _ in range(5):
        u = rng.uniform(-3, 3, nx * nt)
        uh = np.fft.fft2(u.reshape(nx, nt))  # axes (m, l)
        parseval = (mu2 * np.abs(uh) ** 2).sum() / (nx * nt)
        expect = parseval / (2 * D * tau) + 0.5 * mass2 * (u * u).sum()
        assert oracle.action(lat, u) == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("nx,nt", SHAPES)
def test_action_symmetries(nx, nt):
    # Translations in x and t, and the parity v'(l, m) = -v(l, -m), leave S unchanged
    # (periodic lattice).  v -> -v alone is not a symmetry of the nonlinear action.
    rng = np.random.default_rng(7)
    lat = oracle.lattice(nx, nt, nu=0.6, D=1.1, a=0.8, tau=0.7)
    for _ in range(4):
        U = rng.uniform(-4, 4, (nx, nt))
        S = oracle.action(lat, U.reshape(-1))
        for sh in (1, nx - 1):
            assert oracle.action(lat, np.roll(U, sh, axis=0).reshape(-1)) == pytest.approx(S, rel=1e-13)
        assert oracle.action(lat, np.roll(U, 1, axis=1).reshape(-1)) == pytest.approx(S, rel=1e-13)
        parity = -U[(-np.arange(nx)) % nx, :]
        assert oracle.action(lat, parity.reshape(-1)) == pytest.approx(S, rel=1e-13)
    if nx >= 3:
        U = rng.uniform(-4, 4, (nx, nt))
        assert abs(oracle.action(lat, -U.reshape(-1)) - oracle.action(lat, U.reshape(-1))) > 1e-6


@pytest.mark.parametrize("nx,nt", SHAPES)
def test_correlation_of_plane_wave(nx, nt):
    # v(l, m) = cos(2 pi kappa m / Nx + phi_l): P_r = cos(2 pi kappa r / Nx) / 2 for
    # 0 < kappa < Nx/2, and P_r = c^2 for a constant field.
    lat = oracle.lattice(nx, nt)
    m = np.arange(nx)[:, None]
    phi = np.linspace(0.0, 1.0, nt)[None, :]
    for kappa in range(1, (nx + 1) // 2):
        U = np.cos(2 * np.pi * kappa * m / nx + phi)
        P = oracle.correlations(lat, U.reshape(-1))
        r = np.arange(nx // 2 + 1)
        np.testing.assert_allclose(P, 0.5 * np.cos(2 * np.pi * kappa * r / nx), atol=1e-14)
    P = oracle.correlations(lat, np.full(nx * nt, -1.5))
    np.testing.assert_allclose(P, 2.25, rtol=1e-15)


@pytest.mark.parametrize("nx,nt", SHAPES)
def test_correlation_symmetry_and_zero_distance(nx, nt):
    # P_r = P_{Nx - r} is what makes r <= Nx/2 sufficient: check it against the
    # reflected field (P_r of v(-m) equals P_{Nx-r} of v), and P_0 = |v|^2 / d.
    rng = np.random.default_rng(3)
    lat = oracle.lattice(nx, nt)
    U = rng.normal(size=(nx, nt))
    P = oracle.correlations(lat, U.reshape(-1))
    assert P[0] == pytest.approx((U * U).sum() / (nx * nt), rel=1e-14)
    full = [(U * np.roll(U, -r, axis=0)).sum() / (nx * nt) for r in range(nx)]
    for r in range(nx // 2 + 1):
        assert full[r] == pytest.approx(full[(nx - r) % nx], rel=1e-13)
        assert P[r] == pytest.approx(full[r], rel=1e-13)
