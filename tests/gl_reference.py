"""Independent expected values for the oracle's pins (tests only).

* ``gl_box``: tensor-product composite Gauss-Legendre quadrature of
  Z = int exp(-S) and N(r) = int P_r exp(-S) over a box, for lattices with
  d <= 4.  The action is evaluated here with numpy array shifts, written
  from Eq. (Gen2) independently of the oracle's loop form.
* ``linear_limit``: the closed form of the regulated linear limit
  (nonlinear term off, mass2 > 0), from the Fourier symbol of the linear
  residual.  With v_{l,m} = exp(i(w l + k m)) the residual of Eq. (Gen2)
  without advection is
      R = [e^{iw} - 1 + (4 nu tau / a^2) sin^2(k/2)] v = mu(k, w) v,
  so S = 1/2 v^T Q v with eigenvalues lambda = |mu|^2/(D tau) + mass2 at
  k = 2 pi j / Nx, w = 2 pi p / Nt.  Then
      Z    = (2 pi)^{d/2} / prod sqrt(lambda)
      C(r) = (1/d) sum_{j,p} cos(2 pi j r / Nx) / lambda_{jp}.
"""
from __future__ import annotations

import numpy as np


def action_np(U, nu=1.0, D=1.0, a=1.0, tau=1.0, nonlinear=1.0, mass2=0.0):
    """S for configurations U[..., m, l] (m space, l time), periodic."""
    nxt = np.roll(U, -1, axis=-1)      # v(t_{l+1}, x_m)
    right = np.roll(U, -1, axis=-2)    # v(t_l, x_{m+1})
    left = np.roll(U, 1, axis=-2)      # v(t_l, x_{m-1})
    adv = U * (right - left) / (2.0 * a)
    lap = (right - 2.0 * U + left) / (a * a)
    R = nxt - U + tau * (nonlinear * adv - nu * lap)
    return (R * R).sum(axis=(-1, -2)) / (2.0 * D * tau) + 0.5 * mass2 * (U * U).sum(axis=(-1, -2))


def corr_np(U):
    """P_r = (1/d) sum_{l,m} v_{l,m} v_{l,m+r}, r = 0..Nx//2, for U[..., m, l]."""
    nx, nt = U.shape[-2], U.shape[-1]
    out = []
    for r in range(nx // 2 + 1):
        out.append((U * np.roll(U, -r, axis=-2)).sum(axis=(-1, -2)) / (nx * nt))
    return np.stack(out, axis=-1)


def _composite_gl(lo, hi, panels, order):
    x, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(lo, hi, panels + 1)
    xs, ws = [], []
    for p in range(panels):
        a, b = edges[p], edges[p + 1]
        xs.append(0.5 * (b - a) * x + 0.5 * (b + a))
        ws.append(0.5 * (b - a) * w)
    return np.concatenate(xs), np.concatenate(ws)


def gl_box(nx, nt, lo, hi, panels=8, order=8, **params):
    """(Z, N[r]) over the box prod_j [lo_j, hi_j] by tensor Gauss-Legendre."""
    d = nx * nt
    lo = np.broadcast_to(np.asarray(lo, dtype=float), (d,))
    hi = np.broadcast_to(np.asarray(hi, dtype=float), (d,))
    rules = [_composite_gl(lo[j], hi[j], panels, order) for j in range(d)]
    R = nx // 2 + 1
    Z = 0.0
    N = np.zeros(R)
    # loop over the first coordinate, vectorise the rest
    rest = np.meshgrid(*[r[0] for r in rules[1:]], indexing="ij") if d > 1 else []
    wrest = np.ones(1)
    if d > 1:
        wrest = rules[1][1]
        for r in rules[2:]:
            wrest = np.multiply.outer(wrest, r[1])
        wrest = wrest.reshape(-1)
    pts_rest = np.stack([g.reshape(-1) for g in rest], axis=-1) if d > 1 else np.zeros((1, 0))
    for x0, w0 in zip(*rules[0]):
        Y = np.concatenate([np.full((pts_rest.shape[0], 1), x0), pts_rest], axis=1)
        U = Y.reshape(-1, nx, nt)  # coordinate j = m*nt + l
        S = action_np(U, **params)
        f = np.exp(-S) * wrest * w0
        Z += f.sum()
        N += (f[:, None] * corr_np(U)).sum(axis=0)
    return Z, N


def linear_limit(nx, nt, nu=1.0, D=1.0, a=1.0, tau=1.0, mass2=1.0):
    """Closed form (Z, C[r]) of the regulated linear limit on all of R^d."""
    j = np.arange(nx)[:, None]
    p = np.arange(nt)[None, :]
    k = 2 * np.pi * j / nx
    w = 2 * np.pi * p / nt
    mu = np.exp(1j * w) - 1.0 + 4.0 * nu * tau / a ** 2 * np.sin(k / 2) ** 2
    lam = np.abs(mu) ** 2 / (D * tau) + mass2
    d = nx * nt
    Z = (2 * np.pi) ** (d / 2) / np.sqrt(np.prod(lam))
    C = np.array([(np.cos(k * r) / lam).sum() / d for r in range(nx // 2 + 1)])
    return Z, C, lam
