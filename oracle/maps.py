"""Samplers that take the Philox unit point to the field v, written plainly.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

The box sampler (``oracle.integrate``) draws v uniformly in a box.  Two more:

TRANSFORM (Sec. 4): the paper maps the infinite range to (-1, 1) without
saying how.  Our choice is v = y / (1 - y^2) per coordinate, a bijection of
(-1, 1) onto R with dv/dy = (1 + y^2) / (1 - y^2)^2 > 0.  The box is given in
y, inside [-1, 1]^d, and
    int_{T(box)} exp(-S(v)) dv = int_box exp(-S(T(y)) + sum_j ln T'(y_j)) dy,
so the estimator is the box estimator of exp(-S_eff) with
S_eff = S(T(y)) - sum_j ln T'(y_j).

GAUSSIAN (Sec. 5 names a better-concentrated integrand as the way to large
gains; this is importance sampling): v = mean + F z with z standard normal,
drawn from the unit point u in Box-Muller pairs (Box & Muller 1958; the paper
fixes no generator):
    z_{2p} = r cos(2 pi u_{2p+1}),  z_{2p+1} = r sin(2 pi u_{2p+1}),
    r = sqrt(-2 ln u_{2p}),
with u_d the next Philox word when d is odd.  So v ~ N(mean, F F^T) with
density q.  For a box B,
    int_B exp(-S(v)) dv = E_q[ 1_B(v) exp(-S(v)) / q(v) ],
    1 / q(v) = (2 pi)^(d/2) |det F| exp(|z|^2 / 2),
so the weight is exp(-S_eff) with S_eff = S(v) - |z|^2 / 2 (0 outside B) and
the record's log-volume is (d/2) ln(2 pi) + ln |det F|.

The proposal is the linear limit of the action (nonlinear term dropped),
S_lin = v^T A v / 2, whose modes e^{i(w l + k m)} (time slice l, site m) have
A-eigenvalues |e^{iw} - 1 + 4 c_dif sin^2(k/2)|^2 / (D tau) + mass2 with
c_dif = nu tau / a^2 (the symbol of the residual of Eq. (Gen2) without the
advection term).  The constant mode (and any other zero mode) has eigenvalue 0
when mass2 = 0; the proposal adds 1 / sigma0^2 to every eigenvalue so that it
is a proper Gaussian: covariance (A + I / sigma0^2)^-1.

The record layout and the merge are those of ``oracle.integrate``; the shift
m_s is the smallest S_eff among the samples with weight.
"""
from __future__ import annotations

import math

import numpy as np

from . import eval_points, merge, num_r, points, slot_len

BOX, TRANSFORM, GAUSSIAN = 0, 1, 2


def sincospi(x):
    """(sin(pi x), cos(pi x)) for x in [0, 2].  x - k/2 (k = the nearest
    integer to 2x) is exact for the unit coordinates, so only pi * y with
    |y| <= 1/4 rounds; the quarter turns k are applied exactly."""
    x = np.asarray(x, dtype=float)
    k = np.rint(2.0 * x)
    y = x - 0.5 * k
    s0, c0 = np.sin(math.pi * y), np.cos(math.pi * y)
    k = k.astype(np.int64) % 4
    s = np.choose(k, [s0, c0, -s0, -c0])
    c = np.choose(k, [c0, -s0, -c0, s0])
    return s, c


def standard_normals(u, d):
    """z [n, d] from unit points u [n, d + (d odd)], pair by pair: Box-Muller."""
    r = np.sqrt(-2.0 * np.log(u[:, 0::2]))
    s, c = sincospi(2.0 * u[:, 1::2])
    z = np.empty((u.shape[0], 2 * r.shape[1]))
    z[:, 0::2] = r * c
    z[:, 1::2] = r * s
    return z[:, :d]


def transform(y):
    """v = y / (1 - y^2), with 1 - y^2 formed as (1 - y)(1 + y)."""
    y = np.asarray(y, dtype=float)
    return y / ((1.0 - y) * (1.0 + y))


def log_jacobian(y):
    """ln dv/dy = ln(1 + y^2) - 2 ln(1 - y^2), per coordinate."""
    y = np.asarray(y, dtype=float)
    return np.log1p(y * y) - 2.0 * np.log((1.0 - y) * (1.0 + y))


def linear_limit_eigen(lat):
    """Eigenvalues of A on the modes (w_p, k_q), p < Nt, q < Nx, as [Nt, Nx]."""
    nx, nt = lat.nx, lat.nt
    k = 2.0 * np.pi * np.arange(nx)[None, :] / nx
    w = 2.0 * np.pi * np.arange(nt)[:, None] / nt
    c_dif = lat.nu * lat.tau / lat.a ** 2
    sym = np.exp(1j * w) - 1.0 + 4.0 * c_dif * np.sin(k / 2.0) ** 2
    return np.abs(sym) ** 2 / (lat.D * lat.tau) + lat.mass2


def proposal_covariance(lat, zero_mode_sigma: float):
    """(A + I / sigma0^2)^-1 as a real d x d matrix in the coordinate order
    j = m Nt + l, summed over the Fourier modes."""
    nx, nt = lat.nx, lat.nt
    d = nx * nt
    lam = linear_limit_eigen(lat) + 1.0 / zero_mode_sigma ** 2          # [Nt, Nx]
    m = np.arange(d) // nt
    l = np.arange(d) % nt
    dm = m[:, None] - m[None, :]
    dl = l[:, None] - l[None, :]
    w = 2.0 * np.pi * np.arange(nt) / nt
    k = 2.0 * np.pi * np.arange(nx) / nx
    cov = np.zeros((d, d))
    for p in range(nt):
        for q in range(nx):
            cov += np.cos(w[p] * dl + k[q] * dm) / lam[p, q]
    return cov / d


def _fsum_cols(a):
    return np.array([math.fsum(a[:, i]) for i in range(a.shape[1])])


def _slot(n, S_eff, P, inside, log_v):
    """Subvolume record from the samples' S_eff, P_r and in-box flags."""
    R = P.shape[1]
    if inside.any():
        m = float(S_eff[inside].min())
        w = np.where(inside, np.exp(m - np.where(inside, S_eff, m)), 0.0)
    else:
        m = math.inf
        w = np.zeros(S_eff.shape[0])
    w2 = w * w
    out = np.zeros(5 + 3 * R)
    out[0] = n
    out[1] = m
    out[2] = log_v
    out[3] = math.fsum(w)
    out[4] = math.fsum(w2)
    out[5:5 + R] = _fsum_cols(w[:, None] * P)
    out[5 + R:5 + 2 * R] = _fsum_cols(w2[:, None] * P)
    out[5 + 2 * R:] = _fsum_cols(w2[:, None] * P * P)
    return out


def integrate_mapped(lat, lo, hi, samples, seed, job_id=0, sub_id=None, kind=TRANSFORM, mean=None, factor=None):
    """Slots [nsub, 5+3R] and totals [4+2R] of the lattice integral with the
    BOX, TRANSFORM or GAUSSIAN sampler (see the module text), FP64 throughout.
    BOX repeats ``oracle.integrate`` in numpy (a cross-check of the record)."""
    d = lat.nx * lat.nt
    lo = np.asarray(lo, dtype=float).reshape(-1, d)
    hi = np.asarray(hi, dtype=float).reshape(-1, d)
    nsub = lo.shape[0]
    samples = np.broadcast_to(np.asarray(samples, dtype=np.uint64), (nsub,))
    sid = np.arange(nsub, dtype=np.uint32) if sub_id is None else np.asarray(sub_id, dtype=np.uint32)
    if kind == GAUSSIAN:
        factor = np.asarray(factor, dtype=float).reshape(d, d)
        mean = np.zeros(d) if mean is None else np.asarray(mean, dtype=float)
        log_v_gauss = 0.5 * d * math.log(2.0 * math.pi) + np.linalg.slogdet(factor)[1]
    slots = np.zeros((nsub, slot_len(lat.nx)))
    for s in range(nsub):
        n = int(samples[s])
        if n == 0:
            slots[s, 1] = math.inf
            slots[s, 2] = (log_v_gauss if kind == GAUSSIAN else float(np.sum(np.log(hi[s] - lo[s]))))
            continue
        if kind == BOX:
            v = points(d, lo[s], hi[s], int(sid[s]), seed, job_id, 0, n)
            lj = np.zeros(n)
            inside = np.ones(n, dtype=bool)
            log_v = float(np.sum(np.log(hi[s] - lo[s])))
        elif kind == TRANSFORM:
            y = points(d, lo[s], hi[s], int(sid[s]), seed, job_id, 0, n)
            v = transform(y)
            lj = log_jacobian(y).sum(axis=1)
            inside = np.ones(n, dtype=bool)
            log_v = float(np.sum(np.log(hi[s] - lo[s])))
        elif kind == GAUSSIAN:
            dp = d + d % 2
            u = points(dp, np.zeros(dp), np.ones(dp), int(sid[s]), seed, job_id, 0, n)
            z = standard_normals(u, d)
            v = mean + z @ factor.T
            lj = 0.5 * np.sum(z * z, axis=1)
            inside = np.all((v >= lo[s]) & (v < hi[s]), axis=1)
            log_v = log_v_gauss
        else:
            raise ValueError("kind must be BOX, TRANSFORM or GAUSSIAN")
        S, P = eval_points(lat, v)
        slots[s] = _slot(n, S - lj, P, inside, log_v)
    return slots, merge(lat.nx, slots)


__all__ = ["BOX", "TRANSFORM", "GAUSSIAN", "transform", "log_jacobian", "linear_limit_eigen",
           "proposal_covariance", "integrate_mapped", "num_r", "sincospi", "standard_normals"]
