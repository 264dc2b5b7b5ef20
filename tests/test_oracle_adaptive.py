"""Pins of the oracle's adaptive subdivision (Sec. 3): closed forms of the
N-sphere, quadrature of a small lattice, the reduction to a plain estimate when
the test always passes, the dyadic tiling when it never does, and a
hand-counted run of the depth and round limits."""
import math

import numpy as np
import pytest

import oracle
from oracle.adaptive import Convergence, adaptive_integrate, adaptive_nsphere
from gl_reference import gl_box
from workloads import bisected_boxes


def _volumes(out):
    return sum(float(np.prod(h - l)) for l, h in zip(out.leaves_lo, out.leaves_hi))


def _tiles(out, lo, hi):
    """The kept leaves are disjoint and cover the box: their volumes add up,
    and every one of a set of probe points lies in exactly one leaf."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    assert _volumes(out) == pytest.approx(float(np.prod(hi - lo)), rel=1e-12)
    rng = np.random.default_rng(0)
    pts = lo + (hi - lo) * rng.random((500, lo.size))
    L = np.array(out.leaves_lo)
    H = np.array(out.leaves_hi)
    inside = np.all((pts[:, None, :] >= L[None]) & (pts[:, None, :] < H[None]), axis=2)
    assert np.all(inside.sum(axis=1) == 1)


def test_listing1_half_volume_of_the_4_ball():
    # Sec. 3, Listing 1: (half) the volume of the unit 4-ball with a 3-dimensional
    # integrand over [-1,1]^3; the paper printed 2.465467 +- 0.002691.  Exact: pi^2/4.
    res, err, out = adaptive_nsphere(3, 100_000, 1, Convergence(2.0, 0.003, 0.0, 0.0, 8, 1 << 16))
    assert err < 0.01
    assert abs(res - math.pi ** 2 / 4) < 4 * err
    assert abs(2.465467073965016 - math.pi ** 2 / 4) < 4 * 0.002690919078211793
    _tiles(out, [-1] * 3, [1] * 3)


@pytest.mark.parametrize("dims", [1, 2, 5])
def test_half_volumes_of_balls(dims):
    # half the volume of the unit (k+1)-ball: pi^((k+1)/2) / Gamma((k+1)/2 + 1) / 2
    exact = math.pi ** ((dims + 1) / 2) / math.gamma((dims + 1) / 2 + 1) / 2
    res, err, out = adaptive_nsphere(dims, 20_000, 3, Convergence(2.0, 0.01, 0.0, 0.0, 6, 256))
    assert abs(res - exact) < 4 * err
    _tiles(out, [-1] * dims, [1] * dims)


def test_always_converged_is_the_plain_estimate():
    # criterion (3) with a huge threshold holds at once: one round, and the
    # result is the second evaluation of the whole volume (sub_id 3, 2n samples)
    res, err, out = adaptive_nsphere(2, 10_000, 5, Convergence(2.0, 0.0, 0.0, 1e300, 8, 16))
    assert out.stats == dict(rounds=1, evaluated=1, converged=1, kept_depth=0, kept_budget=0, leaves=1,
                             samples=30_000)
    assert (res, err) == oracle.nsphere(2, 20_000, 5, sub_id=3)


def test_factor_rounds_up():
    _, _, out = adaptive_nsphere(1, 1001, 5, Convergence(1.5, 0.0, 0.0, 1e300, 8, 16))
    assert out.stats["samples"] == 1001 + 1502


def test_outside_the_ball_converges_by_criterion_3():
    # over [0.5, 1.3]^2 only the corner near the origin meets the unit disk:
    # halves away from it have f = 0, so max |r| = 0 <= small at once
    _, _, out = adaptive_nsphere(2, 4_000, 2, Convergence(2.0, 0.0, 0.0, 1e-300, 3, 1 << 10), lo=0.5, hi=1.3)
    outside = 0
    for l, h, (r, e) in zip(out.leaves_lo, out.leaves_hi, out.kept):
        if np.linalg.norm(l) >= 1.0:   # the nearest corner is outside the disk
            assert r == 0.0 and e == 0.0
            outside += 1
        else:
            assert r > 0.0
    # the halves away from the corner stop at once; the corner's keeps halving
    assert outside >= 2 and out.stats["converged"] == outside
    assert out.stats["kept_depth"] == out.stats["leaves"] - outside
    _tiles(out, [0.5, 0.5], [1.3, 1.3])


def test_never_converged_lattice_tiles_dyadically():
    # no criterion on: every subvolume is halved along its widest side until
    # max_depth, which for the cube [-5,5]^8 halves coordinates 0, 1, 2 in turn
    lat = oracle.lattice(4, 2)
    totals, out = adaptive_integrate(lat, -5.0, 5.0, 512, 7, Convergence(2.0, 0.0, 0.0, 0.0, 3, 1 << 10))
    assert out.stats["leaves"] == out.stats["kept_depth"] == 8
    assert out.stats["rounds"] == 4 and out.stats["evaluated"] == 1 + 2 + 4 + 8
    lo, hi = bisected_boxes(8, 3)
    got = sorted(zip(map(tuple, out.leaves_lo), map(tuple, out.leaves_hi)))
    want = sorted(zip(map(tuple, lo), map(tuple, hi)))
    assert got == want
    # the totals are the merge of the kept second evaluations, 1024 samples each
    assert totals[2] == 8 * 1024


def test_round_and_depth_limits_by_hand():
    # criteria off, at most 5 subvolumes per round, depth limit 6:
    #   round 1: 1 -> split; round 2: 2 -> both split; rounds 3-6: 4 subvolumes,
    #   the first two split (2 + 2 <= 5), the other two kept for lack of room;
    #   round 7: the 4 at depth 6 are kept at the depth limit.
    _, _, out = adaptive_nsphere(2, 256, 1, Convergence(2.0, 0.0, 0.0, 0.0, 6, 5))
    assert out.stats == dict(rounds=7, evaluated=1 + 2 + 4 * 5, converged=0, kept_depth=4, kept_budget=8,
                             leaves=12, samples=23 * (256 + 512))
    _tiles(out, [-1, -1], [1, 1])


def test_adaptive_lattice_agrees_with_quadrature():
    # 3x1 lattice over [-5,5]^3: the merged kept leaves estimate Z and C(r),
    # against tensor Gauss-Legendre quadrature of the same box
    lat = oracle.lattice(3, 1)
    Zq, Nq = gl_box(3, 1, -5.0, 5.0, panels=16, order=8)
    totals, out = adaptive_integrate(lat, -5.0, 5.0, 20_000, 11, Convergence(2.0, 0.02, 0.0, 0.0, 5, 64))
    assert out.stats["leaves"] > 1
    Z = math.exp(totals[0])
    assert abs(Z - Zq) < 4 * Z * totals[1]
    R = 2
    for r in range(R):
        assert abs(totals[4 + r] - Nq[r] / Zq) < 4 * totals[4 + R + r] + 1e-9
    _tiles(out, [-5] * 3, [5] * 3)


def test_relative_criterion_is_a_ratio():
    # Sec. 4 quotes criterion (1) as ratios (1.025 to 1.085): results 1.00 and
    # 1.03 lie within a factor 1.0305 of each other but not within 1.0295, in
    # plain values and in logarithms alike
    from oracle.adaptive import _criteria_linear, _criteria_log
    for tol, ok in [(0.0305, True), (0.0295, False)]:
        c = Convergence(2.0, tol, 0.0, 0.0, 1, 1)
        [(v, t)] = _criteria_linear(1.0, 1.03, c)
        assert (v <= t) == ok
        [(v, t)] = _criteria_linear(-1.03, -1.0, c)
        assert (v <= t) == ok
        [(v, t)] = _criteria_log(math.log(7.0), math.log(7.0 * 1.03), c)
        assert (v <= t) == ok
    # opposite signs are never within a ratio
    [(v, t)] = _criteria_linear(1.0, -1.0, Convergence(2.0, 0.5, 0.0, 0.0, 1, 1))
    assert v > t
