"""Adaptive subdivision with the convergence test of Sec. 3, written plainly.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

Sec. 3: the volume is subdivided until every subvolume has converged; a
subvolume is evaluated twice, the second time with a user factor more samples,
and has converged when one or more of three criteria holds for the two results:
(1) their absolute relative difference is below a factor, (2) their absolute
difference is below a value, (3) the larger absolute result is below a value.
Sec. 4 quotes the factor of (1) as a ratio (1.025 to 1.085), so (1) reads
|r1 - r2| <= rel_tol * min(|r1|, |r2|): the results lie within a factor
1 + rel_tol of each other.
A subvolume that has not converged is halved along the dimension its
integrand suggests.

The paper leaves open which of the two results a converged subvolume keeps
(here the second), the bookkeeping of the tree (here heap numbers: the whole
volume is node 1, the halves of node h are 2h and 2h + 1, whose evaluations use
sub_id 2h and 2h + 1), and what happens when the subdivision must stop (here a
depth limit and a limit on the subvolumes of one round, halving in order while
both halves fit).  Each round evaluates every open subvolume, one after the
other, and then decides them in order.

Besides the result, the drivers return every decision with its distance from
the threshold that decided it, so a test can tell whether a different rounding
of the results could have flipped it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import integrate, merge, nsphere, slot_len


@dataclass
class Convergence:
    factor: float = 2.0
    rel_tol: float = 0.0
    abs_tol: float = 0.0
    small: float = 0.0
    max_depth: int = 12
    max_leaves: int = 1 << 16


@dataclass
class Outcome:
    stats: dict
    leaves_lo: list = field(default_factory=list)
    leaves_hi: list = field(default_factory=list)
    kept: list = field(default_factory=list)          # what each kept leaf keeps (result or slot)
    margins: list = field(default_factory=list)       # relative distance of each criterion value from its threshold


def _criteria_linear(r1, r2, c):
    """Values and thresholds of criteria (1)-(3) for two plain results."""
    diff = abs(r1 - r2)
    big = max(abs(r1), abs(r2))
    little = min(abs(r1), abs(r2))
    out = []
    if c.rel_tol > 0:
        out.append((diff, c.rel_tol * little))
    if c.abs_tol > 0:
        out.append((diff, c.abs_tol))
    if c.small > 0:
        out.append((big, c.small))
    return out


def _criteria_log(l1, l2, c):
    """The same criteria for positive results given as logarithms:
    |Z1 - Z2| / min(Z1, Z2) = exp(|ln Z1 - ln Z2|) - 1, and |Z1 - Z2| is
    min(Z1, Z2) times that."""
    top = max(l1, l2)
    rel = math.expm1(abs(l1 - l2))
    out = []
    if c.rel_tol > 0:
        out.append((rel, c.rel_tol))
    if c.abs_tol > 0:
        out.append((math.exp(min(l1, l2)) * rel, c.abs_tol))
    if c.small > 0:
        out.append((top, math.log(c.small)))
    return out


def _margin(value, threshold):
    if value == threshold == 0.0:
        return math.inf  # exact zeros on both sides (an integrand that vanishes on the box)
    scale = max(abs(value), abs(threshold), 1e-300)
    return abs(value - threshold) / scale


def _run(lo, hi, n, c, evaluate, criteria):
    """The subdivision loop.  evaluate(lo, hi, n, sub_id) -> (result for the
    criteria, what a kept leaf keeps, split dimension)."""
    n2 = int(math.ceil(c.factor * float(n)))
    front = [(np.array(lo, dtype=float), np.array(hi, dtype=float), 1, 0)]
    out = Outcome(stats=dict(rounds=0, evaluated=0, converged=0, kept_depth=0, kept_budget=0, leaves=0, samples=0))
    st = out.stats
    while front:
        st["rounds"] += 1
        st["evaluated"] += len(front)
        st["samples"] += len(front) * (n + n2)
        evals = []
        for (l, h, heap, depth) in front:
            r1, _, _ = evaluate(l, h, n, 2 * heap)
            r2, keep, sd = evaluate(l, h, n2, 2 * heap + 1)
            crit = criteria(r1, r2, c)
            out.margins.extend(_margin(v, t) for v, t in crit)
            evals.append((any(v <= t for v, t in crit), keep, sd))
        nxt = []
        for (l, h, heap, depth), (ok, keep, sd) in zip(front, evals):
            if not ok and depth < c.max_depth and len(nxt) + 2 <= c.max_leaves:
                mid = 0.5 * (l[sd] + h[sd])
                h_low, l_up = h.copy(), l.copy()
                h_low[sd] = mid
                l_up[sd] = mid
                nxt.append((l, h_low, 2 * heap, depth + 1))
                nxt.append((l_up, h, 2 * heap + 1, depth + 1))
                continue
            if ok:
                st["converged"] += 1
            elif depth >= c.max_depth:
                st["kept_depth"] += 1
            else:
                st["kept_budget"] += 1
            st["leaves"] += 1
            out.leaves_lo.append(l)
            out.leaves_hi.append(h)
            out.kept.append(keep)
        front = nxt
    return out


def adaptive_nsphere(dims, n, seed, conv, job_id=0, lo=-1.0, hi=1.0):
    """(result, abs_err, Outcome) for the N-sphere integrand: the sum of the
    kept results and the root of the sum of their squared errors."""
    lo = np.broadcast_to(np.asarray(lo, dtype=float), (dims,))
    hi = np.broadcast_to(np.asarray(hi, dtype=float), (dims,))

    def evaluate(l, h, m, sub_id):
        r, e, sd = nsphere(dims, m, seed, job_id=job_id, lo=l, hi=h, split=True, sub_id=sub_id)
        return r, (r, e), sd

    out = _run(lo, hi, n, conv, evaluate, _criteria_linear)
    result = sum(r for r, _ in out.kept)
    err = math.sqrt(sum(e * e for _, e in out.kept))
    return result, err, out


def adaptive_integrate(lat, lo, hi, n, seed, conv, job_id=0):
    """(totals, Outcome) for the lattice integral: the test compares Z_s, a
    subvolume is halved along its widest side (the first on ties), and the
    totals merge the kept second evaluations."""
    d = lat.nx * lat.nt
    lo = np.broadcast_to(np.asarray(lo, dtype=float), (d,))
    hi = np.broadcast_to(np.asarray(hi, dtype=float), (d,))

    def evaluate(l, h, m, sub_id):
        slots, _ = integrate(lat, l[None, :], h[None, :], m, seed, job_id=job_id,
                             sub_id=np.array([sub_id], dtype=np.uint32))
        s = slots[0]
        log_z = s[2] - math.log(s[0]) - s[1] + math.log(s[3])
        return log_z, s.copy(), int(np.argmax(h - l))

    out = _run(lo, hi, n, conv, evaluate, _criteria_log)
    totals = merge(lat.nx, np.array(out.kept).reshape(-1, slot_len(lat.nx)))
    return totals, out


__all__ = ["Convergence", "Outcome", "adaptive_nsphere", "adaptive_integrate"]
