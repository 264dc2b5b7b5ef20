"""The C-ABI library loads on the CPU, exports every symbol include/bfi.h
declares, and its host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "bfi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bfi_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(bfi):
    lib = ctypes.CDLL(bfi.LIBRARY_PATH)
    names = _declared_functions()
    assert "bfi_plan_execute" in names and "bfi_integrate" in names
    for name in names:
        assert hasattr(lib, name), name
    # and the binding declares a signature for each of them
    assert set(names) <= set(bfi._SIGNATURES)


def test_record_sizes(bfi):
    for nx in (2, 3, 4, 10, 64):
        R = nx // 2 + 1
        assert bfi.num_r(nx) == R
        assert bfi.slot_len(nx) == oracle.slot_len(nx) == 5 + 3 * R
        assert bfi.totals_len(nx) == oracle.totals_len(nx) == 4 + 2 * R


def test_invalid_arguments_are_rejected_before_any_device_call(bfi):
    bad = [bfi.lattice(1, 2), bfi.lattice(4, 0), bfi.lattice(64, 16), bfi.lattice(4, 2, D=0.0),
           bfi.lattice(4, 2, tau=-1.0), bfi.lattice(4, 2, mass2=-1.0), bfi.lattice(4, 2, nu=float("nan"))]
    for lat in bad:
        with pytest.raises(bfi.BfiError) as e:
            bfi.Plan(lat, [100])
        assert e.value.status == 1
    with pytest.raises(bfi.BfiError) as e:
        bfi.Plan(bfi.lattice(4, 2), [1 << 50])
    assert e.value.status == 1 and "2^48" in str(e.value)


def test_host_merge_matches_oracle_merge(bfi):
    # the library's own FP64 host merge against the oracle's, on oracle records
    lat = oracle.lattice(6, 2)
    d = 12
    lo = np.stack([np.full(d, -3.0), np.full(d, -1.0), np.full(d, 0.0), np.full(d, -2.0)])
    hi = np.stack([np.full(d, 3.0), np.full(d, 1.0), np.full(d, 0.5), np.full(d, 2.0)])
    slots, tot = oracle.integrate(lat, lo, hi, [1000, 3000, 0, 2000], seed=8)
    mine = bfi.merge_host(6, slots)
    np.testing.assert_allclose(mine, tot, rtol=1e-13)
    # one-sample subvolume -> infinite errors, like the oracle
    s1, t1 = oracle.integrate(lat, lo[:1], hi[:1], [1], seed=8)
    m1 = bfi.merge_host(6, s1)
    assert np.isinf(m1[1]) and np.isinf(t1[1]) and m1[0] == pytest.approx(t1[0], rel=1e-15)


def test_stated_error_bound_on_oracle_records(bfi):
    """bfi_error_bound is host arithmetic on a result's records.  In FP32 it
    stays below 1e-6 on Z and C(r) for the 4x2 and 10x2 lattices of the plain,
    paper-shaped and precision workloads over the batching workload's nu range
    [0.1, 10]; for bigger lattices at large actions (S in the tens of
    thousands and more) the compensated action's absolute error grows with S
    and the bound says so.  In FP64 the bound is a few 1e-12 for 10x2 (a
    worst case: the measured agreement with the oracle is ~1e-14) and grows
    with S like exp(-S)'s conditioning."""
    def records(nx, nt, p):
        d = nx * nt
        lo, hi = np.full((2, d), -5.0), np.full((2, d), 5.0)
        lo[1, 0], hi[0, 0] = 0.0, 0.0
        return oracle.integrate(oracle.lattice(nx, nt, **p), lo, hi, [3000, 3000], seed=3)[0]

    for nx, nt in [(4, 2), (10, 2)]:
        for p in [dict(nu=0.1), {}, dict(nu=10.0), dict(nu=0.1, D=1.7, a=0.8, tau=0.6)]:
            slots = records(nx, nt, p)
            lat = bfi.lattice(nx, nt, **p)
            b32 = bfi.error_bound(lat, bfi.FP32, slots, 5.0)
            b64 = bfi.error_bound(lat, bfi.FP64, slots, 5.0)
            assert b32.shape == (1 + nx // 2 + 1,)
            assert np.all(b32 > 0) and np.all(b32 < 1e-6), (nx, nt, p, b32)
            assert b32[0] < 5e-7 and np.all(b32[1:] > b32[0])  # C(r) adds the products' rounding
            assert np.all(b64 > 0) and np.all(b64 < 1e-9) and np.all(b64 < b32)
            if not p:
                assert b64.max() < 1e-11
    small = bfi.error_bound(bfi.lattice(10, 2), bfi.FP32, records(10, 2, {}), 5.0)
    big = bfi.error_bound(bfi.lattice(64, 8, nu=10.0), bfi.FP32, records(64, 8, dict(nu=10.0)), 5.0)
    assert big[0] > small[0] and big.max() > small.max() and big.max() < 1e-4
    slots = records(4, 2, {})
    with pytest.raises(bfi.BfiError):
        bfi.error_bound(bfi.lattice(4, 2), bfi.FP32, slots, -1.0)
    with pytest.raises(bfi.BfiError):
        bfi.error_bound(bfi.lattice(4, 2), bfi.FP32, np.zeros((1, 14)), 5.0)
