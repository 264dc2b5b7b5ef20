"""The N-sphere test integrand of Sec. 3 on the GPU and the line-protocol
program bfi_cli (Listings 1-2): parity with the oracle, the paper's worked
example, and input validation (the latter on the CPU)."""
import math
import subprocess

import numpy as np
import pytest

import oracle
from workloads import bisected_boxes

# The GPU sums per thread, then in a fixed tree per block, then over blocks in
# order; the oracle sums compensated in sample order.  Both are within
# (a few thousand) * eps64 of the exact sum of the same terms.
RESULT_RTOL = 1e-12
ERR_RTOL = 1e-10

CASES = [  # dims, n, seed, lo, hi
    (1, 1000, 3, -1.0, 1.0),
    (2, 200_003, 1, -1.0, 1.0),
    (3, 150_000, 5, [-1, -1, 0], [1, 1, 1]),
    (3, 100_001, 2, [-0.2, -1, -1], [1, 1, 1]),
    (4, 99_999, 7, -0.8, 0.9),
    (5, 65_537, 4, -1.0, 1.0),
    (8, 50_000, 9, -0.5, 0.6),
    (17, 20_000, 6, -0.3, 0.3),
    (32, 10_000, 8, -0.2, 0.25),
    (2, 2, 1, -1.0, 1.0),
]


def _run_cli(bfi, args, stdin, timeout=300):
    return subprocess.run([bfi.CLI_PATH, *args], input=stdin, capture_output=True, text=True, timeout=timeout)


@pytest.mark.gpu
@pytest.mark.parametrize("dims,n,seed,lo,hi", CASES)
def test_nsphere_matches_oracle(bfi, dims, n, seed, lo, hi):
    res, err, sd = bfi.nsphere(dims, n, seed, job_id=seed, lo=lo, hi=hi)
    ores, oerr, osd = oracle.nsphere(dims, n, seed, job_id=seed, lo=lo, hi=hi, split=True)
    assert res == pytest.approx(ores, rel=RESULT_RTOL, abs=1e-300)
    assert err == pytest.approx(oerr, rel=ERR_RTOL, abs=1e-300)
    assert sd == osd


@pytest.mark.gpu
def test_nsphere_sub_id_draws_other_points(bfi):
    a = bfi.nsphere(3, 100_000, 1, sub_id=0)
    b = bfi.nsphere(3, 100_000, 1, sub_id=1)
    assert a[0] != b[0]
    assert abs(a[0] - b[0]) < 6 * math.hypot(a[1], b[1])


@pytest.mark.gpu
def test_nsphere_counter_high_word(bfi):
    # more than 2^32 samples use the counter's third word; the estimate of
    # half the unit 2-ball's volume (pi/2 over [-1,1]) stays unbiased
    n = (1 << 32) + 12345
    res, err, _ = bfi.nsphere(1, n, 3)
    assert abs(res - math.pi / 2) < 5 * err
    assert err == pytest.approx(2 * math.sqrt(2 / 3 - (math.pi / 4) ** 2) / math.sqrt(n), rel=1e-3)


@pytest.mark.gpu
def test_listing2_through_the_line_protocol(bfi):
    # Sec. 3, Listing 2: "1e7 -1 1 -1 1" on standard input gives
    # "result abs_error split_dim"; the paper printed 2.0938 and 4.3551e-4.
    r = _run_cli(bfi, [], "1e7 -1 1 -1 1\n")
    assert r.returncode == 0, r.stderr
    fields = r.stdout.split()
    assert len(fields) == 3
    res, err, sd = float(fields[0]), float(fields[1]), int(fields[2])
    assert err == pytest.approx(4.355051371078182e-04, rel=0.01)
    assert abs(res - 2 * math.pi / 3) < 4 * err
    assert sd in (0, 1)
    # the same line through the binding (seed 1, line 0) is the same estimate
    b = bfi.nsphere(2, 10_000_000, 1, job_id=0)
    assert (res, err, sd) == (float(f"{b[0]:.15e}"), float(f"{b[1]:.15e}"), b[2])


@pytest.mark.gpu
def test_cli_lines_are_independent_jobs(bfi):
    lines = "100000 -1 1 -1 1 -1 1\n\n100000 -1 1 -1 1 -1 1\n1000 -1 1\n"
    r = _run_cli(bfi, ["--seed", "4"], lines)
    assert r.returncode == 0, r.stderr
    out = [l.split() for l in r.stdout.strip().splitlines()]
    assert len(out) == 3
    for k, (dims, n) in enumerate([(3, 100_000), (3, 100_000), (1, 1000)]):
        ores, oerr, osd = oracle.nsphere(dims, n, 4, job_id=k, split=True)
        assert float(out[k][0]) == pytest.approx(ores, rel=1e-12)
        assert float(out[k][1]) == pytest.approx(oerr, rel=1e-10)
        assert int(out[k][2]) == osd


@pytest.mark.gpu
@pytest.mark.parametrize("output", ["logz", "z", "c0", "c1", "c2"])
def test_cli_burgers_matches_oracle(bfi, output):
    # one subvolume of the 4x2 lattice per line; line k is job k of seed 3
    lo, hi = bisected_boxes(8, 1)
    lines = "".join(f"40000 {' '.join(f'{a} {b}' for a, b in zip(lo[s], hi[s]))}\n" for s in range(2))
    lines += "30000 -5 5\n"
    r = _run_cli(bfi, ["--integrand", "burgers", "--lattice", "4x2", "--seed", "3", "--output", output], lines)
    assert r.returncode == 0, r.stderr
    out = [l.split() for l in r.stdout.strip().splitlines()]
    boxes = [(lo[0], hi[0], 40000), (lo[1], hi[1], 40000), (np.full(8, -5.0), np.full(8, 5.0), 30000)]
    lat = oracle.lattice(4, 2)
    for k, (l, h, n) in enumerate(boxes):
        _, tot = oracle.integrate(lat, l[None, :], h[None, :], n, seed=3, job_id=k)
        if output == "logz":
            want = (tot[0], tot[1])
        elif output == "z":
            want = (math.exp(tot[0]), math.exp(tot[0]) * tot[1])
        else:
            r_ = int(output[1:])
            want = (tot[4 + r_], tot[4 + 3 + r_])
        # FP64 parity of the lattice path: 16 eps64 relative to the action scale
        assert float(out[k][0]) == pytest.approx(want[0], rel=1e-11, abs=1e-13)
        assert float(out[k][1]) == pytest.approx(want[1], rel=1e-7, abs=1e-13)
        # the split suggestion is the widest side, first on ties
        assert int(out[k][2]) == int(np.argmax(h - l))


@pytest.mark.gpu
def test_listing1_through_the_wrapper_mode(bfi):
    # Sec. 3, Listing 1: the wrapper integrates (half) the unit 4-ball's volume
    # with the 3-dimensional integrand over [-1,1] and prints "result abs_error"
    args = ["--adaptive", "1", "--integrand", "nsphere", "--dimensions", "3", "--min-extent", "-1",
            "--max-extent", "1", "--samples", "1e5", "--rel-tol", "0.003", "--max-depth", "8"]
    r = _run_cli(bfi, args, "")
    assert r.returncode == 0, r.stderr
    res, err = map(float, r.stdout.split())
    assert err < 0.01 and abs(res - math.pi ** 2 / 4) < 4 * err
    b = bfi.adaptive_nsphere(3, 100_000, 1, bfi.convergence(2.0, 0.003, 0.0, 0.0, 8, 1 << 16))
    assert (res, err) == (float(f"{b[0]:.15g}"), float(f"{b[1]:.15g}"))


@pytest.mark.gpu
def test_wrapper_mode_lattice(bfi):
    args = ["--adaptive", "1", "--integrand", "burgers", "--lattice", "4x2", "--min-extent", "-5",
            "--max-extent", "5", "--samples", "20000", "--rel-tol", "0.05", "--max-depth", "4", "--output", "logz",
            "--seed", "3"]
    r = _run_cli(bfi, args, "")
    assert r.returncode == 0, r.stderr
    logz, rel = map(float, r.stdout.split())
    ctx = bfi.Context(0)
    try:
        t, _ = ctx.adaptive_integrate(bfi.lattice(4, 2), -5.0, 5.0, 20_000, 3,
                                      bfi.convergence(2.0, 0.05, 0.0, 0.0, 4, 1 << 16))
    finally:
        ctx.close()
    assert (logz, rel) == (float(f"{t[0]:.15g}"), float(f"{t[1]:.15g}"))


@pytest.mark.parametrize("args,stdin", [
    (["--adaptive", "1"], ""),
    (["--adaptive", "1", "--dimensions", "3", "--factor", "0.5"], ""),
    (["--adaptive", "1", "--dimensions", "3", "--samples", "1"], ""),
    (["--adaptive", "1", "--dimensions", "3", "--min-extent", "1", "--max-extent", "1"], ""),
    (["--adaptive", "1", "--dimensions", "40"], ""),
    ([], "abc\n"),
    ([], "1e7 -1\n"),
    ([], "1.5 -1 1\n"),
    ([], "1 -1 1\n"),
    ([], "100 1 -1\n"),
    (["--integrand", "cube"], ""),
    (["--integrand", "burgers", "--output", "c9"], ""),
    (["--integrand", "burgers", "--output", "w"], ""),
    (["--lattice", "10"], ""),
    (["--seed"], ""),
])
def test_cli_rejects_bad_input_before_the_device(bfi, args, stdin):
    r = _run_cli(bfi, args, stdin, timeout=60)
    assert r.returncode == 2
    assert r.stdout == ""
    assert r.stderr


def test_nsphere_rejects_bad_arguments(bfi):
    with pytest.raises(bfi.BfiError):
        bfi.nsphere(0, 100, 1)
    with pytest.raises(bfi.BfiError):
        bfi.nsphere(33, 100, 1)
    with pytest.raises(bfi.BfiError):
        bfi.nsphere(2, 1, 1)
    with pytest.raises(bfi.BfiError):
        bfi.nsphere(2, 100, 1, lo=[0, 1], hi=[1, 1])
