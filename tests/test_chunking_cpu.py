"""How a job's budgets are cut into chunks (bfi_chunking_of, host only): the
rule every entry point uses, checked on the CPU through the C ABI.

Chunks are the work units the integrand kernels hand out to CTAs, in index
order.  The cut depends on the budgets alone.  The last subvolumes, up to an
eighth of the samples, are cut into chunks a quarter as long so that the
launch ends on short chunks."""
import numpy as np
import pytest

BLOCK = 256          # threads per CTA of the thread-per-sample kernels
TWO_STAGE_ROWS = 256  # rows per thread from which a chunk screens in two stages


def _rows(c):
    return c // BLOCK


def _check_invariants(samples, ch):
    """What the rule promises, whatever the budgets."""
    samples = np.asarray(samples, dtype=np.uint64)
    nsub, total = samples.size, int(samples.sum())
    cs, ts, tc = ch.chunk_samples, ch.tail_subvolume, ch.tail_chunk_samples
    rows = _rows(cs)
    assert cs % BLOCK == 0 and rows & (rows - 1) == 0 and 4 <= rows <= 2048
    # at least 2048 chunks of the main size whenever there are 4 rows to spare
    if rows > 4:
        assert total // cs >= 2048
    # rows above 512 only while 4096 chunks remain
    if rows > 512:
        assert total // cs >= 4096
    assert 0 <= ts <= nsub
    if ts < nsub:
        tail = int(samples[ts:].sum())
        assert 0 < tail <= min(total // 8, 512 * cs)
        assert tc == max(cs // 4, TWO_STAGE_ROWS * BLOCK) and tc < cs
        assert _rows(tc) >= TWO_STAGE_ROWS
        # the longest such suffix: one more subvolume would break the limit
        if ts > 0:
            assert tail + int(samples[ts - 1]) > min(total // 8, 512 * cs)
    else:
        assert tc == cs
    per = [(int(n) + (tc if s >= ts else cs) - 1) // (tc if s >= ts else cs) for s, n in enumerate(samples)]
    assert ch.chunks == sum(per)


@pytest.mark.parametrize("samples,cs,ts,tc,chunks", [
    # 10x2, 1024 subvolumes x 2^20: 1024 rows, the last 128 subvolumes (2^27 samples) in 256-row chunks
    ([1 << 20] * 1024, 1 << 18, 896, 1 << 16, 896 * 4 + 128 * 16),
    # the 2^34-sample job: 2048 rows; 512 chunks' worth (2^28) is the limit, 16 subvolumes in 512-row chunks
    ([1 << 24] * 1024, 1 << 19, 1008, 1 << 17, 1008 * 32 + 16 * 128),
    # 2^27 samples: 256 rows, no shorter chunk keeps the two-stage screen, so no tail
    ([1 << 21] * 64, 1 << 16, 64, 1 << 16, 2048),
    # 2^28 samples: 512 rows, tail chunks of 256
    ([1 << 24] * 16, 1 << 17, 14, 1 << 16, 14 * 128 + 2 * 256),
    # one subvolume: no suffix of whole subvolumes fits an eighth
    ([1 << 30], 1 << 18, 1, 1 << 18, 4096),
    # small jobs: 4 rows, no tail
    ([30_000, 1, 0, 65_436], 1024, 4, 1024, 30 + 1 + 0 + 64),
])
def test_chunking_of_known_jobs(bfi, samples, cs, ts, tc, chunks):
    ch = bfi.chunking(samples)
    assert (ch.chunk_samples, ch.tail_subvolume, ch.tail_chunk_samples, ch.chunks) == (cs, ts, tc, chunks)
    _check_invariants(samples, ch)


def test_chunking_invariants_on_random_budgets(bfi):
    rng = np.random.default_rng(11)
    for _ in range(300):
        nsub = int(rng.integers(1, 3000))
        scale = 2.0 ** rng.uniform(4, 30)
        samples = np.floor(rng.pareto(1.5, nsub) * scale).astype(np.uint64)
        if rng.random() < 0.3:
            samples[rng.integers(0, nsub, nsub // 4 + 1)] = 0
        if samples.sum() == 0:
            samples[0] = 1
        _check_invariants(samples, bfi.chunking(samples))


def test_chunking_rejects_bad_budgets(bfi):
    with pytest.raises(bfi.BfiError):
        bfi.chunking(np.array([], dtype=np.uint64))
    with pytest.raises(bfi.BfiError):
        bfi.chunking([1 << 48])
    with pytest.raises(bfi.BfiError):
        bfi.chunking([(1 << 48) - 1] * (1 << 15))   # 2^63 in all
