"""The oracle's threaded helpers (host threads over independent batch ranges
or arrays) give the same outputs as its one-thread functions.

The word of a batch depends only on (seed, batch index, attempt), so any split
of the batches over threads must reproduce the sequential result exactly;
these helpers serve the full-size GPU parity tests and the all-cores CPU
baseline."""
import numpy as np
import pytest

import oracle
from paper_2408_06213_gb300 import inputs


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_dice_parallel_equals_sequential(threads):
    bm1, off = inputs.dice_workload(50_003, seed=7)
    ref = oracle.dice(bm1, off, 7)
    assert np.array_equal(oracle.dice_parallel(bm1, off, 7, threads=threads), ref)
    # one roll per batch (the unbatched form)
    ref1 = oracle.dice(bm1[:9_001], None, 11)
    assert np.array_equal(oracle.dice_parallel(bm1[:9_001], None, 11, threads=threads), ref1)


def test_dice_parallel_rejects_bad_offsets():
    bm1, off = inputs.dice_workload(1000, seed=7)
    bad = off.copy()
    bad[5], bad[6] = bad[6], bad[5]
    with pytest.raises(oracle.OracleError):
        oracle.dice_parallel(bm1, bad, 7)


@pytest.mark.parametrize("b", list(inputs.FIXED_BOUNDS) + [1 << 32])
def test_dice_fixed_parallel_equals_sequential(b):
    k = inputs.fixed_k(b) if b != 1 << 32 else 2
    for n in (1, 7, 40_001):
        ref = oracle.dice_fixed(b, k, n, 5)
        assert np.array_equal(oracle.dice_fixed_parallel(b, k, n, 5, threads=4), ref)


@pytest.mark.parametrize("threads", [1, 4])
def test_shuffle_batched_parallel_equals_sequential(threads):
    data, offsets, seeds, _ = inputs.batched_shuffles(n_arrays=300)
    ref = oracle.shuffle_batched(data, offsets, seeds)
    assert np.array_equal(oracle.shuffle_batched_parallel(data, offsets, seeds, threads=threads), ref)
    # another schedule (one word per die)
    nk1 = (0,) * 9
    ref1 = oracle.shuffle_batched(data, offsets, seeds, nk=nk1, k_max=1)
    got1 = oracle.shuffle_batched_parallel(data, offsets, seeds, nk=nk1, k_max=1, threads=threads)
    assert np.array_equal(got1, ref1)


def test_sparse_sample_reference_matches_the_oracle():
    """The dictionary form of the sample used for n beyond what the oracle
    materialises agrees with oracle.sample wherever both run."""
    from _sample_ref import sample_sparse

    for n, m in [(1, 1), (2, 2), (5, 5), (6, 3), (100, 99), (1000, 7), (70000, 3000), (2 ** 21, 500)]:
        assert np.array_equal(sample_sparse(n, m, 9 + m), oracle.sample(n, m, 9 + m)), (n, m)
