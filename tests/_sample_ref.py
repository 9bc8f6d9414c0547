"""A restatement of the partial Fisher-Yates sample for arrays too large to
materialise (test helper): Algorithm 1's first m steps on the virtual
identity array, with the dice from the oracle and only the written slots
stored.  Pinned to oracle.sample by tests/test_oracle_parallel.py."""
import numpy as np

import oracle


def sample_sparse(n, m, seed):
    """The first m steps of Algorithm 1 on the virtual identity array of
    length n, for n too large to materialise: batches as the oracle plans
    them (k = min(k_rule(i), i - stop)), dice from oracle.roll_batch, and a
    dictionary holding only the slots the steps have written."""
    stop = max(n - m, 1)
    slot = {}
    i, g, out = n, 0, []
    while i > stop:
        k = min(oracle.k_rule(i), i - stop)
        digits, _ = oracle.roll_batch([i - q for q in range(k)], seed, g)
        for q, j in enumerate(digits):
            p = i - 1 - q
            vp, vj = slot.get(p, p), slot.get(j, j)
            slot[p], slot[j] = vj, vp
            out.append(slot[p])
        g += 1
        i -= k
    if m == n:
        out.append(slot.get(0, 0))
    return np.array(out[:m], dtype=np.uint32)
