"""The chain-resolution algorithm of the GPU shuffles, modelled in plain
Python and checked against the oracle's sequential swap application.

The GPU kernels apply a swap sequence j[] by four parallel passes instead of
the sequential loop of Algorithm 1 (see csrc/chains.cu).  This model runs
the same passes on the same data structures (list heads, links, the
out-of-order bitmap) one step at a time, with the pushes of pass 1 in an
arbitrary order, as concurrent threads may perform them.  It must give the
sequential result for every swap sequence: exhaustively for n <= 7 (every j
with j[p] in [0, p]) under several push orders, and for random and extreme
sequences at larger n.  The kernels themselves are compared with the oracle
on the GPU (test_gpu_chains.py, test_gpu_shuffle.py, test_gpu_batched.py).
"""
import itertools
import random

import numpy as np

import oracle


def chain_apply(a, j, order):
    """The four passes: push (in `order`), fix parents, roots, gather."""
    n = len(a)
    head = [0] * n
    link = [0] * n
    flagged = [False] * n
    for c in order:  # pass 1
        y = j[c]
        if y == c:  # self-target: not listed, link records c
            link[c] = c
            continue
        old = head[y]
        head[y] = c
        link[c] = old if old else y  # empty list: the link is the target
        if old and old < c:
            flagged[y] = True
    for y in range(n):  # pass 2
        h = head[y]
        if h == 0:
            head[y] = y
        elif flagged[y]:
            members, m = [], h
            while True:
                members.append(m)
                if link[m] == y:
                    break
                m = link[m]
            members.sort()
            for p, q in zip(members, members[1:]):
                link[p] = q
            link[members[-1]] = y
            head[y] = members[0]
    q = head  # pass 3: roots, in decreasing order with path compression
    for x in range(n - 1, -1, -1):
        r = q[x]
        while q[r] != r:
            r = q[r]
        q[x] = r
    out = [a[q[0]]]  # pass 4
    for c in range(1, n):
        lc = link[c]
        out.append(a[q[lc]] if lc >= c else a[lc])
    return out


def _orders(n, rng):
    steps = list(range(1, n))
    yield steps[::-1]  # decreasing, as the kernels mostly push
    yield steps  # increasing: every list out of order
    yield rng.sample(steps, len(steps))


def _check(j, rng):
    n = len(j)
    data = np.arange(100, 100 + n, dtype=np.uint32)
    want = oracle.apply_swaps(data, np.array(j, dtype=np.uint32)).tolist()
    for order in _orders(n, rng):
        assert chain_apply(data.tolist(), j, order) == want, (j, order)


def test_exhaustive_small():
    rng = random.Random(1)
    for n in range(1, 8):
        for tail in itertools.product(*[range(c + 1) for c in range(1, n)]):
            _check([0] + list(tail), rng)


def test_random_and_extreme_sequences():
    rng = random.Random(2)
    for n in (50, 257, 1000, 4099):
        for _ in range(10):
            _check([0] + [rng.randrange(c + 1) for c in range(1, n)], rng)
        _check([0] * n, rng)  # every step targets slot 0
        _check(list(range(n)), rng)  # every step targets itself
        _check([0] + [c - 1 for c in range(1, n)], rng)  # one long chain
