"""Host-side helpers of bench.py that shape its measurements."""
import numpy as np

import bench


def _children(par):
    ch = [[] for _ in range(len(par))]
    for v, p in enumerate(par):
        if p >= 0:
            ch[p].append(v)
    return ch


def _subtree(ch, u):
    out, stack = [u], [u]
    while stack:
        x = stack.pop()
        for c in ch[x]:
            out.append(c)
            stack.append(c)
    return out


def test_subtree_groups_brute_force():
    rng = np.random.default_rng(0)
    for n, cap in ((1, 5), (300, 7), (3000, 50)):
        perm = rng.permutation(n)
        par = np.full(n, -1, np.int64)
        for i in range(1, n):
            par[perm[i]] = perm[rng.integers(0, i)]
        tops, lab, size = bench._subtree_groups(par, cap)
        ch = _children(par)
        for u in range(n):
            assert size[u] == len(_subtree(ch, u))
        for u in tops:
            assert size[u] <= cap and (par[u] < 0 or size[par[u]] > cap)
            assert set(np.flatnonzero(lab == u).tolist()) == set(_subtree(ch, u))
        assert np.array_equal(lab >= 0, size <= cap)


def test_subtree_groups_path():
    # a path 0 <- 1 <- 2 <- ... : the maximal subtree of at most 3 points is {n-3, n-2, n-1}
    n = 10
    par = np.arange(-1, n - 1)
    tops, lab, size = bench._subtree_groups(par, 3)
    assert tops.tolist() == [7]
    assert np.flatnonzero(lab == 7).tolist() == [7, 8, 9]
