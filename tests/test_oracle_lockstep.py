"""Lockstep density (Section 5.5, Table 6): how much the visited sets of the
queries of one group overlap, the sum of their sizes over (group size x the
size of their union).

Pins: the visited set of a beam has exactly the size the beam counts as
evaluations and holds every expanded vertex; a group of one query, or of
the same query repeated, has density 1; disjoint sets give 1/|group|.  The
measurement itself runs the frozen substrate S_0 of a 20,000-point seeded
subset of the in-cache workload (unit vectors, d = 100, T = 8, ef_h = 64):
groups that are subtrees of tree 0 (64 to 512 points, the points themselves
as queries, as in the harvest) against random groups of the same sizes.  It
is a report (printed with -s), not a pin: the paper's figure comes from its
own datasets.
"""
import numpy as np
import pytest

import oracle
from paper_2609_30493_gb300 import synth


def test_density_special_cases():
    a = np.array([1, 2, 3], np.int32)
    b = np.array([4, 5], np.int32)
    assert oracle.lockstep_density([a]) == 1.0
    assert oracle.lockstep_density([a, a, a]) == 1.0
    assert oracle.lockstep_density([a, b]) == pytest.approx(5 / (2 * 5))
    assert oracle.lockstep_density([a, np.array([1, 2, 3, 4], np.int32)]) == \
        pytest.approx(7 / (2 * 4))


@pytest.fixture(scope="module")
def incache_subset():
    ps = synth.vmf_like(20_000, 100, 64, seed=0, kappa=20.0)
    D = oracle.Data(ps.X, 100, 1)
    rts, parents, _ = oracle.sat_forest(D, 8, seed=0)
    s_off, s_ids = oracle.scaffold(20_000, parents)
    return ps, D, rts, parents, s_off, s_ids


def test_visited_matches_beam(incache_subset):
    ps, D, rts, parents, s_off, s_ids = incache_subset
    for p in (0, 777, 12345):
        v = oracle.visited(D, s_off, s_ids, rts, ps.X[p], 64)
        E, Ed, P, Pd, nev = oracle.beam(D, s_off, s_ids, rts, ps.X[p], 64)
        assert len(v) == nev and len(np.unique(v)) == len(v)
        assert set(E.tolist()) <= set(v.tolist())
        assert set(rts.tolist()) <= set(v.tolist())


def _subtrees(parent0, lo, hi):
    n = len(parent0)
    ch = [[] for _ in range(n)]
    root = -1
    for x in range(n):
        if parent0[x] >= 0:
            ch[parent0[x]].append(x)
        else:
            root = x
    order, stack = [], [root]
    while stack:
        u = stack.pop()
        order.append(u)
        stack.extend(ch[u])
    size = np.ones(n, np.int64)
    for u in reversed(order):
        if parent0[u] >= 0:
            size[parent0[u]] += size[u]
    picks = [u for u in range(n) if lo <= size[u] <= hi]
    groups = []
    for u in picks[:4]:
        members, stack = [], [u]
        while stack:
            w = stack.pop()
            members.append(w)
            stack.extend(ch[w])
        groups.append(np.array(members, np.int32))
    return groups


def test_lockstep_density_measured(incache_subset, capsys):
    ps, D, rts, parents, s_off, s_ids = incache_subset
    coherent = _subtrees(parents[0], 64, 512)
    assert coherent, "no tree-0 subtree of 64 to 512 points"
    rng = np.random.default_rng(3)
    random_groups = [rng.choice(D.n, size=len(g), replace=False).astype(np.int32)
                     for g in coherent]

    def density(group):
        sets = [oracle.visited(D, s_off, s_ids, rts, ps.X[p], 64) for p in group]
        dd = oracle.lockstep_density(sets)
        assert 1.0 / len(group) <= dd <= 1.0
        return dd

    dc = [density(g) for g in coherent]
    dr = [density(g) for g in random_groups]
    with capsys.disabled():
        print(f"\nlockstep density, groups of {[len(g) for g in coherent]} points: "
              f"tree-0 subtrees {np.round(dc, 4).tolist()}, random {np.round(dr, 4).tolist()}")
    # every query shares the roots and the first expansions, so even random
    # groups overlap far above 1 / |group|
    assert min(dc + dr) > 4.0 / min(len(g) for g in coherent)


def _preorder(parent0):
    n = len(parent0)
    ch = [[] for _ in range(n)]
    root = -1
    for x in range(n):
        if parent0[x] >= 0:
            ch[parent0[x]].append(x)
        else:
            root = x
    order, stack = [], [root]
    while stack:
        u = stack.pop()
        order.append(u)
        stack.extend(reversed(ch[u]))
    return np.array(order, np.int32)


def test_preorder_windows_share_targets(incache_subset, capsys):
    """Column-batched target loads (Section 5.5) save at most the share of a
    window's gathers that another search of the same window also makes,
    1 - |union| / (sum of sizes) = 1 - 1 / (W x density), and only if the
    searches reached the shared targets at the same moment.  Windows of W
    consecutive points of the tree-0 preorder (the order the harvest kernel
    claims its searches in) against windows of random points: a report, with
    the one property that the preorder's windows share more."""
    ps, D, rts, parents, s_off, s_ids = incache_subset
    pre = _preorder(parents[0])
    assert sorted(pre.tolist()) == list(range(D.n))
    run = pre[5000:5000 + 320]
    rnd = np.random.default_rng(4).choice(D.n, size=len(run), replace=False).astype(np.int32)
    vis_run = [oracle.visited(D, s_off, s_ids, rts, ps.X[p], 64) for p in run]
    vis_rnd = [oracle.visited(D, s_off, s_ids, rts, ps.X[p], 64) for p in rnd]

    def shared(vis, W):
        out = []
        for i in range(0, len(vis) - W + 1, W):
            grp = vis[i:i + W]
            dd = oracle.lockstep_density(grp)
            out.append(1.0 - 1.0 / (W * dd))
        return float(np.mean(out))

    rows = [(W, shared(vis_run, W), shared(vis_rnd, W)) for W in (4, 8, 16)]
    with capsys.disabled():
        print("\nshared share of a window's gathers (W, tree-0 preorder, random): " +
              ", ".join(f"({W}, {a:.3f}, {b:.3f})" for W, a, b in rows))
    for W, a, b in rows:
        assert 0.0 <= b <= 1.0 and 0.0 <= a <= 1.0
    assert rows[-1][1] > rows[-1][2]
