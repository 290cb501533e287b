"""Pins for the oracle's spatial approximation trees and scaffold (Section 1:
T SAT trees [Navarro 2002] whose edges are unioned and symmetrised; Section 3:
S_0 is that union).

Checked by brute force on small inputs, independently of how the oracle
builds the tree: every tree spans the points with n-1 edges; each node's
children satisfy the neighbour condition in key order; each other point of a
node's subtree was rejected by an earlier child and sits under its closest
child; the work count matches its closed form per node; hand-worked
fixtures; the scaffold equals the symmetrised union built here in numpy.
"""
import numpy as np
import pytest

import oracle
from paper_2609_30493_gb300 import synth
from golden import reader


def _children(parent):
    ch = {i: [] for i in range(len(parent))}
    for x, p in enumerate(parent):
        if p >= 0:
            ch[int(p)].append(x)
    return ch


def _subtree(ch, a):
    out, st = [], [a]
    while st:
        u = st.pop()
        out.append(u)
        st.extend(ch[u])
    return out


def check_sat(D, root, parent, evals):
    n = D.n
    assert parent[root] == -1
    assert (parent[np.arange(n) != root] >= 0).all()
    # spanning, acyclic: every point reaches the root
    for x in range(n):
        seen, u = 0, x
        while u != root:
            u = parent[u]
            seen += 1
            assert seen <= n
    ch = _children(parent)
    work = 0
    for a in range(n):
        P = [x for x in _subtree(ch, a) if x != a]
        if not P:
            continue
        N = ch[a]
        key = {x: (oracle.dist(D, x, a), x) for x in P}
        Ns = sorted(N, key=lambda x: key[x])
        # neighbour condition: strictly closer to a than to every earlier child
        for i, x in enumerate(Ns):
            for b in Ns[:i]:
                assert oracle.dist(D, x, a) < oracle.dist(D, x, b)
        sub_of = {}
        for b in N:
            for y in _subtree(ch, b):
                sub_of[y] = b
        for y in P:
            if y in N:
                continue
            # rejected by some child with a smaller key
            assert any(key[b] < key[y] and not (oracle.dist(D, y, a) < oracle.dist(D, y, b))
                       for b in N)
            # and placed under its closest child (ties to the smaller id)
            best = min(N, key=lambda b: (oracle.dist(D, y, b), b))
            # y sits in best's subtree only if y was assigned at node a to best
            # (deeper points were assigned at a as well: subtree(b) minus b is
            # exactly what node a assigned to b)
            assert sub_of[y] == best
        m, k = len(P), len(N)
        work += m + k * (k - 1) // 2 + (m - k) * k
    assert work == evals


@pytest.mark.parametrize("metric,d,n", [(0, 4, 60), (0, 16, 150), (1, 100, 120), (2, 16, 100)])
def test_sat_invariants(metric, d, n):
    if metric == 1:
        ps = synth.vmf_like(n, d, 4, seed=3)
    elif metric == 2:
        ps = synth.uint8_mixture(n, d, 4, seed=3)
    else:
        ps = synth.gaussian_mixture(n, d, 4, seed=3)
    D = oracle.Data(ps.X, d, metric)
    for root in (0, n // 2):
        parent, ev = oracle.sat_tree(D, root)
        check_sat(D, root, parent, ev)


def test_sat_with_duplicates_and_ties():
    rng = np.random.default_rng(0)
    base = rng.integers(0, 3, size=(12, 4)).astype(np.float32)
    X = np.concatenate([base, base[:6], base[:3]])  # repeated points, many ties
    D = oracle.Data(X, 4, 0)
    for root in (0, 5, 20):
        parent, ev = oracle.sat_tree(D, root)
        check_sat(D, root, parent, ev)


@pytest.mark.parametrize("name", ["sat_line.txt", "sat_tie.txt"])
def test_sat_golden(name):
    g = reader.load(name)
    D = oracle.Data(g["X"], g["d"], g["metric"])
    parent, ev = oracle.sat_tree(D, g["root"])
    assert {i: int(p) for i, p in enumerate(parent)} == g["parents"]
    assert ev == g["evals"]


def test_forest_and_scaffold():
    ps = synth.gaussian_mixture(300, 16, 4, seed=1)
    D = oracle.Data(ps.X, 16, 0)
    rts, parents, ev = oracle.sat_forest(D, 4, seed=0)
    assert (rts == oracle.roots(0, 4, 300)).all()
    tot = 0
    for t in range(4):
        p1, e1 = oracle.sat_tree(D, int(rts[t]))
        assert (p1 == parents[t]).all()
        tot += e1
    assert tot == ev
    off, ids = oracle.scaffold(300, parents)
    edges = set()
    for t in range(4):
        for x in range(300):
            p = parents[t, x]
            if p >= 0:
                edges.add((x, int(p)))
                edges.add((int(p), x))
    got = set()
    for u in range(300):
        row = ids[off[u]:off[u + 1]]
        assert (np.diff(row) > 0).all()
        got.update((u, int(v)) for v in row)
    assert got == edges
