"""Pins for the oracle's beam search and occlusion prune (Section 3: beam
search of width ef_h from the tree roots; occlusion prune of the expanded set
to at most R neighbours, after FANNG and DiskANN).

Beam: hand-worked fixture; with ef >= n on a connected graph the pool is the
brute-force (delta, id) order of all points and every point is expanded; at
any ef the pool is sorted, each entry no better than the brute-force entry of
the same rank, and the pool holds the best of what was evaluated.
Prune: hand-worked fixture; no kept edge is alpha-dominated; every dropped
candidate is dominated by an earlier kept one or comes after the R-th keep;
R = 1 keeps the nearest; alpha = 0 keeps only the nearest and a huge
alpha keeps the R nearest.
"""
import numpy as np
import pytest

import oracle
from paper_2609_30493_gb300 import synth
from golden import reader


def _csr(n, edges):
    adj = [set() for _ in range(n)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    off = np.zeros(n + 1, np.int64)
    for u in range(n):
        off[u + 1] = off[u] + len(adj[u])
    ids = np.array([v for u in range(n) for v in sorted(adj[u])], np.int32)
    return off, ids


def test_beam_golden():
    g = reader.load("beam_path.txt")
    D = oracle.Data(g["X"], g["d"], g["metric"])
    off, ids = _csr(len(g["X"]), g["edges"])
    q = np.array(g["query"], np.float32)
    for case in g["cases"]:
        E, Ed, P, Pd, nev = oracle.beam(D, off, ids, np.array([g["root"]]), q, int(case["ef"]))
        assert E.tolist() == [int(v) for v in case["expand"].split(",")]
        assert P.tolist() == [int(v) for v in case["pool"].split(",")]
        assert nev == int(case["evals"])


def _tiny():
    ps = synth.gaussian_mixture(250, 16, 4, seed=2)
    D = oracle.Data(ps.X, 16, 0)
    rts, parents, _ = oracle.sat_forest(D, 3, seed=4)
    off, ids = oracle.scaffold(250, parents)
    return ps, D, rts, off, ids


def test_beam_full_width_is_brute_force():
    ps, D, rts, off, ids = _tiny()
    Q = synth.queries(ps, 5, 9)
    for q in list(Q) + [ps.X[17]]:
        E, Ed, P, Pd, nev = oracle.beam(D, off, ids, rts, q, 250)
        bd = np.array([oracle.dist_vec(D, q, j) for j in range(250)], np.float32)
        order = np.lexsort((np.arange(250), bd))
        assert P.tolist() == order.tolist()
        assert sorted(E.tolist()) == list(range(250))
        assert nev == 250
        # expansion always takes the best unexpanded entry: with a full-width
        # pool the expansion order is increasing in (delta, id) until the
        # frontier forces a worse vertex; the recorded distances are exact
        assert np.array_equal(Ed, bd[E])


@pytest.mark.parametrize("ef", [1, 4, 16, 40])
def test_beam_pool_bounds(ef):
    ps, D, rts, off, ids = _tiny()
    Q = synth.queries(ps, 6, 11)
    for q in Q:
        E, Ed, P, Pd, nev = oracle.beam(D, off, ids, rts, q, ef)
        bd = np.sort(np.array([oracle.dist_vec(D, q, j) for j in range(250)], np.float32))
        assert len(P) == min(ef, nev)
        assert (np.diff(Pd) >= 0).all()
        assert (Pd >= bd[: len(Pd)]).all()
        assert set(P.tolist()) <= set(E.tolist())  # the search ends with all pool entries expanded
        assert len(set(E.tolist())) == len(E)
        assert nev >= len(E)


def test_prune_golden():
    g = reader.load("prune_line.txt")
    D = oracle.Data(g["X"], g["d"], g["metric"])
    cand = np.array(g["cand"], np.int32)
    for case in g["cases"]:
        kept, ev = oracle.prune_list(D, g["p"], cand, g["alpha"], int(case["R"]))
        assert kept.tolist() == [int(v) for v in case["keep"].split(",")]
        assert ev == int(case["evals"])


def _check_prune(D, p, cand, alpha, R, kept):
    a2 = np.float32(alpha) * np.float32(alpha)
    cand = sorted(set(int(c) for c in cand if c != p),
                  key=lambda c: (oracle.dist(D, p, c), c))
    pos = {c: i for i, c in enumerate(cand)}
    assert len(kept) <= R
    assert [pos[k] for k in kept] == sorted(pos[k] for k in kept)  # keep order = rank order
    for i, ki in enumerate(kept):
        for kj in kept[i + 1:]:
            assert np.float32(a2 * np.float32(oracle.dist(D, ki, kj))) > oracle.dist(D, p, kj)
    last = pos[kept[-1]] if kept else -1
    for c in cand:
        if c in kept:
            continue
        dominated = any(pos[k] < pos[c] and
                        np.float32(a2 * np.float32(oracle.dist(D, k, c))) <= oracle.dist(D, p, c)
                        for k in kept)
        assert dominated or (len(kept) == R and pos[c] > last)


@pytest.mark.parametrize("R,alpha", [(1, 1.2), (4, 1.0), (8, 1.2), (16, 1.5), (64, 1.2)])
def test_prune_invariants(R, alpha):
    ps = synth.gaussian_mixture(200, 16, 2, seed=5)
    D = oracle.Data(ps.X, 16, 0)
    rng = np.random.default_rng(R)
    for p in range(0, 200, 23):
        cand = rng.choice(200, size=60, replace=False)
        kept, _ = oracle.prune_list(D, p, cand, alpha, R)
        _check_prune(D, p, cand, alpha, R, kept.tolist())
        if R == 1:
            nearest = min((c for c in cand if c != p), key=lambda c: (oracle.dist(D, p, c), c))
            assert kept.tolist() == [nearest]


def test_prune_extreme_alpha():
    # alpha = 0 removes every candidate after the first keep; a huge alpha
    # removes none, so the prune reduces to the R nearest in (delta, id) order
    ps = synth.gaussian_mixture(120, 16, 2, seed=6)
    D = oracle.Data(ps.X, 16, 0)
    cand = np.arange(1, 120)
    order = sorted(cand.tolist(), key=lambda c: (oracle.dist(D, 0, c), c))
    kept, _ = oracle.prune_list(D, 0, cand, 0.0, 32)
    assert kept.tolist() == order[:1]
    kept, _ = oracle.prune_list(D, 0, cand, 1e6, 32)
    assert kept.tolist() == order[:32]


def test_prune_drops_self_and_repeats():
    ps = synth.gaussian_mixture(50, 16, 2, seed=8)
    D = oracle.Data(ps.X, 16, 0)
    a, _ = oracle.prune_list(D, 3, np.array([3, 5, 5, 7, 9, 7]), 1.2, 8)
    b, _ = oracle.prune_list(D, 3, np.array([5, 7, 9]), 1.2, 8)
    assert a.tolist() == b.tolist()
