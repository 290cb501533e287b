"""Pins for the oracle's FGraft build, final graph, query search and dense
block (Section 3 and Proposition 1; Section 2's brute-force answer key;
Section 5.3's fixed pair sets).

FGraft: B = 0 and B = 1 both give the frozen harvest (Section 3: B <= 1
reproduces Graft); the graph is identical at 1 and N threads
(Proposition 1); S_b grows monotonically; every row of block b equals the
prune of a beam over S_b rebuilt here from the rows of earlier blocks only
(a row of the same or a later block leaking into S_b fails this); rows hold
at most R distinct ids and never the point itself.
Final graph: a hand-worked fixture (an over-degree row whose prune removes a
candidate that the tree-0 spine adds back, rows of exactly R candidates, the
work count); on the tiny workload every row contains the tree-0 spine and is
sorted by (delta, id), a row that needed no prune is exactly C(u) with the
spine, and an over-degree row minus its spine-only vertices equals a prune
of C(u) restated here in plain Python, which passes the prune invariants;
the work counter equals |C(u) U spine(u)| summed plus those prunes' removal
passes.
Search: equals brute force at full width.  Brute force: agrees with a float64
numpy sort wherever the float64 gap exceeds the rounding bound.
Dense block: the float32 top-k equals the float64 top-k up to rank swaps
inside the rounding bound; on integer-valued data they are identical.
"""
import numpy as np
import pytest

import oracle
from golden import reader
from paper_2609_30493_gb300 import synth
from test_oracle_beam_prune import _check_prune


@pytest.fixture(scope="module")
def tiny():
    ps = synth.gaussian_mixture(2000, 16, 8, seed=0)
    D = oracle.Data(ps.X, 16, 0)
    rts, parents, sev = oracle.sat_forest(D, 4, seed=0)
    s_off, s_ids = oracle.scaffold(2000, parents)
    return ps, D, rts, parents, s_off, s_ids


def test_frozen_B0_equals_B1(tiny):
    ps, D, rts, parents, s_off, s_ids = tiny
    A0, c0, k0, _ = oracle.fgraft(D, rts, s_off, s_ids, 16, 32, 0, 1.2)
    A1, c1, k1, _ = oracle.fgraft(D, rts, s_off, s_ids, 16, 32, 1, 1.2)
    assert np.array_equal(A0, A1) and np.array_equal(c0, c1) and k0 == k1


@pytest.mark.parametrize("B", [1, 4])
def test_thread_count_invariance(tiny, B):
    ps, D, rts, parents, s_off, s_ids = tiny
    A1, c1, k1, p1 = oracle.fgraft(D, rts, s_off, s_ids, 16, 32, B, 1.2, nthreads=1)
    A4, c4, k4, p4 = oracle.fgraft(D, rts, s_off, s_ids, 16, 32, B, 1.2, nthreads=4)
    assert np.array_equal(A1, A4) and np.array_equal(c1, c4) and k1 == k4
    assert np.array_equal(p1, p4)


def test_blocks_see_only_earlier_rows(tiny):
    ps, D, rts, parents, s_off, s_ids = tiny
    R, ef, B, alpha = 16, 32, 4, 1.2
    A, cnt, ctr, per = oracle.fgraft(D, rts, s_off, s_ids, R, ef, B, alpha)
    n = 2000
    prev = None
    for b in range(B):
        off, ids = oracle.substrate(n, s_off, s_ids, A, cnt, R, B, b)
        edges = {(u, int(v)) for u in range(n) for v in ids[off[u]:off[u + 1]]}
        if prev is not None:
            assert prev <= edges  # S_b is a subset of S_{b+1}
        prev = edges
        for p in range(b, n, B * 37):
            E, Ed, P, Pd, nev = oracle.beam(D, off, ids, rts, ps.X[p], ef)
            kept, _ = oracle.prune_list(D, p, E, alpha, R)
            assert A[p, :cnt[p]].tolist() == kept.tolist()
            assert (A[p, cnt[p]:] == -1).all()
    assert (cnt <= R).all()
    for p in range(n):
        row = A[p, :cnt[p]]
        assert p not in row and len(set(row.tolist())) == len(row)


def _prune_py(D, p, cand, alpha, R):
    """Section 3's occlusion prune in plain Python (independent of the C
    oracle's prune): candidates minus p, deduplicated, sorted by
    (delta(p, c), id); keep the first alive c*, remove each alive c after it
    with fl(alpha^2 * delta(c*, c)) <= delta(p, c); stop at R kept.  Returns
    (kept ids, candidates examined in the removal passes)."""
    a2 = np.float32(np.float32(alpha) * np.float32(alpha))
    C = sorted({int(c) for c in cand if int(c) != p}, key=lambda c: (oracle.dist(D, p, c), c))
    dp = [np.float32(oracle.dist(D, p, c)) for c in C]
    alive = [True] * len(C)
    kept, ev = [], 0
    for i, c in enumerate(C):
        if not alive[i]:
            continue
        kept.append(c)
        alive[i] = False
        if len(kept) == R:
            break
        for j in range(i + 1, len(C)):
            if alive[j]:
                ev += 1
                if np.float32(a2 * np.float32(oracle.dist(D, c, C[j]))) <= dp[j]:
                    alive[j] = False
    return kept, ev


@pytest.mark.parametrize("R", [2, 3])
def test_final_golden(R):
    g = reader.load("final_spine.txt")
    D = oracle.Data(g["X"], g["d"], g["metric"])
    n = len(g["X"])
    A = np.full((n, R), -1, np.int32)
    cnt = np.zeros(n, np.int32)
    for p, row in g["arows"].items():
        A[p, :len(row)] = row
        cnt[p] = len(row)
    parent0 = np.array([g["parents"][i] for i in range(n)], np.int32)
    case = next(c for c in g["cases"] if int(c["R"]) == R)
    off, ids, ev = oracle.final(D, A, cnt, R, g["alpha"], parent0)
    for u in range(n):
        assert ids[off[u]:off[u + 1]].tolist() == [int(v) for v in case[f"row{u}"].split(",")]
    assert ev == int(case["evals"])


def test_final_graph(tiny):
    ps, D, rts, parents, s_off, s_ids = tiny
    R, alpha = 16, 1.2
    A, cnt, ctr, per = oracle.fgraft(D, rts, s_off, s_ids, R, 32, 4, alpha)
    off, ids, ev = oracle.final(D, A, cnt, R, alpha, parents[0])
    n = 2000
    cand = [set() for _ in range(n)]
    for p in range(n):
        for u in A[p, :cnt[p]]:
            cand[p].add(int(u))
            cand[int(u)].add(p)
    spine = [set() for _ in range(n)]
    for x in range(n):
        if parents[0, x] >= 0:
            spine[x].add(int(parents[0, x]))
            spine[int(parents[0, x])].add(x)
    work, over = 0, 0
    for u in range(n):
        row = ids[off[u]:off[u + 1]].tolist()
        assert len(set(row)) == len(row)
        assert spine[u] <= set(row)
        keys = [(oracle.dist(D, u, v), v) for v in row]
        assert keys == sorted(keys)
        work += len(cand[u] | spine[u])
        if len(cand[u]) <= R:
            assert set(row) == cand[u] | spine[u]
        else:
            over += 1
            kept, pev = _prune_py(D, u, sorted(cand[u]), alpha, R)
            work += pev
            assert set(row) - (spine[u] - set(kept)) == set(kept)
            _check_prune(D, u, sorted(cand[u]), alpha, R, kept)
    assert over > 50  # the over-degree branch is exercised
    assert ev == work


def test_search_full_width_equals_bruteforce(tiny):
    ps, D, rts, parents, s_off, s_ids = tiny
    Q = synth.queries(ps, 20, 1)
    bi, bd = oracle.bruteforce(D, Q, 10)
    si, sd, se = oracle.search(D, s_off, s_ids, rts, Q, 10, 2000)
    assert np.array_equal(bi, si) and np.array_equal(bd, sd)
    assert (se == 2000).all()


def test_bruteforce_matches_float64(tiny):
    ps, D, rts, parents, s_off, s_ids = tiny
    Q = synth.queries(ps, 15, 3)
    bi, bd = oracle.bruteforce(D, Q, 10)
    X64 = ps.X[:, :16].astype(np.float64)
    for qi, q in enumerate(Q[:, :16].astype(np.float64)):
        d64 = ((X64 - q) ** 2).sum(1)
        order = np.lexsort((np.arange(len(d64)), d64))
        ref = order[:10]
        # identical unless two float64 distances are within the fp32 rounding bound
        tol = 30 * 2.0 ** -24 * d64[ref[-1]]
        if np.all(np.diff(np.sort(d64)[:11]) > tol):
            assert bi[qi].tolist() == ref.tolist()
        assert np.allclose(bd[qi], d64[bi[qi]], rtol=30 * 2.0 ** -24)


def test_dense_block_vs_float64():
    ps = synth.vmf_like(3000, 100, 4, seed=2)
    D = oracle.Data(ps.X, 100, 1)
    blocks = synth.intra_cluster_blocks(ps.labels, 2, 128, seed=0)
    i32, d32, _ = oracle.dense_block(D, blocks, 8)
    i64, _, d64 = oracle.dense_block(D, blocks, 8, use_f64=True)
    bound = 2 * (100 + 8) * 2.0 ** -24 * 2  # absolute, for unit vectors
    mism = 0
    for b in range(2):
        for r in range(128):
            if i32[b, r].tolist() != i64[b, r].tolist():
                mism += 1
                # a swap is only allowed between near-ties
                a = d64[b, r]
                assert np.min(np.abs(np.diff(a))) <= 2 * bound or \
                    abs(float(d32[b, r, -1]) - a[-1]) <= 2 * bound
            assert np.all(np.abs(d32[b, r].astype(np.float64) - d64[b, r]) <= 2 * bound) or \
                i32[b, r].tolist() != i64[b, r].tolist()
    assert mism <= 8


def test_dense_block_integer_data_exact():
    rng = np.random.default_rng(1)
    X = rng.integers(-4, 5, size=(300, 16)).astype(np.float32)
    D = oracle.Data(X, 16, 0)
    blocks = np.stack([np.arange(0, 100), np.arange(100, 200)]).astype(np.int32)
    blocks[1, -5:] = -1  # padding
    i32, d32, _ = oracle.dense_block(D, blocks, 12)
    i64, _, d64 = oracle.dense_block(D, blocks, 12, use_f64=True)
    assert np.array_equal(i32, i64)
    assert np.array_equal(d32.astype(np.float64), np.where(i64 >= 0, d64, np.inf))
    assert (i32[1, -5:] == -1).all()


def test_sampled_final_rows_helper_matches_oracle(tiny):
    # the one-row-at-a-time recomputation used by the full-size GPU parity
    # tests gives the oracle's final rows
    import sampled
    ps, D, rts, parents, s_off, s_ids = tiny
    R = 16
    A, cnt, ctr, per = oracle.fgraft(D, rts, s_off, s_ids, R, 32, 4, 1.2)
    off, ids, ev = oracle.final(D, A, cnt, R, 1.2, parents[0])
    users = np.random.default_rng(3).choice(2000, size=150, replace=False)
    got = sampled.final_rows(D, A, cnt, R, 1.2, parents[0], users)
    for u, row in got.items():
        assert ids[off[u]:off[u + 1]].tolist() == row
