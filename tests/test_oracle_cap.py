"""Pins for the scaffold degree cap (Section 6, the ablation the paper reports
as negative): a row longer than K keeps its K nearest entries by
(delta, id).  Checked against float64 distances computed here with numpy
(outside rounding ties at the K-th place), as a subset of the uncapped row,
sorted by id; a cap at or above the largest degree changes nothing."""
import numpy as np

import oracle
from paper_2609_30493_gb300 import synth


def _fixture():
    ps = synth.gaussian_mixture(3000, 24, 6, seed=21)
    D = oracle.Data(ps.X, 24, 0)
    rts, parents, _ = oracle.sat_forest(D, 6, seed=2)
    off, ids = oracle.scaffold(3000, parents)
    return ps, D, off, ids


def test_cap_keeps_nearest():
    ps, D, off, ids = _fixture()
    X64 = ps.X[:, :24].astype(np.float64)
    K = 5
    co, ci = oracle.scaffold_cap(D, off, ids, K)
    capped = 0
    for u in range(D.n):
        row = ids[off[u]:off[u + 1]]
        new = ci[co[u]:co[u + 1]]
        assert len(new) == min(len(row), K)
        assert np.all(np.diff(new) > 0) and set(new.tolist()) <= set(row.tolist())
        if len(row) <= K:
            assert new.tolist() == row.tolist()
            continue
        capped += 1
        d64 = ((X64[row] - X64[u]) ** 2).sum(1)
        kth = np.sort(d64)[K - 1]
        tol = 64 * 2.0 ** -24 * max(kth, 1e-30)
        assert all(d64[row.tolist().index(v)] <= kth + tol for v in new.tolist())
        assert set(row[d64 < kth - tol].tolist()) <= set(new.tolist())
    assert capped > 100


def test_cap_above_max_degree_is_identity():
    ps, D, off, ids = _fixture()
    K = int(np.diff(off).max())
    co, ci = oracle.scaffold_cap(D, off, ids, K)
    assert np.array_equal(co, off) and np.array_equal(ci, ids)
