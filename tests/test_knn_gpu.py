"""Exact k nearest neighbours of the points themselves through the C ABI
(fgraft_knn_exact: the brute force of Section 2 restricted to the points,
which local completeness needs for every point), bit for bit against the
oracle's brute force with the point itself removed: ids, float32 distances
and the order of ties by id, on both float metrics, several lane shapes,
ragged row ranges, duplicate points, fewer points than k, and rows that
collect too many columns and scan every point."""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_30493_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30493_gb300 import build, fgraft
    build.build()
    fgraft.load()
    return fgraft


def _ref(X, d, metric, rows, k):
    D = oracle.Data(X, d, metric)
    oi, od = oracle.bruteforce(D, X[rows], k + 1)
    ids = np.full((len(rows), k), -1, np.int32)
    ds = np.full((len(rows), k), np.inf, np.float32)
    for r, p in enumerate(rows):
        keep = oi[r] != p
        ii, dd = oi[r][keep][:k], od[r][keep][:k]
        ids[r, :len(ii)] = ii
        ds[r, :len(dd)] = dd
    return ids, ds


def _check(fg, X, d, metric, k, row0=0, nrows=None):
    n = X.shape[0]
    nrows = n - row0 if nrows is None else nrows
    gi, gd, st = fg.fgraft_knn_exact(torch.from_numpy(X).cuda(), d, metric, k, row0, nrows,
                                     stats=True)
    ri, rd = _ref(X, d, metric, np.arange(row0, row0 + nrows), k)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    bad = np.flatnonzero((gi != ri).any(1) | (gd != rd).any(1))
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:4] + row0}"
    return st


@pytest.mark.parametrize("case", [("gauss", 3000, 16, 10), ("vmf", 4000, 100, 10),
                                  ("gauss", 700, 40, 1), ("gauss", 700, 40, 32),
                                  ("vmf", 1500, 300, 16), ("vmf", 1200, 960, 10)])
def test_knn_exact_matches_bruteforce(fg, case):
    kind, n, d, k = case
    ps = (synth.gaussian_mixture(n, d, 8, seed=3) if kind == "gauss"
          else synth.vmf_like(n, d, 8, seed=3, kappa=20.0))
    st = _check(fg, ps.X, d, ps.metric, k)
    assert st["rerank_evals"] >= n * min(k, n - 1)


def test_knn_exact_row_ranges(fg):
    ps = synth.vmf_like(5000, 100, 16, seed=4, kappa=20.0)
    for row0, nrows in ((37, 1000), (0, 1), (4999, 1), (128, 256), (4000, 1000)):
        _check(fg, ps.X, 100, ps.metric, 10, row0, nrows)


def test_knn_exact_duplicates_and_tiny(fg):
    ps = synth.gaussian_mixture(1500, 24, 8, seed=5)
    X = np.ascontiguousarray(np.concatenate([ps.X, ps.X[:300], ps.X[100:150]]))
    _check(fg, X, 24, ps.metric, 10)  # ties at distance 0, ordered by id
    small = synth.gaussian_mixture(5, 8, 2, seed=6)
    gi, gd = fg.fgraft_knn_exact(torch.from_numpy(small.X).cuda(), 8, small.metric, 10)
    assert (gi[:, 4:].cpu().numpy() == -1).all() and np.isinf(gd[:, 4:].cpu().numpy()).all()
    _check(fg, small.X, 8, small.metric, 10)


def test_knn_exact_full_scan_rows(fg):
    # 600 copies of one vector plus a few others: every copy has 599 columns
    # at distance 0, more than a row's list holds, so it scans every point
    ps = synth.gaussian_mixture(40, 16, 2, seed=7)
    X = np.ascontiguousarray(np.concatenate([np.repeat(ps.X[:1], 600, axis=0), ps.X[1:]]))
    st = _check(fg, X, 16, ps.metric, 10)
    assert st["full_scan_rows"] >= 600


def test_knn_exact_rejects(fg):
    ps = synth.gaussian_mixture(100, 8, 2, seed=8)
    X = torch.from_numpy(ps.X).cuda()
    for kw in (dict(k=0), dict(k=33), dict(k=5, row0=90, nrows=20), dict(k=5, row0=-1, nrows=5)):
        with pytest.raises(fg.FgraftError):
            fg.fgraft_knn_exact(X, 8, ps.metric, **kw)
    u8 = synth.uint8_mixture(100, 16, 2, seed=9)
    with pytest.raises(fg.FgraftError):
        fg.fgraft_knn_exact(torch.from_numpy(u8.X).cuda(), 16, u8.metric, 5)
    gi, gd = fg.fgraft_knn_exact(X, 8, ps.metric, 5, 10, 0)
    assert gi.shape == (0, 5)
