"""Visited-set log of the harvest searches (Section 5.5, Table 6) through the
C ABI, against the oracle's visited sets on the same substrates S_b: the
same sets, sizes and insertion of the roots first, in every visited-set
layout, for points of the block about to be harvested and for others; the
sizes of a block's sets sum to its harvest evaluations; the log changes
nothing of the build."""
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


@pytest.fixture(scope="module")
def case():
    ps = synth.gaussian_mixture(3000, 16, 8, seed=2)
    T, R, ef, B = 4, 16, 32, 4
    D = oracle.Data(ps.X, ps.d, ps.metric)
    ref = oracle.build_graph(D, T, R, ef, B, 1.2, 0)
    subs = [oracle.substrate(ps.n, ref["s_off"], ref["s_ids"], ref["A"], ref["cnt"], R, B, b)
            for b in range(B + 1)]
    return ps, (T, R, ef, B), D, ref, subs


# (hash_log2, overflow_mode): the occupancy rule's layout, a 128-slot hash
# that moves into the global bitmap, and one whose searches re-run on
# global scratch
@pytest.mark.parametrize("layout", [(0, 0), (7, 1), (7, 2)])
def test_visited_log_matches_oracle(fg, case, layout):
    ps, (T, R, ef, B), D, ref, subs = case
    n = ps.n
    X = torch.from_numpy(ps.X).cuda()
    ix = fg.fgraft_build_scaffold(X, ps.d, fg.Params(T=T, R=R, ef_h=ef, B=B, alpha=1.2,
                                                     seed=0, metric=ps.metric))
    if layout != (0, 0):
        fg.fgraft_index_tune(ix, hash_log2=layout[0], overflow_mode=layout[1])
    rng = np.random.default_rng(1)
    for b in range(B + 1):
        blk = np.arange(b, n, B) if b < B else np.zeros(0, np.int64)
        other = rng.choice(np.setdiff1d(np.arange(n), blk), 25, replace=False)
        pts = np.concatenate([blk, other, [-1, n]]).astype(np.int32)
        ev0 = fg.fgraft_index_counters(ix)["harvest_evals"]
        ids_t, cnt_t = fg.fgraft_harvest_visited(ix, torch.from_numpy(pts).cuda(), 2048)
        short_t, cshort_t = fg.fgraft_harvest_visited(ix, torch.from_numpy(pts).cuda(), 7)
        assert fg.fgraft_index_counters(ix)["harvest_evals"] == ev0
        ids, cnt = ids_t.cpu().numpy(), cnt_t.cpu().numpy()
        assert cnt[-2] == -1 and cnt[-1] == -1
        assert np.array_equal(cshort_t.cpu().numpy(), cnt)
        assert np.array_equal(short_t.cpu().numpy()[:-2], ids[:-2, :7])
        off, sids = subs[b]
        for i, q in enumerate(pts[:-2]):
            v = oracle.visited(D, off, sids, ref["roots"], ps.X[q], ef)
            assert 0 < cnt[i] <= 2048
            assert cnt[i] == len(v), (b, q)
            assert np.array_equal(np.sort(ids[i, :cnt[i]]), np.sort(v)), (b, q)
            assert np.array_equal(ids[i, :T], ref["roots"])
        if b < B:
            fg.fgraft_harvest_block(ix, b)
            ev1 = fg.fgraft_index_counters(ix)["harvest_evals"]
            assert ev1 - ev0 == int(cnt[:len(blk)].sum())
    st = fg.fgraft_index_copy(ix)
    assert np.array_equal(st["rows"].cpu().numpy(), ref["A"])
    assert np.array_equal(st["counts"].cpu().numpy(), ref["cnt"])


def test_visited_log_rejects(fg, case):
    ps, (T, R, ef, B), D, ref, subs = case
    X = torch.from_numpy(ps.X).cuda()
    ix = fg.fgraft_build_scaffold(X, ps.d, fg.Params(T=T, R=R, ef_h=ef, B=B, alpha=1.2,
                                                     seed=0, metric=ps.metric))
    pts = torch.arange(4, dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FgraftError):
        fg.fgraft_harvest_visited(ix, pts, 0)
    ids, cnt = fg.fgraft_harvest_visited(ix, pts[:0], 5)
    assert ids.shape == (0, 5) and cnt.shape == (0,)
