"""Parity in the launch configuration of the paper-scale workload.

n = 400,000 unit vectors, d = 100 (160 MB, more than the L2 cache), angular,
T = 8, B = 8, R = 64, ef_h = 100, alpha = 1.2: the searches of every block are
claimed in tree-0 preorder, and the visited sets start in the small
shared-memory hash chosen for occupancy and continue in global bitmaps.  The
oracle recomputes, one at a time, sampled harvested rows, each from its own
S_b, rebuilt from the scaffold and the rows of earlier blocks, sampled
final-graph rows from the harvested rows, and 200 sampled query searches over
the final graph.
"""
import numpy as np
import pytest
import torch

import oracle
import sampled
from paper_2609_30493_gb300 import synth

pytestmark = pytest.mark.gpu

N, D, T, B, R, EF, ALPHA = 400_000, 100, 8, 8, 64, 100, 1.2


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30493_gb300 import build, fgraft as fg
    build.build()
    ps = synth.vmf_like(N, D, 256, seed=3, kappa=20.0, sizes="zipf")
    X = torch.from_numpy(ps.X).cuda()
    ix = fg.fgraft_build_scaffold(X, D, fg.Params(T=T, R=R, ef_h=EF, B=B, alpha=ALPHA,
                                                  seed=0, metric=fg.ANGULAR_F32))
    coherent = fg.fgraft_index_schedule(ix) is not None
    ctr = fg.fgraft_harvest_all(ix, use_graph=True, counters=True)
    st = {k: v.cpu().numpy() for k, v in fg.fgraft_index_copy(ix).items()}
    f_off, f_ids = fg.fgraft_prune(ix)
    Q = synth.queries(ps, 2_000, 4)
    qi, qd, qe = fg.fgraft_search(ix, torch.from_numpy(Q).cuda(), 10, 64)
    return dict(ps=ps, D=oracle.Data(ps.X, D, oracle.ANGULAR_F32), st=st, ctr=ctr,
                coherent=coherent, f_off=f_off.cpu().numpy(), f_ids=f_ids.cpu().numpy(), Q=Q,
                qi=qi.cpu().numpy(), qd=qd.cpu().numpy(), qe=qe.cpu().numpy())


def test_runs_in_the_large_configuration(built):
    assert built["coherent"]


def test_sampled_rows_per_block(built):
    st, D, ps = built["st"], built["D"], built["ps"]
    rng = np.random.default_rng(7)
    for b in range(B):
        off, ids = oracle.substrate(N, st["s_off"], st["s_ids"], st["rows"], st["counts"], R, B, b)
        pts = b + B * rng.choice((N - b + B - 1) // B, size=6, replace=False)
        for p in pts:
            E, Ed, P, Pd, nev = oracle.beam(D, off, ids, st["roots"], ps.X[p], EF)
            kept, _ = oracle.prune_list(D, int(p), E, ALPHA, R)
            assert st["counts"][p] == len(kept), (b, p)
            assert st["rows"][p, :len(kept)].tolist() == kept.tolist(), (b, p)
            assert (st["rows"][p, len(kept):] == -1).all()


def test_sampled_final_rows(built):
    st, D_ = built["st"], built["D"]
    users = np.random.default_rng(9).choice(N, size=100, replace=False)
    want = sampled.final_rows(D_, st["rows"], st["counts"], R, ALPHA, st["parents"][0], users)
    for u, row in want.items():
        assert built["f_ids"][built["f_off"][u]:built["f_off"][u + 1]].tolist() == row, u


def test_sampled_search(built):
    Q = built["Q"]
    sel = np.random.default_rng(10).choice(len(Q), size=200, replace=False)
    oi, od, oe = oracle.search(built["D"], built["f_off"], built["f_ids"], built["st"]["roots"],
                               Q[sel], 10, 64)
    assert np.array_equal(built["qi"][sel], oi)
    assert np.array_equal(built["qd"][sel], od)
    assert np.array_equal(built["qe"][sel].astype(np.uint32), oe)
