"""Parity in the launch configuration of the paper-scale workload.

n = 400,000 unit vectors, d = 100 (160 MB, more than the L2 cache), angular,
T = 8, B = 8, R = 64, ef_h = 100, alpha = 1.2: the searches of every block are
claimed in tree-0 preorder, and the visited sets start in the small
shared-memory hash chosen for occupancy and continue in global bitmaps.  The
oracle recomputes, one point at a time, sampled harvested rows, each from
its own S_b, rebuilt from the scaffold and the rows of earlier blocks.
"""
import numpy as np
import pytest
import torch

import oracle
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
    return dict(ps=ps, D=oracle.Data(ps.X, D, oracle.ANGULAR_F32), st=st, ctr=ctr,
                coherent=coherent)


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
