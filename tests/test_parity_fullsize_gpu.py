"""Parity at the benchmark's full size, in its launch configuration.

Workload: n = 100,000 unit vectors, d = 100, angular, 64 clusters; T = 8,
B = 8, R = 32, ef_h = 64, alpha = 1.2; the blocks run as one CUDA graph, as
bench.py times them.  The oracle recomputes the whole SAT forest, the
scaffold and the final graph, and, one point at a time, sampled harvested
rows (each from its own S_b, rebuilt from the scaffold and the rows of
earlier blocks only) and sampled query searches.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle_cache
from paper_2609_30493_gb300 import synth

pytestmark = pytest.mark.gpu

N, D, T, B, R, EF, ALPHA = 100_000, 100, 8, 8, 32, 64, 1.2


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30493_gb300 import build, fgraft as fg
    build.build()
    ps = synth.vmf_like(N, D, 64, seed=0, kappa=20.0)
    X = torch.from_numpy(ps.X).cuda()
    ix = fg.fgraft_build_scaffold(X, D, fg.Params(T=T, R=R, ef_h=EF, B=B, alpha=ALPHA,
                                                  seed=0, metric=fg.ANGULAR_F32))
    ctr = fg.fgraft_harvest_all(ix, use_graph=True, counters=True)
    off, ids = fg.fgraft_prune(ix)
    st = {k: v.cpu().numpy() for k, v in fg.fgraft_index_copy(ix).items()}
    Q = synth.queries(ps, 10_000, 1)
    qi, qd, qe = fg.fgraft_search(ix, torch.from_numpy(Q).cuda(), 10, 64)
    D_ = oracle.Data(ps.X, D, oracle.ANGULAR_F32)
    return dict(ps=ps, D=D_, st=st, ctr=ctr, f_off=off.cpu().numpy(), f_ids=ids.cpu().numpy(),
                Q=Q, qi=qi.cpu().numpy(), qd=qd.cpu().numpy(), qe=qe.cpu().numpy())


def test_forest_and_scaffold_full(built):
    st, D = built["st"], built["D"]
    rts, parents, sev = oracle.sat_forest(D, T, seed=0)
    assert np.array_equal(st["roots"], rts)
    assert np.array_equal(st["parents"], parents)
    assert built["ctr"]["sat_evals"] == sev
    s_off, s_ids = oracle.scaffold(N, parents)
    assert np.array_equal(st["s_off"], s_off)
    assert np.array_equal(st["s_ids"], s_ids)


def test_sampled_rows_per_block(built):
    st, D, ps = built["st"], built["D"], built["ps"]
    rng = np.random.default_rng(5)
    for b in range(B):
        off, ids = oracle.substrate(N, st["s_off"], st["s_ids"], st["rows"], st["counts"], R, B, b)
        pts = b + B * rng.choice((N - b + B - 1) // B, size=12, replace=False)
        for p in pts:
            E, Ed, P, Pd, nev = oracle.beam(D, off, ids, st["roots"], ps.X[p], EF)
            kept, _ = oracle.prune_list(D, int(p), E, ALPHA, R)
            assert st["counts"][p] == len(kept), (b, p)
            assert st["rows"][p, :len(kept)].tolist() == kept.tolist(), (b, p)
            assert (st["rows"][p, len(kept):] == -1).all()


def test_final_graph_full(built):
    st, D = built["st"], built["D"]
    f_off, f_ids, fev = oracle.final(D, st["rows"], st["counts"], R, ALPHA, st["parents"][0])
    assert np.array_equal(built["f_off"], f_off)
    assert np.array_equal(built["f_ids"], f_ids)
    assert built["ctr"]["final_prune_evals"] == fev


def test_sampled_search(built):
    D, Q = built["D"], built["Q"]
    sel = np.random.default_rng(8).choice(len(Q), size=200, replace=False)
    oi, od, oe = oracle.search(D, built["f_off"], built["f_ids"], built["st"]["roots"], Q[sel],
                               10, 64)
    assert np.array_equal(built["qi"][sel], oi)
    assert np.array_equal(built["qd"][sel], od)
    assert np.array_equal(built["qe"][sel].astype(np.uint32), oe)


def test_whole_build_equals_oracle(built):
    st, D, ps, ctr = built["st"], built["D"], built["ps"], built["ctr"]
    g = oracle_cache.build_graph(D, ps.X, T, R, EF, B, ALPHA, seed=0)
    assert np.array_equal(st["roots"], g["roots"])
    assert np.array_equal(st["counts"], g["cnt"])
    assert np.array_equal(st["rows"], g["A"])
    for k in ("sat_evals", "harvest_evals", "prune_evals", "final_prune_evals", "expansions"):
        assert ctr[k] == g["counters"][k], k
    assert np.array_equal(built["f_off"], g["f_off"])
    assert np.array_equal(built["f_ids"], g["f_ids"])
