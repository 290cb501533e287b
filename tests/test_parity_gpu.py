"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

Integer and index results (tree parents, scaffold, harvested rows, final
graph, search ids, dense-block ids) must match bit for bit, float distances
must match bit for bit too (both sides use the same fixed float32 order),
and the algorithmic counters must be equal.
"""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _np(t):
    return t.cpu().numpy()


def _build_both(fg, ps, T, R, ef, B, alpha=1.2, seed=0, use_graph=False, hash_log2=0,
                overflow_mode=0, cap=0):
    X = _dev(ps.X)
    p = fg.Params(T=T, R=R, ef_h=ef, B=B, alpha=alpha, seed=seed, metric=ps.metric)
    ix, c0 = fg.fgraft_build_scaffold(X, ps.d, p, counters=True)
    if hash_log2 or overflow_mode:
        fg.fgraft_index_tune(ix, hash_log2=hash_log2, overflow_mode=overflow_mode)
    ctr = fg.fgraft_harvest_all(ix, use_graph=use_graph, counters=True)
    off, ids = fg.fgraft_prune(ix)
    st = fg.fgraft_index_copy(ix)
    D = oracle.Data(ps.X, ps.d, ps.metric)
    ref = oracle.build_graph(D, T, R, ef, B, alpha, seed, cap=cap)
    return ix, ctr, st, (off, ids), D, ref


def _compare(ctr, st, fin, ref, check_final=True):
    assert np.array_equal(_np(st["roots"]), ref["roots"])
    assert np.array_equal(_np(st["parents"]), ref["parents"])
    assert np.array_equal(_np(st["s_off"]), ref["s_off"])
    assert np.array_equal(_np(st["s_ids"]), ref["s_ids"])
    cnt = _np(st["counts"])
    rows = _np(st["rows"])
    bad = np.flatnonzero((cnt != ref["cnt"]) | (rows != ref["A"]).any(1))
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:5]}"
    rc = ref["counters"]
    for k in ("sat_evals", "harvest_evals", "prune_evals", "expansions"):
        assert ctr[k] == rc[k], (k, ctr[k], rc[k])
    if check_final:
        off, ids = fin
        assert np.array_equal(_np(off), ref["f_off"])
        assert np.array_equal(_np(ids), ref["f_ids"])
        assert ctr["final_prune_evals"] == rc["final_prune_evals"]


@pytest.mark.parametrize("B", [1, 4])
def test_tiny_gauss_parity(fg, B):
    ps = synth.gaussian_mixture(2000, 16, 8, seed=0)
    ix, ctr, st, fin, D, ref = _build_both(fg, ps, T=4, R=16, ef=32, B=B)
    _compare(ctr, st, fin, ref)
    # the final graph is computed once per index; a later call copies it out
    off2, ids2 = fg.fgraft_prune(ix)
    assert torch.equal(off2, fin[0]) and torch.equal(ids2, fin[1])
    assert fg.fgraft_index_counters(ix)["final_prune_evals"] == ref["counters"]["final_prune_evals"]
    Q = synth.queries(ps, 200, 1)
    for ef_s in (10, 32, 64):
        gi, gd, ge = fg.fgraft_search(ix, _dev(Q), 10, ef_s)
        oi, od, oe = oracle.search(D, ref["f_off"], ref["f_ids"], ref["roots"], Q, 10, ef_s)
        assert np.array_equal(_np(gi), oi)
        assert np.array_equal(_np(gd), od)
        assert np.array_equal(_np(ge).astype(np.uint32), oe)


def test_graph_capture_same_graph(fg):
    ps = synth.gaussian_mixture(2000, 16, 8, seed=0)
    ix, ctr, st, fin, D, ref = _build_both(fg, ps, T=4, R=16, ef=32, B=4, use_graph=True)
    _compare(ctr, st, fin, ref)


@pytest.mark.parametrize("case", [
    dict(kind="vmf", n=3000, d=100, k=16, T=8, R=32, ef=64, B=8),
    dict(kind="gauss", n=1500, d=960, k=8, T=4, R=16, ef=32, B=2),
    dict(kind="u8", n=2500, d=128, k=8, T=8, R=32, ef=64, B=8),
    dict(kind="gauss", n=1200, d=3, k=4, T=3, R=8, ef=16, B=3),
    dict(kind="gauss", n=1300, d=129, k=4, T=4, R=12, ef=40, B=2),
    dict(kind="vmf", n=1700, d=300, k=8, T=5, R=24, ef=100, B=5),
    dict(kind="u8", n=900, d=20, k=4, T=2, R=10, ef=20, B=3),
])
def test_shapes_parity(fg, case):
    if case["kind"] == "vmf":
        ps = synth.vmf_like(case["n"], case["d"], case["k"], seed=3)
    elif case["kind"] == "u8":
        ps = synth.uint8_mixture(case["n"], case["d"], case["k"], seed=3)
    else:
        ps = synth.gaussian_mixture(case["n"], case["d"], case["k"], seed=3)
    ix, ctr, st, fin, D, ref = _build_both(fg, ps, case["T"], case["R"], case["ef"], case["B"])
    _compare(ctr, st, fin, ref)


@pytest.mark.parametrize("case", [
    dict(kind="vmf", n=3000, d=100, k=16, T=8, R=32, ef=64, B=8),
    dict(kind="gauss", n=1300, d=129, k=4, T=4, R=12, ef=40, B=2),
    dict(kind="gauss", n=1200, d=3, k=4, T=3, R=8, ef=16, B=3),
])
def test_prune_lane_groups_parity(fg, case):
    # the prune with every dominance test on the lane groups (no tensor-core
    # Gram) gives the same graphs
    try:
        fg.fgraft_tune_prune(False)
        if case["kind"] == "vmf":
            ps = synth.vmf_like(case["n"], case["d"], case["k"], seed=4)
        else:
            ps = synth.gaussian_mixture(case["n"], case["d"], case["k"], seed=4)
        ix, ctr, st, fin, D, ref = _build_both(fg, ps, case["T"], case["R"], case["ef"],
                                               case["B"])
        _compare(ctr, st, fin, ref)
    finally:
        fg.fgraft_tune_prune(True)


def test_prune_tune_rejects(fg):
    with pytest.raises(fg.FgraftError):
        fg._check(fg.load().fgraft_tune_prune(2))


@pytest.mark.parametrize("mode", [1, 2])
def test_overflow_is_exact(fg, mode):
    # a 128-slot visited set overflows for most queries; moving to the global
    # bitmap (mode 1) or re-running on global scratch (mode 2) must give the
    # same graph and counters
    ps = synth.gaussian_mixture(2000, 16, 8, seed=0)
    ix, ctr, st, fin, D, ref = _build_both(fg, ps, T=4, R=16, ef=32, B=4, hash_log2=7,
                                           overflow_mode=mode)
    if mode == 2:
        assert ctr["reruns"] > 0
    else:
        assert ctr["reruns"] == 0
    _compare(ctr, st, fin, ref)
    Q = synth.queries(ps, 100, 1)
    gi, gd, ge = fg.fgraft_search(ix, _dev(Q), 10, 32)
    oi, od, oe = oracle.search(D, ref["f_off"], ref["f_ids"], ref["roots"], Q, 10, 32)
    assert np.array_equal(_np(gi), oi) and np.array_equal(_np(gd), od)


def test_edge_cases(fg):
    # few points, duplicates (ties everywhere), R = 1, ef = 1, T = n
    rng = np.random.default_rng(0)
    base = rng.integers(0, 3, size=(40, 4)).astype(np.float32)
    X = np.concatenate([base, base[:20], base[:5]])
    ps = synth.PointSet(X, 4, 0, np.zeros(len(X), np.int32), np.zeros((1, 4)),
                        dict(kind="gauss", sigma=1.0))
    for T, R, ef, B in [(3, 1, 1, 2), (4, 8, 16, 3), (2, 4, 128, 1)]:
        ix, ctr, st, fin, D, ref = _build_both(fg, ps, T, R, ef, B)
        _compare(ctr, st, fin, ref)
    tiny = synth.gaussian_mixture(5, 8, 1, seed=1)
    ix, ctr, st, fin, D, ref = _build_both(fg, tiny, T=5, R=3, ef=4, B=2)
    _compare(ctr, st, fin, ref)


def test_prune_lists_parity(fg):
    ps = synth.vmf_like(3000, 100, 8, seed=4)
    D = oracle.Data(ps.X, 100, 1)
    rng = np.random.default_rng(2)
    nl, R = 300, 16
    owners = rng.integers(0, 3000, size=nl).astype(np.int32)
    lens = rng.integers(0, 200, size=nl)
    # 1500: a long list sorted and pruned in shared memory; 5000: one too
    # long for it, in global scratch
    lens[:4] = [0, 1, 1500, 5000]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    cand = rng.integers(0, 3000, size=int(off[-1])).astype(np.int32)
    cand[off[5]] = owners[5]  # the owner itself appears in a list
    out, cnt = fg.fgraft_prune_lists(_dev(ps.X), 100, 1, _dev(owners), _dev(off), _dev(cand),
                                     1.2, R)
    out, cnt = _np(out), _np(cnt)
    for i in range(nl):
        kept, _ = oracle.prune_list(D, int(owners[i]), cand[off[i]:off[i + 1]], 1.2, R)
        assert cnt[i] == len(kept)
        assert out[i, :cnt[i]].tolist() == kept.tolist()
        assert (out[i, cnt[i]:] == -1).all()


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("metric,d,k", [(1, 100, 32), (0, 960, 64), (0, 16, 10), (1, 300, 20)])
def test_dense_block_parity(fg, metric, d, k, precision):
    ps = synth.vmf_like(4000, d, 4, seed=5) if metric == 1 else \
        synth.gaussian_mixture(4000, d, 4, seed=5)
    blocks = synth.intra_cluster_blocks(ps.labels, 3, 1000, seed=1)
    blocks[2, -7:] = -1
    gi, gd, st = fg.fgraft_dense_block_dist(_dev(ps.X), d, metric, _dev(blocks), k,
                                            precision=precision, stats=True,
                                            err64=precision >= 1)
    D = oracle.Data(ps.X, d, metric)
    oi, od, _ = oracle.dense_block(D, blocks, k)
    assert np.array_equal(_np(gi), oi)
    assert np.array_equal(_np(gd), od)
    if precision >= 1:
        assert 0.0 < st[0] <= 1.0 and st[1] > 0.0
        # the filter's error stays inside its bound on every recomputed pair
        assert 0.0 < st[4] <= 1.0
        assert st[5] >= 0.0


def test_dense_block_uint8_parity(fg):
    ps = synth.uint8_mixture(3000, 128, 4, seed=5)
    blocks = synth.intra_cluster_blocks(ps.labels, 3, 700, seed=2)
    blocks[1, -9:] = -1
    gi, gd = fg.fgraft_dense_block_dist(_dev(ps.X), 128, fg.L2_U8, _dev(blocks), 32)
    oi, od, _ = oracle.dense_block(oracle.Data(ps.X, 128, fg.L2_U8), blocks, 32)
    assert np.array_equal(_np(gi), oi) and np.array_equal(_np(gd), od)
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_dense_block_dist(_dev(ps.X), 128, fg.L2_U8, _dev(blocks), 32, precision=1)


def test_api_rejects_bad_arguments(fg):
    ps = synth.gaussian_mixture(100, 16, 2, seed=0)
    X = _dev(ps.X)
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_build_scaffold(X, 16, fg.Params(T=0, R=8, ef_h=8, B=1, alpha=1.2))
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_build_scaffold(X, 16, fg.Params(T=2, R=8, ef_h=200, B=1, alpha=1.2))
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_build_scaffold(X, 17, fg.Params(T=2, R=8, ef_h=8, B=1, alpha=-1.0))
    ix = fg.fgraft_build_scaffold(X, 16, fg.Params(T=2, R=8, ef_h=8, B=3, alpha=1.2))
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_harvest_block(ix, 2)  # out of order
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_prune(ix)  # blocks missing
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_search(ix, X[:4], 10, 16)  # no final graph yet


@pytest.mark.parametrize("use_graph", [False, True])
def test_profile_hooks(fg, use_graph):
    ps = synth.gaussian_mixture(2000, 16, 8, seed=0)
    X = _dev(ps.X)
    ix = fg.fgraft_build_scaffold(X, 16, fg.Params(T=4, R=16, ef_h=32, B=4, alpha=1.2))
    fg.fgraft_index_profile(ix, True)
    before = fg.fgraft_kernel_launches()
    fg.fgraft_harvest_all(ix, use_graph=use_graph)
    ms, nl = fg.fgraft_index_harvest_ms(ix)
    assert nl == 4 and ms > 0.0
    assert fg.fgraft_kernel_launches() - before > 4


@pytest.mark.parametrize("split,finish", [(2, 1), (64, 16), (700, 2048), (300, 100)])
def test_sat_multi_cta_nodes(fg, split, finish):
    # force the multi-CTA SAT path for small nodes too, with tiled selection
    # steps down to lists of `finish` points; the forest must not change
    try:
        fg.fgraft_tune_sat(split, finish)
        ps = synth.vmf_like(2500, 100, 8, seed=6)
        ix, ctr, st, fin, D, ref = _build_both(fg, ps, T=6, R=16, ef=32, B=2)
        _compare(ctr, st, fin, ref)
    finally:
        fg.fgraft_tune_sat(16384, 512)


def test_n20000_parity(fg):
    # the top tree nodes (19,999 points) take the default multi-CTA path
    ps = synth.vmf_like(20000, 100, 32, seed=9)
    ix, ctr, st, fin, D, ref = _build_both(fg, ps, T=8, R=32, ef=64, B=8)
    _compare(ctr, st, fin, ref)


def test_harvest_block_multi_equals_single(fg):
    # three independent builds harvested block by block together give the
    # rows and final graphs of their separate builds
    sets = [(synth.gaussian_mixture(1500, 16, 4, seed=11), 16, fg.L2_F32),
            (synth.vmf_like(1800, 100, 6, seed=12), 100, fg.ANGULAR_F32),
            (synth.gaussian_mixture(900, 33, 3, seed=13), 33, fg.L2_F32)]
    p = dict(T=4, R=16, ef_h=32, B=4, alpha=1.2)
    multi, single = [], []
    for ps, d, metric in sets:
        X = _dev(ps.X)
        multi.append(fg.fgraft_build_scaffold(X, d, fg.Params(metric=metric, **p)))
        single.append(fg.fgraft_build_scaffold(X, d, fg.Params(metric=metric, **p)))
    for b in range(4):
        fg.fgraft_harvest_block_multi(multi, b)
    for ix in single:
        for b in range(4):
            fg.fgraft_harvest_block(ix, b)
    for im, is_ in zip(multi, single):
        cm, cs = fg.fgraft_index_copy(im), fg.fgraft_index_copy(is_)
        assert torch.equal(cm["rows"], cs["rows"]) and torch.equal(cm["counts"], cs["counts"])
        om, os_ = fg.fgraft_prune(im), fg.fgraft_prune(is_)
        assert torch.equal(om[0], os_[0]) and torch.equal(om[1], os_[1])
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_harvest_block_multi(multi, 0)  # already past block 0


def test_many_builds_share_one_launch(fg):
    # five angular builds of different sizes share one search launch per
    # block, two uint8 builds another; rows, counters and final graphs equal
    # their separate builds, and one of them equals the oracle
    sets = [(synth.vmf_like(n, 100, 6, seed=30 + i), 100, fg.ANGULAR_F32)
            for i, n in enumerate((1500, 4000, 700, 2500, 3000))]
    sets += [(synth.uint8_mixture(n, 20, 4, seed=40 + i), 20, fg.L2_U8)
             for i, n in enumerate((1200, 2600))]
    p = dict(T=4, R=24, ef_h=64, B=3, alpha=1.2)
    multi, single = [], []
    for ps, d, metric in sets:
        X = _dev(ps.X)
        multi.append(fg.fgraft_build_scaffold(X, d, fg.Params(metric=metric, **p)))
        single.append(fg.fgraft_build_scaffold(X, d, fg.Params(metric=metric, **p)))
    for b in range(3):
        fg.fgraft_harvest_block_multi(multi, b)
    for ix in single:
        for b in range(3):
            fg.fgraft_harvest_block(ix, b)
    for im, is_ in zip(multi, single):
        cm, cs = fg.fgraft_index_copy(im), fg.fgraft_index_copy(is_)
        assert torch.equal(cm["rows"], cs["rows"]) and torch.equal(cm["counts"], cs["counts"])
        om, os_ = fg.fgraft_prune(im), fg.fgraft_prune(is_)
        assert torch.equal(om[0], os_[0]) and torch.equal(om[1], os_[1])
        ctm, cts = fg.fgraft_index_counters(im), fg.fgraft_index_counters(is_)
        for k in ("harvest_evals", "prune_evals", "expansions", "final_prune_evals"):
            assert ctm[k] == cts[k], k
    ps, d, metric = sets[1]
    ref = oracle.build_graph(oracle.Data(ps.X, d, metric), 4, 24, 64, 3, 1.2, 0)
    om = fg.fgraft_prune(multi[1])
    assert np.array_equal(_np(om[0]), ref["f_off"]) and np.array_equal(_np(om[1]), ref["f_ids"])


@pytest.mark.parametrize("kind,cap", [("gauss", 3), ("vmf", 6), ("u8", 5)])
def test_scaffold_cap_parity(fg, kind, cap):
    # Section 6's ablation: scaffold rows capped at their cap nearest entries
    if kind == "gauss":
        ps = synth.gaussian_mixture(2000, 16, 8, seed=7)
    elif kind == "vmf":
        ps = synth.vmf_like(2500, 100, 8, seed=7)
    else:
        ps = synth.uint8_mixture(1500, 32, 6, seed=7)
    try:
        fg.fgraft_tune_scaffold_cap(cap)
        ix, ctr, st, fin, D, ref = _build_both(fg, ps, T=6, R=16, ef=32, B=4, cap=cap)
    finally:
        fg.fgraft_tune_scaffold_cap(0)
    assert int(np.diff(_np(st["s_off"])).max()) <= cap
    _compare(ctr, st, fin, ref)


def _check_preorder(parent, pre):
    # pre is a preorder of the tree: a permutation in which every subtree
    # occupies one contiguous range that starts at its root
    n = parent.size
    assert np.array_equal(np.sort(pre), np.arange(n))
    kids = [[] for _ in range(n)]
    roots = []
    for v, u in enumerate(parent.tolist()):
        (roots if u < 0 else kids[u]).append(v)
    order, k = list(roots), 0
    while k < len(order):
        order.extend(kids[order[k]])
        k += 1
    assert len(order) == n
    size = np.ones(n, dtype=np.int64)
    for v in reversed(order):
        if parent[v] >= 0:
            size[parent[v]] += size[v]
    u = parent[parent >= 0]
    v = np.flatnonzero(parent >= 0)
    assert (pre[u] < pre[v]).all()
    assert (pre[v] + size[v] <= pre[u] + size[u]).all()


@pytest.mark.parametrize("B", [1, 8, 64])
def test_coherent_schedule_is_tree0_preorder(fg, B):
    # the harvest claims each block's searches in a preorder of tree 0
    ps = synth.vmf_like(20000, 100, 32, seed=21)
    X = _dev(ps.X)
    try:
        fg.fgraft_tune_schedule(1)
        ix = fg.fgraft_build_scaffold(X, 100, fg.Params(T=4, R=16, ef_h=32, B=B, alpha=1.2,
                                                        metric=fg.ANGULAR_F32))
    finally:
        fg.fgraft_tune_schedule(2)
    sched = fg.fgraft_index_schedule(ix)
    assert sched is not None
    pre, qorder = _np(sched[0]), _np(sched[1])
    n = ps.X.shape[0]
    parent0 = _np(fg.fgraft_index_copy(ix)["parents"]).reshape(-1)[:n]
    _check_preorder(parent0, pre)
    start = 0
    for b in range(B):
        pts = np.arange(b, n, B)
        want = (pts[np.argsort(pre[pts], kind="stable")] - b) // B
        assert np.array_equal(qorder[start:start + pts.size], want), b
        start += pts.size
    assert start == n


def test_coherent_schedule_same_graph(fg):
    # the schedule moves work, never results: id order and tree-0 preorder
    # give the same rows, counters and final graph
    ps = synth.vmf_like(20000, 100, 32, seed=22)
    X = _dev(ps.X)
    out = []
    try:
        for coherent in (False, True):
            fg.fgraft_tune_schedule(coherent)
            p = fg.Params(T=8, R=32, ef_h=64, B=8, alpha=1.2, metric=fg.ANGULAR_F32)
            ix = fg.fgraft_build_scaffold(X, 100, p)
            assert (fg.fgraft_index_schedule(ix) is not None) == coherent
            ctr = fg.fgraft_harvest_all(ix, use_graph=True, counters=True)
            st = fg.fgraft_index_copy(ix)
            out.append((ctr, st["rows"], st["counts"], *fg.fgraft_prune(ix)))
    finally:
        fg.fgraft_tune_schedule(2)
    a, b = out
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        assert torch.equal(x, y)


def test_many_blocks_fall_back_to_id_order(fg):
    # more than 64 blocks: searches in id order, same parity with the oracle
    ps = synth.gaussian_mixture(1500, 16, 4, seed=23)
    try:
        fg.fgraft_tune_schedule(1)
        ix, ctr, st, fin, D, ref = _build_both(fg, ps, T=4, R=16, ef=32, B=100)
    finally:
        fg.fgraft_tune_schedule(2)
    assert fg.fgraft_index_schedule(ix) is None
    _compare(ctr, st, fin, ref)
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_tune_schedule(3)


def test_schedule_auto_by_size(fg):
    # the default picks the preorder only for vectors larger than the L2 cache
    ps = synth.gaussian_mixture(3000, 16, 4, seed=24)
    ix = fg.fgraft_build_scaffold(_dev(ps.X), 16, fg.Params(T=4, R=16, ef_h=32, B=4,
                                                            alpha=1.2, metric=fg.L2_F32))
    assert fg.fgraft_index_schedule(ix) is None


def test_auto_visited_layout_same_graph(fg):
    # at n = 200,000 the automatic layout takes a hash smaller than 2^12
    # slots (more searches in flight, more of them continuing in the global
    # bitmap); the rows and counters equal those of the explicit 2^12 hash
    ps = synth.vmf_like(200_000, 100, 64, seed=25)
    X = _dev(ps.X)
    out = []
    for hl2 in (0, 12):
        p = fg.Params(T=8, R=32, ef_h=64, B=4, alpha=1.2, metric=fg.ANGULAR_F32)
        ix = fg.fgraft_build_scaffold(X, 100, p)
        if hl2:
            fg.fgraft_index_tune(ix, hash_log2=hl2)
        ctr = fg.fgraft_harvest_all(ix, use_graph=True, counters=True)
        st = fg.fgraft_index_copy(ix)
        out.append((ctr, st["rows"], st["counts"], *fg.fgraft_prune(ix)))
        del ix
    a, b = out
    for k in ("harvest_evals", "prune_evals", "expansions", "final_prune_evals"):
        assert a[0][k] == b[0][k], k
    for x, y in zip(a[1:], b[1:]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("precision", [1, 2])
def test_dense_block_edge_cases(fg, precision):
    # blocks of fewer than k + 1 members (every column is a candidate), a
    # single-member block, a block of repeated points (ties everywhere: the
    # filter cannot separate them, so every column is reranked), and more
    # blocks than one launch group holds
    ps = synth.vmf_like(6000, 100, 8, seed=9)
    X = ps.X.copy()
    X[100:400] = X[100]  # 300 copies of one point
    lab = ps.labels
    blocks = synth.intra_cluster_blocks(lab, 70, 64, seed=3)
    blocks[0, 20:] = -1           # 20 members, k = 32
    blocks[1, 1:] = -1            # one member
    blocks[2, :] = np.arange(100, 164)  # all identical
    blocks[3, :40] = np.arange(100, 140)  # 40 copies + 24 others
    gi, gd = fg.fgraft_dense_block_dist(_dev(X), 100, 1, _dev(blocks), 32, precision=precision)
    oi, od, _ = oracle.dense_block(oracle.Data(X, 100, 1), blocks, 32)
    assert np.array_equal(_np(gi), oi)
    assert np.array_equal(_np(gd), od)


def _emulated_min(X, blocks, d, fp8):
    """Smallest approximate angular distance per row, with the rounding the
    Gram kernel applies (float32 block mean: eight partial sums over the rows
    r = w, w + 8, .. of the block, added in order; centred rows rounded to
    BF16, or to E4M3 after scaling the row's largest magnitude to 448), the
    products and sums in float64."""
    nb, bs = blocks.shape
    out = np.full((nb, bs), np.inf)
    for b in range(nb):
        ids = blocks[b]
        valid = ids >= 0
        rows = X[ids[valid], :d].astype(np.float32)
        parts = []
        for w in range(8):
            s = np.zeros(d, np.float32)
            for r in range(w, bs, 8):
                if ids[r] >= 0:
                    s = (s + X[ids[r], :d].astype(np.float32)).astype(np.float32)
            parts.append(s)
        s = parts[0]
        for w in range(1, 8):
            s = (s + parts[w]).astype(np.float32)
        mu = (s * np.float32(np.float32(1.0) / np.float32(len(rows)))).astype(np.float32)
        c = torch.from_numpy((rows - mu).astype(np.float32))
        if fp8:
            mx = c.abs().max(dim=1).values
            scale = torch.where(mx > 0, mx / 448.0, torch.ones_like(mx))
            q = (c * (1.0 / scale)[:, None]).to(torch.float8_e4m3fn).double() * scale.double()[:, None]
        else:
            q = c.to(torch.bfloat16).double()
        x2 = (rows.astype(np.float64) ** 2).sum(1)
        n = (c.double() ** 2).sum(1).numpy()
        g = (q @ q.T).numpy()
        dist = 0.5 * (n[:, None] + n[None, :] - 2 * g) + 0.5 * (1 - x2)[:, None] + 0.5 * (1 - x2)[None, :]
        np.fill_diagonal(dist, np.inf)
        out[b, np.nonzero(valid)[0]] = dist.min(1)
    return out


@pytest.mark.parametrize("precision", [1, 2])
def test_dense_gram_only_matches_emulation(fg, precision):
    ps = synth.vmf_like(5000, 100, 4, seed=11)
    blocks = synth.intra_cluster_blocks(ps.labels, 4, 1024, seed=4)
    blocks[3, -100:] = -1
    got, ms = fg.fgraft_dense_block_gram(_dev(ps.X), 100, 1, _dev(blocks), precision=precision)
    want = _emulated_min(ps.X, blocks, 100, precision == 2)
    got = _np(got).astype(np.float64)
    fin = np.isfinite(want)
    assert np.array_equal(np.isfinite(got), fin)
    assert np.max(np.abs(got[fin] - want[fin])) < 2e-4
    assert ms > 0.0


def test_autotune_settings_give_the_same_graph(fg):
    # the autotuner's candidate settings (warps per CTA, visited-set layout,
    # overflow handling) never change the graph, and the tuned index builds
    # the oracle's graph
    ps = synth.vmf_like(30_000, 100, 16, seed=6)
    X = _dev(ps.X)
    p = fg.Params(T=4, R=32, ef_h=64, B=4, alpha=1.2, seed=0, metric=1)
    graphs = []
    for wpc, hl, ov, ga, ib in [(4, 0, 1, 0, 2), (1, 9, 1, 1, 1), (2, 10, 2, 1, 2),
                                (4, 12, 1, 0, 1), (2, 0, 2, 1, 2), (4, 0, 1, 1, 2)]:
        ix = fg.fgraft_build_scaffold(X, 100, p)
        fg.fgraft_index_set_tuning(ix, warps_per_cta=wpc, hash_log2=hl, overflow_mode=ov,
                                   gather=ga, id_batch=ib)
        fg.fgraft_harvest_all(ix, use_graph=False)
        off, ids = fg.fgraft_prune(ix)
        graphs.append((_np(off), _np(ids)))
    for g in graphs[1:]:
        assert np.array_equal(g[0], graphs[0][0]) and np.array_equal(g[1], graphs[0][1])
    ix = fg.fgraft_build_scaffold(X, 100, p)
    t = fg.fgraft_index_autotune(ix, sample=2000)
    assert t["warps_per_cta"] in (1, 2, 4) and t["overflow_mode"] in (1, 2)
    assert t["gather"] in (0, 1) and t["id_batch"] in (1, 2)
    assert t["us_per_query"] > 0 and t["default_us_per_query"] > 0
    fg.fgraft_harvest_all(ix, use_graph=True)
    off, ids = fg.fgraft_prune(ix)
    assert np.array_equal(_np(off), graphs[0][0]) and np.array_equal(_np(ids), graphs[0][1])
    ref = oracle.build_graph(oracle.Data(ps.X, 100, 1), 4, 32, 64, 4, 1.2, 0)
    assert np.array_equal(_np(off), ref["f_off"]) and np.array_equal(_np(ids), ref["f_ids"])
    # a later index of the same shape starts from the tuned settings
    ix2 = fg.fgraft_build_scaffold(X, 100, p)
    fg.fgraft_harvest_all(ix2, use_graph=False)
    o2, i2 = fg.fgraft_prune(ix2)
    assert np.array_equal(_np(o2), graphs[0][0]) and np.array_equal(_np(i2), graphs[0][1])
    # calibrating on a later block (2 of 4 harvested) writes block 2's rows
    # early, with the values its own harvest gives them: the graph is the same
    ix3 = fg.fgraft_build_scaffold(X, 100, p)
    for b in range(2):
        fg.fgraft_harvest_block(ix3, b)
    t3 = fg.fgraft_index_autotune(ix3, sample=2000)
    assert t3["us_per_query"] > 0
    for b in range(2, 4):
        fg.fgraft_harvest_block(ix3, b)
    o3, i3 = fg.fgraft_prune(ix3)
    assert np.array_equal(_np(o3), ref["f_off"]) and np.array_equal(_np(i3), ref["f_ids"])
    st3 = fg.fgraft_index_copy(ix3)
    assert np.array_equal(_np(st3["rows"]), ref["A"]) and np.array_equal(_np(st3["counts"]), ref["cnt"])


def test_wide_lists_use_both_prune_tiles(fg):
    # ef_h = 100 gives list buffers of 256 entries and R = 64 final rows of
    # more than 128 candidates: the harvest and the final graph take the
    # 128- and 256-candidate tensor-core tiles; the whole graph and every
    # counter equal the oracle's
    ps = synth.vmf_like(12_000, 100, 8, seed=14)
    A, cnt, off, ids, ctr, _ = _build_both_simple(fg, ps, T=4, R=64, ef=100, B=2)
    ref = oracle.build_graph(oracle.Data(ps.X, 100, 1), 4, 64, 100, 2, 1.2, 0)
    assert np.array_equal(A, ref["A"]) and np.array_equal(cnt, ref["cnt"])
    assert np.array_equal(off, ref["f_off"]) and np.array_equal(ids, ref["f_ids"])
    for k in ("harvest_evals", "prune_evals", "final_prune_evals", "expansions", "sat_evals"):
        assert ctr[k] == ref["counters"][k], k
    # the final graph did prune rows past one 128-candidate tile
    indeg = np.bincount(ref["A"][ref["A"] >= 0], minlength=12_000)
    assert ((ref["cnt"] + indeg) > 128).sum() > 100


def _build_both_simple(fg, ps, T, R, ef, B):
    X = _dev(ps.X)
    ix = fg.fgraft_build_scaffold(X, ps.d, fg.Params(T=T, R=R, ef_h=ef, B=B, alpha=1.2, seed=0,
                                                     metric=ps.metric))
    ctr = fg.fgraft_harvest_all(ix, use_graph=True, counters=True)
    off, ids = fg.fgraft_prune(ix)
    st = fg.fgraft_index_copy(ix)
    return _np(st["rows"]), _np(st["counts"]), _np(off), _np(ids), ctr, ix
