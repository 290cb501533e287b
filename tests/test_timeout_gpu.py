"""Bounded tensor-core waits give up cleanly (failure handling of the C ABI).

With the first-wait poll limit at 0 every tensor-core kernel gives up at its
first wait for MMA products: it sets its error flag, waits for the products
in flight with the full bound, frees its tensor memory and returns.  Each
call that reads a flag must return FGRAFT_ETIMEOUT: the SAT's closest-child
assignment (fgraft_build_scaffold), the harvest's occlusion prune
(fgraft_harvest_block with counters), the final graph's prune (fgraft_prune),
the dense blocks (fgraft_dense_block_dist and its Gram-only form) and the
exact k-NN filter (fgraft_knn_exact).  Nothing faults or hangs,
and with the default limit restored the same calls give results bit-equal to
those computed before.
"""
import pytest
import torch

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


def _timeout(fg, fn):
    with pytest.raises(fg.FgraftError) as e:
        fn()
        torch.cuda.synchronize()
    assert e.value.status == 5, str(e.value)


def test_tensor_core_waits_give_up_and_recover(fg):
    ps = synth.vmf_like(20_000, 100, 16, seed=3)
    X = torch.from_numpy(ps.X).cuda()
    p = fg.Params(T=4, R=32, ef_h=64, B=2, alpha=1.2, seed=0, metric=fg.ANGULAR_F32)
    blocks = torch.from_numpy(synth.intra_cluster_blocks(ps.labels, 4, 256, 2)).cuda()

    def whole_build():
        ix = fg.fgraft_build_scaffold(X, 100, p)
        fg.fgraft_harvest_all(ix, use_graph=False)
        return ix, fg.fgraft_prune(ix)

    ix_ref, (off_ref, ids_ref) = whole_build()
    c_ref = fg.fgraft_index_counters(ix_ref)
    dense_ref = [fg.fgraft_dense_block_dist(X, 100, fg.ANGULAR_F32, blocks, 16, precision=pr)
                 for pr in (1, 2)]
    knn_ref = fg.fgraft_knn_exact(X, 100, fg.ANGULAR_F32, 10, 0, 3000)
    ix_h = fg.fgraft_build_scaffold(X, 100, p)          # for the harvest's prune
    ix_f = fg.fgraft_build_scaffold(X, 100, p)          # for the final graph's prune
    for b in range(2):
        fg.fgraft_harvest_block(ix_f, b)
    torch.cuda.synchronize()
    try:
        fg.fgraft_tune_mma_wait(0)
        for pr in (1, 2):
            _timeout(fg, lambda: fg.fgraft_dense_block_dist(X, 100, fg.ANGULAR_F32, blocks, 16,
                                                            precision=pr))
        _timeout(fg, lambda: fg.fgraft_build_scaffold(X, 100, p))
        _timeout(fg, lambda: fg.fgraft_harvest_block(ix_h, 0, counters=True))
        _timeout(fg, lambda: fg.fgraft_prune(ix_f))
        _timeout(fg, lambda: fg.fgraft_knn_exact(X, 100, fg.ANGULAR_F32, 10, 0, 3000))
        _timeout(fg, lambda: fg.fgraft_dense_block_gram(X, 100, fg.ANGULAR_F32, blocks,
                                                        precision=1))
    finally:
        fg.fgraft_tune_mma_wait(-1)
    # the context is intact and the next normal calls are bit-exact
    ix2, (off2, ids2) = whole_build()
    assert torch.equal(off2, off_ref) and torch.equal(ids2, ids_ref)
    assert fg.fgraft_index_counters(ix2) == c_ref
    for pr, (ri, rd) in zip((1, 2), dense_ref):
        gi, gd = fg.fgraft_dense_block_dist(X, 100, fg.ANGULAR_F32, blocks, 16, precision=pr)
        assert torch.equal(gi, ri) and torch.equal(gd, rd)
    ki, kd = fg.fgraft_knn_exact(X, 100, fg.ANGULAR_F32, 10, 0, 3000)
    assert torch.equal(ki, knn_ref[0]) and torch.equal(kd, knn_ref[1])
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_tune_mma_wait(-2)
