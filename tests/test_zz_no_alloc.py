"""The allocation-free list prune, called through the C ABI, gives the same
rows as fgraft_prune_lists on two calls in a row.

It is meant for callers that cannot allocate device memory when they prune:
serving loops that must not touch the allocator, and hosts whose own pool
allocator already owns the device memory.  Its scratch is a fixed device
array that keeps the previous call's contents, so the second call checks
that nothing carries over.  Lists above shared-memory size (more than 1024
candidates) run through that array's key buffers, up to its limit of 4096
candidates per list: a list of exactly 4096 matches the allocating prune, one
of 4097 is rejected, and the next clean call succeeds with the allocating
prune's rows.  This file is collected last so that a run stopping at its
first failure has run every other test before it.
"""
import numpy as np
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


def _lists(n, nl, seed, long_every):
    rng = np.random.default_rng(seed)
    owners = rng.integers(0, n, size=nl).astype(np.int32)
    lens = rng.integers(0, 300, size=nl)
    lens[::long_every] = rng.integers(1025, 4096, size=len(lens[::long_every]))
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    cand = rng.integers(0, n, size=int(off[-1])).astype(np.int32)
    return owners, off, cand


def test_noalloc_prune_matches_allocating_prune(fg):
    ps = synth.vmf_like(5000, 100, 8, seed=12)
    X = torch.from_numpy(ps.X).cuda()
    R = 24
    for call, (nl, seed, every) in enumerate([(700, 1, 97), (450, 2, 53)]):
        owners, off, cand = _lists(5000, nl, seed, every)
        o, f, c = (torch.from_numpy(a).cuda() for a in (owners, off, cand))
        ref_ids, ref_cnt = fg.fgraft_prune_lists(X, 100, 1, o, f, c, 1.2, R)
        got_ids, got_cnt = fg.fgraft_prune_lists_noalloc(X, 100, 1, o, f, c, 1.2, R)
        torch.cuda.synchronize()
        assert torch.equal(got_cnt, ref_cnt), f"call {call}: counts differ"
        assert torch.equal(got_ids, ref_ids), f"call {call}: rows differ"


def test_noalloc_prune_rejects_too_many_lists(fg):
    ps = synth.vmf_like(100, 100, 2, seed=1)
    X = torch.from_numpy(ps.X).cuda()
    nl = 65537
    owners = torch.zeros(nl, dtype=torch.int32, device="cuda")
    off = torch.zeros(nl + 1, dtype=torch.int64, device="cuda")
    cand = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_prune_lists_noalloc(X, 100, 1, owners, off, cand, 1.2, 8)


def test_noalloc_prune_length_limit_and_recovery(fg):
    ps = synth.vmf_like(6000, 100, 8, seed=13)
    X = torch.from_numpy(ps.X).cuda()
    R = 16
    rng = np.random.default_rng(4)

    def lists(lens):
        owners = rng.integers(0, 6000, size=len(lens)).astype(np.int32)
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        cand = rng.integers(0, 6000, size=int(off[-1])).astype(np.int32)
        return tuple(torch.from_numpy(a).cuda() for a in (owners, off, cand))

    # exactly at the limit: same rows as the allocating prune
    o, f, c = lists([4096, 7, 0, 1500, 4096, 33])
    ref = fg.fgraft_prune_lists(X, 100, 1, o, f, c, 1.2, R)
    got = fg.fgraft_prune_lists_noalloc(X, 100, 1, o, f, c, 1.2, R)
    torch.cuda.synchronize()
    assert torch.equal(got[1], ref[1]) and torch.equal(got[0], ref[0])
    # one past the limit: rejected after the call
    o, f, c = lists([12, 4097, 40])
    with pytest.raises(fg.FgraftError, match="EINVAL"):
        fg.fgraft_prune_lists_noalloc(X, 100, 1, o, f, c, 1.2, R)
    # the next clean call starts from cleared counters
    o, f, c = lists([2000, 5, 3000, 90])
    ref = fg.fgraft_prune_lists(X, 100, 1, o, f, c, 1.2, R)
    got = fg.fgraft_prune_lists_noalloc(X, 100, 1, o, f, c, 1.2, R)
    torch.cuda.synchronize()
    assert torch.equal(got[1], ref[1]) and torch.equal(got[0], ref[0])


def test_noalloc_prune_checks_output_tensors(fg):
    ps = synth.vmf_like(100, 100, 2, seed=1)
    X = torch.from_numpy(ps.X).cuda()
    owners = torch.zeros(3, dtype=torch.int32, device="cuda")
    off = torch.tensor([0, 2, 4, 6], dtype=torch.int64, device="cuda")
    cand = torch.tensor([1, 2, 3, 4, 5, 6], dtype=torch.int32, device="cuda")
    bad = [torch.empty((2, 8), dtype=torch.int32, device="cuda"),
           torch.empty((3, 8), dtype=torch.int64, device="cuda"),
           torch.empty((8, 3), dtype=torch.int32, device="cuda").t()]
    for out in bad:
        with pytest.raises(ValueError):
            fg.fgraft_prune_lists_noalloc(X, 100, 1, owners, off, cand, 1.2, 8, out=out)
