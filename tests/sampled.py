"""Oracle recomputation of sampled outputs of a large build, one at a time.

final_rows: the final-graph rows of a few points (Section 3: C(u) = A[u] U
{p : u in A[p]}; pruned to R when longer; the tree-0 parent and children
added; sorted by (delta, id)), from given harvested rows, with the oracle's
distance and list prune.
"""
import numpy as np

import oracle


def final_rows(D, A, cnt, R, alpha, parent0, users):
    users = [int(u) for u in users]
    valid = np.arange(A.shape[1])[None, :] < cnt[:, None]
    hit_p, hit_c = np.nonzero(np.isin(A, users) & valid)
    rev = {u: set() for u in users}
    for p, c in zip(hit_p.tolist(), hit_c.tolist()):
        rev[int(A[p, c])].add(p)
    out = {}
    for u in users:
        C = set(A[u, :cnt[u]].tolist()) | rev[u]
        if len(C) > R:
            kept = oracle.prune_list(D, u, np.array(sorted(C), np.int32), alpha, R)[0].tolist()
        else:
            kept = sorted(C)
        spine = set(np.nonzero(parent0 == u)[0].tolist())
        if parent0[u] >= 0:
            spine.add(int(parent0[u]))
        row = set(kept) | spine
        out[u] = sorted(row, key=lambda v: (oracle.dist(D, u, v), v))
    return out
