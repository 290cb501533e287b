"""CPU oracle for the FGraft builder -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of the method of "Batched Feedback and the
Random-Access Wall in Search-Based Graph Construction" (Section 3 and
Proposition 1), written in C (``fgraft_oracle.c``) and driven from here
through ctypes with numpy arrays.  Only the tests, the smoke check and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library
never calls it, and this package imports nothing from the CUDA path.

Parity status of each function (what pins it, see ``tests/test_oracle_*``):
  splitmix64 / roots  pinned: SplitMix64's published reference outputs for
                      state 0; roots distinct and keyed.
  dist / dist_f64     pinned: exact on integer-valued inputs, within the
                      gamma_d rounding bound of the float64 value otherwise,
                      uint8 exact, symmetric.
  sat_tree / forest   pinned: Navarro's neighbour condition and closest-child
                      assignment checked by brute force, spanning tree with
                      n-1 edges, work count by its closed form.
  scaffold            pinned: edge set equals the symmetrised union of the
                      tree edges built independently in numpy.
  beam                pinned: with ef >= n on a connected graph the pool is
                      the brute-force (delta, id) order and every vertex is
                      expanded; the pool never beats brute force.
  prune_list          pinned: no kept edge is alpha-dominated, every dropped
                      candidate is dominated or R was reached, R = 1 keeps
                      the nearest, huge alpha keeps only the nearest.
  fgraft              pinned: B = 0 and B = 1 give the frozen harvest, the
                      graph is identical at 1 and N threads, S_b grows
                      monotonically, rows hold at most R ids and never p.
  final               pinned: a hand-worked fixture (an over-degree row whose
                      prune removes a candidate the tree-0 spine adds back,
                      rows of exactly R, the work count); every row contains
                      the spine and is sorted; a row with at most R
                      candidates is C(u) with the spine; an over-degree row
                      minus its spine-only vertices equals a plain-Python
                      prune of C(u) and obeys the prune invariants; the work
                      counter equals its definition.
  search              pinned: equals brute force when ef >= n.
  bruteforce          pinned: equals a float64 numpy sort up to rounding ties.
  dense_block         pinned: equals the brute-force sort of the same block.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fgraft_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

L2_F32, ANGULAR_F32, L2_U8 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Data(C.Structure):
    _fields_ = [("X", C.c_void_p), ("n", C.c_int64), ("d", C.c_int32), ("ld", C.c_int64),
                ("metric", C.c_int32)]


class _Counters(C.Structure):
    _fields_ = [("sat_evals", C.c_uint64), ("harvest_evals", C.c_uint64),
                ("prune_evals", C.c_uint64), ("final_prune_evals", C.c_uint64),
                ("expansions", C.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.fgo_dist.restype = C.c_float
            _lib.fgo_dist_vec.restype = C.c_float
            _lib.fgo_dist_f64.restype = C.c_double
            _lib.fgo_splitmix64.restype = C.c_uint64
            _lib.fgo_splitmix64.argtypes = [C.c_uint64]
            _lib.fgo_prune_list.restype = C.c_int32
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class Data:
    """Borrowed view of a point set: X is (n, ld) float32 or uint8, first d used."""

    def __init__(self, X: np.ndarray, d: int | None = None, metric: int = L2_F32):
        if metric == L2_U8:
            X = np.ascontiguousarray(X, dtype=np.uint8)
        else:
            X = np.ascontiguousarray(X, dtype=np.float32)
        self.X = X
        self.n = X.shape[0]
        self.d = X.shape[1] if d is None else d
        self.metric = metric
        self.s = _Data(_p(X), self.n, self.d, X.shape[1], metric)

    @property
    def ref(self):
        return C.byref(self.s)


def dist(D: Data, i: int, j: int) -> float:
    return float(_load().fgo_dist(D.ref, C.c_int64(i), C.c_int64(j)))


def dist_vec(D: Data, q: np.ndarray, j: int) -> float:
    q = np.ascontiguousarray(q, dtype=D.X.dtype)
    return float(_load().fgo_dist_vec(D.ref, _p(q), C.c_int64(j)))


def dist_f64(D: Data, i: int, j: int) -> float:
    return float(_load().fgo_dist_f64(D.ref, C.c_int64(i), C.c_int64(j)))


def splitmix64(z: int) -> int:
    return int(_load().fgo_splitmix64(C.c_uint64(z)))


def roots(seed: int, T: int, n: int) -> np.ndarray:
    out = np.empty(T, np.int32)
    if _load().fgo_roots(C.c_uint64(seed), C.c_int32(T), C.c_int64(n), _p(out)):
        raise ValueError("need 1 <= T <= n")
    return out


def sat_tree(D: Data, root: int):
    parent = np.empty(D.n, np.int32)
    ev = C.c_uint64(0)
    if _load().fgo_sat_tree(D.ref, C.c_int32(root), _p(parent), C.byref(ev)):
        raise MemoryError("oracle SAT allocation failed")
    return parent, int(ev.value)


def sat_forest(D: Data, T: int, seed: int):
    r = np.empty(T, np.int32)
    parents = np.empty((T, D.n), np.int32)
    ev = C.c_uint64(0)
    if _load().fgo_sat_forest(D.ref, C.c_int32(T), C.c_uint64(seed), _p(r), _p(parents),
                              C.byref(ev)):
        raise ValueError("oracle SAT forest failed")
    return r, parents, int(ev.value)


def scaffold(n: int, parents: np.ndarray):
    parents = np.ascontiguousarray(parents, np.int32)
    T = parents.shape[0]
    nnz = C.c_int64(0)
    lib = _load()
    lib.fgo_scaffold(C.c_int64(n), C.c_int32(T), _p(parents), None, None, C.byref(nnz))
    off = np.empty(n + 1, np.int64)
    ids = np.empty(max(nnz.value, 1), np.int32)
    lib.fgo_scaffold(C.c_int64(n), C.c_int32(T), _p(parents), _p(off), _p(ids), C.byref(nnz))
    return off, ids[: nnz.value]


def scaffold_cap(D: Data, off: np.ndarray, ids: np.ndarray, K: int):
    """Section 6's ablation: every scaffold row longer than K keeps its K
    nearest entries by (delta, id); rows stay sorted by id."""
    off = np.ascontiguousarray(off, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    nnz = C.c_int64(0)
    lib = _load()
    lib.fgo_scaffold_cap(D.ref, _p(off), _p(ids), C.c_int32(K), None, None, C.byref(nnz))
    o = np.empty(D.n + 1, np.int64)
    out = np.empty(max(nnz.value, 1), np.int32)
    lib.fgo_scaffold_cap(D.ref, _p(off), _p(ids), C.c_int32(K), _p(o), _p(out), C.byref(nnz))
    return o, out[: nnz.value]


def beam(D: Data, off: np.ndarray, ids: np.ndarray, rts: np.ndarray, q: np.ndarray, ef: int):
    """One beam search; returns (E_ids, E_d, pool_ids, pool_d, n_eval)."""
    off = np.ascontiguousarray(off, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    rts = np.ascontiguousarray(rts, np.int32)
    q = np.ascontiguousarray(q, dtype=D.X.dtype)
    E_ids = np.empty(D.n, np.int32)
    E_d = np.empty(D.n, np.float32)
    P_ids = np.empty(ef, np.int32)
    P_d = np.empty(ef, np.float32)
    ne, pl, nev = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _load().fgo_beam(D.ref, _p(off), _p(ids), _p(rts), C.c_int32(len(rts)), _p(q),
                     C.c_int32(ef), _p(E_ids), _p(E_d), C.byref(ne), _p(P_ids), _p(P_d),
                     C.byref(pl), C.byref(nev))
    return (E_ids[: ne.value], E_d[: ne.value], P_ids[: pl.value], P_d[: pl.value],
            int(nev.value))


def visited(D: Data, off: np.ndarray, ids: np.ndarray, rts: np.ndarray, q: np.ndarray, ef: int):
    """The visited set of one beam search (ids in visiting order)."""
    off = np.ascontiguousarray(off, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    rts = np.ascontiguousarray(rts, np.int32)
    q = np.ascontiguousarray(q, dtype=D.X.dtype)
    out = np.empty(D.n, np.int32)
    nv = C.c_int64(0)
    _load().fgo_visited(D.ref, _p(off), _p(ids), _p(rts), C.c_int32(len(rts)), _p(q),
                        C.c_int32(ef), _p(out), C.byref(nv))
    return out[: nv.value].copy()


def lockstep_density(sets):
    """Lockstep density of a group of queries searched together (Section 5.5,
    Table 6): the visited sets' summed sizes over (group size x the size of
    their union).  1 when every query visits the same vertices, 1/|group|
    when no vertex is shared."""
    union = np.unique(np.concatenate(sets)) if sets else np.empty(0, np.int32)
    total = sum(len(v) for v in sets)
    return total / (len(sets) * max(len(union), 1))


def prune_list(D: Data, p: int, cand: np.ndarray, alpha: float, R: int):
    """Occlusion prune of an explicit candidate list; returns (kept ids, evals)."""
    cand = np.ascontiguousarray(cand, np.int32)
    out = np.empty(max(R, 1), np.int32)
    ev = C.c_uint64(0)
    k = _load().fgo_prune_list(D.ref, C.c_int32(p), _p(cand), C.c_int64(len(cand)),
                               C.c_float(alpha), C.c_int32(R), _p(out), C.byref(ev))
    return out[:k].copy(), int(ev.value)


def fgraft(D: Data, rts, s_off, s_ids, R: int, ef_h: int, B: int, alpha: float,
           nthreads: int = 0):
    """Harvest all blocks.  Returns (A [n,R] -1 padded, cnt [n], counters dict,
    per-block harvest evaluations)."""
    rts = np.ascontiguousarray(rts, np.int32)
    s_off = np.ascontiguousarray(s_off, np.int64)
    s_ids = np.ascontiguousarray(s_ids, np.int32)
    A = np.empty((D.n, R), np.int32)
    cnt = np.empty(D.n, np.int32)
    ctr = _Counters()
    nb = max(B, 1)
    per = np.zeros(nb, np.uint64)
    _load().fgo_fgraft(D.ref, C.c_int32(len(rts)), _p(rts), _p(s_off), _p(s_ids), C.c_int32(R),
                       C.c_int32(ef_h), C.c_int32(B), C.c_float(alpha), C.c_int32(nthreads),
                       _p(A), _p(cnt), C.byref(ctr), _p(per))
    c = {f: int(getattr(ctr, f)) for f, _ in _Counters._fields_}
    return A, cnt, c, per


def substrate(n: int, s_off, s_ids, A, cnt, R: int, B: int, b: int):
    s_off = np.ascontiguousarray(s_off, np.int64)
    s_ids = np.ascontiguousarray(s_ids, np.int32)
    A = np.ascontiguousarray(A, np.int32)
    cnt = np.ascontiguousarray(cnt, np.int32)
    nnz = C.c_int64(0)
    lib = _load()
    args = (C.c_int64(n), _p(s_off), _p(s_ids), _p(A), _p(cnt), C.c_int32(R), C.c_int32(B),
            C.c_int32(b))
    # one call into a buffer of the largest possible size: the scaffold plus
    # both directions of every harvested row
    off = np.empty(n + 1, np.int64)
    ids = np.empty(max(len(s_ids) + 2 * int(cnt.astype(np.int64).sum()), 1), np.int32)
    lib.fgo_substrate(*args, _p(off), _p(ids), C.byref(nnz))
    return off, ids[: nnz.value]


def final(D: Data, A, cnt, R: int, alpha: float, parent0):
    A = np.ascontiguousarray(A, np.int32)
    cnt = np.ascontiguousarray(cnt, np.int32)
    parent0 = np.ascontiguousarray(parent0, np.int32)
    nnz = C.c_int64(0)
    ev = C.c_uint64(0)
    lib = _load()
    lib.fgo_final(D.ref, _p(A), _p(cnt), C.c_int32(R), C.c_float(alpha), _p(parent0), None,
                  None, C.byref(nnz), C.byref(ev))
    off = np.empty(D.n + 1, np.int64)
    ids = np.empty(max(nnz.value, 1), np.int32)
    lib.fgo_final(D.ref, _p(A), _p(cnt), C.c_int32(R), C.c_float(alpha), _p(parent0), _p(off),
                  _p(ids), C.byref(nnz), C.byref(ev))
    return off, ids[: nnz.value], int(ev.value)


def search(D: Data, off, ids, rts, Q: np.ndarray, k: int, ef_s: int, nthreads: int = 0):
    off = np.ascontiguousarray(off, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    rts = np.ascontiguousarray(rts, np.int32)
    Q = np.ascontiguousarray(Q, dtype=D.X.dtype)
    nq = Q.shape[0]
    oi = np.empty((nq, k), np.int32)
    od = np.empty((nq, k), np.float32)
    oe = np.empty(nq, np.uint32)
    _load().fgo_search(D.ref, _p(off), _p(ids), _p(rts), C.c_int32(len(rts)), _p(Q),
                       C.c_int64(nq), C.c_int64(Q.shape[1]), C.c_int32(k), C.c_int32(ef_s),
                       _p(oi), _p(od), _p(oe), C.c_int32(nthreads))
    return oi, od, oe


def bruteforce(D: Data, Q: np.ndarray, k: int, nthreads: int = 0):
    Q = np.ascontiguousarray(Q, dtype=D.X.dtype)
    nq = Q.shape[0]
    oi = np.empty((nq, k), np.int32)
    od = np.empty((nq, k), np.float32)
    _load().fgo_bruteforce(D.ref, _p(Q), C.c_int64(nq), C.c_int64(Q.shape[1]), C.c_int32(k),
                           _p(oi), _p(od), C.c_int32(nthreads))
    return oi, od


def dense_block(D: Data, block_ids: np.ndarray, k: int, use_f64: bool = False,
                nthreads: int = 0):
    """Per-row top-k over each block's pairs; returns (ids, d32, d64-or-None)."""
    block_ids = np.ascontiguousarray(block_ids, np.int32)
    nb, bs = block_ids.shape
    oi = np.empty((nb, bs, k), np.int32)
    od = np.empty((nb, bs, k), np.float32)
    o64 = np.empty((nb, bs, k), np.float64) if use_f64 else None
    _load().fgo_dense_block(D.ref, _p(block_ids), C.c_int64(nb), C.c_int32(bs), C.c_int32(k),
                            C.c_int32(1 if use_f64 else 0), _p(oi), _p(od),
                            _p(o64) if use_f64 else None, C.c_int32(nthreads))
    return oi, od, o64


def build_graph(D: Data, T: int, R: int, ef_h: int, B: int, alpha: float, seed: int,
                nthreads: int = 0, cap: int = 0):
    """The whole FGraft pipeline: SAT forest, scaffold (rows capped at `cap`
    nearest when cap > 0, Section 6), B harvest blocks, final graph."""
    rts, parents, sat_ev = sat_forest(D, T, seed)
    s_off, s_ids = scaffold(D.n, parents)
    if cap > 0:
        s_off, s_ids = scaffold_cap(D, s_off, s_ids, cap)
    A, cnt, ctr, per = fgraft(D, rts, s_off, s_ids, R, ef_h, B, alpha, nthreads)
    f_off, f_ids, fev = final(D, A, cnt, R, alpha, parents[0])
    ctr["sat_evals"] = sat_ev
    ctr["final_prune_evals"] = fev
    return dict(roots=rts, parents=parents, s_off=s_off, s_ids=s_ids, A=A, cnt=cnt,
                counters=ctr, per_block_evals=per, f_off=f_off, f_ids=f_ids)
