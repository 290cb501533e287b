"""Python binding of libfgraft (ctypes).  Argument marshalling only: every step
runs in the CUDA library, and a missing library raises instead of falling
back to anything else.

Names mirror the C ABI of include/fgraft.h.  Tensors are torch CUDA tensors;
work is enqueued on torch's current stream of the tensors' device.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

from . import build as _build

L2_F32, ANGULAR_F32, L2_U8 = 0, 1, 2
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EOVERFLOW", 5: "ETIMEOUT"}


class FgraftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Params(C.Structure):
    _fields_ = [("T", C.c_int32), ("R", C.c_int32), ("ef_h", C.c_int32), ("B", C.c_int32),
                ("alpha", C.c_float), ("seed", C.c_uint64), ("metric", C.c_int32)]


class _Counters(C.Structure):
    _fields_ = [("sat_evals", C.c_uint64), ("harvest_evals", C.c_uint64),
                ("prune_evals", C.c_uint64), ("final_prune_evals", C.c_uint64),
                ("expansions", C.c_uint64), ("ids_scanned", C.c_uint64), ("reruns", C.c_uint64)]


_lib = None

EXPORTS = ["fgraft_build_scaffold", "fgraft_harvest_block", "fgraft_harvest_all", "fgraft_prune",
           "fgraft_prune_lists", "fgraft_search", "fgraft_dense_block_dist", "fgraft_index_copy",
           "fgraft_index_sizes", "fgraft_index_counters", "fgraft_index_tune",
           "fgraft_index_profile", "fgraft_index_harvest_ms", "fgraft_kernel_launches",
           "fgraft_tune_sat", "fgraft_tune_prune", "fgraft_prune_lists_noalloc",
           "fgraft_harvest_block_multi", "fgraft_tune_scaffold_cap", "fgraft_tune_schedule",
           "fgraft_index_schedule", "fgraft_tune_mma_wait", "fgraft_dense_block_gram",
           "fgraft_index_autotune", "fgraft_tuning_table_save", "fgraft_tuning_table_load",
           "fgraft_index_set_tuning", "fgraft_harvest_visited", "fgraft_knn_exact",
           "fgraft_index_destroy", "fgraft_last_error"]


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libfgraft.so (built by paper_2609_30493_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: run paper_2609_30493_gb300.build.build()")
        lib = C.CDLL(_build.LIB)
        lib.fgraft_last_error.restype = C.c_char_p
        lib.fgraft_index_destroy.restype = None
        lib.fgraft_kernel_launches.restype = C.c_uint64
        for name in EXPORTS:
            if name not in ("fgraft_last_error", "fgraft_index_destroy", "fgraft_kernel_launches"):
                getattr(lib, name).restype = C.c_int
        _lib = lib
    return _lib


def _check(status: int):
    if status != 0:
        raise FgraftError(status, load().fgraft_last_error().decode())


def _stream(dev=None):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _elem(metric: int):
    return torch.uint8 if metric == L2_U8 else torch.float32


@dataclass
class Params:
    T: int
    R: int
    ef_h: int
    B: int
    alpha: float
    seed: int = 0
    metric: int = L2_F32

    def c(self) -> _Params:
        return _Params(self.T, self.R, self.ef_h, self.B, self.alpha, self.seed, self.metric)


class Index:
    """Owns an fgraft_index*; X (borrowed by the library) is kept alive here."""

    def __init__(self, handle, X, d, params: Params):
        self.handle = handle
        self.X = X
        self.d = d
        self.params = params

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.fgraft_index_destroy(h)

    def sizes(self):
        n, nnz, fnnz = C.c_int64(), C.c_int64(), C.c_int64()
        T, R, bd = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().fgraft_index_sizes(self.handle, C.byref(n), C.byref(T), C.byref(R),
                                         C.byref(nnz), C.byref(fnnz), C.byref(bd)))
        return dict(n=n.value, T=T.value, R=R.value, scaffold_nnz=nnz.value,
                    final_nnz=fnnz.value, blocks_done=bd.value)


def _counters_dict(c: _Counters) -> dict:
    return {f: int(getattr(c, f)) for f, _ in _Counters._fields_}


def fgraft_build_scaffold(X: torch.Tensor, d: int, params: Params, counters: bool = False):
    """X: (n, ld) CUDA tensor (float32 or uint8), row stride a multiple of 16 bytes."""
    assert X.is_cuda and X.dim() == 2 and X.is_contiguous()
    assert X.dtype == _elem(params.metric)
    h = C.c_void_p()
    ctr = _Counters()
    p = params.c()
    _check(load().fgraft_build_scaffold(_ptr(X), C.c_int64(X.shape[0]), C.c_int32(d),
                                        C.c_int64(X.shape[1]), C.byref(p), _stream(X.device),
                                        C.byref(h), C.byref(ctr) if counters else None))
    ix = Index(h, X, d, params)
    return (ix, _counters_dict(ctr)) if counters else ix


def fgraft_harvest_block(ix: Index, b: int, counters: bool = False):
    ctr = _Counters()
    _check(load().fgraft_harvest_block(ix.handle, C.c_int32(b), _stream(ix.X.device),
                                       C.byref(ctr) if counters else None))
    return _counters_dict(ctr) if counters else None


def fgraft_harvest_all(ix: Index, use_graph: bool = True, counters: bool = False):
    ctr = _Counters()
    _check(load().fgraft_harvest_all(ix.handle, C.c_int32(1 if use_graph else 0),
                                     _stream(ix.X.device), C.byref(ctr) if counters else None))
    return _counters_dict(ctr) if counters else None


def fgraft_harvest_block_multi(ixs, b: int):
    """Block b of every index in ixs: one persistent search launch per group of
    indices that share a kernel shape, then the per-index prunes."""
    arr = (C.c_void_p * max(len(ixs), 1))(*[ix.handle for ix in ixs])
    dev = ixs[0].X.device if ixs else None
    _check(load().fgraft_harvest_block_multi(arr, C.c_int32(len(ixs)), C.c_int32(b),
                                             _stream(dev)))


def fgraft_prune(ix: Index, counters: bool = False):
    """Final graph; returns (offsets int64 [n+1], ids int32) CUDA tensors.  A row holds at
    most R + (tree-0 degree) ids, so n*R + 2(n-1) bounds the total."""
    n = ix.X.shape[0]
    cap = n * ix.params.R + 2 * (n - 1)
    off = torch.empty(n + 1, dtype=torch.int64, device=ix.X.device)
    ids = torch.empty(max(cap, 1), dtype=torch.int32, device=ix.X.device)
    need = C.c_int64()
    ctr = _Counters()
    _check(load().fgraft_prune(ix.handle, _stream(ix.X.device),
                               C.byref(ctr) if counters else None, _ptr(off), _ptr(ids),
                               C.c_int64(cap), C.byref(need)))
    out = (off, ids[: need.value])
    return (*out, _counters_dict(ctr)) if counters else out


def fgraft_index_counters(ix: Index) -> dict:
    ctr = _Counters()
    _check(load().fgraft_index_counters(ix.handle, _stream(ix.X.device), C.byref(ctr)))
    return _counters_dict(ctr)


def fgraft_index_tune(ix: Index, hash_log2: int = 0, warps_per_cta: int = 0,
                      overflow_mode: int = 0):
    _check(load().fgraft_index_tune(ix.handle, C.c_int32(hash_log2), C.c_int32(warps_per_cta),
                                    C.c_int32(overflow_mode)))


def fgraft_index_profile(ix: Index, enable: bool = True):
    _check(load().fgraft_index_profile(ix.handle, C.c_int32(1 if enable else 0)))


def fgraft_index_harvest_ms(ix: Index, with_prune: bool = False):
    """(sum of harvest-kernel milliseconds, number of harvest launches) since profiling
    began; with_prune adds the summed milliseconds of the re-run and prune kernels."""
    ms, nl, pm = C.c_double(), C.c_int32(), C.c_double()
    _check(load().fgraft_index_harvest_ms(ix.handle, _stream(ix.X.device), C.byref(ms),
                                          C.byref(nl), C.byref(pm)))
    return (ms.value, nl.value, pm.value) if with_prune else (ms.value, nl.value)


def fgraft_tune_prune(tensor_cores: bool = True):
    _check(load().fgraft_tune_prune(C.c_int32(1 if tensor_cores else 0)))


class _Tuning(C.Structure):
    _fields_ = [("warps_per_cta", C.c_int32), ("hash_log2", C.c_int32),
                ("overflow_mode", C.c_int32), ("gather", C.c_int32), ("id_batch", C.c_int32),
                ("us_per_query", C.c_float), ("default_us_per_query", C.c_float)]


def fgraft_index_autotune(ix: Index, sample: int = 16384) -> dict:
    """Time the harvest launch configurations on a calibration sample of block
    0 and keep the fastest for this index (and its shape in the process
    table).  Returns the chosen settings and the timings."""
    t = _Tuning()
    _check(load().fgraft_index_autotune(ix.handle, C.c_int32(sample), _stream(ix.X.device),
                                        C.byref(t)))
    return {f: getattr(t, f) for f, _ in _Tuning._fields_}


def fgraft_index_set_tuning(ix: Index, warps_per_cta: int = 4, hash_log2: int = 0,
                            overflow_mode: int = 1, gather: int = 0, id_batch: int = 2):
    """Explicit harvest launch settings (results do not depend on them)."""
    t = _Tuning(warps_per_cta, hash_log2, overflow_mode, gather, id_batch, 0.0, 0.0)
    _check(load().fgraft_index_set_tuning(ix.handle, C.byref(t)))


def fgraft_tuning_table_save(path: str):
    _check(load().fgraft_tuning_table_save(C.c_char_p(os.fsencode(path))))


def fgraft_tuning_table_load(path: str):
    _check(load().fgraft_tuning_table_load(C.c_char_p(os.fsencode(path))))


def fgraft_tune_mma_wait(polls: int = -1):
    """Polls of a tensor-core kernel's first wait for its MMA products before it
    gives up (0: at once, which tests the FGRAFT_ETIMEOUT path; -1: default)."""
    _check(load().fgraft_tune_mma_wait(C.c_int32(polls)))


def fgraft_tune_scaffold_cap(cap: int = 0):
    _check(load().fgraft_tune_scaffold_cap(C.c_int32(cap)))


def fgraft_tune_schedule(coherent=2):
    """0 / False: id order; 1 / True: tree-0 preorder; 2: preorder when X exceeds L2."""
    _check(load().fgraft_tune_schedule(C.c_int32(int(coherent))))


def fgraft_index_schedule(ix: Index):
    """(pre, qorder) int32 CUDA tensors of the coherent harvest schedule, or None when
    the index runs its searches in id order."""
    n = ix.X.shape[0]
    pre = torch.empty(n, dtype=torch.int32, device=ix.X.device)
    qorder = torch.empty(n, dtype=torch.int32, device=ix.X.device)
    coh = C.c_int32()
    _check(load().fgraft_index_schedule(ix.handle, _ptr(pre), _ptr(qorder), C.byref(coh),
                                        _stream(ix.X.device)))
    return (pre, qorder) if coh.value else None


def fgraft_tune_sat(big_node_min: int = 0, finish_len: int = 0):
    _check(load().fgraft_tune_sat(C.c_int32(big_node_min), C.c_int32(finish_len)))


def fgraft_kernel_launches() -> int:
    return int(load().fgraft_kernel_launches())


def fgraft_index_copy(ix: Index):
    """Returns dict of CUDA tensors: roots, parents [T,n], s_off, s_ids, rows [n,R], counts."""
    s = ix.sizes()
    n, T, R = s["n"], s["T"], s["R"]
    dev = ix.X.device
    out = dict(roots=torch.empty(T, dtype=torch.int32, device=dev),
               parents=torch.empty((T, n), dtype=torch.int32, device=dev),
               s_off=torch.empty(n + 1, dtype=torch.int64, device=dev),
               s_ids=torch.empty(max(s["scaffold_nnz"], 1), dtype=torch.int32, device=dev),
               rows=torch.empty((n, R), dtype=torch.int32, device=dev),
               counts=torch.empty(n, dtype=torch.int32, device=dev))
    _check(load().fgraft_index_copy(ix.handle, _ptr(out["roots"]), _ptr(out["parents"]),
                                    _ptr(out["s_off"]), _ptr(out["s_ids"]), _ptr(out["rows"]),
                                    _ptr(out["counts"]), _stream(dev)))
    out["s_ids"] = out["s_ids"][: s["scaffold_nnz"]]
    return out


def fgraft_knn_exact(X: torch.Tensor, d: int, metric: int, k: int, row0: int = 0,
                     nrows: int = None, stats: bool = False):
    """Exact k nearest neighbours of points row0 .. row0 + nrows - 1 among all
    rows of X (self excluded), by the canonical float32 distance with ties by
    id.  Returns (ids (nrows, k) int32, dist (nrows, k) float32[, stats])."""
    n = X.shape[0]
    if nrows is None:
        nrows = n - row0
    ids = torch.empty((nrows, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((nrows, k), dtype=torch.float32, device=X.device)
    st = (C.c_double * 4)()
    _check(load().fgraft_knn_exact(_ptr(X), C.c_int64(n), C.c_int32(d), C.c_int64(X.shape[1]),
                                   C.c_int32(metric), C.c_int64(row0), C.c_int64(nrows),
                                   C.c_int32(k), _ptr(ids), _ptr(dist),
                                   st if stats else None, _stream(X.device)))
    if stats:
        return ids, dist, {"rerank_evals": st[0], "full_scan_rows": st[1],
                           "filter_ms": st[2], "rerank_ms": st[3]}
    return ids, dist


def fgraft_harvest_visited(ix: Index, points: torch.Tensor, cap: int):
    """Visited sets of the next block's harvest searches for the given points:
    returns (ids (np, cap) int32, cnt (np,) int32); row i holds the first
    min(cnt[i], cap) vertices point i's search evaluates, cnt[i] = |V_i|
    (-1 for an id outside [0, n))."""
    assert points.is_cuda and points.dtype == torch.int32 and points.dim() == 1
    points = points.contiguous()
    np_ = points.shape[0]
    ids = torch.empty((np_, cap), dtype=torch.int32, device=ix.X.device)
    cnt = torch.empty(np_, dtype=torch.int32, device=ix.X.device)
    _check(load().fgraft_harvest_visited(ix.handle, _ptr(points), C.c_int64(np_),
                                         C.c_int32(cap), _ptr(ids), _ptr(cnt),
                                         _stream(ix.X.device)))
    return ids, cnt


def fgraft_search(ix: Index, Q: torch.Tensor, k: int, ef_s: int):
    """Q: (nq, ldq) CUDA tensor of the index's element type.  Returns (ids, dist, evals)."""
    assert Q.is_cuda and Q.dim() == 2 and Q.is_contiguous() and Q.dtype == ix.X.dtype
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device=Q.device)
    dist = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
    ev = torch.empty(nq, dtype=torch.int32, device=Q.device)
    _check(load().fgraft_search(ix.handle, _ptr(Q), C.c_int64(nq), C.c_int64(Q.shape[1]),
                                C.c_int32(k), C.c_int32(ef_s), _ptr(ids), _ptr(dist), _ptr(ev),
                                _stream(Q.device)))
    return ids, dist, ev


def fgraft_prune_lists(X: torch.Tensor, d: int, metric: int, owner: torch.Tensor,
                       cand_off: torch.Tensor, cand_ids: torch.Tensor, alpha: float, R: int):
    nl = owner.shape[0]
    out = torch.empty((nl, R), dtype=torch.int32, device=X.device)
    cnt = torch.empty(nl, dtype=torch.int32, device=X.device)
    _check(load().fgraft_prune_lists(_ptr(X), C.c_int64(X.shape[0]), C.c_int32(d),
                                     C.c_int64(X.shape[1]), C.c_int32(metric), _ptr(owner),
                                     _ptr(cand_off), _ptr(cand_ids), C.c_int64(nl),
                                     C.c_float(alpha), C.c_int32(R), _ptr(out), _ptr(cnt),
                                     _stream(X.device)))
    return out, cnt


def fgraft_prune_lists_noalloc(X: torch.Tensor, d: int, metric: int, owner: torch.Tensor,
                               cand_off: torch.Tensor, cand_ids: torch.Tensor, alpha: float, R: int,
                               out: torch.Tensor = None, cnt: torch.Tensor = None):
    """fgraft_prune_lists without any device allocation inside the library; the
    output tensors may be passed in (preallocated by the caller).  The kernel
    writes nlists * R ids and nlists counts through plain pointers, so passed
    tensors must be contiguous int32 on X's device with exactly those shapes."""
    nl = owner.shape[0]
    if out is None:
        out = torch.empty((nl, R), dtype=torch.int32, device=X.device)
    if cnt is None:
        cnt = torch.empty(nl, dtype=torch.int32, device=X.device)
    for name, t, shape in (("out", out, (nl, R)), ("cnt", cnt, (nl,))):
        if (tuple(t.shape) != shape or t.dtype != torch.int32 or not t.is_contiguous()
                or t.device != X.device):
            raise ValueError(f"{name} must be a contiguous int32 tensor of shape {shape} "
                             f"on {X.device}")
    _check(load().fgraft_prune_lists_noalloc(_ptr(X), C.c_int64(X.shape[0]), C.c_int32(d),
                                             C.c_int64(X.shape[1]), C.c_int32(metric),
                                             _ptr(owner), _ptr(cand_off), _ptr(cand_ids),
                                             C.c_int64(nl), C.c_float(alpha), C.c_int32(R),
                                             _ptr(out), _ptr(cnt), _stream(X.device)))
    return out, cnt


def fgraft_dense_block_dist(X: torch.Tensor, d: int, metric: int, block_ids: torch.Tensor, k: int,
                            precision: int = 0, stats: bool = False, err64: bool = False):
    """Per-row top-k of every block's pairs.  precision 0: float32 on CUDA cores;
    1: BF16 tensor-core filter and exact float32 rerank; 2: the same with an
    FP8 (E4M3, per-row scale) filter.  With stats=True also
    returns (rerank fraction, Gram ms, select ms, prep ms, max |approx - f64| / bound,
    max |canonical - f64|); the last two only with err64=True (slower)."""
    nb, bs = block_ids.shape
    ids = torch.empty((nb, bs, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((nb, bs, k), dtype=torch.float32, device=X.device)
    st = (C.c_double * 6)()
    st[4] = 1.0 if err64 else 0.0
    _check(load().fgraft_dense_block_dist(_ptr(X), C.c_int64(X.shape[0]), C.c_int32(d),
                                          C.c_int64(X.shape[1]), C.c_int32(metric),
                                          _ptr(block_ids), C.c_int64(nb), C.c_int32(bs),
                                          C.c_int32(k), C.c_int32(precision), _ptr(ids),
                                          _ptr(dist), st if stats else None, _stream(X.device)))
    return (ids, dist, tuple(st)) if stats else (ids, dist)


def fgraft_dense_block_gram(X: torch.Tensor, d: int, metric: int, block_ids: torch.Tensor,
                            precision: int = 1):
    """Raw dense-block rate: the tensor-core Gram of every block reduced to the
    smallest approximate distance per row.  Returns (out_min (nb, bs) float32,
    kernel ms)."""
    nb, bs = block_ids.shape
    out = torch.empty((nb, bs), dtype=torch.float32, device=X.device)
    ms = C.c_double(0.0)
    _check(load().fgraft_dense_block_gram(_ptr(X), C.c_int64(X.shape[0]), C.c_int32(d),
                                          C.c_int64(X.shape[1]), C.c_int32(metric),
                                          _ptr(block_ids), C.c_int64(nb), C.c_int32(bs),
                                          C.c_int32(precision), _ptr(out), C.byref(ms),
                                          _stream(X.device)))
    return out, ms.value


def build_graph(X: torch.Tensor, d: int, params: Params, use_graph: bool = True):
    """Whole FGraft build: scaffold, all blocks, final graph.  Returns (Index, off, ids)."""
    ix = fgraft_build_scaffold(X, d, params)
    fgraft_harvest_all(ix, use_graph)
    off, ids = fgraft_prune(ix)
    return ix, off, ids
