"""Cache of whole oracle builds for the full-size parity tests.

The oracle's result depends only on the data, the build parameters and the
oracle's own source, so it is stored under a hash of the three.  The cache
folder is the one named by the FGRAFT_ORACLE_CACHE environment variable;
without it nothing is stored and the oracle runs every time.
"""
import hashlib
import json
import os

import numpy as np

import oracle

_ORACLE_SRC = os.path.join(os.path.dirname(os.path.abspath(oracle.__file__)), "fgraft_oracle.c")


def _key(X, params):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(X).tobytes())
    h.update(json.dumps(params, sort_keys=True).encode())
    with open(_ORACLE_SRC, "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:24]


def build_graph(D, X, T, R, ef_h, B, alpha, seed, nthreads=0):
    """oracle.build_graph, served from the cache folder when it holds the same
    data, parameters and oracle source."""
    params = dict(T=T, R=R, ef_h=ef_h, B=B, alpha=alpha, seed=seed, d=D.d, metric=D.metric)
    folder = os.environ.get("FGRAFT_ORACLE_CACHE")
    path = os.path.join(folder, f"build-{_key(X, params)}.npz") if folder else None
    if path and os.path.exists(path):
        z = np.load(path)
        g = {k: z[k] for k in z.files if k != "counters"}
        g["counters"] = json.loads(str(z["counters"]))
        return g
    g = oracle.build_graph(D, T, R, ef_h, B, alpha, seed, nthreads=nthreads)
    if path:
        os.makedirs(folder, exist_ok=True)
        arrays = {k: v for k, v in g.items() if isinstance(v, np.ndarray)}
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, counters=json.dumps(g["counters"]), **arrays)
        os.replace(tmp, path)
    return g
