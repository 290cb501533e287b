"""Reader for the hand-worked fixtures in this folder (plain text, one record per line)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    pts, parents, edges, cases, out = {}, {}, [], [], {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            key, rest = tok[0], tok[1:]
            if key == "point":
                pts[int(rest[0])] = [float(v) for v in rest[1:]]
            elif key == "parent":
                parents[int(rest[0])] = int(rest[1])
            elif key == "edge":
                edges.append((int(rest[0]), int(rest[1])))
            elif key == "case":
                cases.append(dict(kv.split("=") for kv in rest))
            elif key == "arow":
                out.setdefault("arows", {})[int(rest[0])] = [int(v) for v in rest[1:]]
            elif key in ("query", "cand"):
                out[key] = [float(v) for v in rest]
            elif key == "alpha":
                out[key] = float(rest[0])
            else:
                out[key] = int(rest[0])
    n = len(pts)
    out["X"] = np.array([pts[i] for i in range(n)], np.float32)
    out["parents"] = parents
    out["edges"] = edges
    out["cases"] = cases
    return out
