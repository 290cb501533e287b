"""The autotuner's tuning table (C ABI, no GPU needed): a JSON round trip
keeps every entry, and files that are not tables, lack a field or hold a
setting out of range are rejected without changing the table."""
import ctypes
import json
import os

import pytest

from paper_2609_30493_gb300 import build


@pytest.fixture(scope="module")
def lib():
    lb = ctypes.CDLL(build.build())
    lb.fgraft_last_error.restype = ctypes.c_char_p
    return lb


def _entry(**kw):
    e = {"metric": 1, "d": 100, "ef_h": 100, "R": 64, "log2_n": 21, "T": 8, "B": 8,
         "warps_per_cta": 2, "hash_log2": 11, "overflow_mode": 1, "us_per_query": 0.5}
    e.update(kw)
    return e


def test_table_round_trip(lib, tmp_path):
    src = tmp_path / "in.json"
    entries = [_entry(), _entry(d=960, ef_h=64, R=32, log2_n=19, warps_per_cta=4, hash_log2=0,
                                overflow_mode=2, us_per_query=3.25), _entry(T=32, B=1)]
    src.write_text(json.dumps({"fgraft_tuning": 1, "entries": entries}))
    assert lib.fgraft_tuning_table_load(os.fsencode(str(src))) == 0
    out = tmp_path / "out.json"
    assert lib.fgraft_tuning_table_save(os.fsencode(str(out))) == 0
    got = json.loads(out.read_text())
    assert got["fgraft_tuning"] == 1
    key = ("metric", "d", "ef_h", "R", "log2_n", "T", "B")
    have = {tuple(e[k] for k in key): e for e in got["entries"]}
    for e in entries:
        g = have[tuple(e[k] for k in key)]
        for f in ("warps_per_cta", "hash_log2", "overflow_mode"):
            assert g[f] == e[f]
        assert abs(g["us_per_query"] - e["us_per_query"]) < 1e-5


@pytest.mark.parametrize("doc", [
    "not json at all",
    json.dumps({"entries": [_entry()]}),
    json.dumps({"fgraft_tuning": 1, "entries": [{k: v for k, v in _entry().items() if k != "R"}]}),
    json.dumps({"fgraft_tuning": 1, "entries": [{k: v for k, v in _entry().items() if k != "B"}]}),
    json.dumps({"fgraft_tuning": 1, "entries": [_entry(warps_per_cta=5)]}),
    json.dumps({"fgraft_tuning": 1, "entries": [_entry(hash_log2=3)]}),
    json.dumps({"fgraft_tuning": 1, "entries": [_entry(overflow_mode=0)]}),
])
def test_table_rejects_bad_files(lib, tmp_path, doc):
    before = tmp_path / "before.json"
    assert lib.fgraft_tuning_table_save(os.fsencode(str(before))) == 0
    bad = tmp_path / "bad.json"
    bad.write_text(doc)
    assert lib.fgraft_tuning_table_load(os.fsencode(str(bad))) == 1
    assert lib.fgraft_last_error()
    after = tmp_path / "after.json"
    assert lib.fgraft_tuning_table_save(os.fsencode(str(after))) == 0
    assert json.loads(before.read_text()) == json.loads(after.read_text())


def test_table_missing_file(lib, tmp_path):
    assert lib.fgraft_tuning_table_load(os.fsencode(str(tmp_path / "none.json"))) == 1
