"""The tuning cache of the tensor-core kernel shapes (host only, no GPU):
a JSON object {"<key>": {"kernel", "cw", "niss", "ms"}} in a file, read by
plans created with autotune and written after a plan measured its
candidates."""
import ctypes
import json

import pytest


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    from paper_1811_06332_gb300 import fmm
    return fmm


def put(F, path, key, vals, ms):
    v = (ctypes.c_int * 3)(*vals)
    return F.lib().fmm_tune_cache_put(str(path).encode(), key.encode(), v, ms)


def get(F, path, key):
    v = (ctypes.c_int * 3)()
    r = F.lib().fmm_tune_cache_get(str(path).encode(), key.encode(), v)
    return r, list(v)


def test_put_get_replace(F, tmp_path):
    path = tmp_path / "a" / "b" / "tune.json"          # directories are created
    k1 = "NVIDIA GB300|p=8|basis=1|prec=3|depth=6"
    k2 = "NVIDIA GB300|p=8|basis=1|prec=2|depth=6"
    assert get(F, path, k1)[0] == 0                     # no file: no entry
    assert put(F, path, k1, (0, 48, 4), 2.58) == F.OK
    assert put(F, path, k2, (0, 32, 4), 3.91) == F.OK
    assert get(F, path, k1) == (1, [0, 48, 4])
    assert get(F, path, k2) == (1, [0, 32, 4])
    assert put(F, path, k1, (1, 96, 1), 2.10) == F.OK   # replaces, keeps the other entry
    assert get(F, path, k1) == (1, [1, 96, 1])
    assert get(F, path, k2) == (1, [0, 32, 4])
    d = json.load(open(path))                           # the file is plain JSON
    assert d[k1] == {"kernel": 1, "cw": 96, "niss": 1, "ms": 2.1}
    assert len(d) == 2
    assert get(F, path, "NVIDIA GB300|p=7|basis=1|prec=3|depth=6")[0] == 0


def test_keys_with_quotes_and_backslashes(F, tmp_path):
    path = tmp_path / "tune.json"
    key = 'GPU "X" \\ model|p=4|basis=1|prec=3|depth=5'
    assert put(F, path, key, (0, 16, 2), 1.0) == F.OK
    assert get(F, path, key) == (1, [0, 16, 2])
    assert json.load(open(path))[key]["cw"] == 16


def test_malformed_or_partial_file(F, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("not json at all")
    assert get(F, path, "k")[0] == 0
    path.write_text('{"k": {"kernel": 0, "cw": 48}}')     # an entry without niss and ms is ignored
    assert get(F, path, "k")[0] == 0
    assert put(F, path, "k", (0, 48, 4), 1.5) == F.OK    # rewritten cleanly
    assert get(F, path, "k") == (1, [0, 48, 4])


def test_unwritable_path_and_bad_arguments(F, tmp_path):
    blocker = tmp_path / "file"
    blocker.write_text("x")
    assert put(F, blocker / "sub" / "tune.json", "k", (0, 48, 4), 1.0) == F.ERR_STATE   # a file in the way
    L = F.lib()
    assert L.fmm_tune_cache_get(None, b"k", (ctypes.c_int * 3)()) == F.ERR_ARG
    assert L.fmm_tune_cache_put(b"x.json", None, (ctypes.c_int * 3)(), 1.0) == F.ERR_ARG
    assert L.fmm_set_tc_shape(None, 0, 48) == F.ERR_ARG
    assert L.fmm_plan_tuning(None, (ctypes.c_int * 8)(), 8) == F.ERR_ARG
