"""Host-side layout of the TF32 form's tensor-core M2L kernel, which streams
each offset's precomputed matrix (no GPU): for every order the kernel
accepts, and every chunk width it can be tuned to, the layout the library computes must keep every copy and MMA operand in
bounds, fit the shared memory, cover the rank triangle |n| + |m| <= p, and
keep the barrier invariant (the issuer count divides the matrix stages; see
test_tc_protocol.py)."""
import ctypes
import os

import numpy as np
import pytest

SMEM_MAX = 227 * 1024     # dynamic shared memory per CTA on sm_103a
TC_PMAX = 96 * 6 * 32     # bound on one part block (hi or lo) of a matrix


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    from paper_1811_06332_gb300 import fmm
    return fmm


def layout(F, p, prec):
    out = (ctypes.c_int * 42)()
    n = F.lib().fmm_tc_layout(p, prec, out, 42)
    assert n == 42, n
    v = list(out)
    keys = ["cw", "nch", "np", "nbst", "niss", "bstage", "mbytes", "smem"]
    d = dict(zip(keys, v[:8]))
    d["kch"] = v[8:14]
    d["nk"] = [v[14:20], v[20:26]]
    d["boff"] = [v[26:32], v[32:38]]
    d["pbytes"] = v[38:40]
    d["poff"] = v[40:42]
    return d


@pytest.mark.parametrize("cw", ["16", "32", "48", "96", None])
def test_layout_invariants(F, cw, monkeypatch):
    if cw is None:
        monkeypatch.delenv("FMM_TC_CHUNK", raising=False)
    else:
        monkeypatch.setenv("FMM_TC_CHUNK", cw)
    for prec, tf in ((F.GEMM_TF32X3, 1),):
        cps = 8 if tf else 16                       # multipole columns per K-step (32 bytes of a row)
        for p in range(1, 9):
            d = layout(F, p, prec)
            nc = (p + 1) ** 2
            rank = [a for a in range(p + 1) for _ in range(2 * a + 1)]
            w = d["cw"]
            if cw is not None:
                assert w == int(cw)
            assert d["nch"] == (nc + w - 1) // w
            assert d["smem"] <= SMEM_MAX, (p, tf, d)
            assert d["nbst"] in (2, 4) and d["niss"] in (2, 4) and d["nbst"] % d["niss"] == 0
            assert 1 <= d["np"] <= (2 if tf else 1)
            for j in range(d["nch"]):
                need = (p - rank[w * j] + 1) ** 2   # multipole columns of chunk j's lowest rank
                assert d["kch"][j] * cps >= need and (d["kch"][j] - 1) * cps < need
                assert sum(d["nk"][t][j] for t in range(d["np"])) == d["kch"][j]
                assert d["nk"][0][j] >= 1            # the first stage initialises every accumulator chunk
                for t in range(d["np"]):
                    assert 0 <= d["nk"][t][j] <= 6
                    end = d["boff"][t][j] + 32 * w * d["nk"][t][j]
                    assert end <= d["pbytes"][t]
            for t in range(d["np"]):
                assert d["pbytes"][t] % 1024 == 0 and 0 < d["pbytes"][t] <= TC_PMAX
                assert 2 * d["pbytes"][t] <= d["bstage"]
            assert d["poff"][0] == 0
            if d["np"] == 2:
                assert d["poff"][1] == 2 * d["pbytes"][0]
            assert d["mbytes"] == 2 * sum(d["pbytes"][:d["np"]])
            assert d["mbytes"] <= 2 * TC_PMAX * (2 if tf else 1)


def test_layout_rejects(F):
    out = (ctypes.c_int * 42)()
    L = F.lib()
    assert L.fmm_tc_layout(9, F.GEMM_TF32X3, out, 42) == F.ERR_ARG
    assert L.fmm_tc_layout(8, F.FP32, out, 42) == F.ERR_ARG
    assert L.fmm_tc_layout(8, F.GEMM_BF16X3, out, 42) == F.ERR_ARG   # the BF16 form: fmm_tc_gen_layout
    assert L.fmm_tc_layout(0, F.GEMM_TF32X3, out, 42) == F.ERR_ARG
    assert L.fmm_tc_layout(8, F.GEMM_TF32X3, out, 8) == 8
