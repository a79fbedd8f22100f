"""C-ABI checks that need no GPU: the library loads, exports every entry
point declared in include/fmm_gb300.h, validates arguments on the host, and
its generated combinatorial tables agree with the oracle."""
import ctypes
import os
import re
import sys

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    from paper_1811_06332_gb300 import fmm
    return fmm


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "fmm_gb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(F):
    L = ctypes.CDLL(F.LIB_PATH)
    syms = declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(F.EXPORTS) == syms


def test_host_validation(F):
    L = F.lib()
    for p in range(11):
        assert L.fmm_ncoef(p, 0) == oracle.ncoef(p, 0)
        assert L.fmm_ncoef(p, 1) == oracle.ncoef(p, 1)
    assert L.fmm_ncoef(11, 0) == F.ERR_ARG
    assert L.fmm_ncoef(3, 2) == F.ERR_ARG
    assert L.fmm_op_m2l(11, 0, 0, 10, None, None, None, 0, None) == F.ERR_ARG
    assert L.fmm_op_m2l(4, 0, 7, 10, None, None, None, 0, None) == F.ERR_ARG
    assert L.fmm_op_m2l(4, 0, 0, 10, None, None, None, 0, None) == F.ERR_ARG
    assert L.fmm_op_m2l(4, 0, 0, -1, None, None, None, 0, None) == F.ERR_ARG
    assert b"null" in L.fmm_last_error(None) or b"n < 0" in L.fmm_last_error(None)
    assert L.fmm_op_dtensor(4, 0, 3, 10, None, None, None) == F.ERR_ARG
    assert L.fmm_op_dtensor(4, 2, 0, 10, None, None, None) == F.ERR_ARG
    assert L.fmm_op_m2m(4, 0, 2, 10, None, None, None, None) == F.ERR_ARG
    assert L.fmm_op_l2p(4, 0, 0, -1, None, None, None, None) == F.ERR_ARG
    assert L.fmm_direct(-1, None, None, None, None, 0, None, None, None, None, None, None) == F.ERR_ARG
    h = ctypes.c_void_p()
    assert L.fmm_create(None, ctypes.byref(h)) == F.ERR_ARG
    bad = F.Config(p=4, basis=0, prec=0, depth=11)
    assert L.fmm_create(ctypes.byref(bad), ctypes.byref(h)) == F.ERR_ARG
    assert not h.value
    assert L.fmm_p2m(None, None) == F.ERR_ARG
    L.fmm_destroy(None)


def _gen():
    sys.path.insert(0, os.path.join(ROOT, "paper_1811_06332_gb300", "csrc"))
    import gen
    return gen


@pytest.mark.parametrize("j", range(0, 9))
def test_generated_maps_match_oracle(j):
    gen = _gen()
    rng = np.random.default_rng(j)
    m = (j + 1) * (j + 2) // 2
    A = rng.uniform(-1, 1, m)
    Dm = np.array([[float(v) for v in row] for row in gen.detracer_rank(j)])
    np.testing.assert_allclose(Dm @ A, oracle.detracer_D(j, A), rtol=1e-12, atol=1e-13)
    # trace expansion agrees with the oracle's rebuild of dependent components
    X = np.array([[float(v) for v in row] for row in gen.expand_rank(j)])
    t = rng.uniform(-1, 1, 2 * j + 1)
    full = np.zeros(oracle.ncoef(j, 0))
    tl = np.zeros(oracle.ncoef(j, 1))
    tl[j * j:] = t
    full_or = oracle.expand_traceless(j, tl)[oracle.ncoef(j - 1, 0) if j else 0:]
    np.testing.assert_allclose(X @ t, full_or, rtol=1e-13, atol=1e-13)
    # reduced representative: supported on nz<=1 and same detraced tensor
    P = np.array([[float(v) for v in row] for row in gen.reduce_rank(j)])
    Ar = P @ A
    emb = np.zeros(m)
    idx = gen.rank_sym(j)
    for k, n in enumerate(gen.rank_tl(j)):
        emb[idx.index(n)] = Ar[k]
    np.testing.assert_allclose(oracle.detracer_D(j, emb), oracle.detracer_D(j, A), rtol=1e-11, atol=1e-12)


def test_generated_dtensor_recurrence_terms():
    """The recurrence used by the CUDA D-tensor kernels, evaluated here in
    plain Python floats, reproduces the oracle's D-tensor (different route:
    Leibniz recurrence versus the closed form of Eq. Detracer3)."""
    gen = _gen()
    p = 10
    r = np.array([0.7, -1.3, 2.1])
    pos = {n: i for i, n in enumerate(gen.sym_list(p))}
    d = np.zeros(len(pos))
    r2 = r @ r
    d[0] = 1 / np.sqrt(r2)
    for k in gen.sym_list(p)[1:]:
        s = 0.0
        for c, ax, src in gen.dtensor_terms(k):
            s += c * (r[ax] if ax is not None else 1.0) * d[pos[src]]
        d[pos[k]] = -s / r2
    D = oracle.dtensor(p, r)
    idx = oracle.indices(p, 0)
    for j in range(p + 1):
        sel = idx.sum(1) == j
        assert np.linalg.norm(d[sel] - D[sel]) / np.linalg.norm(D[sel]) < 1e-13
