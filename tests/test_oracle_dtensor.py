"""Pins for the oracle's multi-index tables and D-tensors (CPU only).

D_n(r) = grad^n r^{-1} is pinned against things other than the oracle's own
formula (Eq. traceless grad + Eq. Detracer3, App. A):
  * the storage table of App. E,
  * textbook closed forms of ranks 0..3 and the rank-2 excerpt printed in
    Sec. 2.2,
  * exact symbolic differentiation of 1/r (sympy) to rank 10,
  * central finite differences (d/dx_i D_k = D_{k+e_i}),
  * homogeneity, parity and the trace-free condition.
"""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pos(p, basis=oracle.SYM):
    return {tuple(n): i for i, n in enumerate(oracle.indices(p, basis))}


def test_storage_counts_match_paper_table():
    rows = np.loadtxt(os.path.join(GOLD, "storage_counts.txt"), dtype=int)
    for p, at_p, total, tl_at_p, tl_total, saving in rows:
        assert oracle.ncoef(p, oracle.SYM) == total
        assert oracle.ncoef(p, oracle.TRACELESS) == tl_total
        idx = oracle.indices(p, oracle.SYM)
        assert (idx.sum(1) == p).sum() == at_p
        idt = oracle.indices(p, oracle.TRACELESS)
        assert (idt.sum(1) == p).sum() == tl_at_p
        assert np.all(idt[:, 2] <= 1)
        assert round(100 * (1 - tl_total / total)) == saving
        # every multi-index appears once
        assert len({tuple(v) for v in idx}) == total


def test_storage_order():
    # rank-concatenated; descending nx then ny inside a rank (symmetric)
    idx = oracle.indices(3, oracle.SYM)
    assert idx[:4].tolist() == [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    assert idx[10:16].tolist() == [[3, 0, 0], [2, 1, 0], [2, 0, 1], [1, 2, 0], [1, 1, 1], [1, 0, 2]]
    idt = oracle.indices(3, oracle.TRACELESS)
    assert idt[9:16].tolist() == [[3, 0, 0], [2, 1, 0], [1, 2, 0], [0, 3, 0],
                                  [2, 0, 1], [1, 1, 1], [0, 2, 1]]


def _closed_form(r):
    """Textbook derivatives of 1/r to rank 3 keyed by multi-index."""
    x = np.asarray(r, dtype=float)
    R2 = x @ x
    R = np.sqrt(R2)
    d = np.eye(3)
    out = {(0, 0, 0): 1 / R}
    for i in range(3):
        n = [0, 0, 0]; n[i] = 1
        out[tuple(n)] = -x[i] / R**3
    for i in range(3):
        for j in range(i, 3):
            n = [0, 0, 0]; n[i] += 1; n[j] += 1
            out[tuple(n)] = (3 * x[i] * x[j] - R2 * d[i, j]) / R**5
    for i in range(3):
        for j in range(i, 3):
            for k in range(j, 3):
                n = [0, 0, 0]; n[i] += 1; n[j] += 1; n[k] += 1
                out[tuple(n)] = -(15 * x[i] * x[j] * x[k]
                                  - 3 * R2 * (x[i] * d[j, k] + x[j] * d[i, k] + x[k] * d[i, j])) / R**7
    return out


@pytest.mark.parametrize("seed", range(5))
def test_dtensor_closed_forms_rank0_3(seed):
    rng = np.random.default_rng(seed)
    r = rng.uniform(-3, 3, 3)
    D = oracle.dtensor(3, r)
    pos = _pos(3)
    for n, v in _closed_form(r).items():
        assert D[pos[n]] == pytest.approx(v, rel=1e-13, abs=1e-15)


def test_dtensor_rank2_excerpt_from_paper():
    rows = np.loadtxt(os.path.join(GOLD, "dtensor_rank2_p5.txt"))
    rng = np.random.default_rng(7)
    pos = _pos(5)
    for _ in range(10):
        r = rng.uniform(-2, 2, 3)
        D = oracle.dtensor(5, r)
        h = r @ r
        u = 1 / np.sqrt(h)
        for row in rows:
            n = tuple(int(v) for v in row[:3])
            axis = n.index(2)
            want = row[3] * u**5 * h + row[4] * u**5 * r[axis] ** 2
            assert D[pos[n]] == pytest.approx(want, rel=1e-13)
        # D_zz = -(D_xx + D_yy)
        assert D[pos[(0, 0, 2)]] == pytest.approx(-(D[pos[(2, 0, 0)]] + D[pos[(0, 2, 0)]]), rel=1e-12)


def test_dtensor_exact_symbolic_rank10():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    f = 1 / sp.sqrt(x**2 + y**2 + z**2)
    pt_q = (sp.Rational(3, 7), sp.Rational(-5, 11), sp.Rational(2, 3))
    subs = dict(zip((x, y, z), pt_q))
    cache = {(0, 0, 0): f}

    def deriv(n):
        if n not in cache:
            nx, ny, nz = n
            if nz:
                cache[n] = sp.diff(deriv((nx, ny, nz - 1)), z)
            elif ny:
                cache[n] = sp.diff(deriv((nx, ny - 1, nz)), y)
            else:
                cache[n] = sp.diff(deriv((nx - 1, ny, nz)), x)
        return cache[n]

    p = 10
    D = oracle.dtensor(p, np.array([float(v) for v in pt_q]))
    idx = oracle.indices(p, oracle.SYM)
    for j in range(p + 1):
        sel = np.where(idx.sum(1) == j)[0]
        exact = np.array([float(sp.N(deriv(tuple(int(v) for v in idx[i])).subs(subs), 30))
                          for i in sel])
        err = np.linalg.norm(D[sel] - exact) / np.linalg.norm(exact)
        assert err < 1e-13, (j, err)


@pytest.mark.parametrize("seed", range(3))
def test_dtensor_finite_differences(seed):
    p = 10
    rng = np.random.default_rng(100 + seed)
    r = rng.uniform(-3, 3, 3)
    r *= 2.5 / np.linalg.norm(r)
    idx = oracle.indices(p, oracle.SYM)
    pos = _pos(p)
    D = oracle.dtensor(p, r)
    h = 1e-4
    for i in range(3):
        e = np.zeros(3); e[i] = h
        Dp, Dm = oracle.dtensor(p, r + e), oracle.dtensor(p, r - e)
        Dp2, Dm2 = oracle.dtensor(p, r + 2 * e), oracle.dtensor(p, r - 2 * e)
        # fourth-order central difference
        fd = (8 * (Dp - Dm) - (Dp2 - Dm2)) / (12 * h)
        for j in range(p):
            sel = np.where(idx.sum(1) == j)[0]
            tgt = []
            for k in sel:
                n = list(idx[k]); n[i] += 1
                tgt.append(D[pos[tuple(n)]])
            tgt = np.array(tgt)
            err = np.linalg.norm(fd[sel] - tgt) / np.linalg.norm(tgt)
            assert err < 1e-8, (i, j, err)


def test_dtensor_homogeneity_parity_tracefree():
    p = 10
    rng = np.random.default_rng(3)
    idx = oracle.indices(p, oracle.SYM)
    pos = _pos(p)
    rank = idx.sum(1)
    for _ in range(5):
        r = rng.uniform(-3, 3, 3)
        D = oracle.dtensor(p, r)
        lam = 1.7
        np.testing.assert_allclose(oracle.dtensor(p, lam * r), lam ** (-rank - 1.0) * D, rtol=1e-12)
        np.testing.assert_allclose(oracle.dtensor(p, -r), (-1.0) ** rank * D, rtol=1e-12)
        for k in oracle.indices(p - 2, oracle.SYM):
            k = tuple(int(v) for v in k)
            s = sum(D[pos[(k[0] + 2 * (a == 0), k[1] + 2 * (a == 1), k[2] + 2 * (a == 2))]]
                    for a in range(3))
            scale = max(abs(D[pos[(k[0] + 2, k[1], k[2])]]), abs(D[pos[(k[0], k[1] + 2, k[2])]]))
            assert abs(s) <= 1e-11 * scale + 1e-300


def test_expand_traceless_roundtrip():
    p = 8
    rng = np.random.default_rng(11)
    At = rng.uniform(-1, 1, oracle.ncoef(p, oracle.TRACELESS))
    A = oracle.expand_traceless(p, At)
    pos = _pos(p)
    idt = oracle.indices(p, oracle.TRACELESS)
    for i, n in enumerate(idt):
        assert A[pos[tuple(n)]] == At[i]
    # the expanded tensor is trace free in every rank
    for k in oracle.indices(p - 2, oracle.SYM):
        k = tuple(int(v) for v in k)
        s = A[pos[(k[0] + 2, k[1], k[2])]] + A[pos[(k[0], k[1] + 2, k[2])]] + A[pos[(k[0], k[1], k[2] + 2)]]
        assert abs(s) < 1e-12
