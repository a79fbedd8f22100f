"""Pins for the oracle's operators P2M, M2M, M2L, L2L, L2P and the direct sum
(CPU only).

  * M2L reproduces the L_x term list printed for p = 3 in Sec. 2.2,
  * M2M is exact (Sec. 2.1): P2M at a child centre then M2M equals P2M at the
    parent centre, in both bases,
  * L2L is an exact shift of the truncated polynomial: composition and
    L2P o L2L = L2P,
  * the traceless (FT) and symmetric chains give the same field,
  * the appendix normalisation (App. B Eq. multipole v1 / field tensor v1 /
    phi v1, restated here in plain Python) gives the same potential and
    gradient as the main-text normalisation,
  * P2M -> M2L -> L2P approaches the direct sum geometrically in p, and the
    longer chain through M2M/L2L agrees with it within truncation error,
  * the direct sum against two-body closed forms and momentum conservation.
"""
import os
from math import factorial

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SYM, TL = oracle.SYM, oracle.TRACELESS


def pos(p, basis=SYM):
    return {tuple(int(v) for v in n): i for i, n in enumerate(oracle.indices(p, basis))}


def cluster(rng, n, centre, half):
    x = rng.uniform(-half, half, (3, n)) + np.asarray(centre)[:, None]
    q = rng.uniform(0.1, 1.0, n)
    return x, q


def test_m2l_worked_example_p3():
    terms = np.loadtxt(os.path.join(GOLD, "m2l_p3_Lx_terms.txt"))
    p = 3
    ps = pos(p)
    rng = np.random.default_rng(0)
    for _ in range(5):
        M = rng.uniform(-1, 1, oracle.ncoef(p, SYM))
        D = rng.uniform(-1, 1, oracle.ncoef(p, SYM))
        L = oracle.m2l_D(p, SYM, M, D)
        want = sum(t[0] * D[ps[tuple(int(v) for v in t[1:4])]] * M[ps[tuple(int(v) for v in t[4:7])]]
                   for t in terms)
        assert L[ps[(1, 0, 0)]] == pytest.approx(want, rel=1e-14)
        # the printed list is complete: zeroing every M it names zeroes L_x
        M2 = M.copy()
        for t in terms:
            M2[ps[tuple(int(v) for v in t[4:7])]] = 0.0
        assert oracle.m2l_D(p, SYM, M2, D)[ps[(1, 0, 0)]] == 0.0


@pytest.mark.parametrize("basis", [SYM, TL])
@pytest.mark.parametrize("p", [1, 3, 6, 10])
def test_m2m_exact(basis, p):
    rng = np.random.default_rng(p)
    x, q = cluster(rng, 20, [0.3, -0.2, 0.1], 0.25)
    zc = np.array([0.25, -0.25, 0.25])
    zp = np.array([0.0, 0.0, 0.0])
    Mc = oracle.p2m(p, basis, x[0], x[1], x[2], q, zc)
    Mshift = oracle.m2m(p, basis, Mc, zc - zp)           # delta = z_child - z_parent
    Mdirect = oracle.p2m(p, basis, x[0], x[1], x[2], q, zp)
    idx = oracle.indices(p, basis)
    for j in range(p + 1):
        sel = idx.sum(1) == j
        err = np.linalg.norm(Mshift[sel] - Mdirect[sel]) / np.linalg.norm(Mdirect[sel])
        assert err < 1e-13, (j, err)


@pytest.mark.parametrize("basis", [SYM, TL])
@pytest.mark.parametrize("p", [2, 5, 8])
def test_l2l_composition_and_l2p(basis, p):
    rng = np.random.default_rng(40 + p)
    L = rng.uniform(-1, 1, oracle.ncoef(p, SYM))
    if basis == TL:
        # a trace-free local expansion: take the M2L of something
        x, q = cluster(rng, 10, [0, 0, 0], 0.5)
        M = oracle.p2m(p, TL, x[0], x[1], x[2], q, np.zeros(3))
        L = oracle.m2l(p, TL, M, np.array([2.7, -1.9, 3.1]))
    d1, d2 = rng.uniform(-0.3, 0.3, 3), rng.uniform(-0.3, 0.3, 3)
    L12 = oracle.l2l(p, basis, oracle.l2l(p, basis, L, d1), d2)
    Lc = oracle.l2l(p, basis, L, d1 + d2)
    np.testing.assert_allclose(L12, Lc, rtol=1e-12, atol=1e-13 * np.abs(Lc).max())
    rb = rng.uniform(-0.2, 0.2, 3)
    np.testing.assert_allclose(oracle.l2p(p, basis, oracle.l2l(p, basis, L, d1), rb),
                               oracle.l2p(p, basis, L, d1 + rb), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("p", [2, 4, 7, 10])
def test_traceless_equals_symmetric(p):
    rng = np.random.default_rng(50 + p)
    x, q = cluster(rng, 30, [0.1, 0.2, -0.1], 0.5)
    zA, zB = np.zeros(3), np.array([3.0, -2.0, 1.0])
    rb = np.array([0.2, -0.3, 0.4])
    out = []
    for basis in (SYM, TL):
        M = oracle.p2m(p, basis, x[0], x[1], x[2], q, zA)
        L = oracle.m2l(p, basis, M, zB - zA)
        out.append(oracle.l2p(p, basis, L, rb))
    np.testing.assert_allclose(out[1], out[0], rtol=1e-12)


def test_appendix_normalisation_gives_same_field():
    """App. B: M'_n = sum q (-1)^|n|/|n|! r_a^n,
    L_n = sum_m (1/|n|!)(|m|!/m!) M_m grad^{n+m} r^{-1},
    grad^k Phi = sum_n ((|n|+|k|)!/(|k|!|n|!)) (|n|!/n!) r^n L_{n+k};
    for |k| <= 1 this is the same Phi and grad Phi as the main-text chain."""
    p = 5
    rng = np.random.default_rng(60)
    x, q = cluster(rng, 12, [0, 0, 0], 0.5)
    r = np.array([2.5, 1.5, -2.0])
    rb = np.array([0.3, -0.1, 0.25])
    idx = [tuple(int(v) for v in n) for n in oracle.indices(p, SYM)]
    D = dict(zip(idx, oracle.dtensor(p, r)))
    fact = lambda n: factorial(n[0]) * factorial(n[1]) * factorial(n[2])
    Mp = {n: sum(qa * (-1) ** sum(n) / factorial(sum(n)) * xa ** n[0] * ya ** n[1] * za ** n[2]
                 for qa, xa, ya, za in zip(q, *x)) for n in idx}
    La = {}
    for n in idx:
        La[n] = sum(Mp[m] * D[(n[0] + m[0], n[1] + m[1], n[2] + m[2])] * factorial(sum(m))
                    / (factorial(sum(n)) * fact(m)) for m in idx if sum(m) <= p - sum(n))

    def grad_k(k):
        s = 0.0
        for n in idx:
            if sum(n) > p - sum(k):
                continue
            w = factorial(sum(n) + sum(k)) / (factorial(sum(k)) * factorial(sum(n))) \
                * factorial(sum(n)) / fact(n)
            s += w * rb[0] ** n[0] * rb[1] ** n[1] * rb[2] ** n[2] * La[(n[0] + k[0], n[1] + k[1], n[2] + k[2])]
        return s

    app = np.array([grad_k((0, 0, 0)), grad_k((1, 0, 0)), grad_k((0, 1, 0)), grad_k((0, 0, 1))])
    M = oracle.p2m(p, SYM, x[0], x[1], x[2], q, np.zeros(3))
    main = oracle.l2p(p, SYM, oracle.m2l(p, SYM, M, r), rb)
    np.testing.assert_allclose(app, main, rtol=1e-12)


def _direct_at(xs, qs, xt):
    d = xs - xt[:, None]
    R = np.sqrt((d * d).sum(0))
    return np.array([np.sum(qs / R), *(qs * d / R**3).sum(1)])  # Phi, grad Phi


@pytest.mark.parametrize("basis", [SYM, TL])
def test_far_field_error_decreases_with_p(basis):
    rng = np.random.default_rng(70)
    x, q = cluster(rng, 40, [0, 0, 0], 0.5)
    zB = np.array([2.0, 1.0, -1.0])
    rb = rng.uniform(-0.5, 0.5, 3)
    exact = _direct_at(x, q, zB + rb)
    errs = []
    for p in range(0, 11):
        M = oracle.p2m(p, basis, x[0], x[1], x[2], q, np.zeros(3))
        o = oracle.l2p(p, basis, oracle.m2l(p, basis, M, zB), rb)
        errs.append(np.linalg.norm(o[1:] - exact[1:]) / np.linalg.norm(exact[1:]))
    errs = np.array(errs)
    # geometric decay: rho = (r_A + r_B)/|r| with r_A = r_B = sqrt(3)/2
    rho = np.sqrt(3) / np.linalg.norm(zB)
    assert errs[10] < 3e-3 * errs[1]
    assert errs[10] < 50 * rho ** 10
    # monotone on average (every 3-step window decreases)
    assert np.all(errs[3:] < errs[:-3])


@pytest.mark.parametrize("basis", [SYM, TL])
def test_translation_consistency(basis):
    """P2M->M2M->M2L->L2L->L2P and P2M->M2L->L2P at the same p both approach
    the direct sum, and their difference shrinks with p."""
    rng = np.random.default_rng(80)
    x, q = cluster(rng, 25, [0.125, 0.125, 0.125], 0.12)   # inside child A
    zA_child, zA = np.array([0.125, 0.125, 0.125]), np.zeros(3)
    zB_child, zB = np.array([4.125, -0.125, 0.125]), np.array([4.0, 0.0, 0.0])
    rb = rng.uniform(-0.1, 0.1, 3)
    xt = zB_child + rb
    exact = _direct_at(x, q, xt)
    diffs, e_long, e_short = [], [], []
    for p in (2, 4, 6, 8):
        Mc = oracle.p2m(p, basis, x[0], x[1], x[2], q, zA_child)
        long_ = oracle.l2p(p, basis, oracle.l2l(p, basis, oracle.m2l(p, basis, oracle.m2m(p, basis, Mc, zA_child - zA), zB - zA),
                                                 zB_child - zB), rb)
        short = oracle.l2p(p, basis, oracle.m2l(p, basis, Mc, zB_child - zA_child), rb)
        nrm = np.linalg.norm(exact[1:])
        e_long.append(np.linalg.norm(long_[1:] - exact[1:]) / nrm)
        e_short.append(np.linalg.norm(short[1:] - exact[1:]) / nrm)
        diffs.append(np.linalg.norm(long_[1:] - short[1:]) / nrm)
    assert all(b < a for a, b in zip(e_long, e_long[1:]))
    assert all(b < a for a, b in zip(e_short, e_short[1:]))
    assert all(b < a for a, b in zip(diffs, diffs[1:]))
    assert e_long[-1] < 1e-6 and e_short[-1] < 1e-6


def test_l2p_gradient_is_derivative_of_potential():
    p = 7
    rng = np.random.default_rng(90)
    x, q = cluster(rng, 10, [0, 0, 0], 0.5)
    M = oracle.p2m(p, TL, x[0], x[1], x[2], q, np.zeros(3))
    L = oracle.m2l(p, TL, M, np.array([3.0, 0.5, -1.0]))
    rb = np.array([0.1, 0.2, -0.15])
    g = oracle.l2p(p, TL, L, rb)[1:]
    h = 1e-5
    for i in range(3):
        e = np.zeros(3); e[i] = h
        fd = (oracle.l2p(p, TL, L, rb + e)[0] - oracle.l2p(p, TL, L, rb - e)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-7)


def test_direct_two_body_and_momentum():
    x = np.array([0.0, 3.0]); y = np.array([0.0, 4.0]); z = np.array([0.0, 0.0])
    q = np.array([2.0, 5.0])
    pot, acc = oracle.direct(x, y, z, q)
    assert pot[0] == pytest.approx(-5.0 / 5.0) and pot[1] == pytest.approx(-2.0 / 5.0)
    np.testing.assert_allclose(acc[:, 0], 5.0 * np.array([3.0, 4.0, 0.0]) / 125.0)
    np.testing.assert_allclose(acc[:, 1], -2.0 * np.array([3.0, 4.0, 0.0]) / 125.0)
    rng = np.random.default_rng(3)
    n = 300
    x, y, z = rng.uniform(0, 1, (3, n))
    q = rng.uniform(0.1, 1, n)
    pot, acc = oracle.direct(x, y, z, q)
    mom = (q[None, :] * acc).sum(1)
    assert np.abs(mom).max() < 1e-10 * np.abs(q[None, :] * acc).sum()
    # targets subset agrees with the full evaluation
    t = np.array([5, 17, 299])
    pt, at = oracle.direct(x, y, z, q, t)
    np.testing.assert_array_equal(pt, pot[t])
    np.testing.assert_array_equal(at, acc[:, t])


@pytest.mark.parametrize("p", [0, 1, 2, 5, 8])
def test_fused_m2m_is_exact(p):
    """Eq. Detracer2 (fused traceless M2M): P2M at a child centre followed by
    the fused M2M equals P2M at the parent centre, as the M2M of Eq. M2M
    does (the shift is exact; App. B)."""
    rng = np.random.default_rng(90 + p)
    n = 9
    x, y, z = rng.uniform(-0.2, 0.2, (3, n)) + 0.3
    q = rng.uniform(0.1, 1.0, n)
    zc = np.array([0.3, 0.31, 0.29])
    zp = np.array([0.2, 0.45, 0.1])
    Mc = oracle.p2m(p, oracle.TRACELESS, x, y, z, q, zc)
    Mref = oracle.p2m(p, oracle.TRACELESS, x, y, z, q, zp)
    Mf = oracle.m2m_fused(p, Mc, zc - zp)
    assert np.abs(Mf - Mref).max() <= 1e-13 * max(np.abs(Mref).max(), 1.0)
    Mu = oracle.m2m(p, oracle.TRACELESS, Mc, zc - zp)
    assert np.abs(Mf - Mu).max() <= 1e-13 * max(np.abs(Mu).max(), 1.0)
