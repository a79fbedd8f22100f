"""Pins for the oracle's detracer (Eq. Detracer, App. A), CPU only.

  * D = T/(2n-1)!! is the orthogonal projection onto trace-free symmetric
    tensors under the n-fold contraction (checked against a projection built
    with numpy linear algebra from the null space of the trace map),
  * DD = D and TT = (2n-1)!! T,
  * the detracer exchange theorem and its companion identity,
  * T[r^n] = (-1)^n r^{2n+1} grad^n r^{-1} (Eq. traceless grad) links the
    general detracer to the D-tensor route (Eq. Detracer3).
"""
from math import factorial

import numpy as np
import pytest

import oracle


def rank_indices(n):
    return [(nx, ny, n - nx - ny) for nx in range(n, -1, -1) for ny in range(n - nx, -1, -1)]


def weights(n):
    return np.array([factorial(n) / (factorial(a) * factorial(b) * factorial(c))
                     for a, b, c in rank_indices(n)])


def contract(n, A, B):
    """n-fold contraction A.n.B = sum_{|k|=n} n!/k! A_k B_k (App. A)."""
    return float(np.sum(weights(n) * A * B))


def trace_map(n):
    rows = rank_indices(n - 2)
    cols = {k: i for i, k in enumerate(rank_indices(n))}
    T = np.zeros((len(rows), len(cols)))
    for r, (a, b, c) in enumerate(rows):
        for d in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
            T[r, cols[(a + d[0], b + d[1], c + d[2])]] = 1.0
    return T


def dfact(n):
    v = 1
    for i in range(2 * n - 1, 1, -2):
        v *= i
    return v


@pytest.mark.parametrize("n", range(0, 8))
def test_D_is_orthogonal_projection(n):
    rng = np.random.default_rng(n)
    A = rng.uniform(-1, 1, (n + 1) * (n + 2) // 2)
    if n < 2:
        np.testing.assert_allclose(oracle.detracer_D(n, A), A, rtol=1e-15)
        return
    Tm = trace_map(n)
    _, s, vt = np.linalg.svd(Tm)
    N = vt[np.sum(s > 1e-10):].T          # basis of trace-free tensors
    W = np.diag(weights(n))
    P = N @ np.linalg.solve(N.T @ W @ N, N.T @ W)
    np.testing.assert_allclose(oracle.detracer_D(n, A), P @ A, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("n", range(0, 9))
def test_idempotent_and_TT(n):
    rng = np.random.default_rng(10 + n)
    A = rng.uniform(-1, 1, (n + 1) * (n + 2) // 2)
    D1 = oracle.detracer_D(n, A)
    np.testing.assert_allclose(oracle.detracer_D(n, D1), D1, rtol=1e-12, atol=1e-12)
    T1 = oracle.detracer_T(n, A)
    np.testing.assert_allclose(oracle.detracer_T(n, T1), dfact(n) * T1, rtol=1e-12,
                               atol=1e-12 * dfact(n) * np.abs(T1).max())
    if n >= 2:
        np.testing.assert_allclose(trace_map(n) @ T1, 0.0, atol=1e-11 * np.abs(T1).max())


@pytest.mark.parametrize("n", range(0, 9))
def test_exchange_theorem(n):
    rng = np.random.default_rng(20 + n)
    m = (n + 1) * (n + 2) // 2
    A, B = rng.uniform(-1, 1, m), rng.uniform(-1, 1, m)
    TA, TB = oracle.detracer_T(n, A), oracle.detracer_T(n, B)
    lhs = contract(n, A, TB)
    assert lhs == pytest.approx(contract(n, TA, B), rel=1e-11, abs=1e-11)
    assert contract(n, TA, TB) == pytest.approx(dfact(n) * lhs, rel=1e-11, abs=1e-9)


@pytest.mark.parametrize("n", range(0, 11))
def test_detracer_of_r_power_is_gradient(n):
    rng = np.random.default_rng(30 + n)
    r = rng.uniform(-2, 2, 3)
    mono = np.array([r[0] ** a * r[1] ** b * r[2] ** c for a, b, c in rank_indices(n)])
    T = oracle.detracer_T(n, mono)
    D = oracle.dtensor(n, r)
    blk = D[oracle.ncoef(n - 1, oracle.SYM) if n else 0:]
    R = np.linalg.norm(r)
    np.testing.assert_allclose((-1) ** n * R ** (-2 * n - 1) * T, blk, rtol=1e-10,
                               atol=1e-12 * np.abs(blk).max())
