"""Pins for the oracle's adaptive-octree FMM (App. C: MAC, dual-tree
traversal), CPU only."""
import numpy as np
import pytest

import oracle
from paper_1811_06332_gb300 import inputs


@pytest.fixture(scope="module")
def plummer():
    n = 6000
    x, y, z = inputs.plummer(n, 4)
    q = inputs.masses_equal(n)
    pot, acc = oracle.direct(x, y, z, q)
    return x, y, z, q, pot, acc


def err(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def test_theta_zero_is_direct_sum(plummer):
    x, y, z, q, pref, aref = plummer
    pot, acc, st = oracle.fmm_adaptive(x, y, z, q, 32, 0.0, 4, 0)
    assert st["m2l_pairs"] == 0
    np.testing.assert_allclose(pot, pref, rtol=1e-12)
    assert err(acc, aref) < 1e-12


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.7])
def test_lists_cover_every_particle_pair_once(plummer, theta):
    x, y, z, q, _, _ = plummer
    _, _, st = oracle.fmm_adaptive(x, y, z, q, 32, theta, 2, 0)
    assert st["covered_pairs"] == len(x) ** 2
    assert st["m2l_pairs"] > 0


@pytest.mark.parametrize("basis", [0, 1])
def test_error_decreases_with_p_and_theta(plummer, basis):
    x, y, z, q, _, aref = plummer
    e = {(th, p): err(oracle.fmm_adaptive(x, y, z, q, 64, th, p, basis)[1], aref)
         for th in (0.4, 0.7) for p in (2, 4, 6, 8)}
    for th in (0.4, 0.7):
        assert e[(th, 2)] > e[(th, 4)] > e[(th, 6)] > e[(th, 8)]
    for p in (2, 4, 6, 8):
        assert e[(0.4, p)] < e[(0.7, p)]
    assert e[(0.4, 8)] < 3e-6


def test_traceless_equals_symmetric_and_sampled(plummer):
    x, y, z, q, _, _ = plummer
    ps, as_, _ = oracle.fmm_adaptive(x, y, z, q, 64, 0.5, 6, 0)
    pt, at, _ = oracle.fmm_adaptive(x, y, z, q, 64, 0.5, 6, 1)
    assert np.abs(pt - ps).max() < 1e-11 * np.abs(ps).max()
    assert np.abs(at - as_).max() < 1e-10 * np.abs(as_).max()
    s = np.array([0, 11, 3000, 5999])
    pss, ass, _ = oracle.fmm_adaptive(x, y, z, q, 64, 0.5, 6, 1, sample=s)
    np.testing.assert_array_equal(pss, pt[s])
    np.testing.assert_array_equal(ass, at[:, s])


def test_single_leaf_and_duplicates():
    x, y, z = inputs.uniform_cube(40, 3)
    x[5] = x[6]; y[5] = y[6]; z[5] = z[6]      # coincident pair: skipped like the direct sum
    q = inputs.masses_open_unit(40, 3)
    pref, aref = oracle.direct(x, y, z, q)
    pot, acc, st = oracle.fmm_adaptive(x, y, z, q, 64, 0.5, 4, 0)
    assert st["nodes"] == 1 and st["p2p_pairs"] == 1
    np.testing.assert_allclose(pot, pref, rtol=1e-13)
    assert err(acc, aref) < 1e-13
