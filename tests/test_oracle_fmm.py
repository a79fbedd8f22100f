"""Pins for the oracle's uniform-octree FMM (App. C) against the O(N^2)
direct sum (Eq. PhiAB), CPU only."""
import numpy as np
import pytest

import oracle
from paper_1811_06332_gb300 import inputs

SYM, TL = oracle.SYM, oracle.TRACELESS


def rel_force_err(acc, ref):
    return float(np.sqrt(((acc - ref) ** 2).sum() / (ref ** 2).sum()))


@pytest.fixture(scope="module")
def cfg1():
    n = 4096
    x, y, z = inputs.uniform_cube(n, 1)
    q = inputs.masses_open_unit(n, 1)
    pot, acc = oracle.direct(x, y, z, q)
    return x, y, z, q, pot, acc


def test_small_uniform_workload_p4(cfg1):
    x, y, z, q, pot_ref, acc_ref = cfg1
    pot, acc = oracle.fmm_uniform(x, y, z, q, depth=3, p=4, basis=SYM)
    e = rel_force_err(acc, acc_ref)
    assert e < 3e-3, e
    assert np.linalg.norm(pot - pot_ref) / np.linalg.norm(pot_ref) < 2e-4


def test_error_decreases_with_p(cfg1):
    x, y, z, q, _, acc_ref = cfg1
    errs = [rel_force_err(oracle.fmm_uniform(x, y, z, q, 3, p, TL)[1], acc_ref) for p in (2, 4, 6, 8)]
    assert all(b < 0.5 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 5e-4


def test_traceless_equals_symmetric(cfg1):
    x, y, z, q, _, _ = cfg1
    ps, as_ = oracle.fmm_uniform(x, y, z, q, 3, 6, SYM)
    pt, at = oracle.fmm_uniform(x, y, z, q, 3, 6, TL)
    assert np.abs(pt - ps).max() < 1e-12 * np.abs(ps).max()
    assert np.abs(at - as_).max() < 1e-11 * np.abs(as_).max()


@pytest.mark.parametrize("depth", [0, 1])
def test_shallow_tree_is_direct_sum(cfg1, depth):
    x, y, z, q, pot_ref, acc_ref = cfg1
    pot, acc = oracle.fmm_uniform(x, y, z, q, depth, 4, SYM)
    np.testing.assert_allclose(pot, pot_ref, rtol=1e-12)
    np.testing.assert_allclose(acc, acc_ref, rtol=1e-9, atol=1e-9 * np.abs(acc_ref).max())


def test_sampled_matches_full(cfg1):
    x, y, z, q, _, _ = cfg1
    pot, acc = oracle.fmm_uniform(x, y, z, q, 3, 5, TL)
    s = np.array([0, 7, 100, 4095, 2048])
    ps, as_ = oracle.fmm_uniform(x, y, z, q, 3, 5, TL, sample=s)
    np.testing.assert_array_equal(ps, pot[s])
    np.testing.assert_array_equal(as_, acc[:, s])


def test_ragged_and_empty_leaves():
    # 37 particles in a depth-3 tree: most leaves empty, a few crowded
    x, y, z = inputs.uniform_cube(37, 9)
    x[:10] *= 0.1; y[:10] *= 0.1; z[:10] *= 0.1
    q = inputs.masses_open_unit(37, 9)
    pot_ref, acc_ref = oracle.direct(x, y, z, q)
    pot, acc = oracle.fmm_uniform(x, y, z, q, 3, 8, TL)
    assert rel_force_err(acc, acc_ref) < 2e-4


@pytest.mark.parametrize("p", [3, 6])
def test_tg_variant_equals_symmetric_and_traceless(p):
    """The TG variant (symmetric multipoles, traceless locals; Sec. 3) gives
    the field of the SYM and FT variants (equal in exact arithmetic)."""
    n, depth = 2500, 3
    x, y, z = inputs.uniform_cube(n, 81)
    q = inputs.masses_open_unit(n, 81)
    res = [oracle.fmm_uniform(x, y, z, q, depth, p, b) for b in (oracle.SYM, oracle.TRACELESS, oracle.TG)]
    for pot, acc in res[1:]:
        assert np.linalg.norm(pot - res[0][0]) <= 1e-13 * np.linalg.norm(res[0][0])
        assert np.linalg.norm(acc - res[0][1]) <= 1e-13 * np.linalg.norm(res[0][1])
