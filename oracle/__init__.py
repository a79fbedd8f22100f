"""FP64 CPU oracle for the Cartesian FMM operators (arXiv:1811.06332).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow restatement of the
paper's equations against which the CUDA library is checked.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import it; the library under ``paper_1811_06332_gb300/`` never does, and the
two share no code.

Every function here marshals numpy arrays into ``fmm_oracle.c``; the arithmetic
is all in that C file, each routine citing the equation it restates:

* ``dtensor``      -- Eq. traceless grad + Eq. Detracer3 (App. A)
* ``detracer_T``   -- Eq. Detracer (App. A); ``detracer_D`` = T/(2n-1)!!
* ``p2m``          -- Eq. P2M (Sec. 2.1), sign (-r_a)^n as in App. B
* ``m2m``          -- Eq. M2M / M2M part 2 (Sec. 2.1)
* ``m2l``          -- Eq. M2L (Sec. 2.1)
* ``l2l``          -- Eq. L2L (Sec. 2.1)
* ``l2p``          -- Eq. L2P (Sec. 2.1)
* ``direct``       -- Eq. PhiAB (App. B), O(N^2)
* ``fmm_uniform``  -- App. C on a uniform octree with the standard
                      (Chebyshev distance >= 2) separation criterion
* ``fmm_adaptive`` -- App. C on an adaptive octree: MAC
                      theta |z_A - z_B| > r_A + r_B, dual-tree traversal,
                      optionally with one M2L order per pair
* ``adaptive_pairs`` -- per-pair features and truncation-error labels for
                      choosing each pair's order (an addition to the paper)
* ``mlp``          -- the order-choosing MLP: forward, backward, Adam, BF16
                      rounding, order selection (numpy, FP64)

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, finite differences, identities,
the paper's worked example and storage table, direct sums).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

SYM = 0
TRACELESS = 1
TG = 2          # fmm_uniform only: symmetric multipoles, traceless locals (the TG variant)

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_ncoef.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_ncoef.restype = ctypes.c_int
        L.orc_indices.argtypes = [ctypes.c_int, ctypes.c_int, _ip]
        L.orc_indices.restype = ctypes.c_int
        L.orc_expand_traceless.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_detracer_T.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_detracer_D.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_dtensor.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_dtensor_batch.argtypes = [ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp, _dp]
        L.orc_p2m.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_m2m.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        L.orc_m2l.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        L.orc_m2l_D.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        L.orc_m2l_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp, _dp,
                                    _dp, ctypes.c_int]
        L.orc_l2l.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        L.orc_l2p.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
        L.orc_direct.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int64, _i64p,
                                 _dp, _dp, _dp, _dp]
        L.orc_fmm_uniform.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int64, _i64p, _dp, _dp, _dp, _dp]
        L.orc_fmm_uniform.restype = ctypes.c_int
        L.orc_fmm_adaptive.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int64, _i64p, _dp, _dp, _dp, _dp,
                                       _i64p]
        L.orc_fmm_adaptive.restype = ctypes.c_int
        L.orc_fmm_adaptive_orders.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_int64, _i64p, _dp, _dp, _dp, _dp, _i64p]
        L.orc_fmm_adaptive_orders.restype = ctypes.c_int
        L.orc_adaptive_pairs.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]
        L.orc_adaptive_pairs.restype = ctypes.c_int64
        L.orc_ncols_features.restype = ctypes.c_int
        L.orc_pair_error.argtypes = [ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int,
                                     _dp, _dp, _dp]
        L.orc_pair_error.restype = ctypes.c_double
        L.orc_adaptive_tree.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_adaptive_tree.restype = ctypes.c_int64
        L.orc_ncols_labels.restype = ctypes.c_int
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_m2m_fused.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        L.orc_fmm_btree.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int64, _i64p, _dp, _dp, _dp, _dp, _i64p]
        L.orc_fmm_btree.restype = ctypes.c_int
        L.orc_btree.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_btree.restype = ctypes.c_int64
        for name in ("orc_fmm_adaptive_ap", "orc_fmm_adaptive_com"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                          ctypes.c_int64, _i64p, _dp, _dp, _dp, _dp, _i64p]
            f.restype = ctypes.c_int
        L.orc_adaptive_tree_com.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int64,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_adaptive_tree_com.restype = ctypes.c_int64
        L.orc_p2m_dipole.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64] + [_dp] * 8
        L.orc_direct_dipole.argtypes = [ctypes.c_int64] + [_dp] * 7 + [ctypes.c_int64, _i64p] + [_dp] * 4
        L.orc_fmm_uniform_dipole.argtypes = [ctypes.c_int64] + [_dp] * 7 + [ctypes.c_int] * 3 + \
            [ctypes.c_int64, _i64p] + [_dp] * 4
        L.orc_fmm_uniform_dipole.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def ncoef(p: int, basis: int) -> int:
    return lib().orc_ncoef(p, basis)


def indices(p: int, basis: int) -> np.ndarray:
    """Multi-indices (ncoef, 3) in storage order."""
    nc = ncoef(p, basis)
    out = np.zeros((nc, 3), dtype=np.int32)
    lib().orc_indices(p, basis, out.ctypes.data_as(_ip))
    return out


def expand_traceless(p: int, A: np.ndarray) -> np.ndarray:
    A = _f64(A)
    out = np.zeros(ncoef(p, SYM))
    lib().orc_expand_traceless(p, _d(A), _d(out))
    return out


def detracer_T(n: int, A: np.ndarray) -> np.ndarray:
    A = _f64(A)
    out = np.zeros((n + 1) * (n + 2) // 2)
    lib().orc_detracer_T(n, _d(A), _d(out))
    return out


def detracer_D(n: int, A: np.ndarray) -> np.ndarray:
    A = _f64(A)
    out = np.zeros((n + 1) * (n + 2) // 2)
    lib().orc_detracer_D(n, _d(A), _d(out))
    return out


def dtensor(p: int, r) -> np.ndarray:
    r = _f64(r)
    out = np.zeros(ncoef(p, SYM))
    lib().orc_dtensor(p, _d(r), _d(out))
    return out


def dtensor_batch(p: int, r: np.ndarray) -> np.ndarray:
    """r: (3, n) -> D: (ns, n)."""
    r = _f64(r)
    n = r.shape[1]
    out = np.zeros((ncoef(p, SYM), n))
    rx, ry, rz = _f64(r[0]), _f64(r[1]), _f64(r[2])
    lib().orc_dtensor_batch(p, n, _d(rx), _d(ry), _d(rz), _d(out))
    return out


def p2m(p: int, basis: int, x, y, z, q, zc) -> np.ndarray:
    x, y, z, q, zc = (_f64(v) for v in (x, y, z, q, zc))
    out = np.zeros(ncoef(p, basis))
    lib().orc_p2m(p, basis, len(x), _d(x), _d(y), _d(z), _d(q), _d(zc), _d(out))
    return out


def m2m_fused(p: int, M: np.ndarray, delta) -> np.ndarray:
    """Traceless M2M in the fused form of Eq. Detracer2 (traceless storage)."""
    M, delta = _f64(M), _f64(delta)
    out = np.zeros(ncoef(p, TRACELESS))
    lib().orc_m2m_fused(p, _d(M), _d(delta), _d(out))
    return out


def p2m_dipole(p: int, basis: int, x, y, z, px, py, pz, zc) -> np.ndarray:
    """Multipole of point dipoles (App. B): the pure dipole M_{e_i} = -p_i
    of each, shifted by M2M from x_a to zc."""
    x, y, z, px, py, pz, zc = (_f64(v) for v in (x, y, z, px, py, pz, zc))
    out = np.zeros(ncoef(p, basis))
    lib().orc_p2m_dipole(p, basis, len(x), _d(x), _d(y), _d(z), _d(px), _d(py), _d(pz), _d(zc), _d(out))
    return out


def direct_dipole(x, y, z, q, px, py, pz, targets=None):
    """O(N^2) FP64 sum over charges and point dipoles: pot = -Phi,
    acc = grad Phi (Phi the paper's positive potential)."""
    x, y, z, q, px, py, pz = (_f64(v) for v in (x, y, z, q, px, py, pz))
    n = len(x)
    if targets is None:
        nt, tp = n, None
    else:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = len(targets), targets.ctypes.data_as(_i64p)
    pot, ax, ay, az = (np.zeros(nt) for _ in range(4))
    lib().orc_direct_dipole(n, _d(x), _d(y), _d(z), _d(q), _d(px), _d(py), _d(pz), nt, tp, _d(pot), _d(ax),
                            _d(ay), _d(az))
    return pot, np.stack([ax, ay, az])


def fmm_uniform_dipole(x, y, z, q, px, py, pz, depth: int, p: int, basis: int, sample=None):
    """Uniform-octree FMM with point dipoles beside the charges."""
    x, y, z, q, px, py, pz = (_f64(v) for v in (x, y, z, q, px, py, pz))
    n = len(x)
    if sample is None:
        ns, sp, nout = -1, None, n
    else:
        sample = np.ascontiguousarray(sample, dtype=np.int64)
        ns, sp, nout = len(sample), sample.ctypes.data_as(_i64p), len(sample)
    pot, ax, ay, az = (np.zeros(nout) for _ in range(4))
    rc = lib().orc_fmm_uniform_dipole(n, _d(x), _d(y), _d(z), _d(q), _d(px), _d(py), _d(pz), depth, p, basis,
                                      ns, sp, _d(pot), _d(ax), _d(ay), _d(az))
    if rc != 0:
        raise ValueError("orc_fmm_uniform_dipole rejected its arguments")
    return pot, np.stack([ax, ay, az])


def m2m(p: int, basis: int, M: np.ndarray, delta) -> np.ndarray:
    M, delta = _f64(M), _f64(delta)
    out = np.zeros(ncoef(p, basis))
    lib().orc_m2m(p, basis, _d(M), _d(delta), _d(out))
    return out


def m2l(p: int, basis: int, M: np.ndarray, r) -> np.ndarray:
    M, r = _f64(M), _f64(r)
    out = np.zeros(ncoef(p, basis))
    lib().orc_m2l(p, basis, _d(M), _d(r), _d(out))
    return out


def m2l_D(p: int, basis: int, M: np.ndarray, D: np.ndarray) -> np.ndarray:
    M, D = _f64(M), _f64(D)
    out = np.zeros(ncoef(p, basis))
    lib().orc_m2l_D(p, basis, _d(M), _d(D), _d(out))
    return out


def m2l_batch(p: int, basis: int, M: np.ndarray, r: np.ndarray) -> np.ndarray:
    """M: (ncoef, n), r: (3, n) -> L: (ncoef, n)."""
    M = _f64(M)
    n = M.shape[1]
    rx, ry, rz = _f64(r[0]), _f64(r[1]), _f64(r[2])
    out = np.zeros((ncoef(p, basis), n))
    lib().orc_m2l_batch(p, basis, n, _d(M), _d(rx), _d(ry), _d(rz), _d(out), 0)
    return out


def l2l(p: int, basis: int, L: np.ndarray, delta) -> np.ndarray:
    L, delta = _f64(L), _f64(delta)
    out = np.zeros(ncoef(p, basis))
    lib().orc_l2l(p, basis, _d(L), _d(delta), _d(out))
    return out


def l2p(p: int, basis: int, L: np.ndarray, rb) -> np.ndarray:
    """Returns [Phi, dPhi/dx, dPhi/dy, dPhi/dz] (paper's positive sign)."""
    L, rb = _f64(L), _f64(rb)
    out = np.zeros(4)
    lib().orc_l2p(p, basis, _d(L), _d(rb), _d(out))
    return out


def direct(x, y, z, q, targets=None):
    """O(N^2) FP64 sum: pot = -sum q/r, acc = sum q (x_j - x_i)/r^3."""
    x, y, z, q = (_f64(v) for v in (x, y, z, q))
    n = len(x)
    if targets is None:
        nt, tp = n, None
    else:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = len(targets), targets.ctypes.data_as(_i64p)
    pot, ax, ay, az = (np.zeros(nt) for _ in range(4))
    lib().orc_direct(n, _d(x), _d(y), _d(z), _d(q), nt, tp, _d(pot), _d(ax), _d(ay), _d(az))
    return pot, np.stack([ax, ay, az])


def fmm_uniform(x, y, z, q, depth: int, p: int, basis: int, sample=None):
    """Uniform-octree FMM (App. C); returns pot (n,) and acc (3, n).

    With ``sample`` (int64 indices) only those particles are evaluated."""
    x, y, z, q = (_f64(v) for v in (x, y, z, q))
    n = len(x)
    if sample is None:
        ns, sp, nout = -1, None, n
    else:
        sample = np.ascontiguousarray(sample, dtype=np.int64)
        ns, sp, nout = len(sample), sample.ctypes.data_as(_i64p), len(sample)
    pot, ax, ay, az = (np.zeros(nout) for _ in range(4))
    rc = lib().orc_fmm_uniform(n, _d(x), _d(y), _d(z), _d(q), depth, p, basis, ns, sp,
                               _d(pot), _d(ax), _d(ay), _d(az))
    if rc != 0:
        raise ValueError("orc_fmm_uniform rejected its arguments")
    return pot, np.stack([ax, ay, az])


def fmm_adaptive(x, y, z, q, max_leaf: int, theta: float, p: int, basis: int, sample=None, pair_orders=None):
    """Adaptive-octree FMM with the dual-tree traversal and MAC of App. C.

    Returns pot (n,), acc (3, n) and stats {nodes, m2l_pairs, p2p_pairs,
    leaves}; with ``sample`` only those particles are evaluated.  With
    ``pair_orders`` (one int per M2L pair, in the order of
    ``adaptive_pairs``) each pair's M2L is truncated at its own order."""
    x, y, z, q = (_f64(v) for v in (x, y, z, q))
    n = len(x)
    if sample is None:
        ns, sp, nout = -1, None, n
    else:
        sample = np.ascontiguousarray(sample, dtype=np.int64)
        ns, sp, nout = len(sample), sample.ctypes.data_as(_i64p), len(sample)
    pot, ax, ay, az = (np.zeros(nout) for _ in range(4))
    st = np.zeros(5, dtype=np.int64)
    if pair_orders is None:
        po, npo = None, 0
    else:
        pair_orders = np.ascontiguousarray(pair_orders, dtype=np.int8)
        po, npo = pair_orders.ctypes.data, len(pair_orders)
    rc = lib().orc_fmm_adaptive_orders(n, _d(x), _d(y), _d(z), _d(q), max_leaf, float(theta), p, basis, po, npo,
                                       ns, sp, _d(pot), _d(ax), _d(ay), _d(az), st.ctypes.data_as(_i64p))
    if rc != 0:
        raise ValueError("orc_fmm_adaptive rejected its arguments (%d)" % rc)
    keys = ("nodes", "m2l_pairs", "p2p_pairs", "leaves", "covered_pairs")
    return pot, np.stack([ax, ay, az]), dict(zip(keys, st.tolist()))


NFEAT = 12      # features per M2L pair (see fmm_oracle.c)
NLABEL = 9      # labels per pair: orders 2..10


def adaptive_pairs(x, y, z, q, max_leaf: int, theta: float, features=True, labels=False):
    """M2L pairs of the adaptive tree, ordered by (target, source).

    Returns (target, source) node indices and, on request, the (npair, 12)
    features and (npair, 9) labels (log10 force error of the pair's M2L at
    orders 2..10 relative to the total force at the target's particles)
    defined in fmm_oracle.c."""
    x, y, z, q = (_f64(v) for v in (x, y, z, q))
    n = len(x)
    L = lib()
    np_ = L.orc_adaptive_pairs(n, _d(x), _d(y), _d(z), _d(q), max_leaf, float(theta), 0, None, None, None, None)
    if np_ < 0:
        raise ValueError("orc_adaptive_pairs rejected its arguments")
    tgt = np.zeros(np_, dtype=np.int64)
    src = np.zeros(np_, dtype=np.int64)
    feat = np.zeros((np_, NFEAT)) if features else None
    lab = np.zeros((np_, NLABEL)) if labels else None
    got = L.orc_adaptive_pairs(n, _d(x), _d(y), _d(z), _d(q), max_leaf, float(theta), np_, tgt.ctypes.data,
                               src.ctypes.data, feat.ctypes.data if features else None,
                               lab.ctypes.data if labels else None)
    assert got == np_
    return tgt, src, feat, lab


def pair_error(p, src_xyzq, zA, zB, targets):
    """Relative force error of the order-p M2L + L2P of the source particles
    (P2M about zA) at the target points (<= 64) against their exact field."""
    xa, ya, za, qa = (_f64(v) for v in src_xyzq)
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(-1, 3).T)
    zA, zB = _f64(zA), _f64(zB)
    tx, ty, tz = (np.ascontiguousarray(t[k]) for k in range(3))
    e = lib().orc_pair_error(p, len(xa), _d(xa), _d(ya), _d(za), _d(qa), _d(zA), _d(zB), t.shape[1], _d(tx),
                             _d(ty), _d(tz))
    if e < 0:
        raise ValueError("orc_pair_error rejected its arguments")
    return e


def btree(x, y, z, max_leaf: int):
    """The binary median-split tree (App. C): (nn, 4) centre and radius,
    (nn, 2) sorted-position ranges, the sorted order, each node's parent."""
    x, y, z = (_f64(v) for v in (x, y, z))
    n = len(x)
    L = lib()
    nn = L.orc_btree(n, _d(x), _d(y), _d(z), max_leaf, 0, None, None, None, None)
    zr = np.zeros((nn, 4))
    rg = np.zeros((nn, 2), dtype=np.int64)
    order = np.zeros(n, dtype=np.int64)
    par = np.zeros(nn, dtype=np.int64)
    assert L.orc_btree(n, _d(x), _d(y), _d(z), max_leaf, nn, zr.ctypes.data, rg.ctypes.data, order.ctypes.data,
                       par.ctypes.data) == nn
    return zr, rg, order, par


def fmm_btree(x, y, z, q, max_leaf: int, theta: float, p: int, basis: int, sample=None):
    """The FMM on the binary median-split tree (App. C)."""
    x, y, z, q = (_f64(v) for v in (x, y, z, q))
    n = len(x)
    if sample is None:
        ns, sp, nout = -1, None, n
    else:
        sample = np.ascontiguousarray(sample, dtype=np.int64)
        ns, sp, nout = len(sample), sample.ctypes.data_as(_i64p), len(sample)
    pot, ax, ay, az = (np.zeros(nout) for _ in range(4))
    st = np.zeros(5, dtype=np.int64)
    rc = lib().orc_fmm_btree(n, _d(x), _d(y), _d(z), _d(q), max_leaf, float(theta), p, basis, ns, sp, _d(pot),
                             _d(ax), _d(ay), _d(az), st.ctypes.data_as(_i64p))
    if rc != 0:
        raise ValueError("orc_fmm_btree rejected its arguments (%d)" % rc)
    keys = ("nodes", "m2l_pairs", "p2p_pairs", "leaves", "covered_pairs")
    return pot, np.stack([ax, ay, az]), dict(zip(keys, st.tolist()))


def adaptive_tree(x, y, z, max_leaf: int, parents=False, com_q=None):
    """Nodes of the adaptive octree: (nn, 4) centre and radius, (nn, 2)
    sorted-position ranges, the sorted order of the particles and, on
    request, each node's parent (-1 for the root).  With com_q (charges)
    the centres are centres of mass (the AP variant's geometry)."""
    x, y, z = (_f64(v) for v in (x, y, z))
    n = len(x)
    L = lib()
    if com_q is None:
        call = lambda cap, *a: L.orc_adaptive_tree(n, _d(x), _d(y), _d(z), max_leaf, cap, *a)  # noqa: E731
    else:
        qq = _f64(com_q)
        call = lambda cap, *a: L.orc_adaptive_tree_com(n, _d(x), _d(y), _d(z), _d(qq), max_leaf, cap, *a)  # noqa: E731
    nn = call(0, None, None, None, None)
    zr = np.zeros((nn, 4))
    rg = np.zeros((nn, 2), dtype=np.int64)
    order = np.zeros(n, dtype=np.int64)
    par = np.zeros(nn, dtype=np.int64)
    got = call(nn, zr.ctypes.data, rg.ctypes.data, order.ctypes.data, par.ctypes.data)
    assert got == nn
    return (zr, rg, order, par) if parents else (zr, rg, order)


def _adaptive_variant(fn, x, y, z, q, max_leaf, theta, p, sample):
    x, y, z, q = (_f64(v) for v in (x, y, z, q))
    n = len(x)
    if sample is None:
        ns, sp, nout = -1, None, n
    else:
        sample = np.ascontiguousarray(sample, dtype=np.int64)
        ns, sp, nout = len(sample), sample.ctypes.data_as(_i64p), len(sample)
    pot, ax, ay, az = (np.zeros(nout) for _ in range(4))
    st = np.zeros(5, dtype=np.int64)
    rc = fn(n, _d(x), _d(y), _d(z), _d(q), max_leaf, float(theta), p, ns, sp, _d(pot), _d(ax), _d(ay), _d(az),
            st.ctypes.data_as(_i64p))
    if rc != 0:
        raise ValueError("adaptive FMM rejected its arguments (%d)" % rc)
    keys = ("nodes", "m2l_pairs", "p2p_pairs", "leaves", "covered_pairs")
    return pot, np.stack([ax, ay, az]), dict(zip(keys, st.tolist()))


def fmm_adaptive_ap(x, y, z, q, max_leaf: int, theta: float, p: int, sample=None):
    """The AP variant (Sec. 3): traceless, centre-of-mass centres, dipole 0,
    gradient only (pot returned as 0)."""
    return _adaptive_variant(lib().orc_fmm_adaptive_ap, x, y, z, q, max_leaf, theta, p, sample)


def fmm_adaptive_com(x, y, z, q, max_leaf: int, theta: float, p: int, sample=None):
    """The traceless adaptive FMM about centres of mass, dipole kept and the
    potential evaluated (the FT variant on the AP tree)."""
    return _adaptive_variant(lib().orc_fmm_adaptive_com, x, y, z, q, max_leaf, theta, p, sample)
