"""GPU parity of the operator-level entry points against the FP64 oracle.

Tolerances (normwise relative error per result):
  * FP64 kernels: 1e-12 per item and rank (expansions) or per item (fields);
    on random-sign coefficients the condition-aware form below, at 1e-12;
  * FP32 D-tensor: 1e-5 for p <= 8 and 5e-5 for p = 9, 10 (normwise per
    rank; the recurrence loses a few bits to cancellation at high rank);
  * FP32 per-pair M2L: per item and rank, max |L_gpu - L_ref| <= 1e-5 x
    max sum_m |M_m/m! D_{n+m}| (condition-aware: random-sign coefficients
    make single L_n cancel, and at symmetric offsets a D component such as
    3x^2 - r^2 vanishes exactly in the oracle but only to rounding in FP32,
    so a bound relative to |L_n| would measure the input, not the kernel);
    on physical multipoles also normwise per rank <= 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1811_06332_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    from paper_1811_06332_gb300 import fmm
    return fmm


def g(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def rank_err(got, ref, p, basis):
    """max over items and ranks of ||got - ref|| / ||ref|| (rank block)."""
    idx = oracle.indices(p, basis).sum(1)
    worst = 0.0
    for j in range(p + 1):
        sel = idx == j
        num = np.linalg.norm(got[sel] - ref[sel], axis=0)
        den = np.linalg.norm(ref[sel], axis=0)
        ok = den > 0
        if ok.any():
            worst = max(worst, float((num[ok] / den[ok]).max()))
        assert np.all(num[~ok] == 0)
    return worst


def abs_terms(p, basis, M, r):
    """sum_m |M_m/m!| |D_{n+m}(r)| for every output component (oracle, with
    traceless multipoles expanded to full symmetric form first)."""
    n = M.shape[1]
    out = np.zeros((oracle.ncoef(p, basis), n))
    sel = None
    if basis:
        idx_s = [tuple(v) for v in oracle.indices(p, 0)]
        sel = [idx_s.index(tuple(v)) for v in oracle.indices(p, 1)]
    for i in range(n):
        Mf = oracle.expand_traceless(p, M[:, i]) if basis else M[:, i]
        D = np.abs(oracle.dtensor(p, r[:, i]))
        L = oracle.m2l_D(p, 0, np.abs(Mf), D)
        out[:, i] = L[sel] if basis else L
    return out


def cond_err(p, basis, got, ref, den):
    """per item and rank: max |got - ref| / max sum|terms| (condition-aware)."""
    num = np.abs(got - ref)
    rank = oracle.indices(p, basis).sum(1)
    e = 0.0
    for j in range(p + 1):
        sel = rank == j
        e = max(e, float((num[sel].max(0) / den[sel].max(0)).max()))
    return e


def pair_offsets(n, seed):
    r, _, _ = inputs.m2l_pairs(n, seed)
    return r


@pytest.mark.parametrize("p", list(range(0, 11)))
def test_dtensor(F, p):
    n = 1000 + 37
    r = pair_offsets(n, 10 + p) + inputs.random_coefficients(3, n, 5, 1) * 0.4
    ref = oracle.dtensor_batch(p, r)
    for prec, tol in ((F.FP64, 1e-12), (F.FP32, 1e-5 if p <= 8 else 5e-5)):
        D = torch.zeros((oracle.ncoef(p, 0), n), device=DEV,
                        dtype=torch.float64 if prec == F.FP64 else torch.float32)
        F.fmm_op_dtensor(p, prec, g(r), D)
        e = rank_err(D.double().cpu().numpy(), ref, p, 0)
        assert e < tol, (prec, e)


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("p", list(range(0, 11)))
def test_m2l_pair_random(F, p, basis):
    n = 700 + 53   # several blocks of 128 and a ragged tail
    nc = oracle.ncoef(p, basis)
    r = pair_offsets(n, 20 + p)
    M = inputs.random_coefficients(nc, n, 30 + p)
    ref = oracle.m2l_batch(p, basis, M, r)
    den = abs_terms(p, basis, M, r)
    L = torch.zeros((nc, n), device=DEV, dtype=torch.float64)
    F.fmm_op_m2l(p, basis, F.FP64, g(M), g(r), L)
    assert cond_err(p, basis, L.cpu().numpy(), ref, den) < 1e-12
    # accumulate mode adds
    F.fmm_op_m2l(p, basis, F.FP64, g(M), g(r), L, accumulate=True)
    assert cond_err(p, basis, L.cpu().numpy(), 2 * ref, 2 * den) < 1e-12
    # FP32: compare with the oracle run on the float-rounded input
    M32 = M.astype(np.float32)
    ref32 = oracle.m2l_batch(p, basis, M32.astype(np.float64), r)
    L32 = torch.zeros((nc, n), device=DEV, dtype=torch.float32)
    F.fmm_op_m2l(p, basis, F.FP32, g(M32, torch.float32), g(r), L32)
    den32 = abs_terms(p, basis, M32.astype(np.float64), r)
    assert cond_err(p, basis, L32.double().cpu().numpy(), ref32, den32) < 1e-5


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("p", [2, 5, 8, 10])
def test_m2l_pair_physical_multipoles(F, p, basis):
    """Multipoles of 16 unit-mass particles per side-1 cell (the micro-benchmark
    workload): GPU P2M -> GPU M2L against oracle P2M -> oracle M2L."""
    n = 300 + 11
    r, src, q = inputs.m2l_pairs(n, 40 + p)
    nc = oracle.ncoef(p, basis)
    Mref = np.stack([oracle.p2m(p, basis, src[0, :, i], src[1, :, i], src[2, :, i], q[:, i], np.zeros(3))
                     for i in range(n)], 1)
    Lref = oracle.m2l_batch(p, basis, Mref, r)
    per = src.shape[1]
    start = torch.arange(0, (n + 1) * per, per, device=DEV, dtype=torch.int64)
    xs = [g(src[d].T.reshape(-1)) for d in range(3)]
    qs = g(q.T.reshape(-1))
    M = torch.zeros((nc, n), device=DEV, dtype=torch.float64)
    F.fmm_op_p2m(p, basis, start, xs[0], xs[1], xs[2], qs, torch.zeros((3, n), device=DEV, dtype=torch.float64), M)
    assert rank_err(M.cpu().numpy(), Mref, p, basis) < 1e-12
    L = torch.zeros((nc, n), device=DEV, dtype=torch.float64)
    F.fmm_op_m2l(p, basis, F.FP64, M, g(r), L)
    assert rank_err(L.cpu().numpy(), Lref, p, basis) < 1e-12
    M32 = M.float()
    L32 = torch.zeros((nc, n), device=DEV, dtype=torch.float32)
    F.fmm_op_m2l(p, basis, F.FP32, M32, g(r), L32)
    ref32 = oracle.m2l_batch(p, basis, M32.double().cpu().numpy(), r)
    assert rank_err(L32.double().cpu().numpy(), ref32, p, basis) < (1e-5 if p <= 8 else 5e-5)


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("p", [0, 1, 4, 8, 10])
def test_p2m_m2m_l2l_l2p(F, p, basis):
    rng = np.random.default_rng(p + 7 * basis)
    ncell = 97
    counts = rng.integers(0, 20, ncell)
    counts[3] = 0   # an empty cell
    start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    npart = int(start[-1])
    cen = rng.uniform(-1, 1, (3, ncell))
    pos = np.repeat(cen, counts, axis=1) + rng.uniform(-0.25, 0.25, (3, npart))
    q = rng.uniform(0.1, 1, npart)
    nc = oracle.ncoef(p, basis)
    Mref = np.zeros((nc, ncell))
    for c in range(ncell):
        s, e = start[c], start[c + 1]
        Mref[:, c] = oracle.p2m(p, basis, pos[0, s:e], pos[1, s:e], pos[2, s:e], q[s:e], cen[:, c])
    M = torch.full((nc, ncell), 7.0, device=DEV, dtype=torch.float64)  # overwritten
    F.fmm_op_p2m(p, basis, g(start, torch.int64), g(pos[0]), g(pos[1]), g(pos[2]), g(q), g(cen), M)
    assert rank_err(M.cpu().numpy(), Mref, p, basis) < 1e-12
    # M2M with a general shift, accumulating
    delta = rng.uniform(-0.3, 0.3, (3, ncell))
    base = inputs.random_coefficients(nc, ncell, 3)
    ref = base + np.stack([oracle.m2m(p, basis, Mref[:, c], delta[:, c]) for c in range(ncell)], 1)
    Mp = g(base)
    F.fmm_op_m2m(p, basis, M, g(delta), Mp)
    assert rank_err(Mp.cpu().numpy(), ref, p, basis) < 1e-12
    # L2L and L2P on trace-free local expansions (M2L of the multipoles)
    rr = pair_offsets(ncell, 77) * 2.0
    Lref = oracle.m2l_batch(p, basis, Mref, rr)
    Lg = torch.zeros((nc, ncell), device=DEV, dtype=torch.float64)
    F.fmm_op_m2l(p, basis, F.FP64, M, g(rr), Lg)
    ref2 = np.stack([oracle.l2l(p, basis, Lref[:, c], delta[:, c]) for c in range(ncell)], 1)
    Lc = torch.zeros_like(Lg)
    F.fmm_op_l2l(p, basis, Lg, g(delta), Lc)
    assert rank_err(Lc.cpu().numpy(), ref2, p, basis) < 1e-12
    ref3 = np.stack([oracle.l2p(p, basis, Lref[:, c], delta[:, c]) for c in range(ncell)], 1)
    out = torch.zeros((4, ncell), device=DEV, dtype=torch.float64)
    F.fmm_op_l2p(p, basis, Lg, g(delta), out)
    o = out.cpu().numpy()
    assert np.abs(o[0] - ref3[0]).max() <= 1e-12 * np.abs(ref3[0]).max()
    gn = np.linalg.norm(ref3[1:], axis=0)
    dn = np.linalg.norm(o[1:] - ref3[1:], axis=0)
    assert np.all(dn[gn == 0] == 0)     # empty cells, and p = 0 (no gradient terms)
    if (gn > 0).any():
        assert (dn[gn > 0] / gn[gn > 0]).max() < 1e-12

    # FP32 forms of M2M, L2L and L2P (storage and arithmetic in FP32), against
    # the oracle run on the float-rounded inputs.  Every result is a sum of at
    # most C(p+3,3) products of O(1) coefficients and shifts below 1, so the
    # normwise error per rank stays within ~100 float roundings (1e-5), and
    # 5e-5 at p = 10 as for the FP32 D-tensor.
    tol = 1e-5 if p <= 8 else 5e-5
    M32 = M.float()
    Mr = M32.double().cpu().numpy()
    b32 = base.astype(np.float32)
    ref = b32.astype(np.float64) + np.stack([oracle.m2m(p, basis, Mr[:, c], delta[:, c]) for c in range(ncell)], 1)
    Mp32 = g(b32, torch.float32)
    F.fmm_op_m2m(p, basis, M32, g(delta), Mp32)
    assert rank_err(Mp32.double().cpu().numpy(), ref, p, basis) < tol
    L32 = Lg.float()
    Lr = L32.double().cpu().numpy()
    ref2 = np.stack([oracle.l2l(p, basis, Lr[:, c], delta[:, c]) for c in range(ncell)], 1)
    Lc32 = torch.zeros_like(L32)
    F.fmm_op_l2l(p, basis, L32, g(delta), Lc32)
    assert rank_err(Lc32.double().cpu().numpy(), ref2, p, basis) < tol
    ref3 = np.stack([oracle.l2p(p, basis, Lr[:, c], delta[:, c]) for c in range(ncell)], 1)
    out32 = torch.zeros((4, ncell), device=DEV, dtype=torch.float32)
    F.fmm_op_l2p(p, basis, L32, g(delta), out32)
    o = out32.double().cpu().numpy()
    assert np.abs(o[0] - ref3[0]).max() <= tol * np.abs(ref3[0]).max()
    gn = np.linalg.norm(ref3[1:], axis=0)
    dn = np.linalg.norm(o[1:] - ref3[1:], axis=0)
    assert np.all(dn[gn == 0] == 0)
    if (gn > 0).any():
        assert (dn[gn > 0] / gn[gn > 0]).max() < tol


@pytest.mark.parametrize("p", [0, 1, 3, 8, 10])
def test_dtensor_traceless_storage(F, p):
    # the traceless storage of D holds its independent components (nz <= 1);
    # the trace condition rebuilds the rest, which must equal the full tensor
    n = 300 + 11
    r = pair_offsets(n, 40 + p) + inputs.random_coefficients(3, n, 6, 1) * 0.4
    full = oracle.dtensor_batch(p, r)
    nt = oracle.ncoef(p, 1)
    for prec, tol in ((F.FP64, 1e-12), (F.FP32, 1e-5 if p <= 8 else 5e-5)):
        D = torch.zeros((nt, n), device=DEV, dtype=torch.float64 if prec == F.FP64 else torch.float32)
        F.fmm_op_dtensor(p, prec, g(r), D, basis=F.BASIS_TRACELESS)
        Dt = D.double().cpu().numpy()
        rebuilt = np.stack([oracle.expand_traceless(p, Dt[:, i]) for i in range(n)], 1)
        assert rank_err(rebuilt, full, p, 0) < tol, (prec, p)


def test_direct_sum(F):
    n = 3000 + 17
    x, y, z = inputs.uniform_cube(n, 8)
    q = inputs.masses_open_unit(n, 8)
    pref, aref = oracle.direct(x, y, z, q)
    out = torch.zeros((4, n), device=DEV, dtype=torch.float64)
    F.fmm_direct(g(x), g(y), g(z), g(q), out[0], out[1], out[2], out[3])
    o = out.cpu().numpy()
    assert np.abs(o[0] - pref).max() <= 1e-13 * np.abs(pref).max()
    # accelerations: normwise over all particles <= 1e-12; per particle the
    # bound is relative to the sum of the magnitudes of its terms,
    # sum_j q_j / r_ij^2, because a particle's total force can cancel far
    # below its terms (near the centre of the cube), where any two summation
    # orders differ by rounding relative to the terms, not to the total
    assert np.linalg.norm(o[1:] - aref) / np.linalg.norm(aref) < 1e-12
    P = np.stack([x, y, z], 1)
    r2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    mag = (q[None, :] / r2).sum(1)
    assert (np.linalg.norm(o[1:] - aref, axis=0) / mag).max() < 1e-13
    t = np.array([0, 5, n - 1], dtype=np.int64)
    out2 = torch.zeros((4, 3), device=DEV, dtype=torch.float64)
    F.fmm_direct(g(x), g(y), g(z), g(q), out2[0], out2[1], out2[2], out2[3], targets=g(t, torch.int64))
    np.testing.assert_allclose(out2.cpu().numpy(), o[:, t], rtol=1e-14)


def test_empty_batches(F):
    e = torch.zeros((0,), device=DEV, dtype=torch.float64)
    M = torch.zeros((35, 0), device=DEV, dtype=torch.float64)
    r = torch.zeros((3, 0), device=DEV, dtype=torch.float64)
    F.fmm_op_m2l(4, 0, F.FP64, M, r, M)
    F.fmm_op_dtensor(4, F.FP64, r, M)
    F.fmm_op_m2m(4, 0, M, r, M.clone())
    F.fmm_direct(e, e, e, e, e, e, e, e)
    torch.cuda.synchronize()


@pytest.mark.parametrize("p", [0, 1, 2, 4, 7, 8, 10])
def test_fused_m2m_vs_oracle(F, p):
    """Eq. Detracer2 on the GPU (fmm_op_m2m_fused) against the oracle's fused
    form and its shift-then-detrace M2M, 1e-12 per item and rank."""
    rng = np.random.default_rng(200 + p)
    ncell = 131
    counts = rng.integers(1, 12, ncell)
    start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    cen = rng.uniform(-1, 1, (3, ncell))
    pos = np.repeat(cen, counts, axis=1) + rng.uniform(-0.25, 0.25, (3, int(start[-1])))
    q = rng.uniform(0.1, 1, int(start[-1]))
    nc = oracle.ncoef(p, 1)
    M = np.zeros((nc, ncell))
    for c in range(ncell):
        s, e = start[c], start[c + 1]
        M[:, c] = oracle.p2m(p, 1, pos[0, s:e], pos[1, s:e], pos[2, s:e], q[s:e], cen[:, c])
    delta = rng.uniform(-0.3, 0.3, (3, ncell))
    base = inputs.random_coefficients(nc, ncell, 4)
    ref = base + np.stack([oracle.m2m_fused(p, M[:, c], delta[:, c]) for c in range(ncell)], 1)
    ref2 = base + np.stack([oracle.m2m(p, 1, M[:, c], delta[:, c]) for c in range(ncell)], 1)
    Mp = g(base)
    F.fmm_op_m2m_fused(p, g(M), g(delta), Mp)
    got = Mp.cpu().numpy()
    assert rank_err(got, ref, p, 1) < 1e-12
    assert rank_err(got, ref2, p, 1) < 1e-12
    assert F.lib().fmm_m2m_fused_terms(p) > 0
