"""Oracle pins of the binary median-split tree (App. C): leaves of at most
N_bucket particles, every split across the longest axis of the cell's
particles at the median, cells shrink-wrapped (centre = centre of the
particles' bounding box); its lists cover every particle pair once and its
FMM converges to the direct sum."""
import numpy as np
import pytest

import oracle
from paper_1811_06332_gb300 import inputs


def lattice(n, seed):
    """Points with every coordinate drawn from 5 values (seeded): most
    medians fall inside a run of equal coordinates, so the tie rule decides
    which particles go to which child."""
    a = np.floor(inputs.u01(seed, 0, 3 * n) * 5).reshape(3, n)
    return a[0] / 5.0, a[1] / 5.0 * 0.7, a[2] / 5.0 * 1.3


def lattice_cube(n, seed):
    """Every coordinate from the same 5 values: the root's (and many cells')
    bounding-box sides tie, so the rule for equal sides (the first of x, y,
    z) decides the split axis."""
    a = np.floor(inputs.u01(seed, 0, 3 * n) * 5).reshape(3, n)
    return a[0] / 5.0, a[1] / 5.0, a[2] / 5.0


@pytest.mark.parametrize("gen,n,ml", [(inputs.plummer, 5000, 32), (inputs.blobs, 4096, 16), (lattice, 3000, 16),
                                      (lattice_cube, 3000, 16)])
def test_structure_median_splits_and_shrink_wrap(gen, n, ml):
    x, y, z = gen(n, 41)
    P = np.stack([x, y, z], 1)
    zr, rg, order, par = oracle.btree(x, y, z, ml)
    nn = len(zr)
    assert sorted(order.tolist()) == list(range(n))
    kids = {c: [k for k in range(nn) if par[k] == c] for c in range(nn)}
    for c in range(nn):
        idx = order[rg[c, 0]:rg[c, 1]]
        pts = P[idx]
        lo, hi = pts.min(0), pts.max(0)
        np.testing.assert_array_equal(zr[c, :3], (lo + hi) * 0.5)           # shrink-wrapped centre
        assert np.linalg.norm(pts - zr[c, :3], axis=1).max() <= zr[c, 3] * (1 + 1e-12)
        ch = kids[c]
        if not ch:
            assert len(idx) <= ml
            continue
        assert len(idx) > ml and len(ch) == 2
        a, b = ch
        na, nb_ = rg[a, 1] - rg[a, 0], rg[b, 1] - rg[b, 0]
        assert na == len(idx) // 2 and na + nb_ == len(idx)                # median split
        assert rg[a, 0] == rg[c, 0] and rg[b, 1] == rg[c, 1]
        axis = int(np.argmax(hi - lo))                                      # longest axis (first on ties)
        left = P[order[rg[a, 0]:rg[a, 1]], axis]
        right = P[order[rg[b, 0]:rg[b, 1]], axis]
        assert left.max() <= right.min()
    # the same tree built independently with numpy: breadth-first, each split
    # a sort by (coordinate, original index) along the longest side of the
    # bounding box, lower half first; every leaf's particle sequence must
    # match the oracle's final order
    seqs = [np.arange(n)]
    k = 0
    while k < len(seqs):
        sq = seqs[k]
        if len(sq) > ml:
            pts = P[sq]
            ax = int(np.argmax(pts.max(0) - pts.min(0)))
            srt = sq[np.lexsort((sq, pts[:, ax]))]
            h = len(sq) // 2
            seqs += [srt[:h], srt[h:]]
        k += 1
    assert len(seqs) == nn
    for c in range(nn):
        if not kids[c]:
            np.testing.assert_array_equal(order[rg[c, 0]:rg[c, 1]], seqs[c])
        else:
            assert sorted(order[rg[c, 0]:rg[c, 1]].tolist()) == sorted(seqs[c].tolist())


def test_lists_cover_every_pair_and_theta_zero_is_direct():
    n = 3000
    x, y, z = inputs.plummer(n, 42)
    q = inputs.masses_open_unit(n, 42)
    _, _, st = oracle.fmm_btree(x, y, z, q, 32, 0.6, 4, oracle.SYM)
    assert st["covered_pairs"] == n * n
    pot, acc, st0 = oracle.fmm_btree(x, y, z, q, 32, 0.0, 4, oracle.SYM)
    assert st0["m2l_pairs"] == 0
    pd, ad = oracle.direct(x, y, z, q)
    assert np.linalg.norm(acc - ad) <= 1e-13 * np.linalg.norm(ad)


def test_error_decreases_with_p_and_bases_agree():
    n = 5000
    x, y, z = inputs.plummer(n, 43)
    q = inputs.masses_equal(n)
    pd, ad = oracle.direct(x, y, z, q)
    errs = []
    for p in (2, 4, 6, 8):
        _, acc, _ = oracle.fmm_btree(x, y, z, q, 32, 0.6, p, oracle.SYM)
        errs.append(np.sqrt(((acc - ad) ** 2).sum() / (ad ** 2).sum()))
    assert all(a > b for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-4, errs
    _, a0, _ = oracle.fmm_btree(x, y, z, q, 32, 0.6, 6, oracle.SYM)
    _, a1, _ = oracle.fmm_btree(x, y, z, q, 32, 0.6, 6, oracle.TRACELESS)
    assert np.linalg.norm(a1 - a0) <= 1e-12 * np.linalg.norm(a0)
