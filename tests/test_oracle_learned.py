"""Pins of the learned-order oracle (oracle/mlp.py and the per-pair
features, labels and per-pair-order FMM in fmm_oracle.c) against
mathematics that does not come from the oracle itself: closed forms,
finite differences, a library bfloat16 conversion, direct sums."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp
from paper_1811_06332_gb300 import inputs


def _random_blob(seed, scale=0.3):
    u = inputs.u01(seed, 0, mlp.NBLOB)
    b = (u - 0.5) * 2 * scale
    b[:mlp.HDR] = mlp.header(0.0)
    b[mlp.OFF_MU:mlp.OFF_MU + mlp.NF] = (inputs.u01(seed, 1, mlp.NF) - 0.5)
    b[mlp.OFF_SD:mlp.OFF_SD + mlp.NF] = 0.5 + inputs.u01(seed, 2, mlp.NF)
    return b


# ---------------------------------------------------------------- bfloat16
def test_bf16_round_matches_library_conversion():
    torch = pytest.importorskip("torch")
    u = inputs.u01(11, 0, 20000)
    a = np.concatenate([(u - 0.5) * 10.0 ** ((inputs.u01(11, 1, 20000) - 0.5) * 20),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, -2.5e-38, 65504.0]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = mlp.bf16_round(a)
    np.testing.assert_array_equal(got, ref)


def test_bf16_round_ties_to_even():
    # 1 + 2^-8 lies halfway between bf16 neighbours 1 and 1 + 2^-7: even mantissa (1) wins;
    # 1 + 3*2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: even mantissa (1 + 2^-6) wins
    np.testing.assert_array_equal(mlp.bf16_round([1 + 2 ** -8, 1 + 3 * 2 ** -8]), [1.0, 1 + 2 ** -6])


# ---------------------------------------------------------------- forward
def test_forward_hand_built_network():
    """W1 copies the normalised features into the first 12 hidden units,
    W2 and W3 are identities, W4 row k sums units with weight (k+1):
    y_k = (k+1) sum_j relu((f_j - mu_j)/sd_j) + b4_k."""
    d = mlp.unpack(_random_blob(3))
    d = {k: np.array(v) for k, v in d.items()}
    d["W1"][:] = 0.0
    d["W1"][:mlp.NF, :] = np.eye(mlp.NF)
    d["b1"][:] = 0.0
    d["W2"][:] = np.eye(mlp.H); d["b2"][:] = 0.0
    d["W3"][:] = np.eye(mlp.H); d["b3"][:] = 0.0
    d["W4"][:] = 0.0
    for k in range(mlp.NOUT):
        d["W4"][k, :] = k + 1
    d["b4"][:] = np.arange(mlp.NOUT) * 0.25
    blob = mlp.pack(d)
    f = (inputs.u01(5, 0, 7 * mlp.NF).reshape(7, mlp.NF) - 0.5) * 4
    z = (f - d["mu"].astype(np.float32)) / d["sd"].astype(np.float32)
    s = np.maximum(z, 0).sum(1)
    want = s[:, None] * (np.arange(mlp.NOUT) + 1)[None, :] + np.arange(mlp.NOUT) * 0.25
    np.testing.assert_allclose(mlp.forward(blob, f), want, rtol=1e-6, atol=1e-6)


def test_forward_bf16_close_to_fp64():
    blob = _random_blob(4)
    f = (inputs.u01(6, 0, 50 * mlp.NF).reshape(50, mlp.NF) - 0.5) * 4
    y64 = mlp.forward(blob, f)
    y16 = mlp.forward(blob, f, bf16=True)
    # bf16 keeps 8 significant bits: relative perturbation per layer ~2^-8
    assert np.max(np.abs(y16 - y64)) < 0.05 * (1 + np.max(np.abs(y64)))


# ---------------------------------------------------------------- backward
def test_loss_grad_matches_central_differences():
    blob = _random_blob(8).astype(np.float64)
    f = (inputs.u01(9, 0, 13 * mlp.NF).reshape(13, mlp.NF) - 0.5) * 4
    t = (inputs.u01(9, 1, 13 * mlp.NOUT).reshape(13, mlp.NOUT) - 0.5) * 2
    loss, g = mlp.loss_grad(blob, f, t)
    idx = np.unique((inputs.u01(10, 0, 300) * mlp.NPAR).astype(int))
    h = 1e-6
    for i in idx:
        bp, bm = blob.copy(), blob.copy()
        bp[mlp.OFF_PAR + i] += h
        bm[mlp.OFF_PAR + i] -= h
        lp = np.mean((mlp.forward(bp, f) - t) ** 2)
        lm = np.mean((mlp.forward(bm, f) - t) ** 2)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(fd)), (i, fd, g[i])
    assert abs(loss - np.mean((mlp.forward(blob, f) - t) ** 2)) < 1e-15


def test_adam_first_two_steps_closed_form():
    th = np.array([1.0, -2.0, 0.5])
    g1 = np.array([0.3, -0.1, 0.0])
    m = np.zeros(3); v = np.zeros(3)
    th1, m, v = mlp.adam_step(th, g1, m, v, 1, lr=0.01, eps=1e-8)
    # step 1: bias-corrected m = g, v = g^2 -> update lr * g / (|g| + eps)
    np.testing.assert_allclose(th1, th - 0.01 * g1 / (np.abs(g1) + 1e-8), rtol=0, atol=1e-15)
    g2 = np.array([0.1, 0.1, 0.2])
    th2, m, v = mlp.adam_step(th1, g2, m, v, 2, lr=0.01, eps=1e-8)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(th2, th1 - 0.01 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-14, atol=1e-15)


def test_select_lowest_order_meeting_threshold():
    pred = np.array([[-1, -2, -3, -4, -5, -6, -7, -8, -9],    # first <= -4.5: p=6 (col 4 = -5)
                     [0, 0, 0, 0, 0, 0, 0, 0, 0],              # none: fallback p_max
                     [-9, -9, -9, -9, -9, -9, -9, -9, -9]], dtype=float)
    np.testing.assert_array_equal(mlp.select(pred, -5.0, 0.5, 10), [6, 10, 2])
    np.testing.assert_array_equal(mlp.select(pred, -5.0, 0.5, 8), [6, 8, 2])
    # K_B = 100 lowers the threshold by one decade: -4.5 -> -5.5, first <= is p=7 (col 5 = -6)
    np.testing.assert_array_equal(mlp.select(pred, -5.0, 0.5, 10, log10_k=[2.0, 2.0, 2.0]), [7, 10, 2])


def test_chain_pairs_counts_ancestor_lists():
    #        0
    #      1   2
    #     3 4
    parent = np.array([-1, 0, 0, 1, 1])
    tgt = np.array([1, 1, 2, 3, 3, 3, 4])     # node 1 has 2 pairs, 2 one, 3 three, 4 one
    np.testing.assert_array_equal(mlp.chain_pairs(tgt, parent), [0, 2, 1, 5, 3])


# ---------------------------------------------------------------- labels
def test_pair_error_collinear_closed_form():
    """One source particle at z_A + (u,0,0), one target at z_B + (w,0,0),
    z_B - z_A = (D,0,0): the order-p force is the Taylor polynomial of
    -q/(D+s)^2 in s = w - u to degree p-1, so with x = -s/D the relative
    error is |x|^p |(p+1) - p x|."""
    D, u, w, q = 10.0, 1.0, -0.5, 0.7
    zA = np.array([0.3, -0.2, 0.1])
    zB = zA + [D, 0, 0]
    x = -(w - u) / D
    for p in range(2, 11):
        e = O.pair_error(p, ([zA[0] + u], [zA[1]], [zA[2]], [q]), zA, zB, [[zB[0] + w, zB[1], zB[2]]])
        want = abs(x) ** p * abs((p + 1) - p * x)
        assert abs(e - want) <= 1e-12 + 1e-9 * want, (p, e, want)


@pytest.fixture(scope="module")
def plummer_pairs():
    n = 3000
    x, y, z = inputs.plummer(n, 21)
    q = inputs.masses_equal(n)
    tgt, src, feat, lab = O.adaptive_pairs(x, y, z, q, 16, 0.6, features=True, labels=True)
    zr, rg, order, par = O.adaptive_tree(x, y, z, 16, parents=True)
    return (x, y, z, q), tgt, src, feat, lab, zr, rg, order, par


def test_pairs_are_the_m2l_list(plummer_pairs):
    (x, y, z, q), tgt, src, feat, lab, zr, rg, order, par = plummer_pairs
    _, _, st = O.fmm_adaptive(x, y, z, q, 16, 0.6, 2, O.SYM, sample=[0])
    assert len(tgt) == st["m2l_pairs"] > 0
    key = tgt * (tgt.max() + 1) + src
    assert np.all(np.diff(key) > 0)          # sorted by (target, source), no duplicates
    # the MAC holds for every pair and the first feature is its log ratio
    d = np.linalg.norm(zr[tgt, :3] - zr[src, :3], axis=1)
    rho = (np.maximum(zr[src, 3] / d, 1e-6) + np.maximum(zr[tgt, 3] / d, 1e-6))
    assert np.all(0.6 * d > zr[src, 3] + zr[tgt, 3])
    np.testing.assert_allclose(feat[:, 0], np.log(rho), rtol=0, atol=1e-12)
    np.testing.assert_allclose(feat[:, 9], np.log(np.minimum(rg[src, 1] - rg[src, 0], 1024)), atol=1e-12)
    np.testing.assert_allclose(feat[:, 10], np.log(np.minimum(rg[tgt, 1] - rg[tgt, 0], 1024)), atol=1e-12)


def test_shape_features_closed_forms(plummer_pairs):
    """A one-particle node at distance r from its centre has r_A = r and
    multipole q(-r)^(x)j of Frobenius norm |q| r^j: its shape features are
    ln 1 = 0.  Every ratio is at most 1 (the norm of a sum of rank-one
    tensors is at most the sum of the norms, each <= q r_A^j)."""
    (x, y, z, q), tgt, src, feat, lab, zr, rg, order, par = plummer_pairs
    one = (rg[src, 1] - rg[src, 0]) == 1
    assert one.sum() > 10
    np.testing.assert_allclose(feat[one, 3:7], 0.0, atol=1e-9)
    assert np.all(feat[:, 3:9] <= 1e-9)
    assert np.all(feat[:, 3:9] >= np.log(1e-6) - 1e-12)


def test_labels_equal_direct_definition(plummer_pairs):
    """Labels from the tree's M2M-built multipoles equal the definition
    recomputed from the pair's particles (P2M at the source centre), with
    the pair's own field and the total field at the targets taken from the
    oracle's direct sum (pinned separately)."""
    (x, y, z, q), tgt, src, feat, lab, zr, rg, order, par = plummer_pairs
    pick = np.unique((inputs.u01(31, 0, 25) * len(tgt)).astype(int))
    for k in pick:
        A, B = src[k], tgt[k]
        ia = order[rg[A, 0]:rg[A, 1]]
        nb = rg[B, 1] - rg[B, 0]
        sp = np.arange(nb) if nb <= 64 else (np.arange(64) * nb) // 64
        ib = order[rg[B, 0] + sp]
        # own field: A's particles plus B's sample points carrying no charge
        xs = np.concatenate([x[ia], x[ib]]); ys = np.concatenate([y[ia], y[ib]])
        zs = np.concatenate([z[ia], z[ib]]); qs = np.concatenate([q[ia], np.zeros(len(ib))])
        _, g_own = O.direct(xs, ys, zs, qs, targets=np.arange(len(ia), len(ia) + len(ib)))
        _, g_tot = O.direct(x, y, z, q, targets=ib)
        scale = np.sqrt((g_own ** 2).sum() / (g_tot ** 2).sum())
        for p in (2, 5, 10):
            e = O.pair_error(p, (x[ia], y[ia], z[ia], q[ia]), zr[A, :3], zr[B, :3],
                             np.stack([x[ib], y[ib], z[ib]], 1))
            assert abs(np.log10(max(e * scale, 1e-12)) - lab[k, p - 2]) < 1e-8, (k, p)


def test_far_field_share_feature(plummer_pairs):
    """f11 is the log of the pair's share of a sum of positive terms over the
    target's list and its ancestors' lists: every share is <= 1, the shares
    of one target's own list sum to at most 1, and to exactly 1 when no
    ancestor of the target has an M2L list."""
    (x, y, z, q), tgt, src, feat, lab, zr, rg, order, par = plummer_pairs
    assert np.all(feat[:, 11] <= 1e-12)
    share = np.exp(feat[:, 11])
    tot = np.bincount(tgt, weights=share, minlength=len(zr))
    assert np.all(tot <= 1 + 1e-9)
    has_list = np.bincount(tgt, minlength=len(zr)) > 0
    anc_list = np.zeros(len(zr), dtype=bool)
    for c in range(len(zr)):          # parents precede children
        if par[c] >= 0:
            anc_list[c] = anc_list[par[c]] or has_list[par[c]]
    only = has_list & ~anc_list
    assert only.sum() > 0
    np.testing.assert_allclose(tot[only], 1.0, rtol=1e-12)


def test_labels_decrease_with_order(plummer_pairs):
    (x, y, z, q), tgt, src, feat, lab, zr, rg, order, par = plummer_pairs
    m = lab.mean(0)
    assert np.all(np.diff(m) < -0.2)
    # geometric decay: the mean slope is near log10 of a typical separation ratio
    assert -0.8 < np.mean(np.diff(m)) < -0.2


# ---------------------------------------------------------------- per-pair orders
def test_pair_orders_all_p_equal_fixed_p():
    n = 2000
    x, y, z = inputs.plummer(n, 23)
    q = inputs.masses_equal(n)
    tgt, _, _, _ = O.adaptive_pairs(x, y, z, q, 16, 0.6, features=False)
    s = np.arange(0, n, 7)
    pa, aa, _ = O.fmm_adaptive(x, y, z, q, 16, 0.6, 6, O.SYM, sample=s)
    pb, ab, _ = O.fmm_adaptive(x, y, z, q, 16, 0.6, 6, O.SYM, sample=s,
                               pair_orders=np.full(len(tgt), 6, dtype=np.int8))
    np.testing.assert_allclose(pb, pa, rtol=1e-13)
    np.testing.assert_allclose(ab, aa, rtol=1e-12, atol=1e-12 * np.abs(aa).max())


def test_pair_orders_lower_order_equals_lower_p_on_the_far_field():
    """With every pair at order 4 but storage at order 8 the far field is
    the order-4 one: equal to a plain order-4 run up to the extra (exact)
    ranks of P2M/M2M/L2L, which do not change the order-4 terms."""
    n = 2000
    x, y, z = inputs.plummer(n, 24)
    q = inputs.masses_equal(n)
    tgt, _, _, _ = O.adaptive_pairs(x, y, z, q, 16, 0.6, features=False)
    s = np.arange(0, n, 5)
    p4, a4, _ = O.fmm_adaptive(x, y, z, q, 16, 0.6, 4, O.SYM, sample=s)
    pm, am, _ = O.fmm_adaptive(x, y, z, q, 16, 0.6, 8, O.SYM, sample=s,
                               pair_orders=np.full(len(tgt), 4, dtype=np.int8))
    np.testing.assert_allclose(pm, p4, rtol=1e-12)
    np.testing.assert_allclose(am, a4, rtol=1e-11, atol=1e-12 * np.abs(a4).max())


def test_pair_orders_error_between_bounds():
    n = 2000
    x, y, z = inputs.plummer(n, 25)
    q = inputs.masses_equal(n)
    tgt, _, _, _ = O.adaptive_pairs(x, y, z, q, 16, 0.6, features=False)
    s = np.arange(0, n, 3)
    _, ad = O.direct(x, y, z, q, targets=s)
    mixed = np.where(np.arange(len(tgt)) % 2 == 0, 3, 8).astype(np.int8)

    def err(a):
        return np.sqrt(((a - ad) ** 2).sum() / (ad ** 2).sum())

    e3 = err(O.fmm_adaptive(x, y, z, q, 16, 0.6, 8, O.SYM, sample=s, pair_orders=np.full(len(tgt), 3, np.int8))[1])
    e8 = err(O.fmm_adaptive(x, y, z, q, 16, 0.6, 8, O.SYM, sample=s)[1])
    em = err(O.fmm_adaptive(x, y, z, q, 16, 0.6, 8, O.SYM, sample=s, pair_orders=mixed)[1])
    assert e8 < em < e3


def test_pair_orders_rejects_wrong_count():
    n = 500
    x, y, z = inputs.plummer(n, 26)
    q = inputs.masses_equal(n)
    with pytest.raises(ValueError):
        O.fmm_adaptive(x, y, z, q, 16, 0.6, 6, O.SYM, pair_orders=np.full(3, 4, np.int8))
