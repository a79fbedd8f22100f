"""Learned per-pair M2L order on the GPU against the oracle: pair lists,
features, FP64 labels, the FP32 trainer's gradient and Adam step, BF16
tensor-core inference, the per-order M2L, and the whole learned FMM."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp
from paper_1811_06332_gb300 import fmm as F
from paper_1811_06332_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _plummer(n, seed):
    x, y, z = inputs.plummer(n, seed)
    return x, y, z, inputs.masses_equal(n)


def _he_blob(seed, log10_kappa=0.0):
    """Initial parameters: He-uniform weights from the seeded generator,
    zero biases, unit normalisation."""
    b = np.zeros(mlp.NBLOB)
    b[:mlp.HDR] = mlp.header(log10_kappa)
    b[mlp.OFF_SD:mlp.OFF_SD + mlp.NF] = 1.0
    o = mlp.OFF_PAR
    for k, (name, shp) in enumerate(mlp.SHAPES):
        cnt = int(np.prod(shp))
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shp[1])
            b[o:o + cnt] = (inputs.u01(seed, k, cnt) * 2 - 1) * lim
        o += cnt
    return b.astype(np.float32)


def _gpu_to_oracle_index(plan, tgt_o, src_o):
    t, s = plan.pairs()
    nn = int(max(t.max(), s.max(), tgt_o.max(), src_o.max())) + 1
    ko = tgt_o.astype(np.int64) * nn + src_o
    kg = t.astype(np.int64) * nn + s
    idx = np.searchsorted(ko, kg)
    assert np.all(ko[np.minimum(idx, len(ko) - 1)] == kg)
    return idx


@pytest.fixture(scope="module")
def plummer_p10():
    X = _plummer(6000, 41)
    plan = F.Plan(p=10, basis=F.BASIS_SYM, prec=F.FP64, adaptive=True, max_leaf=16, theta=0.6)
    Xd = [_dev(a) for a in X]
    plan.fmm_build_tree(*Xd)
    feat, lab = plan.pair_data(labels=True)
    torch.cuda.synchronize()
    tgt_o, src_o, feat_o, lab_o = O.adaptive_pairs(*X, 16, 0.6, features=True, labels=True)
    idx = _gpu_to_oracle_index(plan, tgt_o, src_o)
    yield X, plan, feat.cpu().numpy(), lab.cpu().numpy(), feat_o, lab_o, idx
    plan.close()


def test_pair_list_equals_oracle(plummer_p10):
    X, plan, feat, lab, feat_o, lab_o, idx = plummer_p10
    assert len(idx) == len(feat_o)
    assert len(np.unique(idx)) == len(idx)     # a permutation: same set of pairs


def test_features_match_oracle(plummer_p10):
    X, plan, feat, lab, feat_o, lab_o, idx = plummer_p10
    ref = feat_o[idx]
    # FP32 geometry and logs against FP64: |d ln| <= ~1e-6 (shape terms from FP64 multipoles)
    err = np.abs(feat - ref)
    assert err.max() < 2e-5, np.unravel_index(err.argmax(), err.shape)


def test_labels_match_oracle(plummer_p10):
    X, plan, feat, lab, feat_o, lab_o, idx = plummer_p10
    ref = lab_o[idx]
    # both FP64; below ~1e-10 the error itself is rounding noise of the direct sum
    m = ref > -9.0
    assert m.mean() > 0.9
    assert np.abs(lab[m] - ref[m]).max() < 1e-6
    assert np.abs(lab[~m] - ref[~m]).max() < 2.0


def _random_samples(seed, n):
    f = (inputs.u01(seed, 0, n * mlp.NF).reshape(n, mlp.NF) - 0.5) * 6
    t = -1 - 4 * inputs.u01(seed, 1, n * mlp.NOUT).reshape(n, mlp.NOUT)
    return f.astype(np.float32), t.astype(np.float32)


def test_mlp_gradient_matches_oracle():
    blob = _he_blob(7)
    blob[mlp.OFF_MU:mlp.OFF_MU + mlp.NF] = 0.25
    blob[mlp.OFF_SD:mlp.OFF_SD + mlp.NF] = 1.5
    f, t = _random_samples(8, 257)
    loss, g = F.fmm_mlp_grad(blob, _dev(f, torch.float32), _dev(t, torch.float32))
    loss_o, g_o = mlp.loss_grad(blob.astype(np.float64), f, t)
    assert abs(loss - loss_o) <= 1e-5 * loss_o
    assert np.abs(g - g_o).max() <= 1e-4 * np.abs(g_o).max()


def test_mlp_one_adam_step_matches_oracle():
    blob = _he_blob(9)
    f, t = _random_samples(10, 300)
    order = torch.arange(300, dtype=torch.int32, device=DEV)
    out, losses = F.fmm_mlp_train(blob, _dev(f, torch.float32), _dev(t, torch.float32), order, epochs=1, batch=300,
                                  lr=1e-3, fit_moments=False)
    _, g_o = mlp.loss_grad(blob.astype(np.float64), f, t)
    th0 = blob[mlp.OFF_PAR:].astype(np.float64)
    th1, _, _ = mlp.adam_step(th0, g_o, np.zeros_like(th0), np.zeros_like(th0), 1, lr=1e-3)
    got = out[mlp.OFF_PAR:].astype(np.float64)
    # step 1 moves each parameter by ~lr sign(g); FP32 gradients may flip the
    # sign only where |g| is at rounding level
    big = np.abs(g_o) > 1e-4 * np.abs(g_o).max()
    assert np.abs(got - th1)[big].max() < 2e-6
    # |step| <= lr, up to the FP32 rounding of parameters of magnitude < 8
    assert np.abs(got - th0).max() <= 1e-3 + 1e-6
    np.testing.assert_array_equal(out[:mlp.OFF_PAR], blob[:mlp.OFF_PAR])


@pytest.mark.parametrize("n", [1, 1000, 100003])
def test_mlp_predict_bf16_matches_oracle(n):
    blob = _he_blob(12)
    blob[mlp.OFF_PAR:] *= 0.7
    blob[mlp.OFF_MU:mlp.OFF_MU + mlp.NF] = 0.1
    blob[mlp.OFF_SD:mlp.OFF_SD + mlp.NF] = 1.3
    f, _ = _random_samples(13, n)
    pred = torch.empty((n, mlp.NOUT), dtype=torch.float32, device=DEV)
    F.fmm_mlp_predict(blob, _dev(f, torch.float32), pred)
    got = pred.cpu().numpy().astype(np.float64)
    ref = mlp.forward(blob, f, bf16=True)
    d = np.abs(got - ref) / (1 + np.abs(ref))
    # same BF16 roundings on both sides; FP32 (tensor core) against FP64
    # accumulation may move a hidden value across a BF16 rounding boundary
    assert np.quantile(d, 0.99) < 1e-3
    assert d.max() < 3e-2


def test_fixed_pair_orders_match_oracle():
    """Per-pair orders from the oracle's labels (the lowest order whose label
    is below 1e-4, else 8) drive both the GPU FMM (FP64, storage order 8) and
    the oracle FMM: equal to 1e-12."""
    X = _plummer(5000, 43)
    tgt_o, src_o, _, lab_o = O.adaptive_pairs(*X, 16, 0.6, features=False, labels=True)
    ords = mlp.select(lab_o, -4.0, 0.0, 8)
    plan = F.Plan(p=8, basis=F.BASIS_SYM, prec=F.FP64, adaptive=True, max_leaf=16, theta=0.6, learned_p=True)
    Xd = [_dev(a) for a in X]
    plan.fmm_build_tree(*Xd)
    idx = _gpu_to_oracle_index(plan, tgt_o, src_o)
    plan.set_pair_orders(ords[idx])
    pot, acc = plan.evaluate(*Xd)
    torch.cuda.synchronize()
    st = plan.stats()
    counts = np.bincount(ords, minlength=9)
    assert st["pairs_per_order"] == counts.tolist()
    pot_o, acc_o, _ = O.fmm_adaptive(*X, 16, 0.6, 8, O.SYM, pair_orders=ords)
    pot, acc = pot.cpu().numpy(), acc.cpu().numpy()
    assert np.max(np.abs(pot - pot_o)) <= 1e-12 * np.max(np.abs(pot_o))
    assert np.sqrt(((acc - acc_o) ** 2).sum(0)).max() <= 1e-12 * np.sqrt((acc_o ** 2).sum(0)).max()
    plan.close()


def test_learned_plan_without_model_is_a_state_error():
    X = _plummer(500, 44)
    plan = F.Plan(p=6, basis=F.BASIS_SYM, prec=F.FP32, adaptive=True, max_leaf=16, theta=0.6, learned_p=True)
    with pytest.raises(F.FMMError) as e:
        plan.evaluate(*[_dev(a) for a in X])
    assert e.value.code == F.ERR_STATE
    bad = _he_blob(1)
    bad[0] = 1.0
    with pytest.raises(F.FMMError) as e:
        plan.set_mlp(bad)
    assert e.value.code == F.ERR_ARG
    plan.close()
    with pytest.raises(F.FMMError) as e:
        F.Plan(p=6, basis=F.BASIS_TRACELESS, prec=F.FP32, adaptive=True, learned_p=True)
    assert e.value.code == F.ERR_UNSUPPORTED


@pytest.fixture(scope="module")
def trained_blob():
    """Model trained on the GPU on a Plummer set (FP64 labels, p = 10)."""
    X = _plummer(16384, 101)
    plan = F.Plan(p=10, basis=F.BASIS_SYM, prec=F.FP64, adaptive=True, max_leaf=16, theta=0.6)
    plan.fmm_build_tree(*[_dev(a) for a in X])
    feat, lab = plan.pair_data(labels=True)
    n = feat.shape[0]
    order = torch.from_numpy(np.argsort(inputs.u01(102, 0, n)).astype(np.int32)).to(DEV)
    blob, losses = F.fmm_mlp_train(_he_blob(103), feat, lab.float(), order, epochs=25, batch=512, lr=2e-3)
    plan.close()
    return blob, losses, feat.cpu().numpy(), lab.cpu().numpy()


def test_training_reduces_loss(trained_blob):
    blob, losses, feat, lab = trained_blob
    print("epoch losses", losses[0], losses[-1])
    # the first epoch's mean already includes the fast initial descent
    assert losses[-1] < 0.6 * losses[0]
    assert np.all(np.isfinite(losses))
    # the oracle forward of the trained FP32 parameters fits the labels
    pred = mlp.forward(blob, feat)
    rmse = np.sqrt(np.mean((pred - lab) ** 2))
    print("train rmse (decades)", rmse)
    assert rmse < 0.35


def test_learned_fmm_meets_target_with_fewer_terms(trained_blob):
    """kappa calibrated on a held-out Plummer set, then the learned orders on
    a third set meet the target with fewer terms than the fixed fallback."""
    from paper_1811_06332_gb300 import order_model
    blob, _, _, _ = trained_blob
    blob, cal = order_model.calibrate(blob, _plummer(16384, 150), 10, 16, 0.6, 1e-4, prec=F.FP64)
    print("calibration", cal)
    X = _plummer(32768, 202)
    Xd = [_dev(a) for a in X]
    plan = F.Plan(p=10, basis=F.BASIS_SYM, prec=F.FP64, adaptive=True, max_leaf=16, theta=0.6, learned_p=True,
                  target_rel_err=1e-4)
    plan.set_mlp(blob)
    pot, acc = plan.evaluate(*Xd)
    st = plan.stats()
    sel = torch.from_numpy(np.arange(0, 32768, 17)).to(DEV)
    ref = torch.empty((4, len(sel)), dtype=torch.float64, device=DEV)
    F.fmm_direct(*Xd, ref[0], ref[1], ref[2], ref[3], targets=sel)
    a = acc[:, sel]
    err = float(torch.sqrt(((a - ref[1:]) ** 2).sum() / (ref[1:] ** 2).sum()))
    cnt = np.array(st["pairs_per_order"])
    mean_p = (cnt * np.arange(len(cnt))).sum() / cnt.sum()
    print("learned: err", err, "orders", cnt.tolist(), "mean", mean_p)
    assert err < 1e-4
    assert mean_p < 8.0
    # the same decisions as the oracle composition (features -> BF16 MLP -> select)
    tgt_o, src_o, feat_o, _ = O.adaptive_pairs(*X, 16, 0.6, features=True, labels=False)
    _, _, _, par = O.adaptive_tree(*X[:3], 16, parents=True)
    lk = np.log10(np.maximum(mlp.chain_pairs(tgt_o, par), 1.0))[tgt_o]
    ords_o = mlp.select(mlp.forward(blob, feat_o.astype(np.float32), bf16=True), -4.0, float(blob[6]), 10,
                        log10_k=lk)
    counts_o = np.bincount(ords_o, minlength=11)
    assert np.abs(cnt - counts_o).sum() <= 0.01 * cnt.sum()
    plan.close()


def test_learned_orders_large_blob_set_match_oracle(trained_blob):
    """2^20 particles of the blob mixture, FP32 learned-order plan (storage
    order 6, the model picks each pair's order): the oracle, run on the same
    tree with the orders the GPU used, agrees on 200 sampled targets within
    the FP32 form's 5e-6."""
    blob = trained_blob[0]
    n = 1 << 20
    x, y, z = inputs.blobs(n, 5)
    q = inputs.masses_equal(n)
    Xd = [_dev(a) for a in (x, y, z, q)]
    plan = F.Plan(p=6, basis=F.BASIS_SYM, prec=F.FP32, adaptive=True, max_leaf=64, theta=0.6, learned_p=True,
                  target_rel_err=1e-4)
    plan.set_mlp(blob)
    pot, acc = plan.evaluate(*Xd)
    plan.sync_status()
    ords = plan.pair_orders()
    tgt_o, src_o = O.adaptive_pairs(x, y, z, q, 64, 0.6, features=False, labels=False)[:2]
    idx = _gpu_to_oracle_index(plan, tgt_o, src_o)
    plan.close()
    ords_o = np.empty(len(idx), dtype=np.int8)
    ords_o[idx] = ords
    cnt = np.bincount(ords, minlength=7)
    print("orders", cnt.tolist())
    assert (cnt > 0).sum() >= 2          # the model mixes orders
    s = np.sort(np.unique((inputs.u01(5, 98, 200) * n).astype(np.int64)))
    pref, aref, _ = O.fmm_adaptive(x, y, z, q, 64, 0.6, 6, O.SYM, sample=s, pair_orders=ords_o)
    p_, a_ = pot.cpu().numpy()[s], acc.cpu().numpy()[:, s]
    ep = np.linalg.norm(p_ - pref) / np.linalg.norm(pref)
    ea = np.linalg.norm(a_ - aref) / np.linalg.norm(aref)
    assert ep < 5e-6 and ea < 5e-6, (ep, ea)
