"""GPU parity of the adaptive-octree FMM (tree from Morton keys, dual-tree
traversal with the App. C MAC, list M2L/P2P as persistent kernels, CUDA
graph replay) against the FP64 oracle built with the same rules."""
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


def g(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def errs(pot, acc, pref, aref):
    ep = np.linalg.norm(pot - pref) / np.linalg.norm(pref)
    ea = np.linalg.norm(acc - aref) / np.linalg.norm(aref)
    return ep, ea


def run(F, x, y, z, q, p, basis, prec, max_leaf, theta, use_graph=False, reps=1):
    plan = F.Plan(p=p, basis=basis, prec=prec, adaptive=True, max_leaf=max_leaf, theta=theta,
                  use_graph=use_graph)
    stream = torch.cuda.Stream() if use_graph else None
    outs = []
    for _ in range(reps):
        if stream is not None:
            with torch.cuda.stream(stream):
                pot, acc = plan.evaluate(g(x), g(y), g(z), g(q), stream=stream)
            stream.synchronize()
        else:
            pot, acc = plan.evaluate(g(x), g(y), g(z), g(q))
        torch.cuda.synchronize()
        outs.append((pot.cpu().numpy(), acc.cpu().numpy()))
    st = plan.stats()
    plan.close()
    return outs, st


@pytest.mark.parametrize("p,basis,max_leaf,theta", [(4, 0, 32, 0.5), (6, 1, 64, 0.5), (3, 0, 16, 0.7)])
def test_plummer_fp64_vs_oracle(F, p, basis, max_leaf, theta):
    n = 6000
    x, y, z = inputs.plummer(n, 4)
    q = inputs.masses_equal(n)
    (res,), st = run(F, x, y, z, q, p, basis, F.FP64, max_leaf, theta)
    pref, aref, ost = oracle.fmm_adaptive(x, y, z, q, max_leaf, theta, p, basis)
    assert (st["cells"], st["leaves"], st["m2l_pairs"], st["p2p_pairs"]) == \
        (ost["nodes"], ost["leaves"], ost["m2l_pairs"], ost["p2p_pairs"])
    ep, ea = errs(res[0], res[1], pref, aref)
    assert ep < 1e-12 and ea < 1e-12, (ep, ea)


def test_theta_zero_and_single_leaf(F):
    n = 3000
    x, y, z = inputs.blobs(n, 5)
    q = inputs.masses_open_unit(n, 5)
    (res,), st = run(F, x, y, z, q, 4, 0, F.FP64, 64, 0.0)
    pref, aref = oracle.direct(x, y, z, q)
    assert st["m2l_pairs"] == 0
    ep, ea = errs(res[0], res[1], pref, aref)
    assert ep < 1e-12 and ea < 1e-11, (ep, ea)
    (res,), st = run(F, x[:50], y[:50], z[:50], q[:50], 4, 0, F.FP64, 64, 0.5)
    pref, aref = oracle.direct(x[:50], y[:50], z[:50], q[:50])
    assert st["cells"] == 1
    ep, ea = errs(res[0], res[1], pref, aref)
    assert ep < 1e-13 and ea < 1e-12


def test_blobs_fp32_graph_replay(F):
    """FP32 form on a blob mixture; the captured graph replays to the same
    numbers as the eager first evaluation."""
    n = 40000
    x, y, z = inputs.blobs(n, 5)
    q = inputs.masses_equal(n)
    outs, st = run(F, x, y, z, q, 6, 0, F.FP32, 64, 0.5, use_graph=True, reps=3)
    assert st["graph"] == 1 and st["m2l_blocks_per_sm"] >= 1
    s = np.sort(np.unique((inputs.u01(5, 93, 300) * n).astype(np.int64)))
    pref, aref, _ = oracle.fmm_adaptive(x, y, z, q, 64, 0.5, 6, 0, sample=s)
    for pot, acc in outs:
        ep, ea = errs(pot[s], acc[:, s], pref, aref)
        assert ep < 5e-6 and ea < 5e-6, (ep, ea)
    np.testing.assert_array_equal(outs[1][1], outs[2][1])


def test_plummer_large_fp32_sampled(F):
    """2^20 Plummer particles, <= 64 per leaf, symmetric p = 6, FP32."""
    n = 1 << 20
    x, y, z = inputs.plummer(n, 4)
    q = inputs.masses_equal(n)
    (res,), st = run(F, x, y, z, q, 6, 0, F.FP32, 64, 0.5)
    s = np.sort(np.unique((inputs.u01(4, 94, 200) * n).astype(np.int64)))
    pref, aref, ost = oracle.fmm_adaptive(x, y, z, q, 64, 0.5, 6, 0, sample=s)
    assert st["m2l_pairs"] == ost["m2l_pairs"] and st["p2p_pairs"] == ost["p2p_pairs"]
    ep, ea = errs(res[0][s], res[1][:, s], pref, aref)
    assert ep < 5e-6 and ea < 5e-6, (ep, ea)


@pytest.mark.parametrize("p,basis", [(10, 0), (8, 1)])
def test_fp32_high_order_deep_tree(F, p, basis):
    """Deep cells (blobs of sigma 0.005, 2^17 particles, 8 per leaf) at high
    order: in physical units D_k(r) ~ |k|!/r^(|k|+1) leaves the FP32 range,
    the scaled units of the FP32 form keep it finite and at FP32 accuracy
    against the FP64 form on the same tree."""
    n = 131072
    x, y, z = inputs.blobs(n, 9, sigma_lo=0.005, sigma_hi=0.006)
    q = inputs.masses_equal(n)
    (r32,), st32 = run(F, x, y, z, q, p, basis, F.FP32, 8, 0.5)
    (r64,), st64 = run(F, x, y, z, q, p, basis, F.FP64, 8, 0.5)
    assert st32["levels"] >= 10   # cells of side <= 2^-10
    assert np.all(np.isfinite(r32[0])) and np.all(np.isfinite(r32[1]))
    ep, ea = errs(r32[0], r32[1], r64[0], r64[1])
    assert ep < 2e-6 and ea < 2e-5, (ep, ea)


@pytest.mark.parametrize("p,max_leaf,theta", [(4, 32, 0.6), (6, 64, 0.5)])
def test_ap_variant_vs_oracle(F, p, max_leaf, theta):
    """The AP variant (Sec. 3): centre-of-mass centres, dipole 0, gradient
    only, against the oracle's AP FMM on the same tree (same lists; 1e-12 on
    the accelerations)."""
    n = 8000
    x, y, z = inputs.plummer(n, 34)
    q = inputs.masses_open_unit(n, 34)
    plan = F.Plan(p=p, basis=F.BASIS_TRACELESS, prec=F.FP64, adaptive=True, max_leaf=max_leaf, theta=theta, ap=True)
    pot, acc = plan.evaluate(g(x), g(y), g(z), g(q))
    torch.cuda.synchronize()
    st = plan.stats()
    plan.close()
    pref, aref, ost = oracle.fmm_adaptive_ap(x, y, z, q, max_leaf, theta, p)
    assert (st["cells"], st["leaves"], st["m2l_pairs"], st["p2p_pairs"]) == \
        (ost["nodes"], ost["leaves"], ost["m2l_pairs"], ost["p2p_pairs"])
    assert not pot.any()
    acc = acc.cpu().numpy()
    assert np.linalg.norm(acc - aref) / np.linalg.norm(aref) < 1e-12
    for bad in (dict(basis=F.BASIS_SYM), dict(prec=F.FP32), dict(adaptive=False)):
        kw = dict(p=p, basis=F.BASIS_TRACELESS, prec=F.FP64, adaptive=True, ap=True)
        kw.update(bad)
        with pytest.raises(F.FMMError):
            F.Plan(**kw)


@pytest.mark.parametrize("p,basis,max_leaf,theta,dist", [(4, 0, 32, 0.5, "plummer"), (6, 1, 64, 0.6, "plummer"),
                                                          (5, 1, 16, 0.5, "lattice"), (4, 1, 16, 0.5, "cube")])
def test_binary_tree_vs_oracle(F, p, basis, max_leaf, theta, dist):
    """The binary median-split tree (App. C) built on the device: the same
    node, leaf and list counts as the oracle's tree, the fields within 1e-12.
    The lattice case draws every coordinate from 5 values, so most medians
    fall inside runs of equal coordinates and the tie rule (by original
    index) decides the tree."""
    if dist == "plummer":
        n = 7000
        x, y, z = inputs.plummer(n, 41)
    else:
        n = 3000
        a = np.floor(inputs.u01(41, 0, 3 * n) * 5).reshape(3, n)   # every coordinate one of 5 values
        if dist == "lattice":
            x, y, z = a[0] / 5.0, a[1] / 5.0 * 0.7, a[2] / 5.0 * 1.3
        else:   # equal extents: the rule for tied sides decides the axis
            x, y, z = a[0] / 5.0, a[1] / 5.0, a[2] / 5.0
    q = inputs.masses_open_unit(n, 41)
    plan = F.Plan(p=p, basis=basis, prec=F.FP64, adaptive=True, max_leaf=max_leaf, theta=theta, binary_tree=True)
    pot, acc = plan.evaluate(g(x), g(y), g(z), g(q))
    torch.cuda.synchronize()
    st = plan.stats()
    plan.close()
    pref, aref, ost = oracle.fmm_btree(x, y, z, q, max_leaf, theta, p, basis)
    assert (st["cells"], st["leaves"], st["m2l_pairs"], st["p2p_pairs"]) == \
        (ost["nodes"], ost["leaves"], ost["m2l_pairs"], ost["p2p_pairs"])
    ep, ea = errs(pot.cpu().numpy(), acc.cpu().numpy(), pref, aref)
    assert ep < 1e-12 and ea < 1e-12, (ep, ea)


def test_binary_tree_configs(F):
    """The binary tree is an FP64 adaptive option; other forms are refused."""
    for bad in (dict(prec=F.FP32), dict(adaptive=False), dict(ap=True), dict(learned_p=True)):
        kw = dict(p=4, basis=F.BASIS_TRACELESS, prec=F.FP64, adaptive=True, binary_tree=True)
        kw.update(bad)
        with pytest.raises(F.FMMError):
            F.Plan(**kw)
