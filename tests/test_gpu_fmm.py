"""GPU parity of the plan-based uniform-octree FMM (fmm_evaluate and the
step-by-step entry points) against the FP64 oracle on the same tree, plus the
direct-sum accuracy and edge cases.

FP64 tolerance: normwise relative error of pot and of acc over all particles
<= 1e-12, and per particle |d acc|/|acc| <= 1e-10 (summation order differs
between the two; single particles can sit where the field nearly cancels).
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


def g(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def errs(pot, acc, pref, aref):
    ep = np.linalg.norm(pot - pref) / max(np.linalg.norm(pref), 1e-300)
    ea = np.linalg.norm(acc - aref) / max(np.linalg.norm(aref), 1e-300)
    per = np.linalg.norm(acc - aref, axis=0) / np.maximum(np.linalg.norm(aref, axis=0), 1e-300)
    return ep, ea, per.max() if per.size else 0.0


def run(F, x, y, z, q, p, basis, depth, prec=None):
    plan = F.Plan(p=p, basis=basis, prec=F.FP64 if prec is None else prec, depth=depth)
    pot, acc = plan.evaluate(g(x), g(y), g(z), g(q))
    torch.cuda.synchronize()
    plan.close()
    return pot.cpu().numpy(), acc.cpu().numpy()


@pytest.mark.parametrize("p,basis", [(4, 0), (4, 1), (8, 1), (8, 0), (10, 1), (2, 0)])
def test_small_uniform_vs_oracle(F, p, basis):
    n, depth = 4096, 3
    x, y, z = inputs.uniform_cube(n, 1)
    q = inputs.masses_open_unit(n, 1)
    pot, acc = run(F, x, y, z, q, p, basis, depth)
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, p, basis)
    ep, ea, per = errs(pot, acc, pref, aref)
    assert ep < 1e-12 and ea < 1e-12 and per < 1e-10, (ep, ea, per)


def test_small_uniform_vs_direct(F):
    n, depth, p = 4096, 3, 4
    x, y, z = inputs.uniform_cube(n, 1)
    q = inputs.masses_open_unit(n, 1)
    pot, acc = run(F, x, y, z, q, p, 0, depth)
    pd, ad = oracle.direct(x, y, z, q)
    assert np.sqrt(((acc - ad) ** 2).sum() / (ad ** 2).sum()) < 3e-3


def test_step_by_step_equals_evaluate(F):
    n, depth, p = 5000, 3, 6
    x, y, z = inputs.uniform_cube(n, 2)
    q = inputs.masses_open_unit(n, 2)
    plan = F.Plan(p=p, basis=1, prec=F.FP64, depth=depth)
    t = [g(a) for a in (x, y, z, q)]
    out = torch.zeros((4, n), device=DEV, dtype=torch.float64)
    with pytest.raises(F.FMMError):
        plan.fmm_p2m()            # before fmm_build_tree: FMM_ERR_STATE
    plan.fmm_build_tree(*t)
    plan.fmm_p2m(); plan.fmm_m2m(); plan.fmm_m2l(); plan.fmm_l2l()
    plan.fmm_l2p(out[0], out[1], out[2], out[3])
    far = out.clone()
    plan.fmm_p2p(out[0], out[1], out[2], out[3])
    pot, acc = plan.evaluate(*t)
    torch.cuda.synchronize()
    assert torch.equal(out[0], pot) and torch.equal(out[1:], acc)
    assert not torch.equal(far, out)
    plan.close()


@pytest.mark.parametrize("prec,p,basis,depth,n", [("FP32", 8, 1, 4, 70000), ("FP32", 6, 0, 3, 9000),
                                                   ("GEMM_BF16X3", 8, 1, 5, 300000), ("FP32", 4, 1, 1, 2000),
                                                   ("FP32", 8, 1, 2, 2500), ("FP32", 5, 1, 2, 9000),
                                                   ("FP64", 5, 1, 3, 6000)])
def test_fused_far_near_field_equals_the_two_steps(F, prec, p, basis, depth, n):
    """fmm_l2p_p2p (one kernel for the FP32 and tensor-core forms on a
    uniform octree; the two steps otherwise) writes exactly what fmm_l2p
    followed by fmm_p2p writes: the same FP32 arithmetic in the same order
    and explicitly rounded FP64 combinations.  Ragged leaves (Poisson counts,
    some empty at depth 5 with 300,000 particles: about 9 per leaf; about 17
    and 39 per leaf at depths 4 and 2; 140 per leaf at depth 2, several
    blocks of 32 targets per leaf).  At depths 0 and 1 (no far field)
    fmm_l2p_p2p runs the two steps."""
    x, y, z = inputs.uniform_cube(n, 70 + depth)
    q = inputs.masses_open_unit(n, 70 + depth)
    plan = F.Plan(p=p, basis=basis, prec=getattr(F, prec), depth=depth)
    t = [g(a) for a in (x, y, z, q)]
    two = torch.full((4, n), 7.0, device=DEV, dtype=torch.float64)
    one = torch.full((4, n), -3.0, device=DEV, dtype=torch.float64)
    plan.fmm_build_tree(*t)
    plan.fmm_p2m(); plan.fmm_m2m(); plan.fmm_m2l(); plan.fmm_l2l()
    plan.fmm_l2p(two[0], two[1], two[2], two[3])
    plan.fmm_p2p(two[0], two[1], two[2], two[3])
    plan.fmm_l2p_p2p(one[0], one[1], one[2], one[3])
    plan.sync_status()
    plan.close()
    assert torch.equal(one, two)


@pytest.mark.parametrize("depth", [0, 1, 2])
def test_shallow_trees(F, depth):
    n = 1500
    x, y, z = inputs.uniform_cube(n, 3)
    q = inputs.masses_open_unit(n, 3)
    pot, acc = run(F, x, y, z, q, 5, 1, depth)
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, 5, 1)
    ep, ea, per = errs(pot, acc, pref, aref)
    assert ep < 1e-12 and ea < 1e-12, (ep, ea)


@pytest.mark.parametrize("n", [0, 1, 2, 9])
def test_tiny_inputs(F, n):
    x, y, z = inputs.uniform_cube(max(n, 1), 4)
    q = inputs.masses_open_unit(max(n, 1), 4)
    x, y, z, q = x[:n], y[:n], z[:n], q[:n]
    pot, acc = run(F, x, y, z, q, 4, 0, 3)
    if n:
        pref, aref = oracle.fmm_uniform(x, y, z, q, 3, 4, 0)
        np.testing.assert_allclose(pot, pref, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(acc, aref, rtol=1e-10, atol=1e-12 * max(np.abs(aref).max(), 1e-300))
        if n == 1:
            assert pot[0] == 0.0 and not acc.any()


def test_crowded_and_boundary(F):
    """All particles in one leaf, others on the cube faces (x = 1 clamps)."""
    n = 700
    x, y, z = inputs.uniform_cube(n, 5)
    x[:400] = 0.3 + 0.01 * x[:400]; y[:400] = 0.6 + 0.01 * y[:400]; z[:400] = 0.1 + 0.01 * z[:400]
    x[400:410] = 1.0; y[410:420] = 0.0; z[420:430] = 1.0
    q = inputs.masses_open_unit(n, 5)
    pot, acc = run(F, x, y, z, q, 6, 1, 3)
    pref, aref = oracle.fmm_uniform(x, y, z, q, 3, 6, 1)
    ep, ea, per = errs(pot, acc, pref, aref)
    assert ep < 1e-12 and ea < 1e-12, (ep, ea)


def test_fp32_near_field(F):
    n, depth, p = 4096, 3, 6
    x, y, z = inputs.uniform_cube(n, 6)
    q = inputs.masses_open_unit(n, 6)
    pot, acc = run(F, x, y, z, q, p, 1, depth, prec=F.FP32)
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, p, 1)
    ep, ea, per = errs(pot, acc, pref, aref)
    assert ep < 1e-6 and ea < 1e-6, (ep, ea)


def test_host_entry_point(F):
    n, depth, p = 3000, 3, 4
    x, y, z = inputs.uniform_cube(n, 7)
    q = inputs.masses_open_unit(n, 7)
    plan = F.Plan(p=p, basis=0, prec=F.FP64, depth=depth)
    out = np.zeros((4, n))
    plan.fmm_evaluate_host(x, y, z, q, out[0], out[1], out[2], out[3])
    pot, acc = plan.evaluate(g(x), g(y), g(z), g(q))
    np.testing.assert_array_equal(out[0], pot.cpu().numpy())
    np.testing.assert_array_equal(out[1:], acc.cpu().numpy())
    plan.close()


def test_full_size_sampled_precision_workload(F):
    """4,194,304 uniform particles, depth 6 (262,144 leaves), traceless p = 8:
    GPU FP64 FMM against the oracle on 64 sampled particles."""
    n, depth, p = 4194304, 6, 8
    x, y, z = inputs.uniform_cube(n, 3)
    q = inputs.masses_equal(n)
    pot, acc = run(F, x, y, z, q, p, 1, depth)
    s = np.sort(np.unique((inputs.u01(3, 90, 64) * n).astype(np.int64)))
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, p, 1, sample=s)
    ep, ea, per = errs(pot[s], acc[:, s], pref, aref)
    assert ep < 1e-12 and ea < 1e-12 and per < 1e-10, (ep, ea, per)


@pytest.mark.parametrize("depth,n", [(5, 131072), (6, 262144)])
def test_tensor_core_form_vs_oracle(F, depth, n):
    """Offset-grouped tensor-core M2L (BF16 hi/lo, three passes, FP32
    accumulation in TMEM; levels >= 5, the levels below on the FP32 grouped
    kernel), traceless p = 8, against the FP64 oracle on 200 sampled
    particles.  Split BF16 products keep ~16 bits per operand; with the
    issuers' accumulators added in FP64 the measured error is below 1e-6
    normwise at these sizes.  Bound: 5e-6 on pot and acc."""
    x, y, z = inputs.uniform_cube(n, 11 + depth)
    q = inputs.masses_equal(n)
    pot, acc = run(F, x, y, z, q, 8, 1, depth, prec=F.GEMM_BF16X3)
    s = np.sort(np.unique((inputs.u01(7, 92, 200) * n).astype(np.int64)))
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, 8, 1, sample=s)
    ep, ea, per = errs(pot[s], acc[:, s], pref, aref)
    assert ep < 5e-6 and ea < 5e-6, (ep, ea, per)


@pytest.mark.parametrize("depth,n,p", [(6, 262144, 8), (7, 1048576, 8), (6, 262144, 6), (5, 131072, 4)])
def test_swapped_tensor_core_kernel_vs_oracle(F, depth, n, p):
    """Kernel shape 2 (the offset's matrix as the A operand, 128 local
    components; the cells of an 8 x 32 tile as N = 256, 8 x 16 on level 5;
    two K-parts of 48 multipole components, or one at p <= 5), traceless,
    against the FP64 oracle on sampled particles: depth 6 and 7 run the
    256-cell tiles on levels 6 and 7 and the 128-cell tiles on level 5.
    Bound: 5e-6 on pot and acc, as for the other shapes."""
    x, y, z = inputs.uniform_cube(n, 31 + depth + p)
    q = inputs.masses_equal(n)
    plan = F.Plan(p=p, basis=1, prec=F.GEMM_BF16X3, depth=depth)
    plan.set_tc_shape(2, 256)
    pot, acc = plan.evaluate(*[g(a) for a in (x, y, z, q)])
    plan.sync_status()
    assert plan.tuning()["kernel"] == 2
    plan.close()
    pot, acc = pot.cpu().numpy(), acc.cpu().numpy()
    s = np.sort(np.unique((inputs.u01(7, 94, 150) * n).astype(np.int64)))
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, p, 1, sample=s)
    ep, ea, per = errs(pot[s], acc[:, s], pref, aref)
    assert ep < 5e-6 and ea < 5e-6, (ep, ea, per)


@pytest.mark.parametrize("depth,n,p", [(6, 262144, 8), (7, 1048576, 8), (6, 262144, 7), (6, 262144, 6),
                                       (5, 131072, 5)])
def test_split_tensor_core_kernel_vs_oracle(F, depth, n, p):
    """Kernel shape 3: the swapped kernel on the first K-part (multipole
    columns 0..47) while the columns >= 48, which reach only the local rows
    of rank <= p - 6, run as FP32 products on the CUDA cores after the
    tensor-core kernel and are added to L (level 5 with its source classes
    split over four blocks per tile, the groups added in order; p = 6..8; at
    p = 5 there are no such columns and it is kernel 2).  Against the FP64 oracle on sampled
    particles, bound 5e-6 as for the other shapes; and equal to kernel 2
    within 1e-5 of the largest value (the two differ only in the rounding
    of those few products)."""
    x, y, z = inputs.uniform_cube(n, 41 + depth + p)
    q = inputs.masses_equal(n)
    X = [g(a) for a in (x, y, z, q)]
    plan = F.Plan(p=p, basis=1, prec=F.GEMM_BF16X3, depth=depth)
    plan.set_tc_shape(3, 256)
    pot, acc = plan.evaluate(*X)
    plan.sync_status()
    assert plan.tuning()["kernel"] == 3
    plan.set_tc_shape(2, 256)
    pot2, acc2 = plan.evaluate(*X)
    plan.sync_status()
    plan.close()
    for a, b in ((pot, pot2), (acc, acc2)):
        assert float((a - b).abs().max()) <= 1e-5 * float(b.abs().max())
    pot, acc = pot.cpu().numpy(), acc.cpu().numpy()
    s = np.sort(np.unique((inputs.u01(7, 97, 150) * n).astype(np.int64)))
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, p, 1, sample=s)
    ep, ea, per = errs(pot[s], acc[:, s], pref, aref)
    assert ep < 5e-6 and ea < 5e-6, (ep, ea, per)


@pytest.mark.parametrize("depth,n", [(5, 131072), (6, 262144)])
def test_tensor_core_tf32_form_vs_oracle(F, depth, n):
    """The same offset-grouped tensor-core M2L with TF32 hi/lo operands
    (kind::tf32, two K-parts per offset), traceless p = 8, against the FP64
    oracle on 200 sampled particles.  The TF32 split keeps ~21 bits per
    operand, so what remains is the FP32 accumulation in TMEM, over twice
    the K-steps of the BF16 form: measured up to 1.3e-6 normwise at these
    sizes (the BF16 form 0.9e-6, the FP32 SIMT form 0.3e-6).  Bound: 5e-6
    on pot and acc."""
    x, y, z = inputs.uniform_cube(n, 21 + depth)
    q = inputs.masses_equal(n)
    pot, acc = run(F, x, y, z, q, 8, 1, depth, prec=F.GEMM_TF32X3)
    s = np.sort(np.unique((inputs.u01(7, 93, 200) * n).astype(np.int64)))
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, 8, 1, sample=s)
    ep, ea, per = errs(pot[s], acc[:, s], pref, aref)
    assert ep < 5e-6 and ea < 5e-6, (ep, ea, per)


@pytest.mark.parametrize("p", [2, 6])
def test_tensor_core_forms_low_order(F, p):
    """Both tensor-core forms at lower orders (fewer N-chunks and K-steps
    than p = 8; at p = 2 the TF32 form streams one K-part per offset, at
    p = 6 two), depth 5, against the FP64 oracle."""
    n, depth = 40000, 5
    x, y, z = inputs.uniform_cube(n, 40 + p)
    q = inputs.masses_open_unit(n, 40 + p)
    s = np.sort(np.unique((inputs.u01(9, 94, 120) * n).astype(np.int64)))
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, p, 1, sample=s)
    for prec, tol in ((F.GEMM_BF16X3, 5e-6), (F.GEMM_TF32X3, 5e-6)):
        pot, acc = run(F, x, y, z, q, p, 1, depth, prec=prec)
        ep, ea, per = errs(pot[s], acc[:, s], pref, aref)
        assert ep < tol and ea < tol, (prec, ep, ea, per)


@pytest.mark.parametrize("form", ["GEMM_BF16X3", "FP32", "FP64"])
def test_m2l_levels_split_equals_m2l(F, form):
    """fmm_m2l_levels over disjoint level ranges covering 2..depth gives
    fmm_m2l's result (levels are independent); up to the order of the FP64
    atomic adds of the split small levels."""
    n, depth, p = 131072, 5, 6
    x, y, z = inputs.uniform_cube(n, 51)
    q = inputs.masses_equal(n)
    X = [g(a) for a in (x, y, z, q)]
    plan = F.Plan(p=p, basis=1, prec=getattr(F, form), depth=depth)
    outs = []
    for split in (False, True):
        o = torch.zeros((4, n), dtype=torch.float64, device="cuda")
        plan.fmm_build_tree(*X)
        plan.fmm_p2m()
        plan.fmm_m2m()
        if split:
            plan.fmm_m2l_levels(2, 4)
            plan.fmm_m2l_levels(5, 9)
        else:
            plan.fmm_m2l()
        plan.fmm_l2l()
        plan.fmm_l2p(o[0], o[1], o[2], o[3])
        plan.fmm_p2p(o[0], o[1], o[2], o[3])
        torch.cuda.synchronize()
        outs.append(o.cpu().numpy())
    with pytest.raises(F.FMMError):
        plan.fmm_m2l_levels(4, 3)
    plan.close()
    np.testing.assert_allclose(outs[1], outs[0], rtol=1e-12, atol=0)


def test_tensor_core_form_rejects_unsupported(F):
    for prec in (F.GEMM_BF16X3, F.GEMM_TF32X3):
        with pytest.raises(F.FMMError):
            F.Plan(p=9, basis=1, prec=prec, depth=4)
        with pytest.raises(F.FMMError):
            F.Plan(p=6, basis=0, prec=prec, depth=4)


@pytest.mark.parametrize("form,shapes", [("GEMM_BF16X3", [(0, 32), (0, 48), (0, 96), (1, 48), (1, 96), (2, 256),
                                                          (3, 256)]),
                                         ("GEMM_TF32X3", [(0, 16), (0, 32), (0, 48)])])
def test_every_tensor_core_shape_vs_oracle(F, form, shapes):
    """Every kernel shape the autotuner may pick (the streamed-matrix kernel
    at each chunk width; for BF16 also the on-chip-matrix kernel) gives the
    oracle's result within the tensor-core forms' 5e-6, depth 5."""
    n, depth = 131072, 5
    x, y, z = inputs.uniform_cube(n, 16)
    q = inputs.masses_equal(n)
    s = np.sort(np.unique((inputs.u01(7, 95, 150) * n).astype(np.int64)))
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, 8, 1, sample=s)
    X = [g(a) for a in (x, y, z, q)]
    plan = F.Plan(p=8, basis=1, prec=getattr(F, form), depth=depth)
    for kern, cw in shapes:
        plan.set_tc_shape(kern, cw)
        t = plan.tuning()
        assert (t["kernel"], t["cw"], t["source"]) == (kern, cw, "set")
        pot, acc = plan.evaluate(*X)
        plan.sync_status()
        ep, ea, per = errs(pot.cpu().numpy()[s], acc.cpu().numpy()[:, s], pref, aref)
        assert ep < 5e-6 and ea < 5e-6, (kern, cw, ep, ea)
    with pytest.raises(F.FMMError):
        plan.set_tc_shape(1 if form == "GEMM_TF32X3" else 2, 48)
    plan.close()


def test_autotuned_plan_and_its_cache(F, tmp_path, monkeypatch):
    """autotune: the first M2L times every candidate and keeps the fastest;
    a second plan of the same configuration reads the choice back from the
    cache file; both agree with the oracle."""
    monkeypatch.setenv("FMM_TUNE_CACHE", str(tmp_path / "tune.json"))
    n, depth = 131072, 5
    x, y, z = inputs.uniform_cube(n, 17)
    q = inputs.masses_equal(n)
    s = np.sort(np.unique((inputs.u01(7, 96, 120) * n).astype(np.int64)))
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, 8, 1, sample=s)
    X = [g(a) for a in (x, y, z, q)]
    plan = F.Plan(p=8, basis=1, prec=F.GEMM_BF16X3, depth=depth, autotune=True)
    assert plan.tuning()["source"] == "default"
    pot, acc = plan.evaluate(*X)
    plan.sync_status()
    t = plan.tuning()
    plan.close()
    assert t["source"] == "autotuned" and len(t["candidates"]) == 7
    best = min(t["candidates"], key=lambda c: c["us"])
    assert (t["kernel"], t["cw"]) == (best["kernel"], best["cw"])
    ep, ea, _ = errs(pot.cpu().numpy()[s], acc.cpu().numpy()[:, s], pref, aref)
    assert ep < 5e-6 and ea < 5e-6
    plan2 = F.Plan(p=8, basis=1, prec=F.GEMM_BF16X3, depth=depth, autotune=True)
    t2 = plan2.tuning()
    assert t2["source"] == "cache" and (t2["kernel"], t2["cw"]) == (t["kernel"], t["cw"])
    pot2, acc2 = plan2.evaluate(*X)
    torch.cuda.synchronize()
    # the same shape; the small levels add partial sums with FP64 atomics
    torch.testing.assert_close(pot2, pot, rtol=1e-12, atol=0)
    torch.testing.assert_close(acc2, acc, rtol=1e-12, atol=1e-300)
    plan2.close()


@pytest.mark.parametrize("basis,depth,p", [(0, 3, 4), (1, 3, 6), (1, 4, 5), (0, 1, 3)])
def test_point_dipoles_vs_oracle(F, basis, depth, p):
    """Charges and point dipoles (App. B, Dipoles) through
    fmm_evaluate_dipoles (FP64) against the oracle's FMM with dipoles on the
    same tree (1e-12), and near its direct sum."""
    n = 5000 + 7 * depth
    x, y, z = inputs.uniform_cube(n, 70 + depth)
    q = inputs.masses_open_unit(n, 70 + depth) - 0.5
    px, py, pz = (inputs.u01(71 + depth, k, n) - 0.5 for k in range(3))
    X = [g(a) for a in (x, y, z, q, px, py, pz)]
    out = torch.full((4, n), 9.0, dtype=torch.float64, device=DEV)
    plan = F.Plan(p=p, basis=basis, prec=F.FP64, depth=depth)
    plan.fmm_evaluate_dipoles(*X, out[0], out[1], out[2], out[3])
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    pref, aref = oracle.fmm_uniform_dipole(x, y, z, q, px, py, pz, depth, p, basis)
    ep, ea, per = errs(o[0], o[1:], pref, aref)
    assert ep < 1e-12 and ea < 1e-12, (ep, ea)
    # dipole moments zero: the charge-only evaluation
    zero = torch.zeros(n, dtype=torch.float64, device=DEV)
    plan.fmm_evaluate_dipoles(*X[:4], zero, zero, zero, out[0], out[1], out[2], out[3])
    pot, acc = plan.evaluate(*X[:4])
    torch.cuda.synchronize()
    # (another P2M kernel: equal up to the summation order)
    assert (torch.linalg.norm(out[0] - pot) / torch.linalg.norm(pot)).item() < 1e-13
    assert (torch.linalg.norm(out[1:] - acc) / torch.linalg.norm(acc)).item() < 1e-13
    plan.close()
    with pytest.raises(F.FMMError):
        F.Plan(p=4, basis=basis, prec=F.FP32, depth=3).fmm_evaluate_dipoles(*X, out[0], out[1], out[2], out[3])


@pytest.mark.parametrize("p,depth", [(4, 3), (8, 4)])
def test_tg_basis_vs_oracle(F, p, depth):
    """The TG variant (symmetric multipoles, traceless locals) in FP64 against
    the oracle's TG FMM on the same tree (1e-12), and equal to the symmetric
    basis up to rounding."""
    n = 6000
    x, y, z = inputs.uniform_cube(n, 90 + p)
    q = inputs.masses_open_unit(n, 90 + p)
    pot, acc = run(F, x, y, z, q, p, F.BASIS_TG, depth)
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, p, oracle.TG)
    ep, ea, per = errs(pot, acc, pref, aref)
    assert ep < 1e-12 and ea < 1e-12, (ep, ea)
    ps, as_ = run(F, x, y, z, q, p, F.BASIS_SYM, depth)
    ep, ea, _ = errs(pot, acc, ps, as_)
    assert ep < 1e-12 and ea < 1e-12
    for prec in (F.FP32, F.GEMM_BF16X3):
        with pytest.raises(F.FMMError):
            F.Plan(p=p, basis=F.BASIS_TG, prec=prec, depth=depth)


@pytest.mark.parametrize("prec,p,depth,n,kern", [("GEMM_BF16X3", 8, 5, 150000, 2), ("GEMM_BF16X3", 8, 5, 150000, 3),
                                                 ("FP32", 6, 4, 40000, None), ("FP64", 4, 3, 6000, None)])
def test_uniform_graph_replay(F, prec, p, depth, n, kern):
    """use_graph on a uniform plan: the first evaluation runs eagerly, the
    second captures the whole step (tree and operators) and later ones
    replay it; with new particle positions in the same arrays the replayed
    step equals an eager plan's result (to the rounding of the atomic FP64
    accumulation of the small levels' grouped M2L, whose order may differ),
    and new output arrays make it capture again."""
    x, y, z = inputs.uniform_cube(n, 80 + depth)
    q = inputs.masses_open_unit(n, 80 + depth)
    x2, y2, z2 = inputs.uniform_cube(n, 90 + depth)
    X = [g(a) for a in (x, y, z, q)]
    stream = torch.cuda.Stream()
    gp = F.Plan(p=p, basis=1, prec=getattr(F, prec), depth=depth, use_graph=True)
    ep = F.Plan(p=p, basis=1, prec=getattr(F, prec), depth=depth)
    if kern is not None:   # kernel 3: the CUDA-core columns' launches (and level 5's group sum) in the graph
        gp.set_tc_shape(kern, 256)
        ep.set_tc_shape(kern, 256)
    out = torch.empty((4, n), device=DEV, dtype=torch.float64)
    with torch.cuda.stream(stream):
        for k in range(3):
            if k == 2:   # new positions, same arrays
                for t, a in zip(X[:3], (x2, y2, z2)):
                    t.copy_(torch.from_numpy(a).to(DEV))
            gp.fmm_evaluate(*X, out[0], out[1], out[2], out[3], stream=stream)
    stream.synchronize()
    assert gp.stats()["graph"] == 1
    ref = torch.empty_like(out)
    ep.fmm_evaluate(*X, ref[0], ref[1], ref[2], ref[3])
    torch.cuda.synchronize()

    def close(a, b):
        d = (a - b).abs().amax(dim=1)
        return bool((d <= 1e-12 * b.abs().amax(dim=1)).all())
    assert close(out, ref)
    out2 = torch.empty_like(out)
    with torch.cuda.stream(stream):
        gp.fmm_evaluate(*X, out2[0], out2[1], out2[2], out2[3], stream=stream)
    stream.synchronize()
    gp.sync_status()
    assert close(out2, ref)
    gp.close()
    ep.close()
