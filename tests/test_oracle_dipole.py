"""Oracle pins of the point-dipole sources (App. B, "Dipoles and higher
order multipoles"): a point dipole p is the limit of charges +q and -q at
x_a +- s with p = 2 q s, so every dipole result must be the limit of the
same computation on charge pairs; the direct-sum field is the closed form
of a dipole field and the gradient of its potential."""
import numpy as np
import pytest

import oracle
from paper_1811_06332_gb300 import inputs


def pairs(x, y, z, px, py, pz, h):
    """Charge pair of each dipole: +1/h at x + h p/2, -1/h at x - h p/2."""
    P = np.stack([px, py, pz])
    X = np.stack([x, y, z])
    plus, minus = X + 0.5 * h * P, X - 0.5 * h * P
    xs = np.concatenate([plus, minus], 1)
    qs = np.concatenate([np.full(len(x), 1.0 / h), np.full(len(x), -1.0 / h)])
    return xs[0], xs[1], xs[2], qs


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("p", [0, 1, 3, 6])
def test_p2m_dipole_is_the_limit_of_charge_pairs(p, basis):
    rng = np.random.default_rng(p + 10 * basis)
    n = 7
    x, y, z = rng.uniform(-0.3, 0.3, (3, n))
    px, py, pz = rng.uniform(-1, 1, (3, n))
    zc = np.array([0.05, -0.02, 0.01])
    M = oracle.p2m_dipole(p, basis, x, y, z, px, py, pz, zc)
    errs = []
    for h in (1e-2, 5e-3):
        Mq = oracle.p2m(p, basis, *pairs(x, y, z, px, py, pz, h), zc)
        errs.append(np.abs(Mq - M).max())
    scale = max(np.abs(M).max(), 1.0)
    # central difference: error O(h^2), a quarter when h halves
    assert errs[1] <= 1e-4 * scale
    if errs[0] > 1e-12 * scale:
        assert errs[1] < 0.3 * errs[0]
    if p == 0:
        assert np.all(M == 0.0)          # a dipole has no charge


def test_direct_dipole_closed_form_and_gradient():
    rng = np.random.default_rng(3)
    n = 40
    x, y, z = rng.uniform(0, 1, (3, n))
    q = np.zeros(n)
    px, py, pz = rng.uniform(-1, 1, (3, n))
    pot, acc = oracle.direct_dipole(x, y, z, q, px, py, pz)
    # closed form of the dipole potential at particle 0
    d = np.stack([x[0] - x[1:], y[0] - y[1:], z[0] - z[1:]])
    r = np.linalg.norm(d, axis=0)
    phi = ((px[1:] * d[0] + py[1:] * d[1] + pz[1:] * d[2]) / r ** 3).sum()
    assert abs(pot[0] + phi) <= 1e-12 * abs(phi)
    # acc = grad Phi: central finite difference of Phi = -pot at particle 0
    h = 1e-5
    g = []
    for k, v in enumerate((x, y, z)):
        vp, vm = v.copy(), v.copy()
        vp[0] += h
        vm[0] -= h
        args_p = [vp if j == k else w for j, w in enumerate((x, y, z))]
        args_m = [vm if j == k else w for j, w in enumerate((x, y, z))]
        fp = -oracle.direct_dipole(*args_p, q, px, py, pz, targets=[0])[0][0]
        fm = -oracle.direct_dipole(*args_m, q, px, py, pz, targets=[0])[0][0]
        g.append((fp - fm) / (2 * h))
    assert np.allclose(acc[:, 0], g, rtol=1e-6, atol=1e-6 * np.abs(g).max())
    # the charge-pair limit
    xs, ys, zs, qs = pairs(x[1:], y[1:], z[1:], px[1:], py[1:], pz[1:], 1e-4)
    xt = np.concatenate([[x[0]], xs]); yt = np.concatenate([[y[0]], ys]); zt = np.concatenate([[z[0]], zs])
    qt = np.concatenate([[0.0], qs])
    pq, aq = oracle.direct(xt, yt, zt, qt, targets=[0])
    assert abs(pq[0] - pot[0]) <= 1e-6 * abs(pot[0])
    assert np.linalg.norm(aq[:, 0] - acc[:, 0]) <= 1e-6 * np.linalg.norm(acc[:, 0])


@pytest.mark.parametrize("basis", [0, 1])
def test_fmm_with_dipoles_converges_to_the_direct_sum(basis):
    n, depth = 3000, 3
    x, y, z = inputs.uniform_cube(n, 61)
    q = inputs.masses_open_unit(n, 61) - 0.5
    px, py, pz = (inputs.u01(62, k, n) - 0.5 for k in range(3))
    pd, ad = oracle.direct_dipole(x, y, z, q, px, py, pz)
    errs = []
    for p in (2, 4, 6):
        pot, acc = oracle.fmm_uniform_dipole(x, y, z, q, px, py, pz, depth, p, basis)
        errs.append(np.sqrt(((acc - ad) ** 2).sum() / (ad ** 2).sum()))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3, errs
    # without dipoles it is the charge-only FMM
    pz0 = np.zeros(n)
    p0, a0 = oracle.fmm_uniform_dipole(x, y, z, q, pz0, pz0, pz0, depth, 4, basis)
    p1, a1 = oracle.fmm_uniform(x, y, z, q, depth, 4, basis)
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_array_equal(a0, a1)
    # traceless and symmetric storage give the same field
    if basis == 1:
        ps, as_ = oracle.fmm_uniform_dipole(x, y, z, q, px, py, pz, depth, 4, 0)
        pt, at = oracle.fmm_uniform_dipole(x, y, z, q, px, py, pz, depth, 4, 1)
        assert np.linalg.norm(at - as_) <= 1e-12 * np.linalg.norm(as_)
