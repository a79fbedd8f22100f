"""Oracle pins of the AP variant (Sec. 3, astrophysics): the fully traceless
form with expansion centres at the centre of mass, where the dipole
vanishes, and only the gradient evaluated."""
import numpy as np
import pytest

import oracle
from paper_1811_06332_gb300 import inputs


def test_centres_are_centres_of_mass_and_radii_enclose():
    n = 4000
    x, y, z = inputs.plummer(n, 31)
    q = inputs.masses_open_unit(n, 31)
    zr, rg, order = oracle.adaptive_tree(x, y, z, 32, com_q=q)
    P = np.stack([x, y, z], 1)
    for c in range(len(zr)):
        idx = order[rg[c, 0]:rg[c, 1]]
        com = (q[idx, None] * P[idx]).sum(0) / q[idx].sum()        # numpy's own sum
        assert np.abs(zr[c, :3] - com).max() <= 1e-12 * max(1.0, np.abs(com).max())
        d = np.linalg.norm(P[idx] - zr[c, :3], axis=1)
        assert d.max() <= zr[c, 3] * (1 + 1e-12)                    # the radius encloses the cell's particles


def test_dipole_about_the_centre_of_mass_vanishes():
    rng = np.random.default_rng(5)
    x, y, z = rng.uniform(-1, 1, (3, 50))
    q = rng.uniform(0.1, 1.0, 50)
    com = np.array([(q * x).sum(), (q * y).sum(), (q * z).sum()]) / q.sum()
    M = oracle.p2m(6, oracle.TRACELESS, x, y, z, q, com)
    assert np.abs(M[1:4]).max() <= 1e-14 * np.abs(M[0])


@pytest.mark.parametrize("p", [4, 6])
def test_ap_gradient_equals_ft_about_the_same_centres_and_converges(p):
    n = 6000
    x, y, z = inputs.plummer(n, 32)
    q = inputs.masses_equal(n)
    pot_ap, acc_ap, st = oracle.fmm_adaptive_ap(x, y, z, q, 32, 0.6, p)
    pot_ft, acc_ft, st2 = oracle.fmm_adaptive_com(x, y, z, q, 32, 0.6, p)
    assert st == st2
    assert np.all(pot_ap == 0.0)                                    # gradient only
    # dropping the (rounding-level) dipole changes the gradient only at rounding level
    assert np.linalg.norm(acc_ap - acc_ft) <= 1e-12 * np.linalg.norm(acc_ft)
    pd, ad = oracle.direct(x, y, z, q)
    err = np.sqrt(((acc_ap - ad) ** 2).sum() / (ad ** 2).sum())
    err_geo = np.sqrt(((oracle.fmm_adaptive(x, y, z, q, 32, 0.6, p, oracle.TRACELESS)[1] - ad) ** 2).sum() /
                      (ad ** 2).sum())
    print("AP p=%d: %.2e, geometric centres %.2e" % (p, err, err_geo))
    # the truncation error of the same p and theta, no worse than with geometric centres
    assert err < {4: 3e-3, 6: 5e-4}[p] and err < 1.5 * err_geo


def test_ap_error_decreases_with_p():
    n = 5000
    x, y, z = inputs.plummer(n, 33)
    q = inputs.masses_equal(n)
    pd, ad = oracle.direct(x, y, z, q)
    errs = []
    for p in (2, 4, 6, 8):
        _, acc, _ = oracle.fmm_adaptive_ap(x, y, z, q, 32, 0.6, p)
        errs.append(np.sqrt(((acc - ad) ** 2).sum() / (ad ** 2).sum()))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
