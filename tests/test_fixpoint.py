"""Host test of the integer fixed-point leaf coordinates of the uniform tree
build (csrc/fmm_fixpoint.h, compiled here as plain C++): for a coordinate x
in [0, 1) and depth d, the leaf index must be floor(x 2^d) and the FP32
offset from the leaf centre the float nearest (ties to even) to
floor(x 2^62) 2^-62 - (i + 1/2) 2^-d, which is x - (i + 1/2) 2^-d itself
whenever x >= 2^-10 or x has no bits below 2^-62.  The reference is exact
rational arithmetic (fractions), rounded to FP32 by hand."""
import os
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1811_06332_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "fmm_fixpoint.h"
int main(int argc, char** argv) {
    const int d = atoi(argv[1]);
    std::vector<double> x;
    double v;
    while (fread(&v, 8, 1, stdin) == 1) x.push_back(v);
    for (double xi : x) {
        int64_t X = 0;
        const int ok = fmm::fix62(xi, X) ? 1 : 0;
        int i = ok ? fmm::fix62_leaf(X, d) : -1;
        float f = ok ? fmm::fix62_offset(X, i, d) : 0.f;
        fwrite(&ok, 4, 1, stdout); fwrite(&i, 4, 1, stdout); fwrite(&f, 4, 1, stdout);
    }
    return 0;
}
"""


def f32_nearest(fr):
    """The float32 nearest to the rational fr (ties to even), normal range."""
    if fr == 0:
        return 0.0
    s = -1 if fr < 0 else 1
    a = abs(fr)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    scaled = a / Fraction(2) ** (e - 23)          # in [2^23, 2^24)
    m, rem = divmod(scaled.numerator, scaled.denominator)
    r2 = 2 * rem
    if r2 > scaled.denominator or (r2 == scaled.denominator and m % 2 == 1):
        m += 1
    return float(s * Fraction(m) * Fraction(2) ** (e - 23))


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    d = tmp_path_factory.mktemp("fix")
    src = d / "fix.cpp"
    src.write_text(PROG)
    exe = d / "fix"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def run(prog, x, d):
    out = subprocess.run([prog, str(d)], input=np.asarray(x, np.float64).tobytes(), capture_output=True,
                         check=True).stdout
    rec = np.frombuffer(out, dtype=np.dtype([("ok", "<i4"), ("i", "<i4"), ("f", "<f4")]))
    assert len(rec) == len(x)
    return rec


def coords(seed):
    rng = np.random.default_rng(seed)
    xs = list(rng.random(3000))                                  # 53-bit grid, as the synthetic inputs
    # arbitrary bit patterns in [2^-70, 1): bits below 2^-62 for the small ones
    e = rng.integers(1023 - 70, 1023, 3000)
    m = rng.integers(0, 1 << 52, 3000, dtype=np.int64)
    xs += [struct.unpack("<d", struct.pack("<Q", (int(a) << 52) | int(b)))[0] for a, b in zip(e, m)]
    xs += [0.0, 5e-324, 2.0 ** -1022, 2.0 ** -62, 2.0 ** -63, 2.0 ** -10, np.nextafter(2.0 ** -10, 0),
           0.5, np.nextafter(1.0, 0), 0.25, 0.375, 2.0 ** -7, 3 * 2.0 ** -8]
    for k in range(0, 64, 7):                                    # leaf boundaries and centres at depth 6
        for v in (k / 64, (k + 0.5) / 64):
            xs += [v, np.nextafter(v, 0), np.nextafter(v, 1)]
    return [v for v in xs if 0 <= v < 1]


@pytest.mark.parametrize("d", [0, 3, 6, 10])
def test_fixpoint_leaf_and_offset_exact(prog, d):
    xs = coords(100 + d)
    rec = run(prog, xs, d)
    assert rec["ok"].all()
    nexact = 0
    for xv, r in zip(xs, rec):
        fx = Fraction(xv)
        i = int(fx * 2 ** d)                                     # floor(x 2^d)
        assert r["i"] == i, (xv, d)
        X = int(fx * 2 ** 62)                                    # floor(x 2^62)
        want = f32_nearest(Fraction(X, 2 ** 62) - Fraction(2 * i + 1, 2 ** (d + 1)))
        assert float(r["f"]) == want, (xv, d, float(r["f"]), want)
        if Fraction(X, 2 ** 62) == fx:
            nexact += 1
            # then it is the nearest float to the exact offset
            assert float(r["f"]) == f32_nearest(fx - Fraction(2 * i + 1, 2 ** (d + 1)))
    assert nexact > len(xs) // 2


def test_fixpoint_rejects_outside_unit_interval(prog):
    bad = [-0.0, -1e-300, -0.5, 1.0, 1.5, 1e300, float("inf"), float("-inf"), float("nan")]
    rec = run(prog, bad, 6)
    assert not rec["ok"].any()
