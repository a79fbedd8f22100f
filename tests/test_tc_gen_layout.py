"""Host-side layout of the BF16 tensor-core M2L kernel that builds every
offset's matrix in shared memory (csrc/fmm_m2l_tcgen.cu), checked without a
GPU: resource limits, bounds of every store and MMA read, and a byte-level
emulation of one matrix stage -- the generator threads' stores, the MMA's
K-major core-matrix reads, the three split products -- against the oracle's
D-tensor and Eq. M2L."""
import ctypes

from math import factorial

import numpy as np
import pytest

import oracle

SMEM_MAX = 227 * 1024


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    from paper_1811_06332_gb300 import fmm
    return fmm


def gen_layout(F, p, cw, niss):
    out = (ctypes.c_int * 19)()
    grp = (ctypes.c_uint32 * (4 * 256))()
    n = F.lib().fmm_tc_gen_layout(p, cw, niss, out, 19, grp, 4 * 256)
    assert n == 19, n
    v = list(out)
    d = dict(zip(["cw", "nch", "bstage", "nb", "niss", "ngroups", "smem"], v[:7]))
    d["kch"], d["coff"] = v[7:13], v[13:19]
    g = np.array(list(grp), dtype=np.uint32).reshape(256, 4)[:d["ngroups"]]
    return d, g


def bf16(x):
    """float32 -> BF16 (round to nearest even), returned as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def rank_tl(r):
    return int(np.floor(np.sqrt(r)))


CASES = [(p, cw, niss) for p in range(1, 9) for cw in (16, 32, 48, 96) for niss in (1, 2)]


@pytest.mark.parametrize("p,cw,niss", CASES)
def test_limits_and_bounds(F, p, cw, niss):
    d, g = gen_layout(F, p, cw, niss)
    nc = (p + 1) ** 2
    assert d["cw"] == cw and d["niss"] == niss
    assert d["nch"] == (nc + cw - 1) // cw and d["nch"] <= 6
    assert d["smem"] <= SMEM_MAX
    assert 2 <= d["nb"] <= 4 and d["nb"] % niss == 0
    assert d["ngroups"] <= 256                      # one generator thread per group
    assert 2 * cw * d["nch"] <= 256                 # one issuer's TMEM accumulators
    assert cw % 16 == 0 and 2 * cw <= 256           # MMA N of both shapes (M = 128)
    assert d["bstage"] % 1024 == 0
    end = 0
    for j in range(d["nch"]):
        need = (p - rank_tl(cw * j) + 1) ** 2        # columns of the chunk's lowest rank
        assert d["kch"][j] * 16 >= need and (d["kch"][j] - 1) * 16 < need
        assert d["coff"][j] == end
        end += (2 * cw // 8) * d["kch"][j] * 256      # 2 cw rows x kch K-steps; last MMA byte read < end
    assert end <= d["bstage"]
    # every store 16-byte aligned, inside its row's chunk, no two stores overlap
    offs = np.concatenate([g[:, 2], g[:, 3]])
    assert np.all(offs % 16 == 0) and np.all(offs + 16 <= end)
    assert len(np.unique(offs)) == len(offs)
    # the groups cover exactly the rank triangle: row r of rank a has
    # ceil((p - a + 1)^2 / 8) groups
    assert len(g) == sum(-(-(p - rank_tl(r) + 1) ** 2 // 8) for r in range(nc))


def decode_stage(stage, d, nc, p):
    """Matrix rows (hi, lo) as the MMAs read them: chunk j, row rr < 2 cw,
    multipole column kk < 16 kch[j] at coff + (rr/8) 256 kch + (kk/8) 128 +
    (rr%8) 16 + (kk%8) 2 bytes."""
    cw = d["cw"]
    hi = np.zeros((nc, 96), dtype=np.float32)
    lo = np.zeros((nc, 96), dtype=np.float32)
    for n in range(nc):
        j, rr = divmod(n, cw)
        kch = d["kch"][j]
        for part, rrow in ((hi, rr), (lo, rr + cw)):
            for kk in range(16 * kch):
                b = d["coff"][j] + (rrow // 8) * 256 * kch + (kk // 8) * 128 + (rrow % 8) * 16 + (kk % 8) * 2
                part[n, kk] = np.array([int.from_bytes(stage[b:b + 2].tobytes(), "little") << 16],
                                       dtype=np.uint32).view(np.float32)[0]
    return hi, lo


@pytest.mark.parametrize("p,cw", [(8, 48), (8, 32), (8, 96), (8, 16), (5, 48), (2, 32), (1, 16)])
def test_stage_emulation_equals_oracle_m2l(F, p, cw):
    d, g = gen_layout(F, p, cw, 1)
    nc, ns = (p + 1) ** 2, oracle.ncoef(p, 0)
    rng = np.random.default_rng(p * 100 + cw)
    o = np.array([3.0, -2.0, 1.0])                      # a well-separated integer offset (cell units)
    D = oracle.dtensor(p, -o).astype(np.float32)         # the kernel's FP32 D vector of r = -o
    dvec = np.zeros(176, dtype=np.float32)
    dvec[:ns] = D
    # generator threads: 8 values per group, split hi + lo in BF16, two stores
    stage = np.zeros(d["bstage"], dtype=np.uint8)
    for w0, w1, ohi, olo in g:
        ix = [(int(w0) >> (8 * e)) & 255 for e in range(4)] + [(int(w1) >> (8 * e)) & 255 for e in range(4)]
        v = np.array([dvec[i] if i < 255 else 0.0 for i in ix], dtype=np.float32)
        h = bf16(v)
        lo_ = bf16(v - h)
        stage[ohi:ohi + 16] = (h.view(np.uint32) >> 16).astype(np.uint16).view(np.uint8)
        stage[olo:olo + 16] = (lo_.view(np.uint32) >> 16).astype(np.uint16).view(np.uint8)
    hi, lo = decode_stage(stage, d, nc, p)
    # the matrix is D_{n+m} on |n| + |m| <= p and zero elsewhere
    idx_t = oracle.indices(p, 1)
    idx_s = [tuple(v) for v in oracle.indices(p, 0)]
    ref = np.zeros((nc, 96))
    for n in range(nc):
        for m in range(nc):
            if idx_t[n].sum() + idx_t[m].sum() <= p:
                ref[n, m] = D[idx_s.index(tuple(idx_t[n] + idx_t[m]))]
    B = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.all((ref == 0) <= (B == 0))                              # zeros stay exactly zero
    assert np.abs(B - ref).max() <= 2.0 ** -16 * np.abs(ref).max()       # hi + lo keeps ~16 bits
    # the three split products with A = M^r / m! (hi + lo) give Eq. M2L
    Mr = rng.standard_normal(nc)
    fact = np.array([factorial(v[0]) * factorial(v[1]) * factorial(v[2]) for v in idx_t], dtype=np.float64)
    A = (Mr / fact).astype(np.float32)
    Ah = bf16(A).astype(np.float64)
    Al = bf16(A - bf16(A)).astype(np.float64)
    L = (hi.astype(np.float64)[:, :nc] @ Ah + lo.astype(np.float64)[:, :nc] @ Ah + hi.astype(np.float64)[:, :nc] @ Al)
    Mfull = np.zeros(ns)
    for m in range(nc):
        Mfull[idx_s.index(tuple(idx_t[m]))] = Mr[m]
    Lref_s = oracle.m2l(p, 0, Mfull, -o)
    Lref = np.array([Lref_s[idx_s.index(tuple(v))] for v in idx_t])
    den = np.abs(Mr / fact) @ np.abs(ref[:, :nc]).T
    assert np.max(np.abs(L - Lref) / np.maximum(den, 1e-300)) < 3e-5


def test_rejects(F):
    out = (ctypes.c_int * 19)()
    L = F.lib()
    assert L.fmm_tc_gen_layout(9, 48, 1, out, 19, None, 0) == F.ERR_ARG
    assert L.fmm_tc_gen_layout(8, 40, 1, out, 19, None, 0) == F.ERR_ARG
    assert L.fmm_tc_gen_layout(8, 48, 3, out, 19, None, 0) == F.ERR_ARG
    assert L.fmm_tc_gen_layout(8, 48, 1, out, 7, None, 0) == 7
