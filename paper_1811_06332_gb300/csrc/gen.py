"""Build-time generator for the CUDA library's tables and unrolled kernels.

Emits, into csrc/_gen/:
  * fmm_tables.h     multi-index tables (App. D) and exact combinatorial maps
                     (detracer, trace expansion, reduced representative),
                     computed here with exact rational arithmetic;
  * pair_P<p>.cu     per-pair D-tensor and M2L kernels for one order p,
                     straight-line code for both bases and both precisions.

Only the Python standard library is used, so the generator runs wherever the
library is built.  Nothing here is shared with the FP64 oracle; the D-tensor
kernels use a different route to grad^n r^{-1} (the Leibniz recurrence
described at gen_dtensor) from the oracle's closed form.
"""
from __future__ import annotations

import os
import sys
from fractions import Fraction
from math import factorial

PMAX = 10
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_gen")


# ----------------------------------------------------------------------------
# multi-index enumeration (App. D) and storage orders
# ----------------------------------------------------------------------------
def rank_sym(j):
    """Rank-j multi-indices: descending nx, then descending ny."""
    return [(nx, ny, j - nx - ny) for nx in range(j, -1, -1) for ny in range(j - nx, -1, -1)]


def rank_tl(j):
    """Independent rank-j multi-indices (nz <= 1): nz = 0 block then nz = 1."""
    return [(j - ny, ny, 0) for ny in range(j + 1)] + [(j - 1 - ny, ny, 1) for ny in range(j)]


def sym_list(p):
    return [n for j in range(p + 1) for n in rank_sym(j)]


def tl_list(p):
    return [n for j in range(p + 1) for n in rank_tl(j)]


def ns(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def nt(p):
    return (p + 1) ** 2


def mfact(n):
    return factorial(n[0]) * factorial(n[1]) * factorial(n[2])


def add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


E = ((1, 0, 0), (0, 1, 0), (0, 0, 1))


# ----------------------------------------------------------------------------
# exact combinatorial maps per rank
# ----------------------------------------------------------------------------
def dfact_odd(k):
    v = 1
    for i in range(2 * k - 1, 1, -2):
        v *= i
    return v


def detracer_rank(j):
    """Matrix of the idempotent detracer D = T/(2j-1)!! on rank-j symmetric
    tensors (rows, cols: rank_sym(j)), from Eq. Detracer of App. A:
    T[A]_n = sum_{m <= n/2} f_{n,m} sum_{|k|=|m|} (|m|!/k!) A_{n-2m+2k}."""
    idx = rank_sym(j)
    col = {n: i for i, n in enumerate(idx)}
    Mx = [[Fraction(0)] * len(idx) for _ in idx]
    for r, n in enumerate(idx):
        for mx in range(n[0] // 2 + 1):
            for my in range(n[1] // 2 + 1):
                for mz in range(n[2] // 2 + 1):
                    m = (mx, my, mz)
                    mm = mx + my + mz
                    f = Fraction((-1) ** mm * dfact_odd(j - mm) * mfact(n),
                                 2 ** mm * mfact(m) * mfact(sub(n, (2 * mx, 2 * my, 2 * mz))))
                    for k in rank_sym(mm):
                        tgt = (n[0] - 2 * mx + 2 * k[0], n[1] - 2 * my + 2 * k[1], n[2] - 2 * mz + 2 * k[2])
                        Mx[r][col[tgt]] += f * Fraction(factorial(mm), mfact(k))
    s = Fraction(1, dfact_odd(j))
    return [[v * s for v in row] for row in Mx]


def expand_rank(j):
    """Matrix X (rank_sym(j) x rank_tl(j)) rebuilding every component of a
    trace-free rank-j tensor from its independent ones by the trace condition
    A_{k+2ez} = -A_{k+2ex} - A_{k+2ey}."""
    idx = rank_sym(j)
    tl = rank_tl(j)
    tcol = {n: i for i, n in enumerate(tl)}
    rows = {}
    for n in idx:  # symmetric order visits both right-hand sides first
        if n[2] <= 1:
            v = [Fraction(0)] * len(tl)
            v[tcol[n]] = Fraction(1)
        else:
            a = rows[(n[0] + 2, n[1], n[2] - 2)]
            b = rows[(n[0], n[1] + 2, n[2] - 2)]
            v = [-x - y for x, y in zip(a, b)]
        rows[n] = v
    return [rows[n] for n in idx]


def solve_exact(A, B):
    """Solves A X = B exactly (A square, Fractions), Gauss-Jordan."""
    n = len(A)
    M = [list(A[i]) + list(B[i]) for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        pv = M[c][c]
        M[c] = [v / pv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [row[n:] for row in M]


def reduce_rank(j):
    """Matrix P (rank_tl(j) x rank_sym(j)) taking any symmetric rank-j tensor
    A to the unique tensor A^r supported on the nz <= 1 components with
    D[A^r] = D[A].  Because grad^k r^{-1} is trace free, contracting it with
    A^r or with A gives the same number, so the traceless M2L, M2M and
    P2M can run over the 2j+1 stored components only."""
    idx = rank_sym(j)
    tl = rank_tl(j)
    Dm = detracer_rank(j)
    pos = {n: i for i, n in enumerate(idx)}
    rows_tl = [pos[n] for n in tl]
    # restriction of D to nz<=1 inputs, read on the independent outputs
    Dr = [[Dm[r][pos[c]] for c in tl] for r in rows_tl]
    # P = Dr^{-1} (D restricted to independent output rows)
    rhs = [[Dm[r][c] for c in range(len(idx))] for r in rows_tl]
    return solve_exact(Dr, rhs)


# ----------------------------------------------------------------------------
# C emission helpers
# ----------------------------------------------------------------------------
def lit(x, T="T"):
    x = float(x)
    if x == int(x) and abs(x) < 1e15:
        return "%s(%d.0)" % (T, int(x))
    return "%s(%.17g)" % (T, x)


def emit_tables():
    L = []
    L.append("// Generated by gen.py: multi-index tables and exact combinatorial maps.")
    L.append("#pragma once")
    L.append("#define FMM_PMAX %d" % PMAX)
    sl, tlst = sym_list(PMAX), tl_list(PMAX)
    L.append("#define FMM_NS_MAX %d" % len(sl))
    L.append("#define FMM_NT_MAX %d" % len(tlst))
    L.append("static const unsigned char fmm_sym_idx[%d][3] = {%s};" % (
        len(sl), ",".join("{%d,%d,%d}" % n for n in sl)))
    L.append("static const unsigned char fmm_tl_idx[%d][3] = {%s};" % (
        len(tlst), ",".join("{%d,%d,%d}" % n for n in tlst)))
    # per-rank dense maps, flattened with offsets
    for name, fn, shape in (("fmm_detr", detracer_rank, lambda j: ((j + 1) * (j + 2) // 2, (j + 1) * (j + 2) // 2)),
                            ("fmm_expand", expand_rank, lambda j: ((j + 1) * (j + 2) // 2, 2 * j + 1)),
                            ("fmm_reduce", reduce_rank, lambda j: (2 * j + 1, (j + 1) * (j + 2) // 2))):
        vals, offs = [], []
        for j in range(PMAX + 1):
            offs.append(len(vals))
            Mx = fn(j)
            r, c = shape(j)
            assert len(Mx) == r and all(len(row) == c for row in Mx), (name, j)
            for row in Mx:
                vals.extend(row)
        offs.append(len(vals))
        L.append("static const int %s_off[%d] = {%s};" % (name, PMAX + 2, ",".join(map(str, offs))))
        L.append("static const double %s_val[%d] = {%s};" % (
            name, len(vals), ",".join("%.17g" % float(v) for v in vals)))
    return "\n".join(L) + "\n"


# ----------------------------------------------------------------------------
# D-tensor by recurrence.
#
# With phi = 1/|x|, d/dx_i phi = -x_i phi / |x|^2, i.e. |x|^2 d_i phi + x_i phi = 0.
# Applying d^(k - e_i) with Leibniz' rule (d_j |x|^2 = 2 x_j, d_j^2 |x|^2 = 2)
# gives, for any axis i with k_i >= 1,
#   |x|^2 D_k = -[ (2k_i - 1) x_i D_{k-e_i} + sum_{j!=i} 2 k_j x_j D_{k-e_j}
#                 + (k_i - 1)^2 D_{k-2e_i} + sum_{j!=i} k_j (k_j - 1) D_{k-2e_j} ],
# with D_k = d^k phi.  Each component costs at most six products.
# ----------------------------------------------------------------------------
def dtensor_terms(k):
    i = max(range(3), key=lambda a: (k[a], -a))
    terms = []  # (coef, axis or None, source index)
    for j in range(3):
        if k[j] == 0:
            continue
        c = (2 * k[j] - 1) if j == i else 2 * k[j]
        terms.append((c, j, sub(k, E[j])))
    for j in range(3):
        c = (k[j] - 1) ** 2 if j == i else k[j] * (k[j] - 1)
        if k[j] >= 2 and c:
            terms.append((c, None, sub(k, tuple(2 * v for v in E[j]))))
    return terms


def gen_dtensor(p, T="T", out="d"):
    """Straight-line code computing out[0..ns(p)) = grad^k |r|^{-1}."""
    pos = {n: i for i, n in enumerate(sym_list(p))}
    xs = ("x", "y", "z")
    L = ["  const T r2 = x * x + y * y + z * z;",
         "  const T ir2 = T(1) / r2;",
         "  %s[0] = fmm_rsqrt(r2);" % out]
    for k in sym_list(p)[1:]:
        parts = []
        for c, ax, src in dtensor_terms(k):
            cc = lit(c, T)
            if ax is None:
                parts.append("%s * %s[%d]" % (cc, out, pos[src]))
            else:
                parts.append("%s * %s * %s[%d]" % (cc, xs[ax], out, pos[src]))
        L.append("  %s[%d] = -ir2 * (%s);" % (out, pos[k], " + ".join(parts)))
    return "\n".join(L)


# ----------------------------------------------------------------------------
# per-pair M2L (Eq. M2L): L_n += sum_{|m| <= p-|n|} (1/m!) M_m D_{n+m}(r)
# ----------------------------------------------------------------------------
def gen_m2l_pair(p, basis, tile):
    syml = sym_list(p)
    pos = {n: i for i, n in enumerate(syml)}
    outs = syml if basis == 0 else tl_list(p)
    tpos = {n: i for i, n in enumerate(tl_list(p))}
    L = []
    for t0 in range(0, len(outs), tile):
        tl_ = outs[t0:t0 + tile]
        minr = min(sum(n) for n in tl_)
        L.append("  {")
        for a, n in enumerate(tl_):
            L.append("    T a%d = accumulate ? Lp[(int64_t)%d * n + t] : T(0);" % (a, t0 + a))
        for b in range(0, p - minr + 1):
            blk = rank_sym(b)
            L.append("    {")
            # load rank-b multipole block (reconstructing dependents in tl)
            for m in blk:
                if basis == 0:
                    L.append("      const T m_%d_%d_%d = __ldg(&Mp[(int64_t)%d * n + t]);" % (m + (pos[m],)))
                elif m[2] <= 1:
                    L.append("      const T m_%d_%d_%d = __ldg(&Mp[(int64_t)%d * n + t]);" % (m + (tpos[m],)))
                else:
                    L.append("      const T m_%d_%d_%d = -m_%d_%d_%d - m_%d_%d_%d;" % (
                        m + (m[0] + 2, m[1], m[2] - 2) + (m[0], m[1] + 2, m[2] - 2)))
            for m in blk:
                users = [(a, n) for a, n in enumerate(tl_) if sum(n) + b <= p]
                if not users:
                    continue
                f = mfact(m)
                mc = "m_%d_%d_%d" % m if f == 1 else "(m_%d_%d_%d * %s)" % (m + (lit(Fraction(1, f)),))
                L.append("      { const T c = %s;" % mc)
                for a, n in users:
                    L.append("        a%d = fma(c, d[%d], a%d);" % (a, pos[add(n, m)], a))
                L.append("      }")
            L.append("    }")
        for a, n in enumerate(tl_):
            L.append("    Lp[(int64_t)%d * n + t] = a%d;" % (t0 + a, a))
        L.append("  }")
    return "\n".join(L)


def emit_pair_file(p):
    """D-tensor kernels and the M2L launcher of order p."""
    L = ['// Generated by gen.py: per-pair D-tensor kernels and M2L dispatch, p = %d.' % p,
         '#include "../fmm_device.cuh"',
         "namespace fmm {",
         ""]
    for basis in (0, 1):
        for T in ("float", "double"):
            L.append("int launch_m2l_pair_p%d_b%d_%s(int64_t n, const void* M, const double* r, void* L,"
                     " int accumulate, cudaStream_t s);" % (p, basis, T))
    L.append("template <typename T> __global__ void __launch_bounds__(128)")
    L.append("dtensor_pair_p%d(int64_t n, const double* __restrict__ r, T* __restrict__ D) {" % p)
    L.append("  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;")
    L.append("  if (t >= n) return;")
    L.append("  const T x = T(r[t]), y = T(r[n + t]), z = T(r[2 * n + t]);")
    L.append("  T d[%d];" % ns(p))
    L.append(gen_dtensor(p))
    L.append("  #pragma unroll")
    L.append("  for (int i = 0; i < %d; ++i) D[(int64_t)i * n + t] = d[i];" % ns(p))
    L.append("}")
    L.append("")
    # traceless storage: D is trace free (harmonic), so the independent
    # components (nz <= 1, traceless order) determine it
    spos = {n: i for i, n in enumerate(sym_list(p))}
    tsel = ", ".join(str(spos[n]) for n in tl_list(p))
    L.append("template <typename T> __global__ void __launch_bounds__(128)")
    L.append("dtensor_pair_tl_p%d(int64_t n, const double* __restrict__ r, T* __restrict__ D) {" % p)
    L.append("  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;")
    L.append("  if (t >= n) return;")
    L.append("  const T x = T(r[t]), y = T(r[n + t]), z = T(r[2 * n + t]);")
    L.append("  T d[%d];" % ns(p))
    L.append(gen_dtensor(p))
    L.append("  constexpr int sel[%d] = {%s};" % (len(tl_list(p)), tsel))
    L.append("  #pragma unroll")
    L.append("  for (int i = 0; i < %d; ++i) D[(int64_t)i * n + t] = d[sel[i]];" % len(tl_list(p)))
    L.append("}")
    L.append("")
    L.append("template <typename T> __device__ __forceinline__ void dtensor_p%d(T x, T y, T z, T* d) {" % p)
    L.append(gen_dtensor(p))
    L.append("}")
    L.append("")
    L.append("int launch_dtensor_p%d(int basis, int prec, int64_t n, const double* r, void* D, cudaStream_t s) {"
             % p)
    L.append("  if (n <= 0) return 0;")
    L.append("  const unsigned g = (unsigned)((n + 127) / 128);")
    L.append("  if (basis == 0 && prec == 0) dtensor_pair_p%d<double><<<g, 128, 0, s>>>(n, r, (double*)D);" % p)
    L.append("  else if (basis == 0) dtensor_pair_p%d<float><<<g, 128, 0, s>>>(n, r, (float*)D);" % p)
    L.append("  else if (prec == 0) dtensor_pair_tl_p%d<double><<<g, 128, 0, s>>>(n, r, (double*)D);" % p)
    L.append("  else dtensor_pair_tl_p%d<float><<<g, 128, 0, s>>>(n, r, (float*)D);" % p)
    L.append("  return 0;")
    L.append("}")
    L.append("int launch_m2l_pair_p%d(int basis, int prec, int64_t n, const void* M, const double* r, void* L,"
             " int accumulate, cudaStream_t s) {" % p)
    L.append("  if (n <= 0) return 0;")
    for basis in (0, 1):
        L.append("  if (basis == %d && prec == 0) return launch_m2l_pair_p%d_b%d_double(n, M, r, L, accumulate, s);"
                 % (basis, p, basis))
        L.append("  if (basis == %d && prec == 1) return launch_m2l_pair_p%d_b%d_float(n, M, r, L, accumulate, s);"
                 % (basis, p, basis))
    L.append("  return -1;")
    L.append("}")
    L.append("")
    L.append("__global__ void dtable_p%d(int noff, const double* __restrict__ o, double* __restrict__ D) {" % p)
    L.append("  const int t = blockIdx.x * blockDim.x + threadIdx.x;")
    L.append("  if (t >= noff) return;")
    L.append("  double d[%d];" % ns(p))
    L.append("  dtensor_p%d<double>(o[3 * t], o[3 * t + 1], o[3 * t + 2], d);" % p)
    L.append("  for (int i = 0; i < %d; ++i) D[(int64_t)t * %d + i] = d[i];" % (ns(p), ns(p)))
    L.append("}")
    L.append("int launch_dtable_p%d(int noff, const double* o, double* D, cudaStream_t s) {" % p)
    L.append("  dtable_p%d<<<(noff + 63) / 64, 64, 0, s>>>(noff, o, D);" % p)
    L.append("  return 0;")
    L.append("}")
    L.append("}  // namespace fmm")
    return "\n".join(L) + "\n"


def emit_m2l_file(p, basis, T):
    """One per-pair M2L kernel (order p, basis, precision) and its launcher."""
    tile = 40 if T == "float" else 24
    L = ['// Generated by gen.py: per-pair M2L (Eq. M2L), p = %d, basis %d, %s.' % (p, basis, T),
         '#include "../fmm_device.cuh"',
         "namespace fmm {",
         "__global__ void __launch_bounds__(128)",
         "m2l_pair_p%d_b%d_%s(int64_t n, const %s* __restrict__ Mp, const double* __restrict__ r,"
         " %s* __restrict__ Lp, int accumulate) {" % (p, basis, T, T, T),
         "  typedef %s T;" % T,
         "  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;",
         "  if (t >= n) return;",
         "  const T x = T(r[t]), y = T(r[n + t]), z = T(r[2 * n + t]);",
         "  T d[%d];" % ns(p),
         gen_dtensor(p),
         gen_m2l_pair(p, basis, tile),
         "}",
         "int launch_m2l_pair_p%d_b%d_%s(int64_t n, const void* M, const double* r, void* L,"
         " int accumulate, cudaStream_t s) {" % (p, basis, T),
         "  m2l_pair_p%d_b%d_%s<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, (const %s*)M, r, (%s*)L,"
         " accumulate);" % (p, basis, T, T, T),
         "  return 0;",
         "}",
         "}  // namespace fmm"]
    return "\n".join(L) + "\n"


def grouped_layout(p, basis):
    """Row/column structure of the offset-grouped M2L matrices
    Kt_r(n, m) = D_{n+m}(r)/m! (cell units): rows n = output components in
    storage order, columns m = multipole components of rank <= p - |n|, which
    form a prefix of the storage order.  Returns (rows, prefix length per
    row, packed offset per row, packed size)."""
    # basis 2 (the TG variant): traceless rows, full symmetric multipole columns
    rows = sym_list(p) if basis == 0 else tl_list(p)
    pre = [(nt(p - sum(n)) if basis == 1 else ns(p - sum(n))) for n in rows]
    off = [0]
    for k in pre:
        off.append(off[-1] + k)
    return rows, pre, off, off[-1]


def grouped_parts(p, basis, budget=200):
    """Splits the output rows so that accumulators + multipole registers of
    one kernel stay within `budget` 32-bit registers."""
    rows, pre, _, _ = grouped_layout(p, basis)
    parts, r0 = [], 0
    while r0 < len(rows):
        r1 = r0 + 1
        while r1 < len(rows) and (r1 + 1 - r0) + pre[r0] <= budget:
            r1 += 1
        parts.append((r0, r1))
        r0 = r1
    return parts


def kstride(p, basis):
    return (grouped_layout(p, basis)[3] + 3) // 4 * 4


def emit_grouped_file(p, basis, T="float"):
    """Offset-grouped M2L over the uniform interaction lists of one level, in
    FP32 (T = float) or FP64 (T = double) arithmetic: one thread per target
    cell, the block's 128 targets share one parity class and hence one
    sequence of 189 offsets; the packed matrix of each offset is staged in
    shared memory and read by every thread at the same address, the source
    multipole sits in registers, and every thread runs the same unrolled
    FMA sequence (no divergence over the rank triangle)."""
    rows, pre, off, ksz = grouped_layout(p, basis)
    kst = kstride(p, basis)
    f64 = T == "double"
    sfx = "64" if f64 else ""
    L = ['// Generated by gen.py: %s offset-grouped M2L, p = %d, basis %d.' % ("FP64" if f64 else "FP32", p, basis),
         '#include "../fmm_device.cuh"',
         "namespace fmm {"]
    # FP64 values take two registers: half the row budget
    parts = grouped_parts(p, basis, budget=100 if f64 else 200)
    for k, (r0, r1) in enumerate(parts):
        klen = off[r1] - off[r0]
        ncol = pre[r0]
        L.append("template <typename OT>   // the type of the stored locals")
        L.append("__global__ void __launch_bounds__(128)")
        L.append("m2l_grp%s_p%d_b%d_r%d(int l, const %s* __restrict__ M, OT* __restrict__ Lt,"
                 " const %s* __restrict__ K, int64_t ncell, OT* __restrict__ part) {" % (sfx, p, basis, k, T, T))
        L.append("  __shared__ __align__(16) %s sK[%d];" % (T, (klen + 3) // 4 * 4))
        L.append("  const int side = 1 << l, hs = side >> 1, bs = (int)blockDim.x;   // 128 or (FP64 small levels) 32")
        L.append("  const int64_t h3 = (int64_t)hs * hs * hs, bpc = (h3 + bs - 1) / bs;")
        L.append("  const int cls = (int)(blockIdx.x / bpc);")
        L.append("  const int64_t t = (int64_t)(blockIdx.x % bpc) * bs + threadIdx.x;")
        L.append("  const bool act = t < h3;")
        L.append("  const int cx = cls & 1, cy = (cls >> 1) & 1, cz = cls >> 2;")
        L.append("  const int ix = 2 * (int)(t % hs) + cx, iy = 2 * (int)((t / hs) % hs) + cy,"
                 " iz = 2 * (int)(t / ((int64_t)hs * hs)) + cz;")
        for a in range(r1 - r0):
            L.append("  %s a%d = 0;" % (T, a))
        L.append("  // offsets of this block: group blockIdx.y of gridDim.y (one group on large levels)")
        L.append("  const int u0 = (int)blockIdx.y * 216 / (int)gridDim.y, u1 = ((int)blockIdx.y + 1) * 216 / (int)gridDim.y;")
        L.append("  #pragma unroll 1")
        L.append("  for (int u = u0; u < u1; ++u) {")
        L.append("    const int ox = -2 - cx + u % 6, oy = -2 - cy + (u / 6) % 6, oz = -2 - cz + u / 36;")
        L.append("    if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;")
        L.append("    const %s* Kg = K + (int64_t)((3 - oz) * 49 + (3 - oy) * 7 + (3 - ox)) * %d + %d;" % (T, kst, off[r0]))
        L.append("    __syncthreads();")
        L.append("    for (int e = threadIdx.x; e < %d; e += bs) sK[e] = __ldg(Kg + e);" % klen)
        L.append("    __syncthreads();")
        L.append("    const int jx = ix + ox, jy = iy + oy, jz = iz + oz;")
        L.append("    if (!act || jx < 0 || jy < 0 || jz < 0 || jx >= side || jy >= side || jz >= side) continue;")
        L.append("    const int64_t s = cell_index(l, jx, jy, jz);")
        for c in range(ncol):
            L.append("    const %s m%d = __ldg(M + (int64_t)%d * ncell + s);" % (T, c, c))
        for r in range(r0, r1):
            base = off[r] - off[r0]
            for c in range(pre[r]):
                L.append("    a%d = fma(sK[%d], m%d, a%d);" % (r - r0, base + c, c, r - r0))
        L.append("  }")
        L.append("  if (!act) return;")
        L.append("  const int64_t tg = (int64_t)cls * h3 + t;")
        L.append("  if (gridDim.y == 1) {")
        for r in range(r0, r1):
            L.append("    Lt[(int64_t)%d * ncell + tg] = (OT)a%d;" % (r, r - r0))
        L.append("  } else if (part) {   // partial sums of this offset group, added in group order afterwards")
        for r in range(r0, r1):
            L.append("    part[((int64_t)blockIdx.y * %d + %d) * ncell + tg] = (OT)a%d;" % (len(rows), r, r - r0))
        L.append("  } else {")
        for r in range(r0, r1):
            L.append("    atomicAdd(Lt + (int64_t)%d * ncell + tg, (OT)a%d);" % (r, r - r0))
        L.append("  }")
        L.append("}")
    L.append("// groups > 1 splits the 216 offset slots of every target over that many")
    L.append("// blocks (small levels).  Without part the partial sums are added into a")
    L.append("// zeroed Lt with atomics; with part (groups x %d x ncell doubles) they are" % len(rows))
    L.append("// stored there and added in group order (the result does not depend on")
    L.append("// scheduling).  bs: threads (targets) per block, 128 or 32.")
    L.append("template <typename OT>")
    L.append("static int launch_m2l_grp%s_t_p%d_b%d(int l, const %s* M, OT* Lt, const %s* K, int64_t ncell,"
             " cudaStream_t s, int groups, int bs, OT* part) {" % (sfx, p, basis, T, T))
    L.append("  const int hs = (1 << l) >> 1;")
    L.append("  const int64_t h3 = (int64_t)hs * hs * hs, bpc = (h3 + bs - 1) / bs;")
    L.append("  if (groups > 1 && !part && cudaMemsetAsync(Lt, 0, (size_t)%d * ncell * sizeof(OT), s) != cudaSuccess) return -1;" % len(rows))
    for k in range(len(parts)):
        L.append("  m2l_grp%s_p%d_b%d_r%d<OT><<<dim3((unsigned)(8 * bpc), (unsigned)groups), bs, 0, s>>>(l, M, Lt, K, ncell, part);"
                 % (sfx, p, basis, k))
    L.append("  if (groups > 1 && part) { launch_sum_parts(part, Lt, (int64_t)%d * ncell, groups, s); return %d; }" % (len(rows), len(parts) + 1))
    L.append("  return %d;" % len(parts))
    L.append("}")
    L.append("int launch_m2l_grp%s_p%d_b%d(int l, const %s* M, double* Lt, const %s* K, int64_t ncell,"
             " cudaStream_t s, int groups, int bs, double* part) {" % (sfx, p, basis, T, T))
    L.append("  return launch_m2l_grp%s_t_p%d_b%d<double>(l, M, Lt, K, ncell, s, groups, bs, part);" % (sfx, p, basis))
    L.append("}")
    if not f64:
        L.append("// FP32 locals (uniform FP32 and tensor-core plans)")
        L.append("int launch_m2l_grpf_p%d_b%d(int l, const float* M, float* Lt, const float* K, int64_t ncell,"
                 " cudaStream_t s, int groups, int bs, float* part) {" % (p, basis))
        L.append("  return launch_m2l_grp_t_p%d_b%d<float>(l, M, Lt, K, ncell, s, groups, bs, part);" % (p, basis))
        L.append("}")
    L.append("}  // namespace fmm")
    return "\n".join(L) + "\n"


def shift_layout(p, basis, upper):
    """Packed layout of the level-independent shift matrices (scaled units).
    M2M (upper=False): row n uses columns of rank <= |n| (a prefix);
    L2L (upper=True): row n uses columns of rank >= |n| (a suffix).
    Returns (rows, (c0, c1) column range per row, packed offset, size)."""
    rows = sym_list(p) if basis == 0 else tl_list(p)
    pre = (lambda k: ns(k)) if basis == 0 else (lambda k: nt(k))
    nc = len(rows)
    rng = []
    for n in rows:
        a = sum(n)
        rng.append((pre(a - 1) if a > 0 else 0, nc) if upper else (0, pre(a)))
    off = [0]
    for c0, c1 in rng:
        off.append(off[-1] + c1 - c0)
    return rows, rng, off, off[-1]


def shift32_ok(p, basis):
    return 2 * (ns(p) if basis == 0 else nt(p)) <= 180


def emit_shift_file(p, basis):
    """FP32 M2M / L2L on one uniform level (scaled units).  M2M: one thread
    per parent, the eight child matrices staged in shared memory in turn.
    L2L: one thread per child, all threads of a block in one child class,
    which selects the matrix.  Expansions stay FP64 in memory; L2L adds its
    FP32 result into the FP64 local expansion."""
    L = ['// Generated by gen.py: FP32 level shifts (M2M, L2L), p = %d, basis %d.' % (p, basis),
         '#include "../fmm_device.cuh"', "namespace fmm {"]
    nc = ns(p) if basis == 0 else nt(p)
    if shift32_ok(p, basis):
        # ---- M2M ----
        rows, rng, off, sz = shift_layout(p, basis, False)
        L.append("__global__ void __launch_bounds__(128)")
        L.append("m2m32_p%d_b%d(int l, const float* __restrict__ W, const double* __restrict__ Mch, int64_t nch,"
                 " double* __restrict__ Mpa, int64_t npa) {" % (p, basis))
        L.append("  __shared__ float sW[%d];" % sz)
        L.append("  const int64_t P = (int64_t)blockIdx.x * 128 + threadIdx.x;")
        L.append("  const bool act = P < npa;")
        L.append("  int ix = 0, iy = 0, iz = 0;")
        L.append("  if (act) cell_coords(l, P, ix, iy, iz);")
        L.append("  const int64_t lin = lin_index(l, ix, iy, iz), blk = (int64_t)1 << (3 * l);")
        for r in range(nc):
            L.append("  float a%d = 0.f;" % r)
        L.append("  #pragma unroll 1")
        L.append("  for (int c = 0; c < 8; ++c) {")
        L.append("    __syncthreads();")
        L.append("    for (int e = threadIdx.x; e < %d; e += 128) sW[e] = W[c * %d + e];" % (sz, sz))
        L.append("    __syncthreads();")
        L.append("    if (!act) continue;")
        L.append("    const int64_t ch = c * blk + lin;")
        for k in range(nc):
            L.append("    const float x%d = (float)Mch[(int64_t)%d * nch + ch];" % (k, k))
        for r in range(nc):
            c0, c1 = rng[r]
            for k in range(c0, c1):
                L.append("    a%d = fmaf(sW[%d], x%d, a%d);" % (r, off[r] + k - c0, k, r))
        L.append("  }")
        L.append("  if (!act) return;")
        for r in range(nc):
            L.append("  Mpa[(int64_t)%d * npa + P] = (double)a%d;" % (r, r))
        L.append("}")
        # ---- M2M, one child class per block row: the eight children of a
        # parent on eight threads (blockIdx.y = child class), their FP32
        # contributions summed afterwards in child order (m2m32_sum) ----
        L.append("__global__ void __launch_bounds__(128)")
        L.append("m2m32c_p%d_b%d(int l, const float* __restrict__ W, const float* __restrict__ Mch, int64_t nch,"
                 " float* __restrict__ part, int64_t npa) {" % (p, basis))
        L.append("  __shared__ float sW[%d];" % sz)
        L.append("  const int c = (int)blockIdx.y;")
        L.append("  for (int e = threadIdx.x; e < %d; e += 128) sW[e] = W[c * %d + e];" % (sz, sz))
        L.append("  __syncthreads();")
        L.append("  const int64_t P = (int64_t)blockIdx.x * 128 + threadIdx.x;")
        L.append("  if (P >= npa) return;")
        L.append("  int ix, iy, iz;")
        L.append("  cell_coords(l, P, ix, iy, iz);")
        L.append("  const int64_t ch = c * ((int64_t)1 << (3 * l)) + lin_index(l, ix, iy, iz);")
        for k in range(nc):
            L.append("  const float x%d = Mch[(int64_t)%d * nch + ch];" % (k, k))
        for r in range(nc):
            c0, c1 = rng[r]
            L.append("  {")
            L.append("    float a = 0.f;")
            for k in range(c0, c1):
                L.append("    a = fmaf(sW[%d], x%d, a);" % (off[r] + k - c0, k))
            L.append("    part[((int64_t)c * %d + %d) * npa + P] = a;" % (nc, r))
            L.append("  }")
        L.append("}")
        # ---- L2L ----
        rows, rng, off, sz = shift_layout(p, basis, True)
        L.append("__global__ void __launch_bounds__(128)")
        L.append("l2l32_p%d_b%d(int l, const float* __restrict__ V, const double* __restrict__ Lpa, int64_t npa,"
                 " double* __restrict__ Lch, int64_t nch) {" % (p, basis))
        L.append("  __shared__ float sV[%d];" % sz)
        L.append("  const int64_t blk = (int64_t)1 << (3 * l), bpc = (blk + 127) / 128;")
        L.append("  const int c = (int)(blockIdx.x / bpc);")
        L.append("  const int64_t lin = (int64_t)(blockIdx.x % bpc) * 128 + threadIdx.x;")
        L.append("  for (int e = threadIdx.x; e < %d; e += 128) sV[e] = V[c * %d + e];" % (sz, sz))
        L.append("  __syncthreads();")
        L.append("  if (lin >= blk) return;")
        L.append("  const int s = 1 << l;")
        L.append("  const int px = (int)(lin % s), py = (int)((lin / s) % s), pz = (int)(lin / ((int64_t)s * s));")
        L.append("  const int64_t P = cell_index(l, px, py, pz), C = c * blk + lin;")
        for k in range(nc):
            L.append("  const float x%d = (float)Lpa[(int64_t)%d * npa + P];" % (k, k))
        # rows in blocks of 16: the block's old values are loaded before its
        # sums, so that the read-modify-writes of a block are one round trip
        # rather than one per row
        for r0 in range(0, nc, 16):
            r1 = min(nc, r0 + 16)
            L.append("  {")
            for r in range(r0, r1):
                L.append("    const double o%d = Lch[(int64_t)%d * nch + C];" % (r, r))
            for r in range(r0, r1):
                c0, c1 = rng[r]
                L.append("    float a%d = 0.f;" % r)
                for k in range(c0, c1):
                    L.append("    a%d = fmaf(sV[%d], x%d, a%d);" % (r, off[r] + k - c0, k, r))
            for r in range(r0, r1):
                L.append("    Lch[(int64_t)%d * nch + C] = o%d + (double)a%d;" % (r, r, r))
            L.append("  }")
        L.append("}")
        # ---- L2L on FP32 locals (uniform FP32 and tensor-core plans): the
        # same sums, read-modify-writes in FP32 ----
        L.append("__global__ void __launch_bounds__(128)")
        L.append("l2l32f_p%d_b%d(int l, const float* __restrict__ V, const float* __restrict__ Lpa, int64_t npa,"
                 " float* __restrict__ Lch, int64_t nch) {" % (p, basis))
        L.append("  __shared__ float sV[%d];" % sz)
        L.append("  const int64_t blk = (int64_t)1 << (3 * l), bpc = (blk + 127) / 128;")
        L.append("  const int c = (int)(blockIdx.x / bpc);")
        L.append("  const int64_t lin = (int64_t)(blockIdx.x % bpc) * 128 + threadIdx.x;")
        L.append("  for (int e = threadIdx.x; e < %d; e += 128) sV[e] = V[c * %d + e];" % (sz, sz))
        L.append("  __syncthreads();")
        L.append("  if (lin >= blk) return;")
        L.append("  const int s = 1 << l;")
        L.append("  const int px = (int)(lin % s), py = (int)((lin / s) % s), pz = (int)(lin / ((int64_t)s * s));")
        L.append("  const int64_t P = cell_index(l, px, py, pz), C = c * blk + lin;")
        for k in range(nc):
            L.append("  const float x%d = Lpa[(int64_t)%d * npa + P];" % (k, k))
        for r0 in range(0, nc, 16):
            r1 = min(nc, r0 + 16)
            L.append("  {")
            for r in range(r0, r1):
                L.append("    const float o%d = Lch[(int64_t)%d * nch + C];" % (r, r))
            for r in range(r0, r1):
                c0, c1 = rng[r]
                L.append("    float a%d = 0.f;" % r)
                for k in range(c0, c1):
                    L.append("    a%d = fmaf(sV[%d], x%d, a%d);" % (r, off[r] + k - c0, k, r))
            for r in range(r0, r1):
                L.append("    Lch[(int64_t)%d * nch + C] = o%d + a%d;" % (r, r, r))
            L.append("  }")
        L.append("}")
    L.append("int launch_l2l32f_p%d_b%d(int l, const float* V, const float* X, int64_t nx, float* Y, int64_t ny,"
             " cudaStream_t s) {" % (p, basis))
    if shift32_ok(p, basis):
        L.append("  l2l32f_p%d_b%d<<<(unsigned)(8 * ((((int64_t)1 << (3 * l)) + 127) / 128)), 128, 0, s>>>"
                 "(l, V, X, nx, Y, ny);" % (p, basis))
        L.append("  return 1;")
    else:
        L.append("  return -1;")
    L.append("}")
    L.append("int launch_shift32_p%d_b%d(int m2m, int l, const float* A, const double* X, int64_t nx, double* Y,"
             " int64_t ny, cudaStream_t s, float* part, const float* X32, float* Y32) {" % (p, basis))
    if shift32_ok(p, basis):
        L.append("  if (m2m && part && X32 && Y32) {")
        L.append("    m2m32c_p%d_b%d<<<dim3((unsigned)((ny + 127) / 128), 8), 128, 0, s>>>(l, A, X32, nx, part, ny);"
                 % (p, basis))
        L.append("    launch_m2m32_sum(%d, ny, part, Y, Y32, s);" % nc)
        L.append("    return 2;")
        L.append("  }")
        L.append("  if (m2m) m2m32_p%d_b%d<<<(unsigned)((ny + 127) / 128), 128, 0, s>>>(l, A, X, nx, Y, ny);"
                 % (p, basis))
        L.append("  else l2l32_p%d_b%d<<<(unsigned)(8 * ((((int64_t)1 << (3 * l)) + 127) / 128)), 128, 0, s>>>"
                 "(l, A, X, nx, Y, ny);" % (p, basis))
        L.append("  return 1;")
    else:
        L.append("  return -1;")
    L.append("}")
    L.append("}  // namespace fmm")
    return "\n".join(L) + "\n"


def emit_shift_dispatch():
    L = ['// Generated by gen.py: dispatch and packed layouts of the FP32 level shifts.',
         '#include "../fmm_device.cuh"', "namespace fmm {"]
    for p in range(PMAX + 1):
        for b in (0, 1):
            L.append("int launch_shift32_p%d_b%d(int m2m, int l, const float* A, const double* X, int64_t nx,"
                     " double* Y, int64_t ny, cudaStream_t s, float* part, const float* X32, float* Y32);" % (p, b))
    for p in range(PMAX + 1):
        for b in (0, 1):
            L.append("int launch_l2l32f_p%d_b%d(int l, const float* V, const float* X, int64_t nx, float* Y,"
                     " int64_t ny, cudaStream_t s);" % (p, b))
    L.append("// L2L on FP32 locals; returns the launches made, -1 without a kernel")
    L.append("int launch_l2l32f(int p, int basis, int l, const float* V, const float* X, int64_t nx, float* Y,"
             " int64_t ny, cudaStream_t s) {")
    for p in range(PMAX + 1):
        for b in (0, 1):
            L.append("  if (p == %d && basis == %d) return launch_l2l32f_p%d_b%d(l, V, X, nx, Y, ny, s);"
                     % (p, b, p, b))
    L.append("  return -1;")
    L.append("}")
    L.append("// part: 8 x nc x ny floats for the per-child M2M (m2m32c + m2m32_sum), which")
    L.append("// reads the children's FP32 copy X32 and writes both Y and its FP32 copy Y32;")
    L.append("// without them the one-thread-per-parent M2M.  Returns the launches made.")
    L.append("int launch_shift32(int p, int basis, int m2m, int l, const float* A, const double* X, int64_t nx,"
             " double* Y, int64_t ny, cudaStream_t s, float* part, const float* X32, float* Y32) {")
    for p in range(PMAX + 1):
        for b in (0, 1):
            L.append("  if (p == %d && basis == %d)" % (p, b))
            L.append("    return launch_shift32_p%d_b%d(m2m, l, A, X, nx, Y, ny, s, part, X32, Y32);" % (p, b))
    L.append("  return -1;")
    L.append("}")
    # packed entry lists (row, column) for host-side packing
    L.append("int shift32_supported(int p, int basis) {")
    for p in range(PMAX + 1):
        for b in (0, 1):
            L.append("  if (p == %d && basis == %d) return %d;" % (p, b, 1 if shift32_ok(p, b) else 0))
    L.append("  return 0;")
    L.append("}")
    L.append("}  // namespace fmm")
    return "\n".join(L) + "\n"


def emit_list_file(p, basis, T):
    """M2L over explicit interaction lists (adaptive trees): one thread per
    target node of a work queue ordered by list length; the D-tensor of each
    (target, source) pair is computed on the fly (physical units), every
    output component accumulates in a register, and expansions are stored
    node-major ([node][ncoef]) so each thread reads one contiguous block.
    Work is handed out in warps of 32 targets from an atomic counter
    (persistent grid)."""
    syml = sym_list(p)
    pos = {n: i for i, n in enumerate(syml)}
    outs = syml if basis == 0 else tl_list(p)
    tpos = {n: i for i, n in enumerate(tl_list(p))}
    nc = len(outs)
    L = ['// Generated by gen.py: list M2L (adaptive trees), p = %d, basis %d, %s.' % (p, basis, T),
         '#include "../fmm_device.cuh"', "namespace fmm {",
         "__global__ void __launch_bounds__(128)",
         "m2l_list_p%d_b%d_%s(int ntarg, const int* __restrict__ order, const int* __restrict__ off,"
         " const int* __restrict__ src, const double* __restrict__ zc, const int4* __restrict__ ic, float scale,"
         " const %s* __restrict__ Mn, int ldm, double* __restrict__ Ln, int ld, int accum,"
         " int* __restrict__ counter) {" % (p, basis, T, T),
         "  typedef %s T;" % T,
         "  const int lane = threadIdx.x & 31;",
         "  for (;;) {",
         "    int base = 0;",
         "    if (lane == 0) base = atomicAdd(counter, 32);",
         "    base = __shfl_sync(0xffffffffu, base, 0);",
         "    if (base >= ntarg) break;",
         "    const int w = base + lane;",
         "    if (w >= ntarg) continue;",
         "    const int t = order[w];"]
    if T == "double":
        L.append("    const double tx = zc[3 * t], ty = zc[3 * t + 1], tz = zc[3 * t + 2];")
    else:
        # centre offsets from the integer node centres: exact integer
        # difference, one FP32 rounding (no FP64 arithmetic per pair).
        # Scaled units (FP32 form): Mt_A = M_A / h_A^|m|, Lt_B = L_B h_B^(|n|+1),
        # so Lt_n = sum_m (h_A/h_B)^|m| Mt_m/m! D_{n+m}(d/h_B); h_c = side/2^level,
        # d/h_B = (ic_B - ic_A) 2^(level_B - 22), h_A/h_B = 2^(level_B - level_A).
        L.append("    const int4 it = ic[t];")
        L.append("    const T sB = ldexpf(1.0f, it.w - 22);")
    for a in range(nc):
        L.append("    T a%d = T(0);" % a)
    L.append("    for (int k = off[t]; k < off[t + 1]; ++k) {")
    L.append("      const int s = src[k];")
    if T == "double":
        L.append("      const T x = T(tx - zc[3 * s]), y = T(ty - zc[3 * s + 1]), z = T(tz - zc[3 * s + 2]);")
    else:
        L.append("      const int4 is = ic[s];")
        L.append("      const T x = T(it.x - is.x) * sB, y = T(it.y - is.y) * sB, z = T(it.z - is.z) * sB;")
        L.append("      const T rho = ldexpf(1.0f, it.w - is.w);")
        L.append("      T rp = T(1);")
    if T == "double":
        L.append("      const T* __restrict__ Ms = Mn + (int64_t)s * ldm;")
    else:
        # FP32 multipoles sit in rows padded to a multiple of 4: 16-byte loads
        L.append("      const float4* __restrict__ Mv = (const float4*)(Mn + (int64_t)s * ldm);")
    L.append("      T d[%d];" % ns(p))
    L.append("  " + gen_dtensor(p).replace("\n", "\n  "))
    for b in range(p + 1):
        blk = rank_sym(b)
        L.append("      {")
        if T == "float" and b > 0:
            L.append("        rp *= rho;")
        stored = [pos[m] for m in blk] if basis == 0 else [tpos[m] for m in blk if m[2] <= 1]
        if T == "float":
            for qv in range(min(stored) // 4, max(stored) // 4 + 1):
                L.append("        const float4 q%d = Mv[%d];" % (qv, qv))

        def mload(i):
            return ("q%d.%s" % (i // 4, "xyzw"[i % 4])) if T == "float" else ("Ms[%d]" % i)
        for m in blk:
            if basis == 0:
                L.append("        const T m_%d_%d_%d = %s;" % (m + (mload(pos[m]),)))
            elif m[2] <= 1:
                L.append("        const T m_%d_%d_%d = %s;" % (m + (mload(tpos[m]),)))
            else:
                L.append("        const T m_%d_%d_%d = -m_%d_%d_%d - m_%d_%d_%d;" % (
                    m + (m[0] + 2, m[1], m[2] - 2) + (m[0], m[1] + 2, m[2] - 2)))
        for m in blk:
            users = [(a, n) for a, n in enumerate(outs) if sum(n) + b <= p]
            if not users:
                continue
            f = mfact(m)
            mc = "m_%d_%d_%d" % m if f == 1 else "(m_%d_%d_%d * %s)" % (m + (lit(Fraction(1, f)),))
            if T == "float" and b > 0:
                mc = "(%s * rp)" % mc
            L.append("        { const T c = %s;" % mc)
            for a, n in users:
                L.append("          a%d = fma(c, d[%d], a%d);" % (a, pos[add(n, m)], a))
            L.append("        }")
        L.append("      }")
    L.append("    }")
    L.append("    double* __restrict__ Lt = Ln + (int64_t)t * ld;")
    L.append("    if (accum) {")
    for a in range(nc):
        L.append("      Lt[%d] += (double)a%d;" % (a, a))
    L.append("    } else {")
    for a in range(nc):
        L.append("      Lt[%d] = (double)a%d;" % (a, a))
    L.append("    }")
    L.append("  }")
    L.append("}")
    L.append("int launch_m2l_list_p%d_b%d_%s(int ntarg, const int* order, const int* off, const int* src,"
             " const double* zc, const int4* ic, float scale, const void* M, int ldm, double* Ln, int ld,"
             " int accum, int* counter, int blocks, cudaStream_t s) {" % (p, basis, T))
    L.append("  m2l_list_p%d_b%d_%s<<<blocks, 128, 0, s>>>(ntarg, order, off, src, zc, ic, scale, (const %s*)M,"
             " ldm, Ln, ld, accum, counter);" % (p, basis, T, T))
    L.append("  return 0;")
    L.append("}")
    L.append("}  // namespace fmm")
    return "\n".join(L) + "\n"


def emit_list_dispatch():
    L = ['// Generated by gen.py: dispatch of the list M2L kernels.', '#include "../fmm_device.cuh"',
         "namespace fmm {"]
    for p in range(PMAX + 1):
        for b in (0, 1):
            for T in ("float", "double"):
                L.append("int launch_m2l_list_p%d_b%d_%s(int ntarg, const int* order, const int* off, const int* src,"
                         " const double* zc, const int4* ic, float scale, const void* M, int ldm, double* Ln,"
                         " int ld, int accum, int* counter, int blocks, cudaStream_t s);" % (p, b, T))
    L.append("int launch_m2l_list(int p, int basis, int prec, int ntarg, const int* order, const int* off,"
             " const int* src, const double* zc, const int4* ic, float scale, const void* M, int ldm, double* Ln,"
             " int ld, int accum, int* counter, int blocks, cudaStream_t s) {")
    for p in range(PMAX + 1):
        for b in (0, 1):
            for k, T in ((0, "double"), (1, "float")):
                L.append("  if (p == %d && basis == %d && prec == %d) return launch_m2l_list_p%d_b%d_%s(ntarg, order,"
                         " off, src, zc, ic, scale, M, ldm, Ln, ld, accum, counter, blocks, s);" % (p, b, k, p, b, T))
    L.append("  return -1;")
    L.append("}")
    L.append("}  // namespace fmm")
    return "\n".join(L) + "\n"


def emit_grouped_dispatch():
    L = ['// Generated by gen.py: dispatch and layout of the FP32 and FP64 offset-grouped M2L.',
         '#include "../fmm_device.cuh"', "namespace fmm {"]
    for p in range(PMAX + 1):
        for b in (0, 1):
            L.append("int launch_m2l_grp_p%d_b%d(int l, const float* M, double* Lt, const float* K, int64_t ncell,"
                     " cudaStream_t s, int groups, int bs, double* part);" % (p, b))
            L.append("int launch_m2l_grpf_p%d_b%d(int l, const float* M, float* Lt, const float* K, int64_t ncell,"
                     " cudaStream_t s, int groups, int bs, float* part);" % (p, b))
            L.append("int launch_m2l_grp64_p%d_b%d(int l, const double* M, double* Lt, const double* K,"
                     " int64_t ncell, cudaStream_t s, int groups, int bs, double* part);" % (p, b))
        L.append("int launch_m2l_grp64_p%d_b2(int l, const double* M, double* Lt, const double* K,"
                 " int64_t ncell, cudaStream_t s, int groups, int bs, double* part);" % p)
    L.append("// Levels with fewer target blocks than about four per SM split the offsets")
    L.append("// of every target over up to 27 blocks.")
    L.append("int launch_m2l_grp(int p, int basis, int l, const float* M, double* Lt, const float* K,"
             " int64_t ncell, cudaStream_t s) {")
    L.append("  static int sms = 0;")
    L.append("  if (!sms) { int d = 0; cudaGetDevice(&d); cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);"
             " if (sms <= 0) sms = 1; }")
    L.append("  const int64_t hs = (int64_t)1 << (l - 1), blocks = 8 * ((hs * hs * hs + 127) / 128);")
    L.append("  int64_t g = (4 * (int64_t)sms + blocks - 1) / blocks;")
    L.append("  const int groups = (int)(g < 1 ? 1 : g > 27 ? 27 : g);")
    for p in range(PMAX + 1):
        for b in (0, 1):
            L.append("  if (p == %d && basis == %d) return launch_m2l_grp_p%d_b%d(l, M, Lt, K, ncell, s, groups, 128, nullptr);"
                     % (p, b, p, b))
    L.append("  return -1;")
    L.append("}")
    L.append("int grouped_nrows(int p, int basis);")
    L.append("// The same with FP32 locals, deterministic: the split small levels write")
    L.append("// their groups' partial sums to part and add them in group order (no atomic")
    L.append("// adds); without room in part (part_cap floats) a level runs unsplit.")
    L.append("static int grpf_split(int l) {")
    L.append("  static int sms = 0;")
    L.append("  if (!sms) { int d = 0; cudaGetDevice(&d); cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);"
             " if (sms <= 0) sms = 1; }")
    L.append("  const int64_t hs = (int64_t)1 << (l - 1), blocks = 8 * ((hs * hs * hs + 127) / 128);")
    L.append("  const int64_t g = (4 * (int64_t)sms + blocks - 1) / blocks;")
    L.append("  return (int)(g < 1 ? 1 : g > 27 ? 27 : g);")
    L.append("}")
    L.append("int64_t m2l_grpf_part_elems(int p, int basis, int l) {")
    L.append("  const int g = grpf_split(l);")
    L.append("  return g > 1 ? (int64_t)g * grouped_nrows(p, basis) * ((int64_t)1 << (3 * l)) : 0;")
    L.append("}")
    L.append("int launch_m2l_grpf(int p, int basis, int l, const float* M, float* Lt, const float* K,"
             " int64_t ncell, cudaStream_t s, float* part, int64_t part_cap) {")
    L.append("  int groups = grpf_split(l);")
    L.append("  if (!part || (int64_t)groups * grouped_nrows(p, basis) * ncell > part_cap) groups = 1;")
    for p in range(PMAX + 1):
        for b in (0, 1):
            L.append("  if (p == %d && basis == %d) return launch_m2l_grpf_p%d_b%d(l, M, Lt, K, ncell, s, groups, 128, part);"
                     % (p, b, p, b))
    L.append("  return -1;")
    L.append("}")
    L.append("// The FP64 form stays deterministic: levels with fewer than two 128-target")
    L.append("// blocks per SM take blocks of 32, and levels with fewer target blocks than")
    L.append("// about four per SM split the offsets over up to 27 groups whose partial sums")
    L.append("// go to part and are added in group order (no atomic adds); without room in")
    L.append("// part (part_cap doubles) the level runs unsplit.")
    L.append("static int grp64_split(int l, int* bs_out) {")
    L.append("  static int sms = 0;")
    L.append("  if (!sms) { int d = 0; cudaGetDevice(&d); cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);"
             " if (sms <= 0) sms = 1; }")
    L.append("  const int64_t hs = (int64_t)1 << (l - 1), h3 = hs * hs * hs, blocks128 = 8 * ((h3 + 127) / 128);")
    L.append("  const int bs = blocks128 >= 2 * (int64_t)sms ? 128 : 32;")
    L.append("  const int64_t blocks = 8 * ((h3 + bs - 1) / bs);")
    L.append("  const int64_t g = (4 * (int64_t)sms + blocks - 1) / blocks;")
    L.append("  *bs_out = bs;")
    L.append("  return (int)(g < 1 ? 1 : g > 27 ? 27 : g);")
    L.append("}")
    L.append("int grouped_nrows(int p, int basis) {")
    for p in range(PMAX + 1):
        for b in (0, 1, 2):
            L.append("  if (p == %d && basis == %d) return %d;" % (p, b, len(grouped_layout(p, b)[0])))
    L.append("  return -1;")
    L.append("}")
    L.append("// doubles of part that level l needs for its split (0: the level runs unsplit)")
    L.append("int64_t m2l_grp64_part_elems(int p, int basis, int l) {")
    L.append("  int bs = 0;")
    L.append("  const int g = grp64_split(l, &bs);")
    L.append("  return g > 1 ? (int64_t)g * grouped_nrows(p, basis) * ((int64_t)1 << (3 * l)) : 0;")
    L.append("}")
    L.append("int launch_m2l_grp64(int p, int basis, int l, const double* M, double* Lt, const double* K,"
             " int64_t ncell, cudaStream_t s, double* part, int64_t part_cap) {")
    L.append("  int bs = 0;")
    L.append("  int groups = grp64_split(l, &bs);")
    L.append("  if (!part || (int64_t)groups * grouped_nrows(p, basis) * ncell > part_cap) groups = 1;")
    for p in range(PMAX + 1):
        for b in (0, 1, 2):
            L.append("  if (p == %d && basis == %d) return launch_m2l_grp64_p%d_b%d(l, M, Lt, K, ncell, s, groups, bs, part);"
                     % (p, b, p, b))
    L.append("  return -1;")
    L.append("}")
    L.append("int grouped_kstride(int p, int basis) {")
    for p in range(PMAX + 1):
        for b in (0, 1, 2):
            L.append("  if (p == %d && basis == %d) return %d;" % (p, b, kstride(p, b)))
    L.append("  return -1;")
    L.append("}")
    L.append("}  // namespace fmm")
    return "\n".join(L) + "\n"


def emit_ctables():
    """Statically initialised __constant__ copies of the small index tables
    (one copy per translation unit that includes the header)."""
    sl, tlst = sym_list(PMAX), tl_list(PMAX)
    L = ["// Generated by gen.py: device constant tables (internal linkage).", "#pragma once",
         "namespace fmm {"]
    L.append("static __constant__ unsigned char c_sym_idx[%d][3] = {%s};" % (
        len(sl), ",".join("{%d,%d,%d}" % n for n in sl)))
    L.append("static __constant__ unsigned char c_tl_idx[%d][3] = {%s};" % (
        len(tlst), ",".join("{%d,%d,%d}" % n for n in tlst)))
    L.append("static __constant__ double c_invfact[%d] = {%s};" % (
        PMAX + 2, ",".join("%.17g" % (1.0 / factorial(i)) for i in range(PMAX + 2))))
    rows = []
    for a in range(PMAX + 1):
        rows.append("{" + ",".join("%d.0" % (factorial(a) // (factorial(b) * factorial(a - b)) if b <= a else 0)
                                  for b in range(PMAX + 1)) + "}")
    L.append("static __constant__ double c_binom[%d][%d] = {%s};" % (PMAX + 1, PMAX + 1, ",".join(rows)))
    L.append("}  // namespace fmm")
    return "\n".join(L) + "\n"


def write_if_changed(path, text):
    if os.path.exists(path):
        with open(path) as f:
            if f.read() == text:
                return False
    with open(path + ".tmp", "w") as f:
        f.write(text)
    os.replace(path + ".tmp", path)
    return True


def generate(out=OUT):
    os.makedirs(out, exist_ok=True)
    files = []
    p_t = os.path.join(out, "fmm_tables.h")
    write_if_changed(p_t, emit_tables())
    files.append(p_t)
    p_c = os.path.join(out, "fmm_ctables.cuh")
    write_if_changed(p_c, emit_ctables())
    files.append(p_c)
    for p in range(0, PMAX + 1):
        fp = os.path.join(out, "pair_P%d.cu" % p)
        write_if_changed(fp, emit_pair_file(p))
        files.append(fp)
        for basis in (0, 1):
            for T in ("float", "double"):
                fm = os.path.join(out, "m2l_P%d_b%d_%s.cu" % (p, basis, T))
                write_if_changed(fm, emit_m2l_file(p, basis, T))
                files.append(fm)
            fg = os.path.join(out, "grp_P%d_b%d.cu" % (p, basis))
            write_if_changed(fg, emit_grouped_file(p, basis))
            files.append(fg)
            fg64 = os.path.join(out, "grp64_P%d_b%d.cu" % (p, basis))
            write_if_changed(fg64, emit_grouped_file(p, basis, "double"))
            files.append(fg64)
        fg2 = os.path.join(out, "grp64_P%d_b2.cu" % p)
        write_if_changed(fg2, emit_grouped_file(p, 2, "double"))
        files.append(fg2)
    for p in range(0, PMAX + 1):
        for basis in (0, 1):
            fs = os.path.join(out, "shift_P%d_b%d.cu" % (p, basis))
            write_if_changed(fs, emit_shift_file(p, basis))
            files.append(fs)
    for p in range(0, PMAX + 1):
        for basis in (0, 1):
            for T in ("float", "double"):
                fl = os.path.join(out, "list_P%d_b%d_%s.cu" % (p, basis, T))
                write_if_changed(fl, emit_list_file(p, basis, T))
                files.append(fl)
    fld = os.path.join(out, "list_dispatch.cu")
    write_if_changed(fld, emit_list_dispatch())
    files.append(fld)
    fsd = os.path.join(out, "shift_dispatch.cu")
    write_if_changed(fsd, emit_shift_dispatch())
    files.append(fsd)
    fd = os.path.join(out, "grp_dispatch.cu")
    write_if_changed(fd, emit_grouped_dispatch())
    files.append(fd)
    return files


if __name__ == "__main__":
    for f in generate(sys.argv[1] if len(sys.argv) > 1 else OUT):
        print(f)
