// Adaptive-octree FMM (App. C with an octree): tree construction from Morton
// keys, enclosing radii, directed dual-tree traversal with the multipole
// acceptance criterion theta |z_A - z_B| > r_A + r_B, interaction lists in
// CSR form, and the tree forms of P2M, M2M, L2L, L2P and P2P.  Expansions
// are kept node-major ([node][ncoef]) in physical units and public storage
// (full symmetric, or independent traceless components).
//
// Geometry (bounding cube, centres, radii, MAC) is evaluated with explicitly
// rounded FP64 operations (no fused multiply-add) in the same order as the
// plain C formulation, so the tree and the lists do not depend on the
// compiler's contraction choices.
#include "fmm_internal.h"

namespace fmm {

// ---------------------------------------------------------------------------
// bounding cube: lo[3], side, scale = 2^21 / side
// ---------------------------------------------------------------------------
__global__ void k_bbox_partial(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ z, double* __restrict__ part) {
    __shared__ double s[6][256];
    double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308};
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const double v[3] = {x[i], y[i], z[i]};
        for (int d = 0; d < 3; ++d) { lo[d] = fmin(lo[d], v[d]); hi[d] = fmax(hi[d], v[d]); }
    }
    for (int d = 0; d < 3; ++d) { s[d][threadIdx.x] = lo[d]; s[3 + d][threadIdx.x] = hi[d]; }
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o)
            for (int d = 0; d < 3; ++d) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + o]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_bbox_final(int nblk, const double* __restrict__ part, double* __restrict__ box) {
    if (threadIdx.x || blockIdx.x) return;
    double lo[3] = {1e308, 1e308, 1e308}, hi[3] = {-1e308, -1e308, -1e308};
    for (int b = 0; b < nblk; ++b)
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], part[b * 6 + d]);
            hi[d] = fmax(hi[d], part[b * 6 + 3 + d]);
        }
    double side = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double e = __dsub_rn(hi[d], lo[d]);
        if (e > side) side = e;
    }
    if (side == 0.0) side = 1.0;
    side = __dmul_rn(side, 1.0 + 1e-12);
    box[0] = lo[0]; box[1] = lo[1]; box[2] = lo[2];
    box[3] = side;
    box[4] = __ddiv_rn(2097152.0, side);
}

__device__ __forceinline__ uint64_t spread21(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void k_morton(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ z, const double* __restrict__ box, uint64_t* __restrict__ key,
                         int* __restrict__ val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v[3] = {x[i], y[i], z[i]};
    uint64_t k = 0;
    for (int d = 0; d < 3; ++d) {
        int64_t c = (int64_t)floor(__dmul_rn(__dsub_rn(v[d], box[d]), box[4]));
        c = c < 0 ? 0 : (c > 2097151 ? 2097151 : c);
        k |= spread21((uint64_t)c) << d;
    }
    key[i] = k;
    val[i] = (int)i;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint64 key, int value), 8-bit digits.
// Tiles of 2048 elements per block (8 warps x 8 rounds x 32); stable local
// ranks from __match_any_sync within a round plus running per-warp counts.
// ---------------------------------------------------------------------------
constexpr int RS_TILE = 2048;

__global__ void __launch_bounds__(256) k_rs_hist(int64_t n, const uint64_t* __restrict__ key, int shift,
                                                 int nblk, int* __restrict__ hist) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * RS_TILE;
    for (int k = threadIdx.x; k < RS_TILE; k += 256) {
        const int64_t i = b + k;
        if (i < n) atomicAdd(&h[(int)((key[i] >> shift) & 255ull)], 1);
    }
    __syncthreads();
    hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(256) k_rs_scatter(int64_t n, const uint64_t* __restrict__ kin,
                                                    const int* __restrict__ vin, uint64_t* __restrict__ kout,
                                                    int* __restrict__ vout, int shift, int nblk,
                                                    const int* __restrict__ base) {
    __shared__ int cnt[8][256];
    __shared__ int wbase[8][256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < 256 * 8; d += 256) (&cnt[0][0])[d] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE + w * 256;
    int loc[8], dig[8];
    uint64_t kk[8];
    int vv[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t i = t0 + r * 32 + lane;
        const bool act = i < n;
        kk[r] = act ? kin[i] : 0;
        vv[r] = act ? vin[i] : 0;
        const int d = act ? (int)((kk[r] >> shift) & 255ull) : 256 + lane;   // inactive lanes never match
        dig[r] = d;
        const unsigned m = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(m & ((1u << lane) - 1u));
        int c0 = 0;
        if (act) c0 = cnt[w][d];
        __syncwarp();
        loc[r] = c0 + rank;
        if (act && rank == 0) cnt[w][d] = c0 + __popc(m);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps for every digit
    {
        const int d = threadIdx.x;
        int s = 0;
        for (int ww = 0; ww < 8; ++ww) { wbase[ww][d] = s; s += cnt[ww][d]; }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t i = t0 + r * 32 + lane;
        if (i < n) {
            const int d = dig[r];
            const int64_t o = (int64_t)base[d * nblk + blockIdx.x] + wbase[w][d] + loc[r];
            kout[o] = kk[r];
            vout[o] = vv[r];
        }
    }
}

// Sorts (key, val) by key bits [0, bits), 8 bits per pass; buffers
// alternate.  Returns 1 when the result is in (k1, v1) (an odd number of
// passes), 0 when it is in (k0, v0).  Scratch: hist (256 * nblk + 1 ints)
// and scan scratch.
int radix_sort(int64_t n, uint64_t* k0, int* v0, uint64_t* k1, int* v1, int bits, int* hist, int* hsum,
               int* scratch, cudaStream_t s) {
    if (n <= 1) return 0;
    const int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    const int passes = (bits + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = 8 * ps;
        uint64_t* ki = (ps & 1) ? k1 : k0;
        int* vi = (ps & 1) ? v1 : v0;
        uint64_t* ko = (ps & 1) ? k0 : k1;
        int* vo = (ps & 1) ? v0 : v1;
        k_rs_hist<<<nblk, 256, 0, s>>>(n, ki, shift, nblk, hist);
        count_launch();
        scan_excl_int(hist, hsum, (int64_t)256 * nblk, scratch, s);
        k_rs_scatter<<<nblk, 256, 0, s>>>(n, ki, vi, ko, vo, shift, nblk, hsum);
        count_launch();
    }
    return passes & 1;
}

// ---------------------------------------------------------------------------
// tree construction, level by level
// ---------------------------------------------------------------------------
// For each node of the level with more than max_leaf particles (and level
// below 21): the octant ranges by binary search on the sorted keys.
__global__ void k_split_count(int lb, int le, int max_leaf, const int* __restrict__ lev,
                              const int* __restrict__ nb, const int* __restrict__ ne,
                              const uint64_t* __restrict__ key, int* __restrict__ bounds, int* __restrict__ nch) {
    const int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    const int b = nb[c], e = ne[c], L = lev[c];
    int* bd = bounds + 9 * (c - lb);
    if (e - b <= max_leaf || L >= 21) { nch[c - lb] = 0; return; }
    const int shift = 3 * (20 - L);
    bd[0] = b;
    bd[8] = e;
    for (int o = 1; o < 8; ++o) {   // first position whose octant digit is >= o
        int lo = b, hi = e;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int)((key[mid] >> shift) & 7ull) < o) lo = mid + 1; else hi = mid;
        }
        bd[o] = lo;
    }
    int k = 0;
    for (int o = 0; o < 8; ++o) k += bd[o + 1] > bd[o];
    nch[c - lb] = k;
}

__global__ void k_split_write(int lb, int le, const int* __restrict__ bounds, const int* __restrict__ nch,
                              const int* __restrict__ choff, int* __restrict__ lev, int* __restrict__ ix,
                              int* __restrict__ iy, int* __restrict__ iz, int* __restrict__ nb, int* __restrict__ ne,
                              int* __restrict__ child0, int* __restrict__ nchild, int* __restrict__ parent) {
    const int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    const int k = nch[c - lb];
    nchild[c] = k;
    if (!k) { child0[c] = -1; return; }
    const int base = le + choff[c - lb];
    child0[c] = base;
    const int* bd = bounds + 9 * (c - lb);
    int j = 0;
    for (int o = 0; o < 8; ++o) {
        if (bd[o + 1] <= bd[o]) continue;
        const int ch = base + j++;
        lev[ch] = lev[c] + 1;
        ix[ch] = 2 * ix[c] + (o & 1);
        iy[ch] = 2 * iy[c] + ((o >> 1) & 1);
        iz[ch] = 2 * iz[c] + ((o >> 2) & 1);
        nb[ch] = bd[o];
        ne[ch] = bd[o + 1];
        parent[ch] = c;
        child0[ch] = -1;
        nchild[ch] = 0;
    }
}

__device__ __forceinline__ double dist3_rn(const double* a, const double* b) {
    const double dx = __dsub_rn(a[0], b[0]), dy = __dsub_rn(a[1], b[1]), dz = __dsub_rn(a[2], b[2]);
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__global__ void k_centres(int nn, const int* __restrict__ lev, const int* __restrict__ ix, const int* __restrict__ iy,
                          const int* __restrict__ iz, const double* __restrict__ box, double* __restrict__ zc) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nn) return;
    const double h = __ddiv_rn(box[3], (double)(1ull << lev[c]));
    zc[3 * c] = __dadd_rn(box[0], __dmul_rn((double)ix[c] + 0.5, h));
    zc[3 * c + 1] = __dadd_rn(box[1], __dmul_rn((double)iy[c] + 0.5, h));
    zc[3 * c + 2] = __dadd_rn(box[2], __dmul_rn((double)iz[c] + 0.5, h));
}

// Centres of mass of the nodes [lb, lb + n) (one level, children done), the
// AP variant's expansion centres: a leaf sums q_a x_a and q_a over its
// particles in sorted order, a cell sums Q_c z_c and Q_c over its children
// in octant order, z = S / Q; explicitly rounded FP64 in the oracle's order,
// so both trees have the same centres, radii and lists.  A node of zero
// total charge keeps its geometric centre.
__global__ void k_com(int lb, int le, const int* __restrict__ nb, const int* __restrict__ ne,
                      const int* __restrict__ child0, const int* __restrict__ nchild, const double* __restrict__ xs,
                      const double* __restrict__ ys, const double* __restrict__ zs, const double* __restrict__ qs,
                      double* __restrict__ Q, double* __restrict__ zc) {
    const int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    double q = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    if (nchild[c] == 0) {
        for (int a = nb[c]; a < ne[c]; ++a) {
            q = __dadd_rn(q, qs[a]);
            sx = __dadd_rn(sx, __dmul_rn(qs[a], xs[a]));
            sy = __dadd_rn(sy, __dmul_rn(qs[a], ys[a]));
            sz = __dadd_rn(sz, __dmul_rn(qs[a], zs[a]));
        }
    } else {
        for (int k = 0; k < nchild[c]; ++k) {
            const int ch = child0[c] + k;
            q = __dadd_rn(q, Q[ch]);
            sx = __dadd_rn(sx, __dmul_rn(Q[ch], zc[3 * ch]));
            sy = __dadd_rn(sy, __dmul_rn(Q[ch], zc[3 * ch + 1]));
            sz = __dadd_rn(sz, __dmul_rn(Q[ch], zc[3 * ch + 2]));
        }
    }
    Q[c] = q;
    if (q != 0.0) {
        zc[3 * c] = __ddiv_rn(sx, q);
        zc[3 * c + 1] = __ddiv_rn(sy, q);
        zc[3 * c + 2] = __ddiv_rn(sz, q);
    }
}

// AP: the dipole (rank-1 components 1..3 of the node-major multipoles) set to 0
__global__ void k_zero_dipole(int nn, int nc, double* __restrict__ M) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nn) { M[(int64_t)c * nc + 1] = 0.0; M[(int64_t)c * nc + 2] = 0.0; M[(int64_t)c * nc + 3] = 0.0; }
}

// radii in units of side / 2^22 (the unit of the integer centres), rounded to FP32
__global__ void k_radf(int nn, const double* __restrict__ rad, const double* __restrict__ box,
                       float* __restrict__ radf) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nn) radf[c] = (float)(rad[c] / box[3] * 4194304.0);
}
int ad_radf(int nn, const double* rad, const double* box, float* radf, cudaStream_t s) {
    if (nn > 0) { k_radf<<<(nn + 255) / 256, 256, 0, s>>>(nn, rad, box, radf); count_launch(); }
    return 0;
}

// radii of the nodes [lb, le) (one level), children already done
__global__ void k_radii(int lb, int le, const int* __restrict__ nb, const int* __restrict__ ne,
                        const int* __restrict__ child0, const int* __restrict__ nchild, const double* __restrict__ zc,
                        const double* __restrict__ xs, const double* __restrict__ ys, const double* __restrict__ zs,
                        double* __restrict__ rad) {
    const int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    double r = 0.0;
    const double* z = zc + 3 * c;
    if (nchild[c] == 0) {
        for (int a = nb[c]; a < ne[c]; ++a) {
            const double v[3] = {xs[a], ys[a], zs[a]};
            const double d = dist3_rn(v, z);
            if (d > r) r = d;
        }
    } else {
        for (int k = 0; k < nchild[c]; ++k) {
            const int ch = child0[c] + k;
            const double d = __dadd_rn(dist3_rn(zc + 3 * ch, z), rad[ch]);
            if (d > r) r = d;
        }
    }
    rad[c] = r;
}

// ---------------------------------------------------------------------------
// directed dual-tree traversal, one breadth-first step per launch pair
// ---------------------------------------------------------------------------
// mode per pair: 0 = M2L, 1 = P2P, 2 = self split, 3 = split target, 4 = split source.
// The MAC theta |z_A - z_B| > r_A + r_B is evaluated squared (both sides are
// non-negative), theta^2 |z_A - z_B|^2 > (r_A + r_B)^2, with explicitly rounded
// FP64 operations in the oracle's order: no square root per pair.
__device__ __forceinline__ int trav_mode(int A, int B, double theta, const int* nchild, const double* zc,
                                         const double* rad) {
    const bool la = nchild[A] == 0, lb = nchild[B] == 0;
    if (A == B) return la ? 1 : 2;
    const double* a = zc + 3 * A;
    const double* b = zc + 3 * B;
    const double dx = __dsub_rn(a[0], b[0]), dy = __dsub_rn(a[1], b[1]), dz = __dsub_rn(a[2], b[2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double sr = __dadd_rn(rad[A], rad[B]);
    if (__dmul_rn(__dmul_rn(theta, theta), d2) > __dmul_rn(sr, sr)) return 0;
    if (la && lb) return 1;
    if (!la && (lb || rad[A] >= rad[B])) return 3;
    return 4;
}

// FP32 screen of the MAC, in units of side / 2^22 so that no operand leaves
// FP32's normal range: the centre offset is the exact integer difference of
// the integer centres (below 2^23, exact in FP32), the radii are FP32
// copies in the same unit.  Outside a relative band around the boundary
// (wider than the FP32 rounding plus that of the FP64 centres) the FP32
// comparison gives the FP64 rule's answer; inside it the pair is decided by
// trav_mode in FP64.  Returns 0 (accept), 1 (reject), 2 (undecided).
__device__ __forceinline__ int mac_screen(int A, int B, float theta2, float band, const int4* __restrict__ ic,
                                          const float* __restrict__ radf) {
    const int4 a = ic[A], b = ic[B];
    const float dx = (float)(a.x - b.x), dy = (float)(a.y - b.y), dz = (float)(a.z - b.z);
    const float lhs = theta2 * (dx * dx + dy * dy + dz * dz);
    const float sr = radf[A] + radf[B];
    const float rhs = sr * sr;
    if (lhs > rhs * (1.f + band)) return 0;
    if (lhs < rhs * (1.f - band)) return 1;
    return 2;
}

// decides every pair of the frontier once (mode kept for the write pass)
__global__ void k_trav_count(int nq, const int2* __restrict__ q, double theta, const int* __restrict__ nchild,
                             const double* __restrict__ zc, const double* __restrict__ rad, int* __restrict__ cm,
                             int* __restrict__ cp, int* __restrict__ cq, unsigned char* __restrict__ mode,
                             const int4* __restrict__ ic, const float* __restrict__ radf, float theta2,
                             float band) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nq) return;
    const int A = q[k].x, B = q[k].y;
    int m;
    const int sc = A == B ? 2 : mac_screen(A, B, theta2, band, ic, radf);
    if (sc == 0) {
        m = 0;
    } else if (sc == 1) {
        const bool la = nchild[A] == 0, lb = nchild[B] == 0;
        m = (la && lb) ? 1 : (!la && (lb || rad[A] >= rad[B])) ? 3 : 4;
    } else {
        m = trav_mode(A, B, theta, nchild, zc, rad);
    }
    mode[k] = (unsigned char)m;
    cm[k] = m == 0;
    cp[k] = m == 1;
    cq[k] = m == 2 ? nchild[A] * nchild[A] : m == 3 ? nchild[A] : m == 4 ? nchild[B] : 0;
}

__global__ void k_trav_write(int nq, const int2* __restrict__ q, const unsigned char* __restrict__ mode,
                             const int* __restrict__ nchild, const int* __restrict__ child0,
                             const int* __restrict__ om, const int* __restrict__ op, const int* __restrict__ oq,
                             int mbase, int pbase, int2* __restrict__ m2l, int2* __restrict__ p2p,
                             int2* __restrict__ qn) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nq) return;
    const int A = q[k].x, B = q[k].y;
    const int m = mode[k];
    if (m == 0) { m2l[mbase + om[k]] = make_int2(A, B); return; }
    if (m == 1) { p2p[pbase + op[k]] = make_int2(A, B); return; }
    int o = oq[k];
    if (m == 2) {
        for (int i = 0; i < nchild[A]; ++i)
            for (int j = 0; j < nchild[A]; ++j) qn[o++] = make_int2(child0[A] + i, child0[A] + j);
    } else if (m == 3) {
        for (int i = 0; i < nchild[A]; ++i) qn[o++] = make_int2(child0[A] + i, B);
    } else {
        for (int j = 0; j < nchild[B]; ++j) qn[o++] = make_int2(A, child0[B] + j);
    }
}

// keys for grouping pairs by target: key = target, value = pair index
__global__ void k_pair_keys(int n, const int2* __restrict__ pr, uint64_t* __restrict__ key, int* __restrict__ val) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    key[k] = (uint64_t)pr[k].x;
    val[k] = k;
}
// sorted pairs -> CSR sources and per-target counts; a count is the segment
// end minus the segment start, so only the two boundary threads of each
// target's segment touch its counter (no same-address atomic chains)
__global__ void k_pair_csr(int n, const uint64_t* __restrict__ key, const int* __restrict__ val,
                           const int2* __restrict__ pr, int* __restrict__ src, int* __restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    src[k] = pr[val[k]].y;
    const uint64_t t = key[k];
    if (k == 0 || key[k - 1] != t) atomicAdd(&cnt[(int)t], -k);
    if (k == n - 1 || key[k + 1] != t) atomicAdd(&cnt[(int)t], k + 1);
}

// M2L work order: targets with non-empty lists, longest lists first
__global__ void k_len_keys(int nn, const int* __restrict__ off, uint64_t* __restrict__ key, int* __restrict__ val) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nn) return;
    const int len = off[c + 1] - off[c];
    key[c] = (uint64_t)(0x7fffffff - len);
    val[c] = c;
}

// leaves in particle order: key = first particle
__global__ void k_leaf_keys(int nn, const int* __restrict__ nchild, const int* __restrict__ nb,
                            uint64_t* __restrict__ key, int* __restrict__ val) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nn) return;
    key[c] = nchild[c] ? 0xffffffffull : (uint64_t)nb[c];
    val[c] = c;
}

__global__ void k_gather_sorted(int64_t n, const int* __restrict__ perm, const double* __restrict__ x,
                                const double* __restrict__ y, const double* __restrict__ z,
                                const double* __restrict__ q, double* __restrict__ xs, double* __restrict__ ys,
                                double* __restrict__ zs, double* __restrict__ qs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = perm[i];
    xs[i] = x[o]; ys[i] = y[o]; zs[i] = z[o]; qs[i] = q[o];
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ---------------------------------------------------------------------------
// tree operators (physical units, public storage, node-major expansions)
// ---------------------------------------------------------------------------
// M2M (Eq. M2M / M2M part 2): parents [lb, le) of one level, one warp each;
// the children's shifted full-symmetric sums accumulate in shared memory,
// then (traceless) one detrace; the parent is overwritten.  The binomial
// weights are split into factorials,
//   sum_k C(n,k) (-d)^(n-k) M_k = n! sum_k (M_k / k!) ((-d)^(n-k) / (n-k)!),
// so the inner loop reads shared memory only (per-block tables of 1/k! and
// n! per symmetric position).
template <typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_m2m_tree(int p, int basis, int lb, int le, const int* __restrict__ child0, const int* __restrict__ nchild,
           const double* __restrict__ zc, double* __restrict__ Mn, const double* __restrict__ detr,
           const double* __restrict__ expand, DevOffsets off, const int* __restrict__ lev, double side) {
    // FP32 form: expansions in the scaled units of their cell (side h_c):
    // Mt_m = M_m / h_c^|m|; the child's (h/2) terms gain 2^-|k|, the shift
    // uses delta / h_parent.  FP64 form: physical units.
    constexpr bool SCALED = sizeof(T) == 4;
    __shared__ double sX[WARPS][FMM_NS_MAX], sA[WARPS][FMM_NT_MAX];
    __shared__ T sXt[WARPS][FMM_NS_MAX], sY[WARPS][FMM_NS_MAX];
    __shared__ T sP[WARPS][3][FMM_PMAX + 1];
    __shared__ T sInvF[FMM_NS_MAX], sFac[FMM_NS_MAX];
    __shared__ int sIdx[FMM_NS_MAX];
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const int nx = c_sym_idx[s][0], ny = c_sym_idx[s][1], nz = c_sym_idx[s][2];
        const double inv = c_invfact[nx] * c_invfact[ny] * c_invfact[nz];
        sInvF[s] = T(inv);
        sFac[s] = T(1.0 / inv);   // nx! ny! nz! (exact: factorials up to 10! are integers below 2^24)
        sIdx[s] = nx | (ny << 8) | (nz << 16);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lb + blockIdx.x * WARPS + w;
    if (c >= le || nchild[c] == 0) return;
    for (int s = lane; s < ns; s += 32) sY[w][s] = T(0);
    for (int k = 0; k < nchild[c]; ++k) {
        const int ch = child0[c] + k;
        __syncwarp();
        if (basis) {
            for (int t = lane; t < nc; t += 32) sA[w][t] = Mn[(int64_t)ch * nc + t];
            __syncwarp();
            expand_tl_warp(p, sA[w], sX[w], expand, off, lane);
            __syncwarp();
            for (int s = lane; s < ns; s += 32)
                sXt[w][s] = T(SCALED ? ldexp(sX[w][s], -(c_sym_idx[s][0] + c_sym_idx[s][1] + c_sym_idx[s][2]))
                                     : sX[w][s]) * sInvF[s];
        } else {
            for (int s = lane; s < ns; s += 32) {
                const double v = Mn[(int64_t)ch * nc + s];
                sXt[w][s] = T(SCALED ? ldexp(v, -(c_sym_idx[s][0] + c_sym_idx[s][1] + c_sym_idx[s][2])) : v) *
                            sInvF[s];
            }
        }
        if (lane < 3) {
            const double hinv = SCALED ? ldexp(1.0 / side, lev[c]) : 1.0;
            const double md = -(zc[3 * ch + lane] - zc[3 * c + lane]) * hinv;
            double v = 1.0;
            sP[w][lane][0] = T(1);
            for (int j = 1; j <= p; ++j) { v *= md; sP[w][lane][j] = T(v * c_invfact[j]); }
        }
        __syncwarp();
        for (int s = lane; s < ns; s += 32) {
            const int id = sIdx[s];
            const int nx = id & 255, ny = (id >> 8) & 255, nz = id >> 16;
            T v = T(0);
            for (int kx = 0; kx <= nx; ++kx)
                for (int ky = 0; ky <= ny; ++ky) {
                    const T wxy = sP[w][0][nx - kx] * sP[w][1][ny - ky];
                    for (int kz = 0; kz <= nz; ++kz) v += wxy * sP[w][2][nz - kz] * sXt[w][pos_sym(kx, ky, kz)];
                }
            sY[w][s] += v * sFac[s];
        }
    }
    __syncwarp();
    if (!basis) {
        for (int s = lane; s < ns; s += 32) Mn[(int64_t)c * nc + s] = (double)sY[w][s];
        return;
    }
    for (int s = lane; s < ns; s += 32) sX[w][s] = (double)sY[w][s];
    __syncwarp();
    for (int t = lane; t < nc; t += 32) {
        const int nx = c_tl_idx[t][0], nz = c_tl_idx[t][2];
        const int j = c_tl_idx[t][0] + c_tl_idx[t][1] + nz;
        const int cols = (j + 1) * (j + 2) / 2;
        const int row = (j - nx) * (j - nx + 1) / 2 + nz;
        const double* R = detr + off.detr[j] + row * cols;
        const double* Ys = &sX[w][ns_of(j - 1)];
        double v = 0.0;
        for (int s2 = 0; s2 < cols; ++s2) v += R[s2] * Ys[s2];
        Mn[(int64_t)c * nc + t] = v;
    }
}

// L2L (Eq. L2L): children [lb, le) of one level, one warp each, add the
// parent's shifted expansion.
template <typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_l2l_tree(int p, int basis, int lb, int le, const int* __restrict__ parent, const double* __restrict__ zc,
           double* __restrict__ Ln, const double* __restrict__ expand, DevOffsets off, const int* __restrict__ lev,
           double side) {
    // FP32 form: Lt_n = L_n h_c^(|n|+1); the shift uses delta / h_parent and
    // the child's (h/2) output gains 2^-(|n|+1).  FP64 form: physical units.
    constexpr bool SCALED = sizeof(T) == 4;
    __shared__ double sX[WARPS][FMM_NS_MAX], sA[WARPS][FMM_NT_MAX];
    __shared__ T sXt[WARPS][FMM_NS_MAX];
    __shared__ T sP[WARPS][3][FMM_PMAX + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lb + blockIdx.x * WARPS + w;
    if (c >= le) return;
    const int pa = parent[c];
    const int ns = ns_of(p), nc = ncoef_of(p, basis);
    if (basis) {
        for (int t = lane; t < nc; t += 32) sA[w][t] = Ln[(int64_t)pa * nc + t];
        __syncwarp();
        expand_tl_warp(p, sA[w], sX[w], expand, off, lane);
    } else {
        for (int s = lane; s < ns; s += 32) sX[w][s] = Ln[(int64_t)pa * nc + s];
    }
    if (lane < 3) {
        const double hinv = SCALED ? ldexp(1.0 / side, lev[pa]) : 1.0;
        const double d = (zc[3 * c + lane] - zc[3 * pa + lane]) * hinv;
        double v = 1.0;
        sP[w][lane][0] = T(1);
        for (int j = 1; j <= p; ++j) { v *= d; sP[w][lane][j] = T(v * c_invfact[j]); }
    }
    __syncwarp();
    for (int s = lane; s < ns; s += 32) sXt[w][s] = T(sX[w][s]);
    __syncwarp();
    for (int o = lane; o < nc; o += 32) {
        int nx, ny, nz;
        if (basis) { nx = c_tl_idx[o][0]; ny = c_tl_idx[o][1]; nz = c_tl_idx[o][2]; }
        else { nx = c_sym_idx[o][0]; ny = c_sym_idx[o][1]; nz = c_sym_idx[o][2]; }
        const int rem = p - nx - ny - nz;
        T v = T(0);
        for (int kx = 0; kx <= rem; ++kx)
            for (int ky = 0; ky <= rem - kx; ++ky) {
                const T wxy = sP[w][0][kx] * sP[w][1][ky];
                for (int kz = 0; kz <= rem - kx - ky; ++kz)
                    v += wxy * sP[w][2][kz] * sXt[w][pos_sym(nx + kx, ny + ky, nz + kz)];
            }
        // accumulation into the FP64 expansion
        Ln[(int64_t)c * nc + o] += SCALED ? ldexp((double)v, -(nx + ny + nz + 1)) : (double)v;
    }
}

// FP64 P2P over the near-field lists: one warp per target leaf taken from an
// atomic work counter (persistent grid); lane groups split the staged
// sources; positions relative to the target leaf centre.  Accumulates into
// caller order.  (The FP32 form has its own kernel, k_ad_p2p32.)
template <typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_p2p_tree(int nwork, const int* __restrict__ work, const int* __restrict__ off, const int* __restrict__ src,
           const int* __restrict__ nb, const int* __restrict__ ne, const double* __restrict__ zc,
           const double* __restrict__ xs, const double* __restrict__ ys, const double* __restrict__ zs,
           const double* __restrict__ qs, const int* __restrict__ perm, double* __restrict__ pot,
           double* __restrict__ ax, double* __restrict__ ay, double* __restrict__ az, int* __restrict__ counter) {
    __shared__ T sx[WARPS][32], sy[WARPS][32], sz[WARPS][32], sq[WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nwork) break;
        const int c = work[item];
        const double cx = zc[3 * c], cy = zc[3 * c + 1], cz = zc[3 * c + 2];
        const int b = nb[c], e = ne[c];
        for (int t0 = b; t0 < e; t0 += 32) {
            const int tn = min(32, e - t0);
            int tp = 1;
            while (tp < tn) tp <<= 1;
            const int G = 32 / tp, grp = lane / tp, tl = lane % tp;
            const int ti = t0 + tl;
            const bool act = tl < tn;
            const T xi = act ? T(xs[ti] - cx) : T(0), yi = act ? T(ys[ti] - cy) : T(0), zi = act ? T(zs[ti] - cz) : T(0);
            T ph = 0, gx = 0, gy = 0, gz = 0;
            for (int k = off[c]; k < off[c + 1]; ++k) {
                const int S = src[k];
                for (int s0 = nb[S]; s0 < ne[S]; s0 += 32) {
                    __syncwarp();
                    const int sj = s0 + lane;
                    if (sj < ne[S]) {
                        sx[w][lane] = T(xs[sj] - cx); sy[w][lane] = T(ys[sj] - cy);
                        sz[w][lane] = T(zs[sj] - cz); sq[w][lane] = T(qs[sj]);
                    }
                    __syncwarp();
                    const int cnt = min(32, ne[S] - s0);
                    if (act) {
                        for (int j = grp; j < cnt; j += G) {
                            const T dx = sx[w][j] - xi, dy = sy[w][j] - yi, dz = sz[w][j] - zi;
                            const T r2 = dx * dx + dy * dy + dz * dz;
                            const T ir = r2 > T(0) ? fmm_rsqrt(r2) : T(0);   // self and coincident pairs: 0
                            const T qir = sq[w][j] * ir, qir3 = qir * ir * ir;
                            ph += qir; gx += qir3 * dx; gy += qir3 * dy; gz += qir3 * dz;
                        }
                    }
                }
            }
            for (int o = tp; o < 32; o <<= 1) {
                ph += __shfl_xor_sync(0xffffffffu, ph, o); gx += __shfl_xor_sync(0xffffffffu, gx, o);
                gy += __shfl_xor_sync(0xffffffffu, gy, o); gz += __shfl_xor_sync(0xffffffffu, gz, o);
            }
            if (act && grp == 0) {
                const int o = perm[ti];
                pot[o] -= (double)ph; ax[o] += (double)gx; ay[o] += (double)gy; az[o] += (double)gz;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
#define G256(n) (unsigned)(((int64_t)(n) + 255) / 256), 256, 0, s
int ad_bbox(int64_t n, const double* x, const double* y, const double* z, double* part, double* box, cudaStream_t s) {
    const int nblk = 256;
    k_bbox_partial<<<nblk, 256, 0, s>>>(n, x, y, z, part);
    k_bbox_final<<<1, 32, 0, s>>>(nblk, part, box);
    count_launch(); count_launch();
    return 0;
}
int ad_morton(int64_t n, const double* x, const double* y, const double* z, const double* box, uint64_t* key,
              int* val, cudaStream_t s) {
    if (n) { k_morton<<<G256(n)>>>(n, x, y, z, box, key, val); count_launch(); }
    return 0;
}
int ad_gather(int64_t n, const int* perm, const double* x, const double* y, const double* z, const double* q,
              double* xs, double* ys, double* zs, double* qs, cudaStream_t s) {
    if (n) { k_gather_sorted<<<G256(n)>>>(n, perm, x, y, z, q, xs, ys, zs, qs); count_launch(); }
    return 0;
}
int ad_split_count(int lb, int le, int max_leaf, const int* lev, const int* nb, const int* ne, const uint64_t* key,
                   int* bounds, int* nch, cudaStream_t s) {
    k_split_count<<<G256(le - lb)>>>(lb, le, max_leaf, lev, nb, ne, key, bounds, nch);
    count_launch();
    return 0;
}
int ad_split_write(int lb, int le, const int* bounds, const int* nch, const int* choff, int* lev, int* ix, int* iy,
                   int* iz, int* nb, int* ne, int* child0, int* nchild, int* parent, cudaStream_t s) {
    k_split_write<<<G256(le - lb)>>>(lb, le, bounds, nch, choff, lev, ix, iy, iz, nb, ne, child0, nchild, parent);
    count_launch();
    return 0;
}
int ad_centres(int nn, const int* lev, const int* ix, const int* iy, const int* iz, const double* box, double* zc,
               cudaStream_t s) {
    k_centres<<<G256(nn)>>>(nn, lev, ix, iy, iz, box, zc);
    count_launch();
    return 0;
}
int ad_com(int lb, int le, const int* nb, const int* ne, const int* child0, const int* nchild, const double* xs,
           const double* ys, const double* zs, const double* qs, double* Q, double* zc, cudaStream_t s) {
    if (le <= lb) return 0;
    k_com<<<(le - lb + 255) / 256, 256, 0, s>>>(lb, le, nb, ne, child0, nchild, xs, ys, zs, qs, Q, zc);
    count_launch();
    return 0;
}
int ad_zero_dipole(int nn, int nc, double* M, cudaStream_t s) {
    if (nn <= 0 || nc < 4) return 0;
    k_zero_dipole<<<(nn + 255) / 256, 256, 0, s>>>(nn, nc, M);
    count_launch();
    return 0;
}

int ad_radii(int lb, int le, const int* nb, const int* ne, const int* child0, const int* nchild, const double* zc,
             const double* xs, const double* ys, const double* zs, double* rad, cudaStream_t s) {
    k_radii<<<G256(le - lb)>>>(lb, le, nb, ne, child0, nchild, zc, xs, ys, zs, rad);
    count_launch();
    return 0;
}
int ad_trav_count(int nq, const int2* q, double theta, const int* nchild, const double* zc, const double* rad,
                  int* cm, int* cp, int* cq, unsigned char* mode, const int4* ic, const float* radf, float band,
                  cudaStream_t s) {
    k_trav_count<<<G256(nq)>>>(nq, q, theta, nchild, zc, rad, cm, cp, cq, mode, ic, radf,
                               (float)(theta * theta), band);
    count_launch();
    return 0;
}
int ad_trav_write(int nq, const int2* q, const unsigned char* mode, const int* nchild, const int* child0,
                  const int* om, const int* op, const int* oq, int mbase, int pbase, int2* m2l, int2* p2p, int2* qn,
                  cudaStream_t s) {
    k_trav_write<<<G256(nq)>>>(nq, q, mode, nchild, child0, om, op, oq, mbase, pbase, m2l, p2p, qn);
    count_launch();
    return 0;
}
int ad_pair_keys(int n, const int2* pr, uint64_t* key, int* val, cudaStream_t s) {
    if (n) { k_pair_keys<<<G256(n)>>>(n, pr, key, val); count_launch(); }
    return 0;
}
int ad_pair_csr(int n, const uint64_t* key, const int* val, const int2* pr, int* src, int* cnt, cudaStream_t s) {
    if (n) { k_pair_csr<<<G256(n)>>>(n, key, val, pr, src, cnt); count_launch(); }
    return 0;
}
int ad_len_keys(int nn, const int* off, uint64_t* key, int* val, cudaStream_t s) {
    k_len_keys<<<G256(nn)>>>(nn, off, key, val);
    count_launch();
    return 0;
}
int ad_leaf_keys(int nn, const int* nchild, const int* nb, uint64_t* key, int* val, cudaStream_t s) {
    k_leaf_keys<<<G256(nn)>>>(nn, nchild, nb, key, val);
    count_launch();
    return 0;
}
__global__ void k_f64_to_f32_rows(int64_t rows, int nc, int ldm, const double* __restrict__ a, float* __restrict__ b) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * ldm) return;
    const int64_t r = t / ldm;
    const int j = (int)(t % ldm);
    b[t] = j < nc ? (float)a[r * nc + j] : 0.f;
}
int ad_to_f32_rows(int64_t rows, int nc, int ldm, const double* a, float* b, cudaStream_t s) {
    if (rows > 0) { k_f64_to_f32_rows<<<G256(rows * ldm)>>>(rows, nc, ldm, a, b); count_launch(); }
    return 0;
}
int ad_to_f32(int64_t n, const double* a, float* b, cudaStream_t s) {
    if (n) { k_f64_to_f32<<<G256(n)>>>(n, a, b); count_launch(); }
    return 0;
}
int ad_m2m(int prec, int p, int basis, int lb, int le, const int* child0, const int* nchild, const double* zc,
           double* Mn, const DevTables& T, const int* lev, double side, cudaStream_t s) {
    if (le <= lb) return 0;
    constexpr int W = 4;
    const unsigned g = (unsigned)((le - lb + W - 1) / W);
    if (prec)
        k_m2m_tree<float, W><<<g, W * 32, 0, s>>>(p, basis, lb, le, child0, nchild, zc, Mn, T.detr, T.expand,
                                                  T.offsets(), lev, side);
    else
        k_m2m_tree<double, W><<<g, W * 32, 0, s>>>(p, basis, lb, le, child0, nchild, zc, Mn, T.detr, T.expand,
                                                   T.offsets(), lev, side);
    count_launch();
    return 0;
}
int ad_l2l(int prec, int p, int basis, int lb, int le, const int* parent, const double* zc, double* Ln,
           const DevTables& T, const int* lev, double side, cudaStream_t s) {
    if (le <= lb) return 0;
    constexpr int W = 4;
    const unsigned g = (unsigned)((le - lb + W - 1) / W);
    if (prec)
        k_l2l_tree<float, W><<<g, W * 32, 0, s>>>(p, basis, lb, le, parent, zc, Ln, T.expand, T.offsets(), lev,
                                                  side);
    else
        k_l2l_tree<double, W><<<g, W * 32, 0, s>>>(p, basis, lb, le, parent, zc, Ln, T.expand, T.offsets(), lev,
                                                   side);
    count_launch();
    return 0;
}
int ad_p2p(int nwork, const int* work, const int* off, const int* src, const int* nb, const int* ne,
           const double* zc, const double* xs, const double* ys, const double* zs, const double* qs,
           const int* perm, double* pot, double* ax, double* ay, double* az, int* counter, int blocks,
           cudaStream_t s) {
    if (nwork <= 0) return 0;
    constexpr int W = 4;
    k_p2p_tree<double, W><<<blocks, W * 32, 0, s>>>(nwork, work, off, src, nb, ne, zc, xs, ys, zs, qs, perm, pot, ax,
                                                    ay, az, counter);
    count_launch();
    return 0;
}
#undef G256

}  // namespace fmm
