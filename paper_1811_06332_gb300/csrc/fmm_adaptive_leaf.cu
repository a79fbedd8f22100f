// Leaf kernels of the adaptive-octree FMM, specialised per order p and per
// arithmetic type (double for FMM_FP64, float for FMM_FP32):
//   P2M (Eq. P2M)  A_m = sum_a q_a (-(x_a - z))^m about the leaf centre z,
//                  SYM: M = A, TRACELESS: Mbar = D[A] (independent comps);
//   L2P (Eq. L2P)  Phi = sum_k (x - z)^k / k! L_k and its gradient;
//   P2P            near field over the leaf pairs of the interaction lists.
// Expansions are node-major ([node][ncoef]); the FP64 form keeps them in
// physical units, the FP32 form in the scaled units of their cell (side
// h = side/2^level): Mt_m = M_m / h^|m|, Lt_n = L_n h^(|n|+1), which keeps
// every power of a cell size inside the FP32 range at any depth and order.
//
// The FP32 form reads particles as FP32 offsets from the centre of their own
// leaf (pos32), and takes the offset between two node centres from their
// integer coordinates (ic = (2i+1) 2^(21-level) per axis, in units of
// side/2^22): an exact integer difference rounded once to FP32.  No FP64
// arithmetic runs per particle pair or per source, which matters on a part
// whose FP64 rate is 1/64 of its FP32 rate.
#include "fmm_adaptive.h"

namespace fmm {

// pos32[a] = (x_a - z_c, y_a - z_c, z_a - z_c, q_a) for the leaf c holding a
__global__ void k_ad_pos32(int nleaf, const int* __restrict__ leaf, const int* __restrict__ nb,
                           const int* __restrict__ ne, const double* __restrict__ zc, const double* __restrict__ xs,
                           const double* __restrict__ ys, const double* __restrict__ zs,
                           const double* __restrict__ qs, float4* __restrict__ pos32) {
    const int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (k >= nleaf) return;
    const int c = leaf[k];
    const double cx = zc[3 * c], cy = zc[3 * c + 1], cz = zc[3 * c + 2];
    for (int a = nb[c] + lane; a < ne[c]; a += 32)
        pos32[a] = make_float4((float)(xs[a] - cx), (float)(ys[a] - cy), (float)(zs[a] - cz), (float)qs[a]);
}

// ic[c] = integer centre of node c (see above), w = level
__global__ void k_ad_icentre(int nn, const int* __restrict__ lev, const int* __restrict__ ix,
                             const int* __restrict__ iy, const int* __restrict__ iz, int4* __restrict__ ic) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nn) return;
    const int sh = 21 - lev[c];
    ic[c] = make_int4((2 * ix[c] + 1) << sh, (2 * iy[c] + 1) << sh, (2 * iz[c] + 1) << sh, lev[c]);
}

// ---------------------------------------------------------------------------
// P2M: one warp per leaf; lane owns the column (nx, ny) of multi-indices and
// walks nz upward (one product per component and particle).
// ---------------------------------------------------------------------------
template <int P, typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_ad_p2m(int basis, int nleaf, const int* __restrict__ leaf, const int* __restrict__ nb, const int* __restrict__ ne,
         const double* __restrict__ zc, const double* __restrict__ xs, const double* __restrict__ ys,
         const double* __restrict__ zs, const double* __restrict__ qs, const float4* __restrict__ pos32,
         double* __restrict__ Mn, const T* __restrict__ detr, DevOffsets off, const int* __restrict__ lev,
         double side) {
    // FP32 form (pos32 given): moments in the leaf's scaled units,
    // Mt_m = sum_a q_a (-(x_a - z)/h)^m with h = side / 2^level
    constexpr int NS = (P + 1) * (P + 2) * (P + 3) / 6;
    constexpr int NCOL = (P + 1) * (P + 2) / 2;
    constexpr int KC = (NCOL + 31) / 32;
    __shared__ T sx[WARPS][32], sy[WARPS][32], sz[WARPS][32], sq[WARPS][32];
    __shared__ T sA[WARPS][NS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.x * WARPS + w;
    if (k >= nleaf) return;
    const int c = leaf[k];
    const int b = nb[c], e = ne[c];
    T acc[KC][P + 1];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk)
#pragma unroll
        for (int j = 0; j <= P; ++j) acc[kk][j] = T(0);
    int cnx[KC], cny[KC];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
        int col = lane + 32 * kk, nx = 0;
        while (nx <= P && col >= P + 1 - nx) { col -= P + 1 - nx; ++nx; }
        cnx[kk] = nx;
        cny[kk] = col;
    }
    double cx = 0.0, cy = 0.0, cz = 0.0;
    if (!pos32) { cx = zc[3 * c]; cy = zc[3 * c + 1]; cz = zc[3 * c + 2]; }
    const float hinv = pos32 ? (float)ldexp(1.0 / side, lev[c]) : 1.f;
    for (int a0 = b; a0 < e; a0 += 32) {
        const int a = a0 + lane;
        __syncwarp();
        if (a < e) {
            if (pos32) {
                const float4 v = pos32[a];
                sx[w][lane] = T(-v.x * hinv); sy[w][lane] = T(-v.y * hinv); sz[w][lane] = T(-v.z * hinv);
                sq[w][lane] = T(v.w);
            } else {
                sx[w][lane] = T(cx - xs[a]); sy[w][lane] = T(cy - ys[a]); sz[w][lane] = T(cz - zs[a]);
                sq[w][lane] = T(qs[a]);
            }
        }
        __syncwarp();
        const int cnt = min(32, e - a0);
        for (int i = 0; i < cnt; ++i) {
            const T rx = sx[w][i], ry = sy[w][i], rz = sz[w][i], qa = sq[w][i];
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                if (lane + 32 * kk < NCOL) {
                    T wgt = qa;
                    for (int t = 0; t < cnx[kk]; ++t) wgt *= rx;
                    for (int t = 0; t < cny[kk]; ++t) wgt *= ry;
                    const int rem = P - cnx[kk] - cny[kk];
#pragma unroll
                    for (int j = 0; j <= P; ++j)
                        if (j <= rem) { acc[kk][j] += wgt; wgt *= rz; }
                }
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
        if (lane + 32 * kk < NCOL) {
            const int rem = P - cnx[kk] - cny[kk];
#pragma unroll
            for (int j = 0; j <= P; ++j)
                if (j <= rem) sA[w][pos_sym(cnx[kk], cny[kk], j)] = acc[kk][j];
        }
    }
    __syncwarp();
    if (!basis) {
        for (int s = lane; s < NS; s += 32) Mn[(int64_t)c * NS + s] = (double)sA[w][s];
        return;
    }
    constexpr int NT = (P + 1) * (P + 1);
    for (int t = lane; t < NT; t += 32) {
        const int nx = c_tl_idx[t][0], nz = c_tl_idx[t][2];
        const int j = nx + c_tl_idx[t][1] + nz;
        const int cols = (j + 1) * (j + 2) / 2;
        const int row = (j - nx) * (j - nx + 1) / 2 + nz;
        const T* R = detr + off.detr[j] + row * cols;
        const T* As = &sA[w][ns_of(j - 1)];
        T v = T(0);
        for (int s = 0; s < cols; ++s) v += R[s] * As[s];
        Mn[(int64_t)c * NT + t] = (double)v;
    }
}

// ---------------------------------------------------------------------------
// L2P: one warp per leaf, lanes over particles; the full symmetric local
// expansion (dependent traceless components rebuilt) in shared memory.
// Overwrites pot = -Phi and acc = grad Phi in caller order.
// ---------------------------------------------------------------------------
template <int P, typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_ad_l2p(int basis, int nleaf, const int* __restrict__ leaf, const int* __restrict__ nb, const int* __restrict__ ne,
         const double* __restrict__ zc, const double* __restrict__ xs, const double* __restrict__ ys,
         const double* __restrict__ zs, const float4* __restrict__ pos32, const int* __restrict__ perm,
         const double* __restrict__ Ln, const T* __restrict__ expand, DevOffsets off,
         double* __restrict__ pot, double* __restrict__ ax, double* __restrict__ ay, double* __restrict__ az,
         const int* __restrict__ lev, double side) {
    // FP32 form (pos32 given): scaled units of the leaf, Lt_n = L_n h^(|n|+1):
    // Phi = (1/h) sum_k (r/h)^k/k! Lt_k, grad = (1/h^2) sum_k (r/h)^k/k! Lt_{k+e_i}
    constexpr int NS = (P + 1) * (P + 2) * (P + 3) / 6;
    constexpr int NT = (P + 1) * (P + 1);
    __shared__ T sA[WARPS][NT];
    __shared__ T sL[WARPS][NS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.x * WARPS + w;
    if (k >= nleaf) return;
    const int c = leaf[k];
    const int b = nb[c], e = ne[c];
    if (b == e) return;
    if (basis) {
        for (int t = lane; t < NT; t += 32) sA[w][t] = T(Ln[(int64_t)c * NT + t]);
        __syncwarp();
        for (int s = lane; s < NS; s += 32) {
            const int nx = c_sym_idx[s][0], nz = c_sym_idx[s][2];
            const int j = nx + c_sym_idx[s][1] + nz;
            const int row = (j - nx) * (j - nx + 1) / 2 + nz;
            const T* E = expand + off.expand[j] + row * (2 * j + 1);
            T v = T(0);
            for (int t = 0; t < 2 * j + 1; ++t) v += E[t] * sA[w][j * j + t];
            sL[w][s] = v;
        }
    } else {
        for (int s = lane; s < NS; s += 32) sL[w][s] = T(Ln[(int64_t)c * NS + s]);
    }
    __syncwarp();
    double cx = 0.0, cy = 0.0, cz = 0.0;
    if (!pos32) { cx = zc[3 * c]; cy = zc[3 * c + 1]; cz = zc[3 * c + 2]; }
    const double hinv_d = pos32 ? ldexp(1.0 / side, lev[c]) : 1.0;
    const float hinv = (float)hinv_d;
    const T* L = sL[w];
    for (int a0 = b; a0 < e; a0 += 32) {
        const int a = a0 + lane;
        if (a >= e) break;
        T rx, ry, rz;
        if (pos32) {
            const float4 v = pos32[a];
            rx = T(v.x * hinv); ry = T(v.y * hinv); rz = T(v.z * hinv);
        } else {
            rx = T(xs[a] - cx); ry = T(ys[a] - cy); rz = T(zs[a] - cz);
        }
        T fx[P + 1], fy[P + 1], fz[P + 1];
        fx[0] = fy[0] = fz[0] = T(1);
#pragma unroll
        for (int kk = 1; kk <= P; ++kk) {
            fx[kk] = fx[kk - 1] * rx * T(1.0 / kk);
            fy[kk] = fy[kk - 1] * ry * T(1.0 / kk);
            fz[kk] = fz[kk - 1] * rz * T(1.0 / kk);
        }
        T ph = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll
        for (int kx = 0; kx <= P; ++kx) {
            T xp = 0, xgx = 0, xgy = 0, xgz = 0;
#pragma unroll
            for (int ky = 0; ky <= P - kx; ++ky) {
                T s_p = 0, s_gx = 0, s_gy = 0, s_gz = 0;
#pragma unroll
                for (int kz = 0; kz <= P - kx - ky; ++kz) {
                    s_p += fz[kz] * L[pos_sym(kx, ky, kz)];
                    if (kx + ky + kz < P) {
                        s_gx += fz[kz] * L[pos_sym(kx + 1, ky, kz)];
                        s_gy += fz[kz] * L[pos_sym(kx, ky + 1, kz)];
                        s_gz += fz[kz] * L[pos_sym(kx, ky, kz + 1)];
                    }
                }
                xp += fy[ky] * s_p; xgx += fy[ky] * s_gx; xgy += fy[ky] * s_gy; xgz += fy[ky] * s_gz;
            }
            ph += fx[kx] * xp; gx += fx[kx] * xgx; gy += fx[kx] * xgy; gz += fx[kx] * xgz;
        }
        const int o = perm[a];
        pot[o] = -(double)ph * hinv_d;
        ax[o] = (double)gx * hinv_d * hinv_d;
        ay[o] = (double)gy * hinv_d * hinv_d;
        az[o] = (double)gz * hinv_d * hinv_d;
    }
}

// ---------------------------------------------------------------------------
// FP32 P2P over the near-field lists: one warp per target leaf from an
// atomic work counter (persistent grid).  Targets in blocks of up to 32: tp
// lanes per target set (4 or 8) hold NT targets each (8, 16, 24 or 32
// slots), the 32 / tp lane groups split the staged sources and are summed by
// shuffles, so a shared load of one source serves NT interactions.
// Sources of up to 32 source leaves are taken together: a warp prefix sum of
// their counts maps lane g of a chunk to (leaf, particle) by a fixed
// five-step search, so every staged chunk holds 32 sources (float4: offset
// from the target leaf centre via the integer centres, charge) whatever the
// leaf sizes.  r = 0 pairs (the particle itself, coincident points)
// contribute nothing: they occur only among the target leaf's own
// particles, so only the chunks that hold them take the r^2 == 0 select.
// Accumulates into caller order.
// ---------------------------------------------------------------------------
template <bool GUARD>
__device__ __forceinline__ void p2p_acc(const float4 s, float xi, float yi, float zi, float& ph, float& gx,
                                        float& gy, float& gz) {
    const float dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ir = GUARD ? (r2 > 0.f ? fmm_rsqrt(r2) : 0.f) : fmm_rsqrt(r2);
    const float qir = s.w * ir, qir3 = qir * ir * ir;
    ph += qir;
    gx = fmaf(qir3, dx, gx);
    gy = fmaf(qir3, dy, gy);
    gz = fmaf(qir3, dz, gz);
}

// Stages chunk [c0, c0 + 32) of the concatenated sources of one batch of
// source leaves into ss (lane l holds leaf l of the batch: start sb, count
// excl/incl prefix, centre offset o*).  Returns the number staged.
__device__ __forceinline__ int p2p_stage(float4* ss, int lane, int c0, int total, int incl, int excl, int sb,
                                         float ox, float oy, float oz, const float4* __restrict__ pos32) {
    const int g = min(c0 + lane, total - 1);
    int i = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, i + step - 1);
        if (v <= g) i += step;
    }
    const int sbi = __shfl_sync(0xffffffffu, sb, i), exi = __shfl_sync(0xffffffffu, excl, i);
    const float oxi = __shfl_sync(0xffffffffu, ox, i), oyi = __shfl_sync(0xffffffffu, oy, i),
                ozi = __shfl_sync(0xffffffffu, oz, i);
    __syncwarp();
    if (c0 + lane < total) {
        const float4 v = pos32[sbi + (g - exi)];
        ss[lane] = make_float4(v.x + oxi, v.y + oyi, v.z + ozi, v.w);
    }
    __syncwarp();
    return min(32, total - c0);
}

// Near field of targets [t0, t0 + tn) of leaf c from all its source leaves
// [k0, k1): lane (grp, tl) holds targets t0 + tl + tp j, j < NT.
template <int NT>
__device__ __forceinline__ void ad_p2p_block(int c, int4 ct, int k0, int k1, int t0, int tn, int tp, int lane,
                                             float4* ss, const int* __restrict__ src, const int* __restrict__ nb,
                                             const int* __restrict__ ne, const int4* __restrict__ ic, float scale,
                                             const float4* __restrict__ pos32, const int* __restrict__ perm,
                                             double* __restrict__ pot, double* __restrict__ ax,
                                             double* __restrict__ ay, double* __restrict__ az) {
    const int G = 32 / tp, grp = lane / tp, tl = lane % tp;
    float4 pt[NT];
    float ph[NT], gx[NT], gy[NT], gz[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int k = tl + tp * j;
        pt[j] = k < tn ? pos32[t0 + k] : make_float4(0.f, 0.f, 0.f, 0.f);
        ph[j] = 0.f; gx[j] = 0.f; gy[j] = 0.f; gz[j] = 0.f;
    }
    for (int kb = k0; kb < k1; kb += 32) {
        // metadata of up to 32 source leaves, one per lane
        const int kk = kb + lane;
        int cntS = 0, sb = 0;
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (kk < k1) {
            const int S = src[kk];
            const int4 cs = ic[S];
            ox = (float)(cs.x - ct.x) * scale;
            oy = (float)(cs.y - ct.y) * scale;
            oz = (float)(cs.z - ct.z) * scale;
            sb = nb[S];
            cntS = ne[S] - sb;
        }
        int incl = cntS;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31), excl = incl - cntS;
        // the target leaf's own particles in this batch: [s0, s1) of the concatenation
        const unsigned selfm = __ballot_sync(0xffffffffu, kk < k1 && src[kk < k1 ? kk : k0] == c);
        int s0 = total, s1 = total;
        if (selfm) {
            const int sl = __ffs(selfm) - 1;
            s0 = __shfl_sync(0xffffffffu, excl, sl);
            s1 = __shfl_sync(0xffffffffu, incl, sl);
        }
        for (int c0 = 0; c0 < total; c0 += 32) {
            const int cnt = p2p_stage(ss, lane, c0, total, incl, excl, sb, ox, oy, oz, pos32);
            if (c0 < s1 && c0 + 32 > s0) {
                for (int k = grp; k < cnt; k += G) {
                    const float4 sv = ss[k];
#pragma unroll
                    for (int j = 0; j < NT; ++j) p2p_acc<true>(sv, pt[j].x, pt[j].y, pt[j].z, ph[j], gx[j], gy[j], gz[j]);
                }
            } else {
#pragma unroll 2
                for (int k = grp; k < cnt; k += G) {
                    const float4 sv = ss[k];
#pragma unroll
                    for (int j = 0; j < NT; ++j)
                        p2p_acc<false>(sv, pt[j].x, pt[j].y, pt[j].z, ph[j], gx[j], gy[j], gz[j]);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j)
        for (int o = tp; o < 32; o <<= 1) {
            ph[j] += __shfl_xor_sync(0xffffffffu, ph[j], o); gx[j] += __shfl_xor_sync(0xffffffffu, gx[j], o);
            gy[j] += __shfl_xor_sync(0xffffffffu, gy[j], o); gz[j] += __shfl_xor_sync(0xffffffffu, gz[j], o);
        }
    if (grp == 0) {
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int k = tl + tp * j;
            if (k < tn) {
                const int o = perm[t0 + k];
                pot[o] -= (double)ph[j]; ax[o] += (double)gx[j]; ay[o] += (double)gy[j]; az[o] += (double)gz[j];
            }
        }
    }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_ad_p2p32(int nwork, const int* __restrict__ work, const int* __restrict__ off, const int* __restrict__ src,
           const int* __restrict__ nb, const int* __restrict__ ne, const int4* __restrict__ ic, float scale,
           const float4* __restrict__ pos32, const int* __restrict__ perm, double* __restrict__ pot,
           double* __restrict__ ax, double* __restrict__ ay, double* __restrict__ az, int* __restrict__ counter) {
    __shared__ float4 ss[WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nwork) break;
        const int c = work[item];
        const int4 ct = ic[c];
        const int b = nb[c], e = ne[c];
        const int k0 = off[c], k1 = off[c + 1];
        for (int t0 = b; t0 < e; t0 += 32) {
            const int tn = min(32, e - t0);
            if (tn <= 8)
                ad_p2p_block<2>(c, ct, k0, k1, t0, tn, 4, lane, ss[w], src, nb, ne, ic, scale, pos32, perm, pot, ax,
                                ay, az);
            else if (tn <= 16)
                ad_p2p_block<2>(c, ct, k0, k1, t0, tn, 8, lane, ss[w], src, nb, ne, ic, scale, pos32, perm, pot, ax,
                                ay, az);
            else if (tn <= 24)
                ad_p2p_block<3>(c, ct, k0, k1, t0, tn, 8, lane, ss[w], src, nb, ne, ic, scale, pos32, perm, pot, ax,
                                ay, az);
            else
                ad_p2p_block<4>(c, ct, k0, k1, t0, tn, 8, lane, ss[w], src, nb, ne, ic, scale, pos32, perm, pot, ax,
                                ay, az);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int ad_pos32(int nleaf, const int* leaf, const int* nb, const int* ne, const double* zc, const double* xs,
             const double* ys, const double* zs, const double* qs, float4* pos32, cudaStream_t s) {
    if (nleaf <= 0) return 0;
    k_ad_pos32<<<(unsigned)(((int64_t)nleaf * 32 + 255) / 256), 256, 0, s>>>(nleaf, leaf, nb, ne, zc, xs, ys, zs, qs,
                                                                            pos32);
    count_launch();
    return 0;
}

int ad_icentre(int nn, const int* lev, const int* ix, const int* iy, const int* iz, int4* ic, cudaStream_t s) {
    if (nn <= 0) return 0;
    k_ad_icentre<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(nn, lev, ix, iy, iz, ic);
    count_launch();
    return 0;
}

#define AD_P_SWITCH(P_, CALL) \
    switch (P_) {             \
        case 0: CALL(0); break; case 1: CALL(1); break; case 2: CALL(2); break; case 3: CALL(3); break; \
        case 4: CALL(4); break; case 5: CALL(5); break; case 6: CALL(6); break; case 7: CALL(7); break; \
        case 8: CALL(8); break; case 9: CALL(9); break; default: CALL(10); break; }

int ad_p2m_leaf(int prec, int p, int basis, int nleaf, const int* leaf, const int* nb, const int* ne,
                const double* zc, const double* xs, const double* ys, const double* zs, const double* qs,
                const float4* pos32, double* Mn, const DevTables& Tb, const int* lev, double side, cudaStream_t s) {
    if (nleaf <= 0) return 0;
    constexpr int W = 4;
    const unsigned g = (unsigned)((nleaf + W - 1) / W);
#define C64(P) k_ad_p2m<P, double, W><<<g, W * 32, 0, s>>>(basis, nleaf, leaf, nb, ne, zc, xs, ys, zs, qs, nullptr, \
                                                            Mn, Tb.detr, Tb.offsets(), lev, side)
#define C32(P) k_ad_p2m<P, float, W><<<g, W * 32, 0, s>>>(basis, nleaf, leaf, nb, ne, zc, xs, ys, zs, qs, pos32, \
                                                           Mn, Tb.detr32, Tb.offsets(), lev, side)
    if (prec == 0) { AD_P_SWITCH(p, C64) } else { AD_P_SWITCH(p, C32) }
#undef C64
#undef C32
    count_launch();
    return 0;
}

int ad_l2p_leaf(int prec, int p, int basis, int nleaf, const int* leaf, const int* nb, const int* ne,
                const double* zc, const double* xs, const double* ys, const double* zs, const float4* pos32,
                const int* perm, const double* Ln, const DevTables& Tb, double* pot, double* ax, double* ay,
                double* az, const int* lev, double side, cudaStream_t s) {
    if (nleaf <= 0) return 0;
    constexpr int W = 4;
    const unsigned g = (unsigned)((nleaf + W - 1) / W);
#define C64(P) k_ad_l2p<P, double, W><<<g, W * 32, 0, s>>>(basis, nleaf, leaf, nb, ne, zc, xs, ys, zs, nullptr, \
                                                            perm, Ln, Tb.expand, Tb.offsets(), pot, ax, ay, az, \
                                                            lev, side)
#define C32(P) k_ad_l2p<P, float, W><<<g, W * 32, 0, s>>>(basis, nleaf, leaf, nb, ne, zc, xs, ys, zs, pos32, \
                                                           perm, Ln, Tb.expand32, Tb.offsets(), pot, ax, ay, az, \
                                                           lev, side)
    if (prec == 0) { AD_P_SWITCH(p, C64) } else { AD_P_SWITCH(p, C32) }
#undef C64
#undef C32
    count_launch();
    return 0;
}

int ad_p2p32(int nwork, const int* work, const int* off, const int* src, const int* nb, const int* ne, const int4* ic,
             float scale, const float4* pos32, const int* perm, double* pot, double* ax, double* ay, double* az,
             int* counter, int blocks, cudaStream_t s) {
    if (nwork <= 0) return 0;
    constexpr int W = 4;
    k_ad_p2p32<W><<<(unsigned)blocks, W * 32, 0, s>>>(nwork, work, off, src, nb, ne, ic, scale, pos32, perm, pot, ax,
                                                     ay, az, counter);
    count_launch();
    return 0;
}

}  // namespace fmm
